// Split-band fused FP32 marches for N = M P (P = 2 here with M = 4096 or
// 2048, P = 4 in fused4t_kernel.cuh with M = 4096): one row per cluster of
// 2P CTAs, CTA rank c = b P + h advances band b on the samples x[P m + h]
// (m < M), i.e. one of the P interleaved sub-sequences of its band.  The
// formulas below are written for M = 4096; they hold for any M.
//
// The length-N transform is split as N = 4096 x P (decimation in time over
// the P sub-sequences):
//   F_h[k]        = sum_m x[P m + h] W_4096^{m k}            (local, in CTA h)
//   X[k + 4096 r] = sum_h W_P^{h r} (W_N^{h k} F_h[k])       (across the band's CTAs)
// and back:
//   H_h[k]        = W_N^{-h k} sum_r W_P^{-h r} X'[k + 4096 r]
//   x'[P m + h]   = sum_k H_h[k] W_4096^{-m k}               (local)
// with X' = D X, D = (P(q) - 1)/N the propagator increment of the
// real-space increment form of Eq. fov10 (see fused2_kernel.cuh).  Every CTA
// uses the same thread -> k map, so a spectral exchange is "thread t of every
// CTA of the band swaps the values of its 16 frequencies", indexed by thread
// and value pair in the exchange buffers (see fused3_kernel.cuh) so that
// consecutive lanes hit consecutive 16-byte words.  The band coupling swaps
// psi_p with the CTA of the other band that holds the same samples.
#pragma once

#include <cooperative_groups.h>

#include "fused3_kernel.cuh"

namespace bpm {

// P = 2 with one spectral exchange per step.
//
// For P = 2 the forward combine, the propagator increment and the inverse
// combine above reduce, per local frequency k, to
//   X_r = F_0 + (-1)^r W_N^k F_1,   Y_r = D(k + M r) X_r        (r = 0, 1)
//   H_0 = Y_0 + Y_1,                H_1 = W_N^{-k} (Y_0 - Y_1)
// so each CTA only needs its peer's local spectrum F: one exchange of M
// values per CTA instead of two all-to-all rounds.  D(k) and D(k + M) are
// tabulated in FP64 and rounded once each, relative to themselves.  (The
// circulant form E_0 F_h + E_1 W^{+-k} F_{1-h}, E_{0,1} = D(k) +- D(k + M),
// saves the twiddles but rounds a small D(k) relative to the large
// D(k + M) it is paired with; repeated every step, that pushed 20000-step
// marches past the FP32 tolerance.)  Both exchanges of the step (F within
// the band, psi_p across the bands) are asynchronous remote stores that
// complete on the receiver's mbarrier (see fused3_kernel.cuh), double
// buffered by exchange parity (the step's, or for Forest-Ruth that of
// 3 step + stage); no cluster-wide barrier runs inside the march.
// Thread t sends and receives the slots of thread t, so each warp has its
// own barrier per exchange and parity and waits only for the same warp of
// the sender.
// Buffer reuse: a half is rewritten two exchanges later, by a sender that
// has by then received values the receiver computed from that half.
// PHB: strain-slice buffers (2 for the second-order step, N = 4096 only)
template <int LM, int PHB = 1>
struct F4ECfg {
  static constexpr int M = 1 << LM;
  static constexpr int N = 2 * M;
  static constexpr int T = M / 16;
  // N = 8192 stores the strain slice per part (this CTA's samples
  // contiguous); N = 4096 keeps the natural order of the other kernels of
  // that size, so the CTA takes the whole slice and reads every second cell
  static constexpr bool NAT = LM < 12;
  static constexpr int PH = NAT ? N : M;
  static constexpr int PADM = M + (M >> 4);
  static constexpr int WARPS = T / 32;
  static constexpr int OFF_BUF = 0;                        // [PADM]
  static constexpr int OFF_G = OFF_BUF + PADM * 8;         // [2][M] peer's F
  static constexpr int OFF_C = OFF_G + 2 * M * 8;          // [2][M] other band's psi_p
  static constexpr int OFF_PH = OFF_C + 2 * M * 8;         // [PHB][PH] strain slices
  static constexpr int OFF_E1 = OFF_PH + PHB * PH * 8;     // [16][T] D(k_j + M)
  static constexpr int OFF_MBAR = OFF_E1 + M * 8;          // [2] strain-slice barriers
  static constexpr int OFF_GBAR = OFF_MBAR + 16;           // [2][WARPS] F barriers
  static constexpr int OFF_CBAR = OFF_GBAR + 16 * WARPS;   // [2][WARPS] psi_p barriers
  static constexpr int OFF_PPEER = OFF_CBAR + 16 * WARPS;  // [2] peer's band-power part
  static constexpr int OFF_RECPH = OFF_PPEER + 16;
  static constexpr int OFF_RED = OFF_RECPH + 16;           // [WARPS] double
  static constexpr int OFF_PART = OFF_RED + WARPS * 8;
  static constexpr int OFF_SROW = (OFF_PART + 8 + 15) / 16 * 16;   // [2] row heads
  static constexpr int SMEM = OFF_SROW + 2 * 16;
  static_assert(SMEM <= 232448, "fits one SM");
  static_assert(LM == 11 || LM == 12, "N = 4096 or 8192");
  // layout checks: fits one SM (227 KB); bulk-copy and 16-byte store
  // targets 16-byte aligned; mbarriers 8-byte aligned
  static_assert(OFF_G % 16 == 0 && OFF_C % 16 == 0 && OFF_PH % 16 == 0,
                "16-byte stores and bulk copy");
  static_assert(OFF_MBAR % 8 == 0 && OFF_GBAR % 8 == 0 && OFF_CBAR % 8 == 0 &&
                    OFF_PPEER % 8 == 0,
                "mbarrier and 8-byte store alignment");
};

// Spectral index of position `pos` of the local forward transform's output
// (digit-reversed over the pass radices 16, ..., 16, RL).
template <int LM>
__device__ __forceinline__ int local_freq(int pos) {
  using F = F2Cfg<LM>;
  int rem = pos, len = F::N, freq = 0, mult = 1;
#pragma unroll
  for (int p = 0; p < F::NP; ++p) {
    const int r = F::radix(p), stride = len / r;
    freq += (rem / stride) * mult;
    rem %= stride;
    mult *= r;
    len = stride;
  }
  return freq;
}

// Table position of thread t's point j of the last pass (the local
// transform's output order), where the plan's split tables hold D(k_j) and
// D(k_j + M).  (The Forest-Ruth stage tables are kept in thread order
// instead: entry j T + t.)
template <int LM>
__host__ __device__ __forceinline__ int f4e_table_pos(int t, int j) {
  using F = F2Cfg<LM>;
  constexpr int R = F::radix(F::NP - 1);
  return f2_pos<LM, F::NP - 1>(f2_group<LM, F::NP - 1, true>(t, j / R), j % R);
}

__device__ __forceinline__ void st_async_f64(uint32_t raddr, double v, uint32_t rbar) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(raddr),
      "l"(__double_as_longlong(v)), "r"(rbar)
      : "memory");
}

// HALF = true: the second-order (Verlet) step, as in the 2-CTA cluster
// kernel: after the psi_p swap a CTA holds both bands at its samples,
// applies step n's second half-coupling to both and step n + 1's first half
// to its own band (a loop over shared memory); the launch's first half-step
// reads the other band from global memory.  Step n + 1's slice: at N = 4096
// a second slice buffer, fetched a step ahead; at N = 8192 there is no room
// for one, so the CTA's part of it is copied into the half of the peer
// spectrum buffer that step n has finished with (gx[n & 1]: read by this
// step's combine, rewritten by the peer only at step n + 2, after it has
// received this CTA's step n + 1 spectrum), issued once every thread is past
// the combine and awaited at the coupling.
// Separable slices: the column phasors of the CTA's samples stay in the
// slice buffer for the launch (position m holds column 2m + h), and every
// slice copy above carries the step's row head instead, into row-head slot
// 0 (slot 1 for the next step's), on the same barriers.
// SCH, the operator splitting of Eq. split-op (as in fused2_kernel.cuh):
// kSchFirst the first-order step, kSchVerlet the second-order step above,
// kSchForestRuth (N = 8192) the fourth-order step as in fused4s_kernel.cuh:
// three propagations per step with the tables of t dz, (1 - 2t) dz, t dz
// (the row's prop_split holds those of t dz, then those of (1 - 2t) dz, in
// thread order) and the inner couplings (1 - t)/2, in (am1, b), on the
// step's slice after the first two; the next slice is staged in the peer
// spectrum half of the last propagation, whose couplings read it.
template <int LM, bool EX, int SCH = kSchFirst>
__global__ void __cluster_dims__(4, 1, 1) __launch_bounds__(F4ECfg<LM>::T, 1)
    fused4e_march_kernel(const RowDescF32* __restrict__ rows, int n_rows, int steps,
                         const float4* __restrict__ tw, int* __restrict__ status) {
  namespace cg = cooperative_groups;
  constexpr bool HALF = SCH != kSchFirst;           // couples before propagating
  constexpr int STAGES = SCH == kSchForestRuth ? 3 : 1;
  static_assert(SCH != kSchForestRuth || LM == 12, "the fourth-order form is N = 8192's");
  // second-order step with the next slice staged in the peer spectrum
  // buffer (N = 8192) instead of a second slice buffer (N = 4096)
  constexpr bool HALF_G = HALF && LM == 12;
  using C = F4ECfg<LM, (HALF && !HALF_G) ? 2 : 1>;
  using F = F2Cfg<LM>;
  constexpr int L = LM, M = C::M, N = C::N, T = C::T, NP = F::NP;
  extern __shared__ __align__(128) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();

  const int c = int(cluster.block_rank());
  const int band = c >> 1, h = c & 1;
  const int row = blockIdx.x >> 2;
  const int t = threadIdx.x;
  const int lane = t & 31, warp = t >> 5;
  const RowDescF32 d = rows[row < n_rows ? row : 0];
  const bool lead = t == 0;

  float2* buf = reinterpret_cast<float2*>(smem + C::OFF_BUF);
  float2* gx = reinterpret_cast<float2*>(smem + C::OFF_G);
  float2* cb = reinterpret_cast<float2*>(smem + C::OFF_C);
  float2* ph = reinterpret_cast<float2*>(smem + C::OFF_PH);
  float2* e1s = reinterpret_cast<float2*>(smem + C::OFF_E1);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + C::OFF_MBAR);
  uint64_t* gbar = reinterpret_cast<uint64_t*>(smem + C::OFF_GBAR);
  uint64_t* cbar = reinterpret_cast<uint64_t*>(smem + C::OFF_CBAR);
  double* ppeer = reinterpret_cast<double*>(smem + C::OFF_PPEER);
  // the records' common phase, two slots by step parity: the lead writes a
  // record step's phase while a slower warp may still read the previous one
  float2* recph = reinterpret_cast<float2*>(smem + C::OFF_RECPH);
  double* red = reinterpret_cast<double*>(smem + C::OFF_RED);
  double* part = reinterpret_cast<double*>(smem + C::OFF_PART);
  float4* srow0 = reinterpret_cast<float4*>(smem + C::OFF_SROW);
  const bool sep = d.srows != nullptr;
  const uint32_t peer = uint32_t(c ^ 1);       // same band, other half of the samples
  const uint32_t partner = uint32_t(c ^ 2);    // other band, same samples
  const uint32_t g_peer = mapa_u32(smem_u32(gx), peer);
  const uint32_t gbar_peer = mapa_u32(smem_u32(gbar), peer);
  const uint32_t pp_peer = mapa_u32(smem_u32(ppeer), peer);
  const uint32_t c_part = mapa_u32(smem_u32(cb), partner);
  const uint32_t cbar_part = mapa_u32(smem_u32(cbar), partner);

  if (lead) {
    mbar_init(bar);
    if constexpr (HALF) mbar_init(bar + 1);   // N = 8192: the next-slice copies
    for (int i = 0; i < 2 * C::WARPS; ++i) {
      mbar_init(&gbar[i]);
      mbar_init(&cbar[i]);
    }
  }
  fence_mbar_init();

  float2 w0[15], w1[15];
#pragma unroll
  for (int j = 1; j < 16; ++j) {
    const float4 a = __ldg(&tw[2 * (t * j)]);
    w0[j - 1] = make_float2(a.x, a.y);
    const float4 bq = __ldg(&tw[2 * (((t % F::stride(1)) * j) << 4)]);
    w1[j - 1] = make_float2(bq.x, bq.y);
  }
  // Last-pass slice: W_N^{k_j} and D(k_j) in registers, D(k_j + M) in
  // shared memory (table [band][D(k) | D(k + M)][position]).
  const float2* dtab = C::NAT ? d.prop_split : d.prop;
  float2 cw[16], d0[16];
  // Forest-Ruth: a stage's tables, [band][D(k) | D(k + M)][j T + t] in
  // thread order (the row's prop_split), so that a warp's loads are
  // coalesced (each thread rewrites only its own D(k + M) slots)
  [[maybe_unused]] auto load_tables = [&](const float2* tab) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      d0[j] = __ldg(&tab[(band * 2 + 0) * M + j * T + t]);
      e1s[j * T + t] = __ldg(&tab[(band * 2 + 1) * M + j * T + t]);
    }
  };
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int pos = f4e_table_pos<L>(t, j);
    const float4 a = __ldg(&tw[local_freq<L>(pos)]);
    cw[j] = make_float2(a.x, a.y);
    if constexpr (SCH != kSchForestRuth) {
      d0[j] = __ldg(&dtab[(band * 2 + 0) * M + pos]);
      e1s[j * T + t] = __ldg(&dtab[(band * 2 + 1) * M + pos]);
    }
  }
  if constexpr (SCH == kSchForestRuth) load_tables(d.prop_split);

  float2 v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = d.state[band * N + 2 * (t + j * T) + h];
  // separable slices: column 2m + h at position m (the stream keeps it at
  // 2m + h for N = 4096, at h M + m for N = 8192)
  if (sep)
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int m = t + j * T;
      ph[m] = __ldg(&d.scols[C::NAT ? 2 * m + h : h * M + m]);
    }
  cluster.sync();   // every CTA's barriers initialised before any remote store

  const uint32_t slice_bytes = uint32_t(C::PH) * 8u;
  bool timed_out = false;
  double my_part = 0.0;
  // (am1, bb): the step's coupling, or the outer ones of a splitting form;
  // (am1i, bbi): Forest-Ruth's inner couplings
  const float2 am1 = HALF ? d.am1h : d.am1, bb = HALF ? d.bh : d.b;
  [[maybe_unused]] const float2 am1i = d.am1, bbi = d.b;
  const bool pow_on = d.powers != nullptr && d.record_every > 0;
  // step n's slice (the CTA's part of it) into `dst` (separable: its row
  // head into row-head slot `slot`)
  auto fetch = [&](int n, float2* dst, int slot, uint64_t* b) {
    if (sep) bulk_load(srow0 + slot, d.srows + n, kSepHeadBytes, b);
    else bulk_load(dst, d.phasor + size_t(n) * N + (C::NAT ? size_t(0) : size_t(h) * M),
                   slice_bytes, b);
  };
  if constexpr (HALF) {
    // the launch's first half-step on the slice of its first step (buffer
    // 0); later slices are fetched a step ahead into the other buffer
    // (N = 8192: into the free half of the peer spectrum buffer)
    if (lead) fetch(d.n_begin, ph, 0, bar);
    float2 q[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) q[j] = d.state[(band ^ 1) * N + 2 * (t + j * T) + h];
    if (!mbar_wait(bar, 0u)) timed_out = true;
    const SepHead sh = sep ? sep_head(srow0) : SepHead{};
    auto first_half = [&](auto S) {
      constexpr bool SEP = decltype(S)::value;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int m = t + j * T;
        v[j] = couple_cell(v[j], q[j], slice_at<SEP>(ph, sh, (SEP || !C::NAT) ? m : 2 * m + h, 2 * m + h),
                           band, am1, slice_b<SEP>(bb, sh, band));
      }
    };
    if (sep) first_half(BoolC<true>{});
    else first_half(BoolC<false>{});
  }

  const bool rec_on = d.record_every > 0 && (d.records != nullptr || d.powers != nullptr);
  RecSteps rsteps(d.record_every, d.n_begin);
  for (int it = 0; it < steps; ++it) {
    const int n = d.n_begin + it;
    const RecSteps::Step rs = rsteps.next();
    const bool rec = rec_on && rs.at;
    // the previous step was a record: its band-power part rides on this step's G
    const bool part_due = pow_on && rs.prev;
    if (lead && rec) {
      double ang = fmod(double(n + 1 - d.n_phase0) * d.gphase, 6.283185307179586);
      double sa, ca;
      sincos(ang, &sa, &ca);
      recph[(n + 1) & 1] = make_float2(float(ca), float(sa));
    }
    // one stage of the step (Forest-Ruth: three; the others: one, with no
    // loop around it)
    auto stage = [&](const int sg) {
    // exchange index of the stage: buffer halves and barrier phases
    const int ex = it * STAGES + sg;
    const int half = ex & 1;
    const uint32_t xpar = uint32_t((ex >> 1) & 1);
    if constexpr (SCH == kSchForestRuth) {
      // the stage's tables: (P^t - 1)/N for stages 0 and 2, (P^(1-2t) - 1)/N
      // for stage 1
      if (sg > 0) load_tables(d.prop_split + (sg == 1 ? 4 * M : 0));
    }
    float2 org[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) org[j] = v[j];
    dft<16, false, EX>(v);
    f2_twiddle<false>(v, w0);
    f2_store<L, 0>(buf, v, t);
    __syncthreads();
    if (lead && sg == 0) {
      if constexpr (HALF_G) {
        // this step's slice into the one buffer (phase it + 1: the launch's
        // first half-step took phase 0); the next one goes to L2 now and to
        // the peer spectrum buffer once the combine is done
        fetch(n, ph, 0, bar);
        if (!sep && it + 1 < steps)
          bulk_prefetch_l2(d.phasor + size_t(n + 1) * N + size_t(h) * M, slice_bytes);
      } else if constexpr (HALF) {
        // every thread is past step it - 1's couplings, which read the
        // buffer of slice it - 1: fetch slice it + 1 into it
        if (it + 1 < steps)
          fetch(n + 1, ph + ((it + 1) & 1) * C::PH, (it + 1) & 1, bar + ((it + 1) & 1));
      } else {
        fetch(n, ph, 0, bar);
      }
      if (part_due) {   // rides on the peer's warp-0 F barrier
        double s = 0.0;
        for (int w = 0; w < C::WARPS; ++w) s += red[w];
        my_part = s;
        st_async_f64(pp_peer + uint32_t(half) * 8u, s,
                     gbar_peer + uint32_t(half * C::WARPS) * 8u);
      }
    }
    // each warp's F barrier: its 32 threads' slots from the same warp of the peer
    if (lane == 0)
      mbar_expect_tx(&gbar[half * C::WARPS + warp],
                     32u * 16u * 8u + ((lead && part_due && sg == 0) ? 8u : 0u));
    f2_load<L, 1>(buf, v, t);
    dft<16, false, EX>(v);
    f2_twiddle<false>(v, w1);
    f2_store<L, 1>(buf, v, t);
    // (passes 1 and 2 of warp w address positions [512 w, 512 w + 512) only,
    // the last pass's groups as in f2_group: the barriers between them are
    // the warp's)
    __syncwarp();
    f2_load<L, NP - 1, true>(buf, v, t);
    f2_dft<L, NP - 1, false, EX>(v);             // v[j] = F_h[k_j]
    {
      const uint32_t go = g_peer + uint32_t(half * M) * 8u;
      const uint32_t gbo = gbar_peer + uint32_t(half * C::WARPS + warp) * 8u;
#pragma unroll
      for (int pp = 0; pp < 8; ++pp)
        st_async_v4(go + uint32_t(xpair(pp, t, T)) * 8u, v[2 * pp], v[2 * pp + 1], gbo);
    }
    // (no barrier before the inverse pass rewrites buf: each thread's
    // last-pass positions are its own in both directions)
    if (!timed_out && !mbar_wait_cluster(&gbar[half * C::WARPS + warp], xpar)) timed_out = true;
    if (lead && part_due && sg == 0 && h == 0)
      d.powers[2 * rs.pslot + band] = (my_part + ppeer[half]) * d.dx_um;
    {
      const float2* gi = gx + half * M;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float4 g2 = *reinterpret_cast<const float4*>(gi + xpair(j >> 1, t, T));
        const float2 gp = (j & 1) ? make_float2(g2.z, g2.w) : make_float2(g2.x, g2.y);
        const float2 f0 = h ? gp : v[j], f1 = h ? v[j] : gp;
        const float2 w1 = cmul_f(f1, cw[j].x, cw[j].y);         // W^k F_1
        const float2 x0 = cadd(f0, w1), x1 = csub(f0, w1);
        const float2 a = d0[j], b = e1s[j * T + t];
        const float2 y0 = make_float2(fmaf(a.x, x0.x, -(a.y * x0.y)), fmaf(a.x, x0.y, a.y * x0.x));
        const float2 y1 = make_float2(fmaf(b.x, x1.x, -(b.y * x1.y)), fmaf(b.x, x1.y, b.y * x1.x));
        v[j] = h ? cmul_f(csub(y0, y1), cw[j].x, -cw[j].y) : cadd(y0, y1);
      }
    }
    f2_dft<L, NP - 1, true, EX>(v);
    f2_store<L, NP - 1, true>(buf, v, t);
    if (HALF_G && sg == STAGES - 1) {
      // the next-slice copy of a splitting form waits for every thread to be
      // past the combine, the last reader of gx[half]
      __syncthreads();
      if (lead && it + 1 < steps) fetch(n + 1, gx + half * M, 1, bar + 1);
    } else {
      __syncwarp();
    }
    f2_load<L, 1>(buf, v, t);
    f2_twiddle<true>(v, w1);
    dft<16, true, EX>(v);
    f2_store<L, 1>(buf, v, t);
    __syncthreads();
    f2_load<L, 0>(buf, v, t);
    f2_twiddle<true>(v, w0);
    dft<16, true, EX>(v);
    {
      if (lane == 0) mbar_expect_tx(&cbar[half * C::WARPS + warp], 32u * 16u * 8u);
      const uint32_t co = c_part + uint32_t(half * M) * 8u;
      const uint32_t cbo = cbar_part + uint32_t(half * C::WARPS + warp) * 8u;
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = cadd(org[j], v[j]);
#pragma unroll
      for (int pp = 0; pp < 8; ++pp)
        st_async_v4(co + uint32_t(xpair(pp, t, T)) * 8u, v[2 * pp], v[2 * pp + 1], cbo);
    }
    // first order: the step's slice, its row head and the coupling
    // coefficient while the psi_p stores are in flight (the 16-point N = 4096
    // split: 26.5 -> 25.3 ms per 8000-step solve; at N = 8192 this order
    // measured 1 % slower, so there they follow the psi_p wait)
    constexpr bool EARLY = !HALF && LM == 11;
    [[maybe_unused]] SepHead sh1{};
    [[maybe_unused]] float2 bs1 = bb;
    if constexpr (EARLY) {
      if (!timed_out && !mbar_wait(bar, uint32_t(it & 1))) timed_out = true;
      if (sep) {
        sh1 = sep_head(srow0);
        bs1 = slice_b<true>(bb, sh1, band);
      }
    }
    if (!timed_out && !mbar_wait_cluster(&cbar[half * C::WARPS + warp], xpar)) timed_out = true;
    if constexpr (HALF) {
      const bool last = sg == STAGES - 1;
      const bool next = last && it + 1 < steps;
      if constexpr (HALF_G) {
        if (sg == 0 && !timed_out && !mbar_wait(bar, uint32_t((it + 1) & 1))) timed_out = true;
        if (next && !timed_out && !mbar_wait(bar + 1, uint32_t(it & 1))) timed_out = true;
      } else {
        if (next && !timed_out &&
            !mbar_wait(bar + ((it + 1) & 1), uint32_t(((it + 1) >> 1) & 1)))
          timed_out = true;
      }
      const float2* ci = cb + half * M;
      // (separable: the couplings read the column phasors of buffer 0 and
      // the row heads of steps it and it + 1)
      const float2* phc = (HALF_G || sep) ? ph : ph + (it & 1) * C::PH;
      const SepHead shc = sep ? sep_head(srow0 + (HALF_G ? 0 : (it & 1))) : SepHead{};
      if (STAGES > 1 && !last) {
        // Forest-Ruth, after the first two propagations: the inner
        // couplings ((1 - t)/2) on this step's slice
        auto couple_inner = [&](auto S) {
          constexpr bool SEP = decltype(S)::value;
          const float2 bs = slice_b<SEP>(bbi, shc, band);
#pragma unroll
          for (int pp = 0; pp < 8; ++pp) {
            const float4 q2 = *reinterpret_cast<const float4*>(ci + xpair(pp, t, T));
            const int m0 = t + 2 * pp * T, m1 = t + (2 * pp + 1) * T;
            const int c0 = (SEP || !C::NAT) ? m0 : 2 * m0 + h;
            const int c1 = (SEP || !C::NAT) ? m1 : 2 * m1 + h;
            v[2 * pp] = couple_cell(v[2 * pp], make_float2(q2.x, q2.y),
                                    slice_at<SEP>(phc, shc, c0, 2 * m0 + h), band, am1i, bs);
            v[2 * pp + 1] = couple_cell(v[2 * pp + 1], make_float2(q2.z, q2.w),
                                        slice_at<SEP>(phc, shc, c1, 2 * m1 + h), band, am1i, bs);
          }
        };
        if (sep) couple_inner(BoolC<true>{});
        else couple_inner(BoolC<false>{});
      } else {
        const float2* phn = sep ? ph : HALF_G ? gx + half * M : ph + ((it + 1) & 1) * C::PH;
        const SepHead shn =
            (sep && next) ? sep_head(srow0 + (HALF_G ? 1 : ((it + 1) & 1))) : SepHead{};
        const float2 g = rec ? recph[(n + 1) & 1] : make_float2(1.f, 0.f);
        const int slot = rec ? rs.slot : 0;
        float2* r0 = (rec && d.records) ? d.records + size_t(slot) * 2 * N + band * N : nullptr;
        double s = 0.0;
        // a loop over shared memory (three couplings per point unrolled over
        // 16 points would overflow the instruction cache); buf is free once
        // every thread is past the inverse pass 0, and again for the next
        // step once every thread has taken its points back
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 16; ++j) buf[t + j * T] = v[j];
        auto three_halves = [&](auto S) {
          constexpr bool SEP = decltype(S)::value;
          const float2 bc = slice_b<SEP>(bb, shc, band), bo = slice_b<SEP>(bb, shc, band ^ 1);
          const float2 bn = slice_b<SEP>(bb, shn, band);
#pragma unroll 1
          for (int pp = 0; pp < 8; ++pp) {
            const float4 q2 = *reinterpret_cast<const float4*>(ci + xpair(pp, t, T));
#pragma unroll
            for (int k = 0; k < 2; ++k) {
              const int j = 2 * pp + k;
              const int m = t + j * T;
              const int cell = (SEP || !C::NAT) ? m : 2 * m + h;
              const float2 p = buf[m], q = k ? make_float2(q2.z, q2.w) : make_float2(q2.x, q2.y);
              const float2 e = slice_at<SEP>(phc, shc, cell, 2 * m + h);
              float2 c = couple_cell(p, q, e, band, am1, bc);   // step it, second half
              if (rec) {
                s = pow_acc(s, c);
                if (r0)   // records in natural order
                  r0[2 * m + h] = make_float2(fmaf(c.x, g.x, -(c.y * g.y)), fmaf(c.x, g.y, c.y * g.x));
              }
              if (next) {   // step it + 1, first half, with the other band's value
                const float2 co = couple_cell(q, p, e, band ^ 1, am1, bo);
                c = couple_cell(c, co, slice_at<SEP>(phn, shn, cell, 2 * m + h), band, am1, bn);
              }
              buf[m] = c;
            }
          }
        };
        if (sep) three_halves(BoolC<true>{});
        else three_halves(BoolC<false>{});
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = buf[t + j * T];
        __syncthreads();
        if (rec && d.powers) {
          double ds = s;
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) ds += __shfl_xor_sync(0xffffffffu, ds, off);
          if (lane == 0) red[warp] = ds;   // summed by the lead after the next barrier
        }
      }
    } else {
      if constexpr (!EARLY) {
        if (!timed_out && !mbar_wait(bar, uint32_t(it & 1))) timed_out = true;
        if (sep) {
          sh1 = sep_head(srow0);
          bs1 = slice_b<true>(bb, sh1, band);
        }
      }
      const float2* ci = cb + half * M;
      const SepHead sh = sh1;
      auto couple_all = [&](auto S) {
        constexpr bool SEP = decltype(S)::value;
        const float2 bs = SEP ? bs1 : bb;
#pragma unroll
        for (int pp = 0; pp < 8; ++pp) {
          const float4 q2 = *reinterpret_cast<const float4*>(ci + xpair(pp, t, T));
          const int m0 = t + 2 * pp * T, m1 = t + (2 * pp + 1) * T;
          const int c0 = (SEP || !C::NAT) ? m0 : 2 * m0 + h;
          const int c1 = (SEP || !C::NAT) ? m1 : 2 * m1 + h;
          v[2 * pp] = couple_cell(v[2 * pp], make_float2(q2.x, q2.y),
                                  slice_at<SEP>(ph, sh, c0, 2 * m0 + h), band, am1, bs);
          v[2 * pp + 1] = couple_cell(v[2 * pp + 1], make_float2(q2.z, q2.w),
                                      slice_at<SEP>(ph, sh, c1, 2 * m1 + h), band, am1, bs);
        }
      };
      if (sep) couple_all(BoolC<true>{});
      else couple_all(BoolC<false>{});

      if (rec) {
        const int slot = rs.slot;
        const float2 g = recph[(n + 1) & 1];
        double s = 0.0;
        float2* r0 = d.records ? d.records + size_t(slot) * 2 * N + band * N : nullptr;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float2 p = v[j];
          s = pow_acc(s, p);
          if (r0)
            r0[2 * (t + j * T) + h] =
                make_float2(fmaf(p.x, g.x, -(p.y * g.y)), fmaf(p.x, g.y, p.y * g.x));
        }
        if (d.powers) {
          double ds = s;
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) ds += __shfl_xor_sync(0xffffffffu, ds, off);
          if (lane == 0) red[warp] = ds;   // summed by the lead after the next barrier
        }
      }
    }
    };
    if constexpr (STAGES == 1) {
      stage(0);
    } else {
#pragma unroll 1
      for (int sg = 0; sg < STAGES; ++sg) stage(sg);
    }   // (the Forest-Ruth step ends on the t dz tables, which its next step
        // starts with)
  }

  __syncthreads();
  // the band power of a record in the launch's last step has no next step
  // to ride on: exchange it through the cluster's shared memory
  const bool last_due = pow_on && steps > 0 && ((d.n_begin + steps) % d.record_every) == 0;
  if (lead && last_due) {
    double s = 0.0;
    for (int w = 0; w < C::WARPS; ++w) s += red[w];
    *part = s;
  }
  cluster.sync();
  if (lead && last_due && h == 0)
    d.powers[2 * ((d.n_begin + steps) / d.record_every - 1) + band] =
        (*part + *cluster.map_shared_rank(part, int(peer))) * d.dx_um;
#pragma unroll
  for (int j = 0; j < 16; ++j) d.state[band * N + 2 * (t + j * T) + h] = v[j];
  // Error path: after an expired wait a thread skips its later waits and the
  // march runs on to the end of the launch; the lead still issues one slice
  // copy per step on its barrier, so waiting (again bounded) for the last
  // step's phase leaves no copy of its own in flight when the CTA exits.
  if (timed_out) {
    if constexpr (HALF_G) {
      // the slice copies: phase `steps` of bar (phase 0 was the launch's
      // first half-step), phase steps - 2 of the next-slice barrier
      if (lead && steps >= 2) mbar_wait(bar + 1, uint32_t(steps & 1));
      give_up_after_march(bar, uint32_t(steps & 1), lead, status);
    } else if constexpr (HALF) {   // the last slice copy: step steps - 1, in its buffer
      give_up_after_march(bar + ((steps - 1) & 1), uint32_t(((steps - 1) >> 1) & 1), lead, status);
    } else {
      give_up_after_march(bar, uint32_t((steps - 1) & 1), lead, status);
    }
  }
  cluster.sync();   // peers may still read our shared memory
}

}  // namespace bpm
