// N = 4096 as a half-band split (as in fused4_kernel.cuh, P = 2, M = 2048)
// with 8 points per thread: 256 threads per CTA, two warps per scheduler.
//
// The 4-CTA cluster layout is the one of fused4e_march_kernel<11>: CTA rank
// c = 2 band + h holds the samples x[2 m + h] of band b; one exchange of the
// local spectrum F with the other half of the band per step, then
//   X_r = F_0 + (-1)^r W_N^k F_1,   Y_r = D(k + M r) X_r,
//   H_0 = Y_0 + Y_1,                H_1 = W_N^{-k} (Y_0 - Y_1),
// and one swap of psi_p with the CTA of the other band.  The local
// 2048-point transform runs as radix 8, 8, 8, 4 passes (decimation in
// frequency, digit-reversed output; the inverse mirrors it), so each thread
// does half the serial work of the 16-point form and each scheduler has two
// warps to issue from, at the price of one more shared-memory pass per
// transform.  Passes 1-3 of a warp stay within its own 256 positions (see
// s4_group), so of the eight passes of a step only the two next to pass 0
// end in a CTA barrier; the others end in the warp's own.  Thread t sends
// and receives the slots of thread t in both exchanges, so each warp has
// its own pair of exchange barriers and waits only for the same warp of
// the peer (the peer's slowest warp no longer holds up the others).  The propagator
// increments D(k), D(k + M) come from the plan's half-band tables, which are
// stored in the 16-point form's output order: each thread looks its
// frequencies up once per launch.
#pragma once

#include <cooperative_groups.h>

#include "fused4_kernel.cuh"

namespace bpm {

// Pass structure of a 2^LM-point transform with 8 points per thread.
template <int LM>
struct F8Cfg {
  static constexpr int N = 1 << LM;
  static constexpr int E = 8;
  static constexpr int T = N / E;
  static constexpr int NP = (LM + 2) / 3;
  static constexpr int RL = 1 << (LM - 3 * (NP - 1));
  __host__ __device__ static constexpr int radix(int p) { return p < NP - 1 ? 8 : RL; }
  __host__ __device__ static constexpr int len(int p) { return N >> (3 * p); }
  __host__ __device__ static constexpr int stride(int p) { return len(p) / radix(p); }
  __host__ __device__ static constexpr int groups(int p) { return E / radix(p); }
};

template <int LM, int P>
__device__ __forceinline__ int f8_pos(int gi, int j) {
  using C = F8Cfg<LM>;
  constexpr int S = C::stride(P), L = C::len(P);
  return (gi / S) * L + (gi % S) + j * S;
}

// Shared-memory address of transform position p: within each row of 16
// float2 (eight 16-byte bank pairs twice), the position is XOR-ed with
// 4 ((p >> 5) & 3) + ((p >> 4) & 3).  With it the half-warps of all four
// pass patterns (stride 256 and 32: consecutive; stride 4: 32 a + b + 4 j;
// stride 1: 4 l + j) touch 16 distinct bank pairs; a pad of one slot per 16
// left the stride-4 pass 2-way conflicted.
__device__ __forceinline__ int swz8(int p) { return p ^ (((p >> 3) & 12) | ((p >> 4) & 3)); }

template <int LM, int P>
__device__ __forceinline__ void f8_store(float2* buf, const float2* v, int t) {
  using C = F8Cfg<LM>;
  constexpr int R = C::radix(P), G = C::groups(P);
#pragma unroll
  for (int i = 0; i < G; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) buf[swz8(f8_pos<LM, P>(t + i * C::T, j))] = v[i * R + j];
}

template <int LM, int P>
__device__ __forceinline__ void f8_load(const float2* buf, float2* v, int t) {
  using C = F8Cfg<LM>;
  constexpr int R = C::radix(P), G = C::groups(P);
#pragma unroll
  for (int i = 0; i < G; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) v[i * R + j] = buf[swz8(f8_pos<LM, P>(t + i * C::T, j))];
}

template <int LM, int P, bool INV, bool EX>
__device__ __forceinline__ void f8_dft(float2* v) {
  using C = F8Cfg<LM>;
  constexpr int R = C::radix(P), G = C::groups(P);
#pragma unroll
  for (int i = 0; i < G; ++i) dft<R, INV, EX>(v + i * R);
}

// radix-8 twiddle pass with register twiddles w[j-1] = W^{o j}
template <bool INV>
__device__ __forceinline__ void f8_twiddle(float2* v, const float2* w) {
#pragma unroll
  for (int j = 1; j < 8; ++j) {
    const float2 t = w[j - 1];
    v[j] = INV ? cmul_f(v[j], t.x, -t.y) : cmul_f(v[j], t.x, t.y);
  }
}

// Spectral index of position `pos` of the forward transform's output.
template <typename Cfg>
__host__ __device__ __forceinline__ int cfg_freq(int pos) {
  int rem = pos, len = Cfg::N, freq = 0, mult = 1;
#pragma unroll
  for (int p = 0; p < Cfg::NP; ++p) {
    const int r = Cfg::radix(p), stride = len / r;
    freq += (rem / stride) * mult;
    rem %= stride;
    mult *= r;
    len = stride;
  }
  return freq;
}

// Position of frequency k in the 16-point form's output order (radices 16,
// 16, 8 for 2048 points): the inverse of local_freq<11>.
__host__ __device__ __forceinline__ int pos16_of_freq2048(int k) {
  return (k & 15) * 128 + ((k >> 4) & 15) * 8 + (k >> 8);
}

// PHB: strain-slice buffers (2 for the second-order step, which couples
// with the slices of two steps at a time)
template <int PHB = 1>
struct F4SCfg {
  static constexpr int M = 2048;
  static constexpr int N = 2 * M;
  static constexpr int T = M / 8;
  static constexpr int PADM = M + (M >> 4);
  static constexpr int WARPS = T / 32;
  static constexpr int OFF_BUF = 0;                        // [PADM]
  static constexpr int OFF_G = OFF_BUF + PADM * 8;         // [2][M] peer's F
  static constexpr int OFF_C = OFF_G + 2 * M * 8;          // [2][M] other band's psi_p
  static constexpr int OFF_PH = OFF_C + 2 * M * 8;         // [PHB][N] strain slices (natural order)
  static constexpr int OFF_E1 = OFF_PH + PHB * N * 8;      // [8][T] D(k_j + M)
  static constexpr int OFF_MBAR = OFF_E1 + M * 8;          // [PHB] strain-slice barriers
  static constexpr int OFF_GBAR = OFF_MBAR + 8 * PHB;      // [2][WARPS] F barriers
  static constexpr int OFF_CBAR = OFF_GBAR + 16 * WARPS;   // [2][WARPS] psi_p barriers
  static constexpr int OFF_PPEER = OFF_CBAR + 16 * WARPS;  // [2] peer's band-power part
  static constexpr int OFF_RECPH = OFF_PPEER + 16;
  static constexpr int OFF_RED = OFF_RECPH + 16;           // [WARPS] double
  static constexpr int OFF_PART = OFF_RED + WARPS * 8;
  static constexpr int OFF_SROW = (OFF_PART + 8 + 15) / 16 * 16;   // [2] row heads
  static constexpr int SMEM = OFF_SROW + 2 * 16;
  static_assert(SMEM <= 232448, "fits one SM");
  static_assert(OFF_G % 16 == 0 && OFF_C % 16 == 0 && OFF_PH % 16 == 0,
                "16-byte stores and bulk copy");
  static_assert(OFF_MBAR % 8 == 0 && OFF_GBAR % 8 == 0 && OFF_CBAR % 8 == 0 &&
                    OFF_PPEER % 8 == 0,
                "mbarrier and 8-byte store alignment");
};

// Groups of the last pass (radix 4, two per thread), chosen so that passes
// 1, 2 and 3 of warp w all stay within positions [256 w, 256 w + 256): group
// i of thread t is 64 (t / 32) + 32 i + t mod 32.  Pass 1 (stride 32) and
// pass 2 (stride 4) of warp w already address only that block, so between
// passes 1, 2 and 3 (in both directions) a warp waits for itself alone; only
// the passes to and from pass 0 (stride 256) need the whole CTA.
__host__ __device__ __forceinline__ int s4_group(int t, int i) {
  return (t >> 5) * 64 + i * 32 + (t & 31);
}

// Table position of thread t's point j of the last pass: the 16-point
// form's output position of its frequency k_j, where the plan's half-band
// tables hold D(k_j) and D(k_j + M).  (The Forest-Ruth stage tables are kept
// in thread order instead: entry j T + t.)
__host__ __device__ __forceinline__ int s4_table_pos(int t, int j) {
  using F = F8Cfg<11>;
  return pos16_of_freq2048(cfg_freq<F>(s4_group(t, j / F::RL) * F::RL + j % F::RL));
}

__device__ __forceinline__ void s4_store_last(float2* buf, const float2* v, int t) {
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) buf[swz8(s4_group(t, i) * 4 + j)] = v[i * 4 + j];
}

__device__ __forceinline__ void s4_load_last(const float2* buf, float2* v, int t) {
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) v[i * 4 + j] = buf[swz8(s4_group(t, i) * 4 + j)];
}

// SCH, the operator splitting of Eq. split-op (as in fused2_kernel.cuh):
// kSchFirst the first-order step; kSchVerlet the second-order step: after
// the psi_p swap a CTA holds both bands at its samples, so it applies step
// n's second half-coupling to both and step n + 1's first half to its own
// band (8 points per thread: in registers); the launch's first half-step
// reads the other band from global memory; kSchForestRuth the fourth-order
// step: the same with three propagations per step (t dz, (1 - 2t) dz, t dz,
// each with its own half-band tables: the row's prop_split holds those of t
// dz then those of (1 - 2t) dz) and the inner couplings ((1 - t)/2, in
// (am1, b)) after the first two; (am1h, bh) are the outer couplings (t/2).
// The splitting forms fetch step n + 1's slice a step ahead into the second
// buffer (separable slices: its row head into the second row-head slot);
// records are taken after step n's last coupling.
template <bool EX, int SCH = kSchFirst>
__global__ void __cluster_dims__(4, 1, 1) __launch_bounds__(F4SCfg<>::T, 1)
    fused4s_march_kernel(const RowDescF32* __restrict__ rows, int n_rows, int steps,
                         const float4* __restrict__ tw, int* __restrict__ status) {
  namespace cg = cooperative_groups;
  constexpr bool HALF = SCH != kSchFirst;           // couples before propagating
  constexpr int STAGES = SCH == kSchForestRuth ? 3 : 1;
  using C = F4SCfg<HALF ? 2 : 1>;
  using F = F8Cfg<11>;
  constexpr int L = 11, M = C::M, N = C::N, T = C::T, NP = F::NP, RL = F::RL;
  static_assert(NP == 4 && RL == 4, "2048 = 8 x 8 x 8 x 4");
  static_assert(T == 256, "the interval masks take T = 2^8");
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
  float4* srow = reinterpret_cast<float4*>(smem + C::OFF_SROW);
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
    if constexpr (HALF) mbar_init(bar + 1);
    for (int i = 0; i < 2 * C::WARPS; ++i) {
      mbar_init(&gbar[i]);
      mbar_init(&cbar[i]);
    }
  }
  fence_mbar_init();

  // twiddles of passes 0, 1, 2: W_{len(p)}^{o j}, o = t mod stride(p),
  // from the W_N table (N = 2M): index 2 o j M / len(p)
  float2 w0[7], w1[7], w2[7];
#pragma unroll
  for (int j = 1; j < 8; ++j) {
    const float4 a = __ldg(&tw[2 * ((t % F::stride(0)) * j) * (M / F::len(0))]);
    w0[j - 1] = make_float2(a.x, a.y);
    const float4 b1 = __ldg(&tw[2 * ((t % F::stride(1)) * j) * (M / F::len(1))]);
    w1[j - 1] = make_float2(b1.x, b1.y);
    const float4 b2 = __ldg(&tw[2 * ((t % F::stride(2)) * j) * (M / F::len(2))]);
    w2[j - 1] = make_float2(b2.x, b2.y);
  }
  // Last-pass slice: W_N^{k_j} and D(k_j) in registers, D(k_j + M) in shared
  // memory; the plan's table [band][D(k) | D(k + M)][position] is in the
  // 16-point form's output order.
  float2 cw[8], d0[8];
  // Forest-Ruth: a stage's tables, [band][D(k) | D(k + M)][j T + t] in
  // thread order, so that a warp's loads are coalesced (each thread
  // rewrites only its own D(k + M) slots)
  [[maybe_unused]] auto load_tables = [&](const float2* tab) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      d0[j] = __ldg(&tab[(band * 2 + 0) * M + j * T + t]);
      e1s[j * T + t] = __ldg(&tab[(band * 2 + 1) * M + j * T + t]);
    }
  };
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int k = cfg_freq<F>(s4_group(t, j / RL) * RL + j % RL);
    const float4 a = __ldg(&tw[k]);
    cw[j] = make_float2(a.x, a.y);
    if constexpr (SCH != kSchForestRuth) {
      const int p16 = s4_table_pos(t, j);
      d0[j] = __ldg(&d.prop_split[(band * 2 + 0) * M + p16]);
      e1s[j * T + t] = __ldg(&d.prop_split[(band * 2 + 1) * M + p16]);
    }
  }
  if constexpr (SCH == kSchForestRuth) load_tables(d.prop_split);

  float2 v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = d.state[band * N + 2 * (t + j * T) + h];
  // separable slices: the phasor of column 2m + h at position m of the slice
  // buffer for the launch (each thread reads its own points: no conflicts)
  if (sep)
#pragma unroll
    for (int j = 0; j < 8; ++j) ph[t + j * T] = __ldg(&d.scols[2 * (t + j * T) + h]);
  cluster.sync();   // every CTA's barriers initialised before any remote store

  const uint32_t slice_bytes = uint32_t(N) * 8u;
  bool timed_out = false;
  double my_part = 0.0;
  // (am1, bb): the step's coupling, or the outer ones of a splitting form;
  // (am1i, bbi): Forest-Ruth's inner couplings
  const float2 am1 = HALF ? d.am1h : d.am1, bb = HALF ? d.bh : d.b;
  [[maybe_unused]] const float2 am1i = d.am1, bbi = d.b;
  const bool pow_on = d.powers != nullptr && d.record_every > 0;
  const bool rec_on = d.record_every > 0 && (d.records != nullptr || d.powers != nullptr);
  RecSteps rsteps(d.record_every, d.n_begin);
  // step n's slice into buffer `slot` (separable: its row head into row-head
  // slot `slot`; the column phasors stay in buffer 0)
  auto fetch = [&](int n, int slot) {
    if (sep) bulk_load(srow + slot, d.srows + n, kSepHeadBytes, bar + slot);
    else bulk_load(ph + slot * N, d.phasor + size_t(n) * N, slice_bytes, bar + slot);
  };
  if constexpr (HALF) {
    // the launch's first half-step, on the slice of its first step
    if (lead) fetch(d.n_begin, 0);
    float2 q[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) q[j] = d.state[(band ^ 1) * N + 2 * (t + j * T) + h];
    if (!mbar_wait(bar, 0u)) timed_out = true;
    const SepHead sh = sep ? sep_head(srow) : SepHead{};
    auto first_half = [&](auto S) {
      constexpr bool SEP = decltype(S)::value;
      const uint32_t msk = SEP ? sep_mask<1, 8, 8>(sh, t, h) : 0u;
      const float2 bs = slice_b<SEP>(bb, sh, band);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int m = t + j * T;
        v[j] = couple_at<SEP>(v[j], q[j], ph, SEP ? m : 2 * m + h, msk, j, band, am1, bs);
      }
    };
    if (sep) first_half(BoolC<true>{});
    else first_half(BoolC<false>{});
  }

  for (int it = 0; it < steps; ++it) {
    const int n = d.n_begin + it;
    const RecSteps::Step rs = rsteps.next();
    const bool rec = rec_on && rs.at;
    // the previous step was a record: its band-power part rides on this step's F
    const bool part_due = pow_on && rs.prev;
    const int rslot = rs.slot, pslot = rs.pslot;
    if (lead && rec) {
      double ang = fmod(double(n + 1 - d.n_phase0) * d.gphase, 6.283185307179586);
      double sa, ca;
      sincos(ang, &sa, &ca);
      recph[(n + 1) & 1] = make_float2(float(ca), float(sa));
    }
    // one stage of the step (Forest-Ruth: three; the others: one, with no
    // loop around it, which measured 2.5 % faster than a loop of one)
    auto stage = [&](const int sg) {
    // exchange index of the stage: buffer halves and barrier phases
    const int ex = it * STAGES + sg;
    const int half = ex & 1;
    const uint32_t xpar = uint32_t((ex >> 1) & 1);
    if constexpr (SCH == kSchForestRuth) {
      // the stage's tables: (P^t - 1)/N for stages 0 and 2, (P^(1-2t) - 1)/N
      // for stage 1 (each thread rewrites only its own D(k + M) slots)
      if (sg > 0) load_tables(d.prop_split + (sg == 1 ? 4 * M : 0));
    }
    float2 org[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) org[j] = v[j];
    dft<8, false, EX>(v);
    f8_twiddle<false>(v, w0);
    f8_store<L, 0>(buf, v, t);
    __syncthreads();
    if (lead && sg == 0) {
      // the step's slice (separable: its row head); the splitting forms:
      // every thread is past step it - 1's couplings, which read the other
      // buffer: fetch step it + 1's slice into it
      if constexpr (HALF) {
        if (it + 1 < steps) fetch(n + 1, (it + 1) & 1);
      } else {
        fetch(n, 0);
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
                     32u * 8u * 8u + ((lead && part_due && sg == 0) ? 8u : 0u));
    f8_load<L, 1>(buf, v, t);
    dft<8, false, EX>(v);
    f8_twiddle<false>(v, w1);
    f8_store<L, 1>(buf, v, t);
    __syncwarp();
    f8_load<L, 2>(buf, v, t);
    dft<8, false, EX>(v);
    f8_twiddle<false>(v, w2);
    f8_store<L, 2>(buf, v, t);
    __syncwarp();
    s4_load_last(buf, v, t);
    f8_dft<L, NP - 1, false, EX>(v);              // v[j] = F_h[k_j]
    {
      const uint32_t go = g_peer + uint32_t(half * M) * 8u;
      const uint32_t gbo = gbar_peer + uint32_t(half * C::WARPS + warp) * 8u;
#pragma unroll
      for (int pp = 0; pp < 4; ++pp)
        st_async_v4(go + uint32_t(xpair(pp, t, T)) * 8u, v[2 * pp], v[2 * pp + 1], gbo);
    }
    // (no barrier before the inverse pass rewrites buf: each thread's
    // last-pass positions are its own in both directions)
    if (!timed_out && !mbar_wait_cluster(&gbar[half * C::WARPS + warp], xpar)) timed_out = true;
    if (lead && part_due && sg == 0 && h == 0)
      d.powers[2 * pslot + band] = (my_part + ppeer[half]) * d.dx_um;
    {
      const float2* gi = gx + half * M;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float4 g2 = *reinterpret_cast<const float4*>(gi + xpair(j >> 1, t, T));
        const float2 gp = (j & 1) ? make_float2(g2.z, g2.w) : make_float2(g2.x, g2.y);
        const float2 f0 = h ? gp : v[j], f1 = h ? v[j] : gp;
        const float2 w1k = cmul_f(f1, cw[j].x, cw[j].y);        // W^k F_1
        const float2 x0 = cadd(f0, w1k), x1 = csub(f0, w1k);
        const float2 a = d0[j], b = e1s[j * T + t];
        const float2 y0 = make_float2(fmaf(a.x, x0.x, -(a.y * x0.y)), fmaf(a.x, x0.y, a.y * x0.x));
        const float2 y1 = make_float2(fmaf(b.x, x1.x, -(b.y * x1.y)), fmaf(b.x, x1.y, b.y * x1.x));
        v[j] = h ? cmul_f(csub(y0, y1), cw[j].x, -cw[j].y) : cadd(y0, y1);
      }
    }
    f8_dft<L, NP - 1, true, EX>(v);
    s4_store_last(buf, v, t);
    __syncwarp();
    f8_load<L, 2>(buf, v, t);
    f8_twiddle<true>(v, w2);
    dft<8, true, EX>(v);
    f8_store<L, 2>(buf, v, t);
    __syncwarp();
    f8_load<L, 1>(buf, v, t);
    f8_twiddle<true>(v, w1);
    dft<8, true, EX>(v);
    f8_store<L, 1>(buf, v, t);
    __syncthreads();
    f8_load<L, 0>(buf, v, t);
    f8_twiddle<true>(v, w0);
    dft<8, true, EX>(v);
    {
      if (lane == 0) mbar_expect_tx(&cbar[half * C::WARPS + warp], 32u * 8u * 8u);
      const uint32_t co = c_part + uint32_t(half * M) * 8u;
      const uint32_t cbo = cbar_part + uint32_t(half * C::WARPS + warp) * 8u;
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = cadd(org[j], v[j]);
#pragma unroll
      for (int pp = 0; pp < 4; ++pp)
        st_async_v4(co + uint32_t(xpair(pp, t, T)) * 8u, v[2 * pp], v[2 * pp + 1], cbo);
    }
    // first order: the step's slice, and from its row head the interval mask
    // and the coupling coefficient, while the psi_p stores are in flight
    // (they depend on the slice alone)
    [[maybe_unused]] uint32_t msk1 = 0u;
    [[maybe_unused]] float2 bs1 = bb;
    if constexpr (!HALF) {
      if (!timed_out && !mbar_wait(bar, uint32_t(it & 1))) timed_out = true;
      if (sep) {
        const SepHead sh = sep_head(srow);
        msk1 = sep_mask<1, 8, 8>(sh, t, h);   // T = 256
        bs1 = slice_b<true>(bb, sh, band);
      }
    }
    if (!timed_out && !mbar_wait_cluster(&cbar[half * C::WARPS + warp], xpar)) timed_out = true;
    const float2* ci = cb + half * M;
    if constexpr (HALF) {
      // (separable: the column phasors of buffer 0 and the row heads of
      // steps it and it + 1)
      const float2* phc = ph + (sep ? 0 : (it & 1) * N);
      const SepHead shc = sep ? sep_head(srow + (it & 1)) : SepHead{};
      if (sg < STAGES - 1) {
        // Forest-Ruth, after the first two propagations: the inner
        // couplings ((1 - t)/2) on this step's slice
        auto couple_inner = [&](auto S) {
          constexpr bool SEP = decltype(S)::value;
          const float2 bs = slice_b<SEP>(bbi, shc, band);
          const uint32_t msk = SEP ? sep_mask<1, 8, 8>(shc, t, h) : 0u;
#pragma unroll
          for (int pp = 0; pp < 4; ++pp) {
            const float4 q2 = *reinterpret_cast<const float4*>(ci + xpair(pp, t, T));
            const int m0 = t + 2 * pp * T, m1 = t + (2 * pp + 1) * T;
            v[2 * pp] = couple_at<SEP>(v[2 * pp], make_float2(q2.x, q2.y), phc,
                                       SEP ? m0 : 2 * m0 + h, msk, 2 * pp, band, am1i, bs);
            v[2 * pp + 1] = couple_at<SEP>(v[2 * pp + 1], make_float2(q2.z, q2.w), phc,
                                           SEP ? m1 : 2 * m1 + h, msk, 2 * pp + 1, band, am1i, bs);
          }
        };
        if (sep) couple_inner(BoolC<true>{});
        else couple_inner(BoolC<false>{});
      } else {
        const bool next = it + 1 < steps;
        if (next && !timed_out &&
            !mbar_wait(bar + ((it + 1) & 1), uint32_t(((it + 1) >> 1) & 1)))
          timed_out = true;
        const float2* phn = ph + (sep ? 0 : ((it + 1) & 1) * N);
        const SepHead shn = (sep && next) ? sep_head(srow + ((it + 1) & 1)) : SepHead{};
        const float2 g = rec ? recph[(n + 1) & 1] : make_float2(1.f, 0.f);
        const int slot = rec ? rslot : 0;
        float2* r0 = (rec && d.records) ? d.records + size_t(slot) * 2 * N + band * N : nullptr;
        double s = 0.0;
        auto three_halves = [&](auto S) {
          constexpr bool SEP = decltype(S)::value;
          const float2 bc = slice_b<SEP>(bb, shc, band), bo = slice_b<SEP>(bb, shc, band ^ 1);
          const float2 bn = slice_b<SEP>(bb, shn, band);
          const uint32_t mc = SEP ? sep_mask<1, 8, 8>(shc, t, h) : 0u;
          const uint32_t mn = SEP ? sep_mask<1, 8, 8>(shn, t, h) : 0u;
#pragma unroll
          for (int pp = 0; pp < 4; ++pp) {
            const float4 q2 = *reinterpret_cast<const float4*>(ci + xpair(pp, t, T));
#pragma unroll
            for (int k = 0; k < 2; ++k) {
              const int j = 2 * pp + k;
              const int m = t + j * T;
              const int cell = SEP ? m : 2 * m + h;
              const float2 p = v[j], q = k ? make_float2(q2.z, q2.w) : make_float2(q2.x, q2.y);
              // step it, last coupling (this band's and, below, the other band's)
              float2 c = couple_at<SEP>(p, q, phc, cell, mc, j, band, am1, bc);
              if (rec) {
                s = pow_acc(s, c);
                if (r0)   // records in natural order
                  r0[2 * m + h] = make_float2(fmaf(c.x, g.x, -(c.y * g.y)), fmaf(c.x, g.y, c.y * g.x));
              }
              if (next) {   // step it + 1, first coupling, with the other band's value
                const float2 co = couple_at<SEP>(q, p, phc, cell, mc, j, band ^ 1, am1, bo);
                c = couple_at<SEP>(c, co, phn, cell, mn, j, band, am1, bn);
              }
              v[j] = c;
            }
          }
        };
        if (sep) three_halves(BoolC<true>{});
        else three_halves(BoolC<false>{});
        if (rec && d.powers) {
          double ds = s;
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) ds += __shfl_xor_sync(0xffffffffu, ds, off);
          if (lane == 0) red[warp] = ds;   // summed by the lead after the next barrier
        }
      }
    } else {
      auto couple_all = [&](auto S) {
        constexpr bool SEP = decltype(S)::value;
        const float2 bs = SEP ? bs1 : bb;
        const uint32_t msk = SEP ? msk1 : 0u;
#pragma unroll
        for (int pp = 0; pp < 4; ++pp) {
          const float4 q2 = *reinterpret_cast<const float4*>(ci + xpair(pp, t, T));
          const int m0 = t + 2 * pp * T, m1 = t + (2 * pp + 1) * T;
          const int c0 = 2 * m0 + h, c1 = 2 * m1 + h;
          v[2 * pp] = couple_at<SEP>(v[2 * pp], make_float2(q2.x, q2.y), ph, SEP ? m0 : c0, msk,
                                     2 * pp, band, am1, bs);
          v[2 * pp + 1] = couple_at<SEP>(v[2 * pp + 1], make_float2(q2.z, q2.w), ph,
                                         SEP ? m1 : c1, msk, 2 * pp + 1, band, am1, bs);
        }
      };
      if (sep) couple_all(BoolC<true>{});
      else couple_all(BoolC<false>{});
      if (rec) {
        const int slot = rslot;
        const float2 g = recph[(n + 1) & 1];
        double s = 0.0;
        float2* r0 = d.records ? d.records + size_t(slot) * 2 * N + band * N : nullptr;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
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
  for (int j = 0; j < 8; ++j) d.state[band * N + 2 * (t + j * T) + h] = v[j];
  // Error path: as in fused4e_march_kernel (the lead still issues one slice
  // copy per step, so it waits, bounded, for the last step's phase; second
  // order: the copy of step steps - 1's slice, into its buffer).
  if (timed_out) {
    if constexpr (HALF)
      give_up_after_march(bar + ((steps - 1) & 1), uint32_t(((steps - 1) >> 1) & 1), lead, status);
    else
      give_up_after_march(bar, uint32_t((steps - 1) & 1), lead, status);
  }
  cluster.sync();   // peers may still read our shared memory
}

}  // namespace bpm
