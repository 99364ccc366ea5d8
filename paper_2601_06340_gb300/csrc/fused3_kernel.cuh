// Fused FP32 march on a 2-CTA thread-block cluster: one row (one solve) per
// cluster, CTA rank b advances band b (psi_+ or psi_-).  Used where a single
// solve must finish fast: each band gets a whole SM.
//
// Same step as the band-per-thread kernel (real-space increment form of
// Eq. fov10, see fused2_kernel.cuh), with a different placement:
//   * T = N/16 threads per CTA, each owning 16 points of its band; with one
//     CTA per SM a thread can keep in registers its 16 points, the step's
//     original field, its table twiddles and its slice of the propagator
//     table (loaded once per launch);
//   * each CTA sends its psi_p straight into the peer CTA's shared memory
//     with asynchronous 16-byte remote stores that complete on the peer's mbarrier
//     (armed with the expected byte count), and reads the partner band from
//     its own buffer once its barrier completes -- no cluster-wide barrier
//     per step.  The buffer alternates between two halves by exchange
//     parity (the step's, or for Forest-Ruth that of 3 step + stage); a half
//     is rewritten only after the sender has received the receiver's next
//     values, which the receiver sends after consuming the half;
//   * each CTA fetches the strain/mask slice of the step into its own shared
//     memory with a bulk asynchronous copy on an mbarrier (bounded wait).
#pragma once

#include <cooperative_groups.h>

#include "fused2_kernel.cuh"

namespace bpm {

// PHB: strain-slice buffers (2 for the second-order step, which couples
// with the slices of two steps at a time)
template <int LOGN, int PHB = 1>
struct F3Cfg {
  static constexpr int N = 1 << LOGN;
  static constexpr int T = N / 16;
  static constexpr int NP = (LOGN + 3) / 4;
  static constexpr int RL = 1 << (LOGN - 4 * (NP - 1));
  static constexpr int G_LAST = 16 / RL;
  static constexpr int PADN = N + (N >> 4);
  static constexpr int WARPS = T / 32;
  static constexpr int OFF_BUF = 0;                       // [PADN]
  static constexpr int OFF_X = OFF_BUF + PADN * 8;        // [2][N] exchange
  static constexpr int OFF_PH = OFF_X + 2 * N * 8;        // [PHB][N]
  static constexpr int OFF_MBAR = OFF_PH + PHB * N * 8;    // [PHB] strain slice barriers
  static constexpr int OFF_XBAR = OFF_MBAR + 8 * PHB;      // [2][WARPS] exchange barriers
  static constexpr int OFF_RECPH = OFF_XBAR + 16 * WARPS;
  static constexpr int OFF_RED = OFF_RECPH + 16;          // [WARPS] double
  static constexpr int OFF_SROW = (OFF_RED + WARPS * 8 + 15) / 16 * 16;   // [PHB] row heads
  static constexpr int SMEM = OFF_SROW + PHB * 16;
  static_assert(LOGN >= 9 && LOGN <= 12, "cluster kernel covers 512..4096");
  // layout checks: fits one SM (227 KB); bulk-copy and 16-byte store
  // targets 16-byte aligned; mbarriers 8-byte aligned
  static_assert(SMEM <= 232448, "fits one SM");
  static_assert(OFF_X % 16 == 0 && OFF_PH % 16 == 0, "16-byte stores and bulk copy");
  static_assert(OFF_MBAR % 8 == 0 && OFF_XBAR % 8 == 0, "mbarrier alignment");
};

__device__ __forceinline__ uint32_t mapa_u32(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

// Two values per asynchronous remote store.  Exchange buffers keep a
// thread's values in pairs: pair p = (v[2p], v[2p+1]) of thread t sits at
// float2 index p * 2T + 2t (xpair), so one 16-byte st.async carries two values,
// the receiver reads them with one 16-byte load, and consecutive lanes touch
// consecutive 16-byte words (no bank conflicts).
__device__ __forceinline__ void st_async_v4(uint32_t raddr, float2 a, float2 b, uint32_t rbar) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, "
      "[%5];" ::"r"(raddr),
      "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "r"(rbar)
      : "memory");
}

__host__ __device__ constexpr int xpair(int p, int t, int T) { return p * 2 * T + 2 * t; }

// Coupling of one cell (Eq. fov10 with Eqs. fov11, fov12 and the strain
// phase): p = this band's psi_p, q = the other band's, e = exp(i h u) of the
// cell, (0, 0) outside the crystal; band 1 uses the conjugate phase.
// Returns p + (a - 1) p + b e^{+-i h u} q inside, p outside.
__device__ __forceinline__ float2 couple_cell(float2 p, float2 q, float2 e, int band,
                                              float2 am1, float2 bb) {
  const bool inside = (e.x != 0.f) | (e.y != 0.f);
  if (band) e.y = -e.y;
  const float ax = inside ? am1.x : 0.f, ay = inside ? am1.y : 0.f;
  const float cx = fmaf(bb.x, e.x, -(bb.y * e.y)), cy = fmaf(bb.x, e.y, bb.y * e.x);
  float rx = fmaf(ax, p.x, p.x);
  rx = fmaf(-ay, p.y, rx);
  rx = fmaf(cx, q.x, rx);
  rx = fmaf(-cy, q.y, rx);
  float ry = fmaf(ax, p.y, p.y);
  ry = fmaf(ay, p.x, ry);
  ry = fmaf(cx, q.y, ry);
  ry = fmaf(cy, q.x, ry);
  return make_float2(rx, ry);
}

// couple_cell with the inside flag given (separable slices: e is the
// column phasor, the flag the row's interval test).
__device__ __forceinline__ float2 couple_cell_in(float2 p, float2 q, float2 e, bool inside,
                                                 int band, float2 am1, float2 bb) {
  if (band) e.y = -e.y;
  const float ax = inside ? am1.x : 0.f, ay = inside ? am1.y : 0.f;
  const float cx0 = fmaf(bb.x, e.x, -(bb.y * e.y)), cy0 = fmaf(bb.x, e.y, bb.y * e.x);
  const float cx = inside ? cx0 : 0.f, cy = inside ? cy0 : 0.f;
  float rx = fmaf(ax, p.x, p.x);
  rx = fmaf(-ay, p.y, rx);
  rx = fmaf(cx, q.x, rx);
  rx = fmaf(-cy, q.y, rx);
  float ry = fmaf(ax, p.y, p.y);
  ry = fmaf(ay, p.x, ry);
  ry = fmaf(cx, q.y, ry);
  ry = fmaf(cy, q.x, ry);
  return make_float2(rx, ry);
}

// One cell's coupling in either slice form: the stream's phasor ph[c], or
// (SEP) the column phasor ph[c] with bit jj of the thread's interval mask.
template <bool SEP>
__device__ __forceinline__ float2 couple_at(float2 p, float2 q, const float2* ph, int c,
                                            uint32_t msk, int jj, int band, float2 am1,
                                            float2 bb) {
  if constexpr (SEP) return couple_cell_in(p, q, ph[c], (msk >> jj) & 1u, band, am1, bb);
  else return couple_cell(p, q, ph[c], band, am1, bb);
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(
          smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

// Bounded wait with cluster-scope acquire (data written by a peer CTA).
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t b = smem_u32(bar);
  for (int i = 0; i < kWaitPolls; ++i) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(b), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// HALF = false: the first-order step of Eq. fov10.  HALF = true: the
// second-order (Verlet) step of Eq. split-op, half-step coupling on the
// step's slice, propagation, half-step coupling again.  After the psi_p swap
// a CTA holds both bands at its points, so it applies step n's second half
// to both and step n + 1's first half to its own band with no further
// exchange; the launch's first half-step takes the other band from the
// state in global memory.  Records are taken after step n's second half.
// SCH, the operator splitting (as in fused2_kernel.cuh): kSchFirst (HALF =
// false above), kSchVerlet (HALF = true), kSchForestRuth: three
// propagations per step with the tables of t dz, (1 - 2t) dz, t dz (the
// row's prop holds those of t dz, then those of (1 - 2t) dz, in the
// band-per-thread kernels' thread order) and the inner couplings
// (1 - t)/2, in (am1, b), on the step's slice after the first two.
template <int LOGN, bool EX, int SCH = kSchFirst>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(F3Cfg<LOGN>::T, 1)
    fused3_march_kernel(const RowDescF32* __restrict__ rows, int n_rows, int steps,
                        const float4* __restrict__ tw, int* __restrict__ status) {
  namespace cg = cooperative_groups;
  constexpr bool HALF = SCH != kSchFirst;           // couples before propagating
  constexpr int STAGES = SCH == kSchForestRuth ? 3 : 1;
  using C = F3Cfg<LOGN, HALF ? 2 : 1>;
  using F = F2Cfg<LOGN>;   // same pass geometry (E = 16 points per thread)
  constexpr int N = C::N, T = C::T, NP = C::NP, RL = C::RL, GL = C::G_LAST;
  extern __shared__ __align__(128) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();

  const int band = int(cluster.block_rank());
  const int row = blockIdx.x >> 1;
  const int t = threadIdx.x;
  const int lane = t & 31, warp = t >> 5;
  const RowDescF32 d = rows[row < n_rows ? row : 0];
  const bool lead = t == 0;

  float2* buf = reinterpret_cast<float2*>(smem + C::OFF_BUF);
  float2* xb = reinterpret_cast<float2*>(smem + C::OFF_X);
  float2* ph = reinterpret_cast<float2*>(smem + C::OFF_PH);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + C::OFF_MBAR);
  uint64_t* xbar = reinterpret_cast<uint64_t*>(smem + C::OFF_XBAR);
  // the records' common phase, two slots by step parity: the lead writes a
  // record step's phase while a slower warp may still read the previous one
  float2* recph = reinterpret_cast<float2*>(smem + C::OFF_RECPH);
  double* red = reinterpret_cast<double*>(smem + C::OFF_RED);
  float4* srow0 = reinterpret_cast<float4*>(smem + C::OFF_SROW);
  const bool sep = d.srows != nullptr;
  const uint32_t peer = uint32_t(band ^ 1);
  const uint32_t xpeer = mapa_u32(smem_u32(xb), peer);          // peer's exchange buffer
  const uint32_t xbar_peer = mapa_u32(smem_u32(xbar), peer);    // peer's exchange barriers

  if (lead) {
    mbar_init(bar);
    if constexpr (HALF) mbar_init(bar + 1);
    for (int i = 0; i < 2 * C::WARPS; ++i) mbar_init(&xbar[i]);
  }
  fence_mbar_init();

  float2 w0[15], w1[15];
#pragma unroll
  for (int j = 1; j < 16; ++j) {
    const float4 a = __ldg(&tw[t * j]);
    w0[j - 1] = make_float2(a.x, a.y);
    if constexpr (NP >= 3) {
      const float4 b = __ldg(&tw[((t % F::stride(1)) * j) << 4]);
      w1[j - 1] = make_float2(b.x, b.y);
    } else {
      w1[j - 1] = make_float2(0.f, 0.f);
    }
  }
  // this thread's slice of (P - 1)/N in the last pass (for the whole launch;
  // Forest-Ruth reloads it per stage from its stage tables in thread order)
  static_assert(GL * RL == 16 && F::TAIL_WARP == (NP >= 3), "the band-per-thread geometry");
  float2 pr[16];
  auto load_table = [&](const float2* tab) {
#pragma unroll
    for (int k = 0; k < 16; ++k)
      pr[k] = __ldg(&tab[band * N + (SCH == kSchForestRuth ? k * T + t
                                                             : f2_table_pos<LOGN>(t, k))]);
  };
  load_table(d.prop);

  float2 v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = d.state[band * N + t + j * T];
  // separable slices: the column phasors stay in buffer 0 for the launch
  if (sep)
    for (int k = t; k < N; k += T) ph[k] = __ldg(&d.scols[k]);
  cluster.sync();   // peers initialised (mbarriers, shared memory) before any exchange

  const uint32_t slice_bytes = uint32_t(N) * 8u;
  int pending_slot = -1;
  bool timed_out = false;
  // (am1, bb): the step's coupling, or the outer ones of a splitting form;
  // (am1i, bbi): Forest-Ruth's inner couplings
  const float2 am1 = HALF ? d.am1h : d.am1, bb = HALF ? d.bh : d.b;
  [[maybe_unused]] const float2 am1i = d.am1, bbi = d.b;
  // slice of step n into buffer `slot` (separable: the row head only)
  auto fetch = [&](int n, int slot) {
    if (sep) bulk_load(srow0 + slot, d.srows + n, kSepHeadBytes, bar + slot);
    else bulk_load(ph + slot * N, d.phasor + size_t(n) * N, slice_bytes, bar + slot);
  };
  if constexpr (HALF) {
    // the launch's first half-step, on the slice of its first step (buffer
    // 0); later slices are fetched a step ahead into the other buffer
    if (lead) fetch(d.n_begin, 0);
    float2 q[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) q[j] = d.state[(band ^ 1) * N + t + j * T];
    if (!mbar_wait(bar, 0u)) timed_out = true;
    const SepHead sh = sep ? sep_head(srow0) : SepHead{};
    auto first_half = [&](auto S) {
      constexpr bool SEP = decltype(S)::value;
#pragma unroll
      for (int j = 0; j < 16; ++j)
        v[j] = couple_cell(v[j], q[j], slice_at<SEP>(ph, sh, t + j * T, t + j * T), band, am1,
                           slice_b<SEP>(bb, sh, band));
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
    if (lead && rec) {
      double ang = fmod(double(n + 1 - d.n_phase0) * d.gphase, 6.283185307179586);
      double sa, ca;
      sincos(ang, &sa, &ca);
      recph[(n + 1) & 1] = make_float2(float(ca), float(sa));
    }
    // one stage of the step (Forest-Ruth: three; the others: one, with no
    // loop around it)
    auto stage = [&](const int sg) {
    // exchange index of the stage: buffer half and barrier phase
    const int ex = it * STAGES + sg;
    if constexpr (SCH == kSchForestRuth) {
      // the stage's table: (P^t - 1)/N for stages 0 and 2, (P^(1-2t) - 1)/N
      // for stage 1 (read from L2 while the forward passes run)
      if (sg > 0) load_table(d.prop + (sg == 1 ? 2 * N : 0));
    }
    float2 org[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) org[j] = v[j];
    dft<16, false, EX>(v);
    f2_twiddle<false>(v, w0);
    f2_store<LOGN, 0>(buf, v, t);
    __syncthreads();
    if constexpr (HALF) {
      // every thread is past step it - 1's couplings, which read the buffer
      // of slice it - 1: fetch slice it + 1 into it
      if (lead && sg == 0 && it + 1 < steps) fetch(n + 1, (it + 1) & 1);
    } else {
      if (lead) fetch(n, 0);
    }
    if (lead && pending_slot >= 0) {
      double s = 0.0;
      for (int w = 0; w < C::WARPS; ++w) s += red[w];
      d.powers[2 * pending_slot + band] = s * d.dx_um;
      pending_slot = -1;
    }
    // (three passes: pass 1 and the last pass of warp w address positions
    // [512 w, 512 w + 512) only, the last pass's groups as in f2_group, so
    // the barriers between them are the warp's)
    constexpr bool TW = NP >= 3;
    if constexpr (NP >= 3) {
      f2_load<LOGN, 1>(buf, v, t);
      dft<16, false, EX>(v);
      f2_twiddle<false>(v, w1);
      f2_store<LOGN, 1>(buf, v, t);
      tail_sync<TW>();
    }
    {
      constexpr int P = NP - 1;
      f2_load<LOGN, P, TW>(buf, v, t);
      f2_dft<LOGN, P, false, EX>(v);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float2 x = v[k], dd = pr[k];
        v[k] = make_float2(fmaf(x.x, dd.x, -(x.y * dd.y)), fmaf(x.x, dd.y, x.y * dd.x));
      }
      f2_dft<LOGN, P, true, EX>(v);
      f2_store<LOGN, P, TW>(buf, v, t);
      tail_sync<TW>();
    }
    if constexpr (NP >= 3) {
      f2_load<LOGN, 1>(buf, v, t);
      f2_twiddle<true>(v, w1);
      dft<16, true, EX>(v);
      f2_store<LOGN, 1>(buf, v, t);
      __syncthreads();
    }
    f2_load<LOGN, 0>(buf, v, t);
    f2_twiddle<true>(v, w0);
    dft<16, true, EX>(v);
    // send psi_p to the peer (asynchronous remote stores completing on the
    // peer's barrier of this parity); arm our own barrier for the peer's.
    const int half = ex & 1;
    // (per warp: thread t receives the slots of the peer's thread t)
    if (lane == 0) mbar_expect_tx(&xbar[half * C::WARPS + warp], 32u * 16u * 8u);
    const uint32_t xo = xpeer + uint32_t(half * N) * 8u;
    const uint32_t xbo = xbar_peer + uint32_t(half * C::WARPS + warp) * 8u;
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = cadd(org[j], v[j]);
#pragma unroll
    for (int pp = 0; pp < 8; ++pp)
      st_async_v4(xo + uint32_t(xpair(pp, t, T)) * 8u, v[2 * pp], v[2 * pp + 1], xbo);
    // (after one expired wait a thread stops waiting, so a fault costs one
    // bounded wait, not one per step; the host reports BPM_ERR_TIMEOUT)
    if (!timed_out && !mbar_wait_cluster(&xbar[half * C::WARPS + warp], uint32_t((ex >> 1) & 1)))
      timed_out = true;

    const float2* xi = xb + half * N;
    if constexpr (HALF) {
      // (separable: the couplings read the column phasors of buffer 0 and
      // the row heads of steps it and it + 1)
      const float2* phc = ph + (sep ? 0 : (it & 1) * N);
      const SepHead shc = sep ? sep_head(srow0 + (it & 1)) : SepHead{};
      if (STAGES > 1 && sg < STAGES - 1) {
        // Forest-Ruth, after the first two propagations: the inner
        // couplings ((1 - t)/2) on this step's slice (awaited before this
        // step: at the previous step's couplings or the launch's first)
        auto couple_inner = [&](auto S) {
          constexpr bool SEP = decltype(S)::value;
          const float2 bs = slice_b<SEP>(bbi, shc, band);
#pragma unroll
          for (int pp = 0; pp < 8; ++pp) {
            const float4 q2 = *reinterpret_cast<const float4*>(xi + xpair(pp, t, T));
            const int c0 = t + 2 * pp * T, c1 = t + (2 * pp + 1) * T;
            v[2 * pp] = couple_cell(v[2 * pp], make_float2(q2.x, q2.y),
                                    slice_at<SEP>(phc, shc, c0, c0), band, am1i, bs);
            v[2 * pp + 1] = couple_cell(v[2 * pp + 1], make_float2(q2.z, q2.w),
                                        slice_at<SEP>(phc, shc, c1, c1), band, am1i, bs);
          }
        };
        if (sep) couple_inner(BoolC<true>{});
        else couple_inner(BoolC<false>{});
        return;
      }
      const bool next = it + 1 < steps;
      if (next && !timed_out &&
          !mbar_wait(bar + ((it + 1) & 1), uint32_t(((it + 1) >> 1) & 1)))
        timed_out = true;
      const float2* phn = ph + (sep ? 0 : ((it + 1) & 1) * N);
      const SepHead shn = (sep && next) ? sep_head(srow0 + ((it + 1) & 1)) : SepHead{};
      const float2 g = rec ? recph[(n + 1) & 1] : make_float2(1.f, 0.f);
      const int slot = rec ? rs.slot : 0;
      float2* r0 = (rec && d.records) ? d.records + size_t(slot) * 2 * N + band * N : nullptr;
      double s = 0.0;
      // Three couplings per point, unrolled over the thread's 16 points,
      // overflow the instruction cache; they run as a loop over shared
      // memory instead (buf is free once every thread is past the inverse
      // pass 0, and free again for the next step once every thread has
      // taken its points back).
      __syncthreads();
#pragma unroll
      for (int j = 0; j < 16; ++j) buf[t + j * T] = v[j];
      auto three_halves = [&](auto S) {
        constexpr bool SEP = decltype(S)::value;
        const float2 bc = slice_b<SEP>(bb, shc, band), bo = slice_b<SEP>(bb, shc, band ^ 1);
        const float2 bn = slice_b<SEP>(bb, shn, band);
#pragma unroll 1
        for (int pp = 0; pp < 8; ++pp) {
          const float4 q2 = *reinterpret_cast<const float4*>(xi + xpair(pp, t, T));
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const int at = t + (2 * pp + k) * T;
            const float2 p = buf[at], q = k ? make_float2(q2.z, q2.w) : make_float2(q2.x, q2.y);
            const float2 e = slice_at<SEP>(phc, shc, at, at);
            float2 c = couple_cell(p, q, e, band, am1, bc);   // step it, second half
            if (rec) {
              s = pow_acc(s, c);
              if (r0) r0[at] = make_float2(fmaf(c.x, g.x, -(c.y * g.y)), fmaf(c.x, g.y, c.y * g.x));
            }
            if (next) {   // step it + 1, first half, with the other band's value
              const float2 co = couple_cell(q, p, e, band ^ 1, am1, bo);
              c = couple_cell(c, co, slice_at<SEP>(phn, shn, at, at), band, am1, bn);
            }
            buf[at] = c;
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
        if (lane == 0) red[warp] = ds;
        if (lead) pending_slot = slot;
      }
    } else {
      if (!timed_out && !mbar_wait(bar, uint32_t(it & 1))) timed_out = true;
      const SepHead sh = sep ? sep_head(srow0) : SepHead{};
      auto couple_all = [&](auto S) {
        constexpr bool SEP = decltype(S)::value;
        const float2 bs = slice_b<SEP>(bb, sh, band);
#pragma unroll
        for (int pp = 0; pp < 8; ++pp) {
          const float4 q2 = *reinterpret_cast<const float4*>(xi + xpair(pp, t, T));
          const int c0 = t + 2 * pp * T, c1 = t + (2 * pp + 1) * T;
          v[2 * pp] = couple_cell(v[2 * pp], make_float2(q2.x, q2.y),
                                  slice_at<SEP>(ph, sh, c0, c0), band, am1, bs);
          v[2 * pp + 1] = couple_cell(v[2 * pp + 1], make_float2(q2.z, q2.w),
                                      slice_at<SEP>(ph, sh, c1, c1), band, am1, bs);
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
          if (r0) r0[t + j * T] = make_float2(fmaf(p.x, g.x, -(p.y * g.y)), fmaf(p.x, g.y, p.y * g.x));
        }
        if (d.powers) {
          double ds = s;
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) ds += __shfl_xor_sync(0xffffffffu, ds, off);
          if (lane == 0) red[warp] = ds;
          if (lead) pending_slot = slot;
        }
      }
    }
    };
    if constexpr (STAGES == 1) {
      stage(0);
    } else {
#pragma unroll 1
      for (int sg = 0; sg < STAGES; ++sg) stage(sg);
    }   // (the Forest-Ruth step ends on the t dz table, which its next step
        // starts with)
  }

  __syncthreads();
  if (lead && pending_slot >= 0) {
    double s = 0.0;
    for (int w = 0; w < C::WARPS; ++w) s += red[w];
    d.powers[2 * pending_slot + band] = s * d.dx_um;
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) d.state[band * N + t + j * T] = v[j];
  // Error path: after an expired wait a thread skips its later waits and the
  // march runs on to the end of the launch; the lead still issues one slice
  // copy per step on its barrier, so waiting (again bounded) for the last
  // step's phase leaves no copy of its own in flight when the CTA exits.
  if (timed_out) {
    if constexpr (HALF)   // the last slice copy: step steps - 1, in its buffer
      give_up_after_march(bar + ((steps - 1) & 1), uint32_t(((steps - 1) >> 1) & 1), lead, status);
    else
      give_up_after_march(bar, uint32_t((steps - 1) & 1), lead, status);
  }
  cluster.sync();   // the peer may still read our exchange buffer: stay resident
}

}  // namespace bpm
