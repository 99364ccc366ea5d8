// Persistent fused FP32 march (one CTA advances one or more batch rows for
// `steps` z-steps without returning the fields to global memory).
//
// One step of Eq. fov10 (arXiv 2601.06340):
//   psi_p+- = F^-1[ F[psi_+-] exp(i dz^ delta_+-(q)) ]          (bands apart)
//   psi_+   <- psi_p+ + (a-1) psi_p+ + b e^{+i h u} psi_p-       inside Pi
//   psi_-   <- psi_p- + (a-1) psi_p- + b e^{-i h u} psi_p+       inside Pi
// with the common phase exp(i dz^ cos alpha) removed from the march and put
// back (in FP64) when results leave the kernel.
//
// Layout.  N = 2^LOGN points per band.  Each row is handled by T = N/16
// threads that own E = 16 points of each band in registers.  The FFT is a
// mixed-radix decimation-in-frequency transform with passes of radix 16
// (and one last pass of radix 2^(LOGN mod 4) when needed); the output stays
// in digit-reversed order, the propagator table is stored in that order, and
// the inverse is the matching decimation-in-time transform, which restores
// natural order.  Between passes the fields go through shared memory
// (padded by one slot per 16 to avoid bank conflicts).  Three passes are
// fused without a shared-memory round trip:
//   * inverse pass 0 + coupling + record + next step's forward pass 0,
//   * forward last pass + propagator + inverse last pass,
// so a step costs 2 (passes - 1) shared-memory transposes per band.
//
// The strain/mask slice exp(i h u_x[n][.]) (8 bytes per cell, (0,0) outside
// the crystal) is fetched for each step by one bulk asynchronous copy (TMA)
// into shared memory, completing on an mbarrier; the copy is issued early in
// the step and consumed at the coupling, so it overlaps the FFT passes.
// Every wait on that mbarrier is bounded; on expiry the kernel raises a bit
// in the status word and carries on.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bpm_internal.h"
#include "radix.cuh"

namespace bpm {

// PHB: strain-slice buffers per row (2 when the step couples before it
// propagates: the next step's slice is fetched a step ahead)
template <int LOGN, int PHB = 1>
struct FusedCfg {
  static constexpr int N = 1 << LOGN;
  static constexpr int E = N < 16 ? N : 16;          // points per band per thread
  static constexpr int T = N / E;                    // threads per row
  static constexpr int NP = (LOGN + 3) / 4;          // FFT passes
  static constexpr int RL = 1 << (LOGN - 4 * (NP - 1));  // radix of the last pass
  static constexpr int ROWS = T >= 64 ? 1 : 64 / T;  // rows per CTA
  static constexpr int THREADS = T * ROWS;
  static constexpr int PADN = N + (N >> 4);          // padded band length
  static constexpr int WARPS_PER_ROW = T >= 32 ? T / 32 : 1;
  // shared memory layout per CTA (bytes)
  static constexpr int OFF_BUF = 0;                                  // [ROWS][2][PADN] float2
  static constexpr int OFF_PH = OFF_BUF + ROWS * 2 * PADN * 8;       // [ROWS][PHB][N] float2
  static constexpr int OFF_MBAR = OFF_PH + ROWS * PHB * N * 8;       // [ROWS][PHB] u64
  static constexpr int OFF_RECPH = OFF_MBAR + ROWS * PHB * 8;        // [ROWS][2] float2
  static constexpr int OFF_RED = OFF_RECPH + ROWS * 16;              // [ROWS][WARPS][2] double
  static constexpr int OFF_SROW =                                    // [ROWS][PHB] row heads
      (OFF_RED + ROWS * WARPS_PER_ROW * 2 * 8 + 15) / 16 * 16;
  static constexpr int SMEM = OFF_SROW + ROWS * PHB * 16;
  // layout checks: fits one SM (227 KB); bulk-copy and 16-byte store
  // targets 16-byte aligned; mbarriers 8-byte aligned
  static_assert(SMEM <= 232448, "fits one SM");
  static_assert(OFF_PH % 16 == 0 && (N * 8) % 16 == 0, "bulk copy of a slice");
  static_assert(OFF_MBAR % 8 == 0, "mbarrier alignment");

  __host__ __device__ static constexpr int radix(int p) { return p < NP - 1 ? 16 : RL; }
  __host__ __device__ static constexpr int len(int p) { return N >> (4 * p); }
  __host__ __device__ static constexpr int stride(int p) { return len(p) / radix(p); }
  __host__ __device__ static constexpr int groups(int p) { return E / radix(p); }
};

__device__ __forceinline__ int padi(int a) { return a + (a >> 4); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src,
                                          uint32_t bytes, uint64_t* bar) {
  uint32_t b = smem_u32(bar);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile(
      "{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(b),
      "r"(bytes)
      : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(b)
      : "memory");
}

// Asynchronous prefetch of `bytes` of global memory into L2 (16-byte aligned
// address, size a multiple of 16); nothing to wait for.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// ---- separable slices ----------------------------------------------------
// Rows of a plan whose slices take the separable form (bent or unstrained
// slab crystals; SepRow) keep the column phasors of their points in the
// slice buffer for the whole launch and fetch, per step, only the first 16
// bytes of the step's row (one bulk copy on the slice barrier, in place of
// the slice): the row's phase term and its inside interval [lo, hi).  The
// cell's phasor e = col * row enters the coupling only through b e (band +)
// and b conj(e) (band -), so the row phasor is folded into the coupling
// coefficient once per step, (b row) col and (b conj(row)) conj(col): per
// cell the same multiply count as with the stream, the product rounded in
// another order (the two forms agree to FP32 rounding).
constexpr uint32_t kSepHeadBytes = 16;

struct SepHead {
  float2 ph;
  int lo, hi;
};

__device__ __forceinline__ SepHead sep_head(const float4* slot) {
  const float4 h = *slot;
  return {make_float2(h.x, h.y), __float_as_int(h.z), __float_as_int(h.w)};
}

// Bit jj set: the cell of natural column P (t + jj T) + h (T = 2^LOG_T)
// lies in [lo, hi).  Columns P m + h with m in [ceil((lo - h) / P),
// ceil((hi - h) / P)), and m = t + jj T in that range for jj in
// [ceil((mlo - t) / T), ceil((mhi - t) / T)): two clamped shifts per thread
// and step instead of a test per cell (P a power of two; the shifts floor).
__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

template <int LOG_P, int LOG_T, int E>
__device__ __forceinline__ uint32_t sep_mask(const SepHead& sh, int t, int h) {
  constexpr int P = 1 << LOG_P, T = 1 << LOG_T;
  const int mlo = (sh.lo - h + P - 1) >> LOG_P, mhi = (sh.hi - h + P - 1) >> LOG_P;
  const int a = min(max((mlo - t + T - 1) >> LOG_T, 0), E);
  const int b = min(max((mhi - t + T - 1) >> LOG_T, 0), E);
  return ((1u << b) - 1u) & ~((1u << a) - 1u);
}

// The cell's column phasor inside [lo, hi) (natural column j), (0, 0) outside.
__device__ __forceinline__ float2 sep_cell(const SepHead& h, float2 col, int j) {
  const bool in = (j >= h.lo) & (j < h.hi);
  return in ? col : make_float2(0.f, 0.f);
}

// b row (band 0) or b conj(row) (band 1): the coupling coefficient of the
// step with the row phasor folded in.
__device__ __forceinline__ float2 sep_b(float2 bb, const SepHead& h, int band) {
  const float2 r = band ? make_float2(h.ph.x, -h.ph.y) : h.ph;
  return make_float2(fmaf(bb.x, r.x, -(bb.y * r.y)), fmaf(bb.x, r.y, bb.y * r.x));
}

// What the coupling of stream position c (natural column j) multiplies by b:
// the slice's phasor, or (SEP) the column phasor ph[c] inside the interval.
template <bool SEP>
__device__ __forceinline__ float2 slice_at(const float2* ph, const SepHead& sh, int c, int j) {
  if constexpr (SEP) return sep_cell(sh, ph[c], j);
  else return ph[c];
}

// The coupling coefficient to go with slice_at<SEP> for band `band`.
template <bool SEP>
__device__ __forceinline__ float2 slice_b(float2 bb, const SepHead& sh, int band) {
  if constexpr (SEP) return sep_b(bb, sh, band);
  else return bb;
}

// Barrier between two FFT passes: the warp's own when both passes of every
// warp address only positions that warp owns (WARP), else the CTA's.
template <bool WARP>
__device__ __forceinline__ void tail_sync() {
  if constexpr (WARP) __syncwarp();
  else __syncthreads();
}

// The record steps of a march (steps n with n + 1 a multiple of
// record_every), counted instead of found by an integer division every step:
// the division sat on the step's critical path in the single-solve kernels
// (the exchange barriers' expected byte counts depend on it), and counting
// measured 4.8 % faster per 8000-step march of the N = 4096 split.
struct RecSteps {
  int every;   // record_every (0: no records)
  int in;      // steps to the next record step
  int slot;    // that step's record slot, (n + 1) / every - 1
  bool prev;   // the previous step was a record step
  struct Step {
    bool at;     // this step is a record step
    bool prev;   // the previous step of the launch was one
    int slot;    // this step's record slot (at)
    int pslot;   // the previous step's record slot (prev)
  };
  __device__ __forceinline__ RecSteps(int record_every, int n_begin)
      : every(record_every),
        in(record_every > 0 ? record_every - 1 - n_begin % record_every : -1),
        slot(record_every > 0 ? n_begin / record_every : 0),
        prev(false) {}
  // this step's flags and slots, then advance to the next step
  __device__ __forceinline__ Step next() {
    const Step s{in == 0, prev, slot, slot - 1};
    prev = s.at;
    if (s.at) {
      in = every - 1;
      ++slot;
    } else {
      --in;
    }
    return s;
  }
};

// Compile-time flag for generic lambdas that run a loop in both slice forms.
template <bool B>
struct BoolC {
  static constexpr bool value = B;
};

// Poll limit of every bounded mbarrier wait: a try_wait that finds the phase
// incomplete suspends the thread for about 4 us on GB300, so the limit is
// about one second (measured by bpm_selftest_wait_expiry).
constexpr int kWaitPolls = 1 << 18;

// Bounded wait for phase `parity` of the barrier; false on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  uint32_t b = smem_u32(bar);
  for (int i = 0; i < kWaitPolls; ++i) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(b), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Error epilogue of the cluster kernels, out of line so that the march loop's
// code does not change: the lead waits (again bounded) for the phase of the
// launch's last slice copy, and every thread that gave up flags the launch.
static __device__ __noinline__ void give_up_after_march(uint64_t* bar, uint32_t last_parity,
                                                        bool lead, int* status) {
  if (lead) mbar_wait(bar, last_parity);
  atomicOr(status, kStatusWaitTimeout);
}

// ---- per-pass helpers (thread owns groups gi = t + i*T) ------------------
template <int LOGN, int P>
__device__ __forceinline__ int pass_pos(int gi, int j) {
  using C = FusedCfg<LOGN>;
  constexpr int S = C::stride(P), L = C::len(P);
  return (gi / S) * L + (gi % S) + j * S;
}

template <int LOGN, int P>
__device__ __forceinline__ void store_pass(float2* buf, const float2* v, int t) {
  using C = FusedCfg<LOGN>;
  constexpr int R = C::radix(P), G = C::groups(P);
#pragma unroll
  for (int i = 0; i < G; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j)
      buf[padi(pass_pos<LOGN, P>(t + i * C::T, j))] = v[i * R + j];
}

template <int LOGN, int P>
__device__ __forceinline__ void load_pass(const float2* buf, float2* v, int t) {
  using C = FusedCfg<LOGN>;
  constexpr int R = C::radix(P), G = C::groups(P);
#pragma unroll
  for (int i = 0; i < G; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j)
      v[i * R + j] = buf[padi(pass_pos<LOGN, P>(t + i * C::T, j))];
}

// Twiddles after forward pass P (before inverse pass P): element j of group
// gi gets W_{L_P}^{o j}, o = gi mod S_P, i.e. table entry (o j) * 16^P.
template <int LOGN, int P, bool INV>
__device__ __forceinline__ void twiddle_pass(float2* v0, float2* v1, int t,
                                             const float4* __restrict__ tw) {
  using C = FusedCfg<LOGN>;
  constexpr int R = C::radix(P), G = C::groups(P), S = C::stride(P);
#pragma unroll
  for (int i = 0; i < G; ++i) {
    const int o = (t + i * C::T) % S;
#pragma unroll
    for (int j = 1; j < R; ++j) {
      const float4 w = __ldg(&tw[(o * j) << (4 * P)]);
      v0[i * R + j] = mul_tw<INV>(v0[i * R + j], w);
      v1[i * R + j] = mul_tw<INV>(v1[i * R + j], w);
    }
  }
}

template <int LOGN, int P, bool INV>
__device__ __forceinline__ void dft_pass(float2* v0, float2* v1) {
  using C = FusedCfg<LOGN>;
  constexpr int R = C::radix(P), G = C::groups(P);
#pragma unroll
  for (int i = 0; i < G; ++i) {
    dft<R, INV>(v0 + i * R);
    dft<R, INV>(v1 + i * R);
  }
}

// Forward middle pass P (1 <= P <= NP-2): load, DFT, twiddle, store.
template <int LOGN, int P>
__device__ __forceinline__ void fwd_mid(float2* b0, float2* b1, float2* v0,
                                        float2* v1, int t, const float4* tw) {
  load_pass<LOGN, P>(b0, v0, t);
  load_pass<LOGN, P>(b1, v1, t);
  dft_pass<LOGN, P, false>(v0, v1);
  twiddle_pass<LOGN, P, false>(v0, v1, t, tw);
  store_pass<LOGN, P>(b0, v0, t);
  store_pass<LOGN, P>(b1, v1, t);
  __syncthreads();
}

template <int LOGN, int P>
__device__ __forceinline__ void inv_mid(float2* b0, float2* b1, float2* v0,
                                        float2* v1, int t, const float4* tw) {
  load_pass<LOGN, P>(b0, v0, t);
  load_pass<LOGN, P>(b1, v1, t);
  twiddle_pass<LOGN, P, true>(v0, v1, t, tw);
  dft_pass<LOGN, P, true>(v0, v1);
  store_pass<LOGN, P>(b0, v0, t);
  store_pass<LOGN, P>(b1, v1, t);
  __syncthreads();
}

// Last pass: forward DFT, propagator in delta form (x/N + x (P-1)/N), inverse.
template <int LOGN>
__device__ __forceinline__ void last_pass(float2* v0, float2* v1, int t,
                                          const float2* __restrict__ prop) {
  using C = FusedCfg<LOGN>;
  constexpr int P = C::NP - 1, R = C::radix(P), G = C::groups(P);
  constexpr float inv_n = 1.0f / float(C::N);
  dft_pass<LOGN, P, false>(v0, v1);
#pragma unroll
  for (int i = 0; i < G; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int pos = pass_pos<LOGN, P>(t + i * C::T, j);
      const float2 d0 = __ldg(&prop[pos]);
      const float2 d1 = __ldg(&prop[C::N + pos]);
      float2 x = v0[i * R + j];
      v0[i * R + j] = make_float2(fmaf(x.x, inv_n, fmaf(x.x, d0.x, -(x.y * d0.y))),
                                  fmaf(x.y, inv_n, fmaf(x.x, d0.y, x.y * d0.x)));
      x = v1[i * R + j];
      v1[i * R + j] = make_float2(fmaf(x.x, inv_n, fmaf(x.x, d1.x, -(x.y * d1.y))),
                                  fmaf(x.y, inv_n, fmaf(x.x, d1.y, x.y * d1.x)));
    }
  dft_pass<LOGN, P, true>(v0, v1);
}

// Coupling of Eq. fov10 on this thread's cells of both bands, coefficients
// (a - 1, b) of the (fractional) step, e the cells' strain phasors.
// Separable slices (sr != null): ph holds the column phasors, sr this
// step's row head.
template <int LOGN>
__device__ __forceinline__ void couple_both(float2* v0, float2* v1, const float2* ph,
                                            const float4* sr, int t, float2 am1, float2 bb) {
  using C = FusedCfg<LOGN>;
  constexpr int T = C::T, R0 = C::radix(0), G0 = C::groups(0), S0 = C::stride(0);
  SepHead sh{};
  if (sr) sh = sep_head(sr);
  // b for b e and for b conj(e) (separable: with the row phasor folded in)
  const float2 b0 = sr ? sep_b(bb, sh, 0) : bb, b1 = sr ? sep_b(bb, sh, 1) : bb;
#pragma unroll
  for (int i = 0; i < G0; ++i)
#pragma unroll
    for (int j = 0; j < R0; ++j) {
      const int pos = (t + i * T) + j * S0;
      const float2 e = sr ? sep_cell(sh, ph[pos], pos) : ph[pos];
      const bool inside = (e.x != 0.f) | (e.y != 0.f);
      const float ax = inside ? am1.x : 0.f, ay = inside ? am1.y : 0.f;
      // b e and b conj(e)
      const float2 bp = make_float2(fmaf(b0.x, e.x, -(b0.y * e.y)),
                                    fmaf(b0.x, e.y, b0.y * e.x));
      const float2 bm = make_float2(fmaf(b1.x, e.x, b1.y * e.y),
                                    fmaf(b1.y, e.x, -(b1.x * e.y)));
      const float2 p = v0[i * R0 + j], m = v1[i * R0 + j];
      float px = fmaf(ax, p.x, p.x);
      px = fmaf(-ay, p.y, px);
      px = fmaf(bp.x, m.x, px);
      px = fmaf(-bp.y, m.y, px);
      float py = fmaf(ax, p.y, p.y);
      py = fmaf(ay, p.x, py);
      py = fmaf(bp.x, m.y, py);
      py = fmaf(bp.y, m.x, py);
      float mx = fmaf(ax, m.x, m.x);
      mx = fmaf(-ay, m.y, mx);
      mx = fmaf(bm.x, p.x, mx);
      mx = fmaf(-bm.y, p.y, mx);
      float my = fmaf(ax, m.y, m.y);
      my = fmaf(ay, m.x, my);
      my = fmaf(bm.x, p.y, my);
      my = fmaf(bm.y, p.x, my);
      v0[i * R0 + j] = make_float2(px, py);
      v1[i * R0 + j] = make_float2(mx, my);
    }
}

// SCH: the operator splitting of the step, as in fused2_kernel.cuh (0 the
// first-order step of Eq. fov10; 1 Verlet: couple with (am1h, bh),
// propagate, couple with (am1h, bh); 2 Forest-Ruth: couple with (am1h, bh)
// = t/2, then propagate t dz / couple (am1, b) = (1 - t)/2, propagate
// (1 - 2t) dz / couple (am1, b), propagate t dz / couple (am1h, bh), the
// row's table holding the increments of t dz then (1 - 2t) dz per band).
template <int LOGN, int SCH = 0>
__global__ void __launch_bounds__(FusedCfg<LOGN>::THREADS)
    fused_march_kernel(const RowDescF32* __restrict__ rows, int n_rows,
                       int steps, const float4* __restrict__ tw,
                       int* __restrict__ status) {
  constexpr bool HALF = SCH != 0;                  // couples before propagating
  constexpr int STAGES = SCH == 2 ? 3 : 1;
  using C = FusedCfg<LOGN, HALF ? 2 : 1>;
  constexpr int N = C::N, T = C::T, NP = C::NP, R0 = C::radix(0);
  constexpr int G0 = C::groups(0), S0 = C::stride(0);
  extern __shared__ __align__(128) unsigned char smem[];

  const int rl = threadIdx.x / T;
  const int t = threadIdx.x % T;
  const int row = blockIdx.x * C::ROWS + rl;
  const bool active = row < n_rows;
  const RowDescF32 d = rows[active ? row : 0];

  float2* b0 = reinterpret_cast<float2*>(smem + C::OFF_BUF) + rl * 2 * C::PADN;
  float2* b1 = b0 + C::PADN;
  float2* ph0 = reinterpret_cast<float2*>(smem + C::OFF_PH) + rl * (HALF ? 2 : 1) * N;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + C::OFF_MBAR) + rl * (HALF ? 2 : 1);
  // the records' common phase, two slots by step parity: the lead writes a
  // record step's phase while a slower warp may still read the previous one
  float2* recph = reinterpret_cast<float2*>(smem + C::OFF_RECPH) + 2 * rl;
  double* red = reinterpret_cast<double*>(smem + C::OFF_RED) + rl * C::WARPS_PER_ROW * 2;
  float4* srow0 = reinterpret_cast<float4*>(smem + C::OFF_SROW) + rl * (HALF ? 2 : 1);
  const bool sep = d.srows != nullptr;

  if (t == 0) {
    mbar_init(bar);
    if constexpr (HALF) mbar_init(bar + 1);
  }
  fence_mbar_init();
  // separable slices: the column phasors stay in buffer 0 for the launch
  if (sep && active)
    for (int k = t; k < N; k += T) ph0[k] = __ldg(&d.scols[k]);

  // Registers: pass-0 groups of both bands, natural positions gi + j*S0.
  float2 v0[C::E], v1[C::E];
#pragma unroll
  for (int i = 0; i < G0; ++i)
#pragma unroll
    for (int j = 0; j < R0; ++j) {
      const int pos = (t + i * T) + j * S0;
      v0[i * R0 + j] = active ? d.state[pos] : make_float2(0.f, 0.f);
      v1[i * R0 + j] = active ? d.state[N + pos] : make_float2(0.f, 0.f);
    }
  __shared__ int s_abort;
  if (threadIdx.x == 0) s_abort = 0;
  __syncthreads();

  const uint32_t slice_bytes = uint32_t(N) * 8u;
  int pending_slot = -1;            // record whose powers await reduction
  bool timed_out = false;
  // slice of step n into buffer `slot` (separable: the row head only)
  auto fetch = [&](int n, int slot) {
    if (sep) bulk_load(srow0 + slot, d.srows + n, kSepHeadBytes, bar + slot);
    else bulk_load(ph0 + slot * N, d.phasor + size_t(n) * N, slice_bytes, bar + slot);
  };
  if constexpr (HALF) {
    // the first step's slice; later ones are fetched a step ahead
    if (t == 0 && active && steps > 0) fetch(d.n_begin, 0);
  }

  // Error path: a thread whose bounded wait expires raises s_abort; at the
  // next step's first barrier (or after the last step) each row's lead waits
  // once more (again bounded) for its slice copies in flight, so none is in
  // flight when the CTA exits, and the CTA returns.  With one thread per row
  // and no barrier in the step (N <= 16) that thread alone leaves the march.
  const bool rec_on = active && d.record_every > 0 &&
                      (d.records != nullptr || d.powers != nullptr);
  RecSteps rsteps(d.record_every, d.n_begin);
  int it = 0;
  for (; it < steps; ++it) {
    if constexpr (NP == 1) {
      if (timed_out) break;
    }
    const int n = d.n_begin + it;
    // the step's slice (separable: the column phasors and the row head)
    const float2* ph = ph0 + ((HALF && !sep) ? (it & 1) * N : 0);
    const float4* sr = sep ? srow0 + (HALF ? (it & 1) : 0) : nullptr;
    const RecSteps::Step rs = rsteps.next();
    const bool rec = rec_on && rs.at;
    if (t == 0 && rec) {
      // Common phase exp(i (n+1-n_phase0) dz^ cos(alpha)) in FP64, once per row.
      double ang = fmod(double(n + 1 - d.n_phase0) * d.gphase, 6.283185307179586);
      double sa, ca;
      sincos(ang, &sa, &ca);
      recph[(n + 1) & 1] = make_float2(float(ca), float(sa));
    }
    if constexpr (HALF) {
      // one thread per row (N <= 16) has no barrier in the step: it is past
      // its own couplings of step it - 1, so the other buffer is free
      if constexpr (NP == 1) {
        if (t == 0 && active && it + 1 < steps) fetch(n + 1, (it + 1) & 1);
      }
      // the leading coupling, on this step's slice
      if (active) {
        if (!timed_out && !mbar_wait(bar + (it & 1), uint32_t((it >> 1) & 1))) {
          timed_out = true;
          s_abort = 1;
        }
        couple_both<LOGN>(v0, v1, ph, sr, t, d.am1h, d.bh);
      }
    }

#pragma unroll 1
    for (int sg = 0; sg < STAGES; ++sg) {
      // the stage's propagator increments: (P - 1)/N of the whole step, or
      // for Forest-Ruth those of t dz (stages 0, 2) and (1 - 2t) dz (stage 1)
      const float2* tab = d.prop + ((SCH == 2 && sg == 1) ? 2 * N : 0);
      if constexpr (NP == 1) {
        if constexpr (!HALF) {
          if (t == 0 && active) fetch(n, 0);
        }
        last_pass<LOGN>(v0, v1, t, tab);
      } else {
        // forward pass 0: DFT + twiddle, to shared memory
        dft_pass<LOGN, 0, false>(v0, v1);
        twiddle_pass<LOGN, 0, false>(v0, v1, t, tw);
        store_pass<LOGN, 0>(b0, v0, t);
        store_pass<LOGN, 0>(b1, v1, t);
        __syncthreads();
        if (sg == 0) {
          if (s_abort) {   // the same value for every thread (read after the barrier)
            if (t == 0 && active) {
              // slices up to it were issued (HALF), else up to it - 1
              if constexpr (HALF) mbar_wait(bar + (it & 1), uint32_t((it >> 1) & 1));
              else if (it > 0) mbar_wait(bar, uint32_t((it - 1) & 1));
            }
            if (threadIdx.x == 0) atomicOr(status, kStatusWaitTimeout);
            return;
          }
          // every thread of the row has finished the previous step's
          // couplings: the slice buffer they read is free
          if constexpr (HALF) {
            if (t == 0 && active && it + 1 < steps) fetch(n + 1, (it + 1) & 1);
          } else {
            if (t == 0 && active) fetch(n, 0);
          }
          if (t == 0 && pending_slot >= 0) {
            double s0 = 0.0, s1 = 0.0;
            for (int w = 0; w < C::WARPS_PER_ROW; ++w) {
              s0 += red[2 * w];
              s1 += red[2 * w + 1];
            }
            d.powers[2 * pending_slot] = s0 * d.dx_um;
            d.powers[2 * pending_slot + 1] = s1 * d.dx_um;
            pending_slot = -1;
          }
        }
        if constexpr (NP >= 3) fwd_mid<LOGN, 1>(b0, b1, v0, v1, t, tw);
        if constexpr (NP >= 4) fwd_mid<LOGN, 2>(b0, b1, v0, v1, t, tw);
        load_pass<LOGN, NP - 1>(b0, v0, t);
        load_pass<LOGN, NP - 1>(b1, v1, t);
        last_pass<LOGN>(v0, v1, t, tab);
        store_pass<LOGN, NP - 1>(b0, v0, t);
        store_pass<LOGN, NP - 1>(b1, v1, t);
        __syncthreads();
        if constexpr (NP >= 4) inv_mid<LOGN, 2>(b0, b1, v0, v1, t, tw);
        if constexpr (NP >= 3) inv_mid<LOGN, 1>(b0, b1, v0, v1, t, tw);
        load_pass<LOGN, 0>(b0, v0, t);
        load_pass<LOGN, 0>(b1, v1, t);
        twiddle_pass<LOGN, 0, true>(v0, v1, t, tw);
        dft_pass<LOGN, 0, true>(v0, v1);
      }

      // ---- coupling through chi_0, chi_h, the strain phase and the mask --
      if (active) {
        if constexpr (!HALF) {
          if (!mbar_wait(bar, uint32_t(it & 1))) {
            timed_out = true;
            s_abort = 1;
          }
          couple_both<LOGN>(v0, v1, ph, sr, t, d.am1, d.b);
        } else if constexpr (SCH == 1) {
          couple_both<LOGN>(v0, v1, ph, sr, t, d.am1h, d.bh);
        } else {
          const bool last = sg == STAGES - 1;
          couple_both<LOGN>(v0, v1, ph, sr, t, last ? d.am1h : d.am1, last ? d.bh : d.b);
        }
      }
    }   // stages

    // ---- record: coalesced write of psi * g^k, band powers ----------------
    const bool want_pw = rec && d.powers != nullptr;
    const int slot = rec ? rs.slot : 0;
    double s0 = 0.0, s1 = 0.0;
    if (rec) {
      const float2 g = recph[(n + 1) & 1];
      float2* r0 = d.records ? d.records + size_t(slot) * 2 * N : nullptr;
#pragma unroll
      for (int i = 0; i < G0; ++i)
#pragma unroll
        for (int j = 0; j < R0; ++j) {
          const int pos = (t + i * T) + j * S0;
          const float2 p = v0[i * R0 + j], m = v1[i * R0 + j];
          s0 = pow_acc(s0, p);
          s1 = pow_acc(s1, m);
          if (r0) {
            r0[pos] = make_float2(fmaf(p.x, g.x, -(p.y * g.y)), fmaf(p.x, g.y, p.y * g.x));
            r0[N + pos] = make_float2(fmaf(m.x, g.x, -(m.y * g.y)), fmaf(m.x, g.y, m.y * g.x));
          }
        }
    }
    if constexpr (NP == 1) {
      if (want_pw) {
        d.powers[2 * slot] = double(s0) * d.dx_um;
        d.powers[2 * slot + 1] = double(s1) * d.dx_um;
      }
    } else {
      // All lanes of the warp take part in the shuffles (rows that share a
      // warp may record on different steps); offsets stay inside a row.
      constexpr int LANES = T < 32 ? T : 32;
      if (__any_sync(0xffffffffu, want_pw)) {
        double ds0 = s0, ds1 = s1;
#pragma unroll
        for (int off = LANES / 2; off > 0; off >>= 1) {
          ds0 += __shfl_xor_sync(0xffffffffu, ds0, off);
          ds1 += __shfl_xor_sync(0xffffffffu, ds1, off);
        }
        if (want_pw) {
          if ((t & (LANES - 1)) == 0) {
            red[2 * (t / 32)] = ds0;
            red[2 * (t / 32) + 1] = ds1;
          }
          if (t == 0) pending_slot = slot;
        }
      }
    }
  }

  __syncthreads();
  {
    const bool stopped = NP == 1 ? timed_out : s_abort != 0;
    if (stopped && t == 0 && active) {
      if constexpr (HALF) {
        // the copy whose wait expired (step it - 1 for one thread per row,
        // which leaves at the start of step it; the last step otherwise)
        // and, for one thread per row, the one issued a step ahead
        const int last = NP == 1 ? it - 1 : steps - 1;
        if (last >= 0) mbar_wait(bar + (last & 1), uint32_t((last >> 1) & 1));
        if (NP == 1 && it < steps) mbar_wait(bar + (it & 1), uint32_t((it >> 1) & 1));
      } else if (it > 0) {
        mbar_wait(bar, uint32_t((it - 1) & 1));
      }
    }
  }
  if (t == 0 && pending_slot >= 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < C::WARPS_PER_ROW; ++w) {
      s0 += red[2 * w];
      s1 += red[2 * w + 1];
    }
    d.powers[2 * pending_slot] = s0 * d.dx_um;
    d.powers[2 * pending_slot + 1] = s1 * d.dx_um;
  }
  if (active) {
#pragma unroll
    for (int i = 0; i < G0; ++i)
#pragma unroll
      for (int j = 0; j < R0; ++j) {
        const int pos = (t + i * T) + j * S0;
        d.state[pos] = v0[i * R0 + j];
        d.state[N + pos] = v1[i * R0 + j];
      }
  }
  if (s_abort && threadIdx.x == 0) atomicOr(status, kStatusWaitTimeout);
}

}  // namespace bpm
