// Fused FP32 march, band-per-thread layout, for 256 <= N <= 4096.
//
// One step of Eq. fov10 (arXiv 2601.06340) is evaluated as
//   psi_p = psi + F^-1[ ((P(q) - 1)/N) F[psi] ]           (each band alone)
//   psi   <- psi_p + (a - 1) psi_p + b e^{+-i h u} psi_p(other band)   in Pi
// i.e. the free propagation is applied as an increment to the stored field.
// The FFT then only produces the small per-step change (|P - 1| is 0.01 to
// 0.2 on the occupied modes), so its FP32 rounding reaches the field scaled
// by |P - 1| instead of in full, and the field itself is rounded once per
// step.  Measured on the 8000-step Bragg march this takes the weak
// transmitted band from 3e-4 to within 10% of the bound set by storing the
// field in FP32 at all.
//
// Layout.  A row of N points per band is handled by 2T threads, T = N/16:
// in every warp lanes 0-15 own 16 points of psi_+ and lanes 16-31 the same
// 16 positions of psi_-, so the coupling partner is one shuffle away.  The
// thread -> FFT-group map is fixed for the whole launch, so each thread keeps
// its table twiddles (passes before the last) in registers.  The original
// field of the step is parked in shared memory by the thread that owns it
// (no barrier needed).  Passes are radix 16 plus a last pass of radix
// 2^(LOGN mod 4); the last forward pass, the propagator and the first
// inverse pass are fused in registers, and so are the last inverse pass,
// the coupling, the record and the next forward pass.
#pragma once

#include "fused_kernel.cuh"

namespace bpm {

// PHB: strain-slice buffers per row (2 when the step couples before it
// propagates: the second- and fourth-order forms fetch the next step's
// slice a step ahead)
template <int LOGN, int PHB = 1>
struct F2Cfg {
  static constexpr int N = 1 << LOGN;
  static constexpr int E = 16;
  static constexpr int T = N / 16;                    // threads per band
  static constexpr int NP = (LOGN + 3) / 4;
  static constexpr int RL = 1 << (LOGN - 4 * (NP - 1));
  static constexpr int ROWS = (2 * T >= 256) ? 1 : 256 / (2 * T);
  static constexpr int THREADS = 2 * T * ROWS;
  static constexpr int WPR = 2 * T / 32;              // warps per row
  static constexpr int PADN = N + (N >> 4);
  static constexpr int OFF_BUF = 0;                                   // [ROWS][2][PADN]
  static constexpr int OFF_ORG = OFF_BUF + ROWS * 2 * PADN * 8;       // [ROWS][2][N]
  static constexpr int OFF_PH = OFF_ORG + ROWS * 2 * N * 8;           // [ROWS][PHB][N]
  static constexpr int OFF_MBAR = OFF_PH + ROWS * PHB * N * 8;        // [ROWS][PHB]
  static constexpr int OFF_RECPH = OFF_MBAR + ROWS * PHB * 8;
  static constexpr int OFF_RED = OFF_RECPH + ROWS * 16;               // [ROWS][WPR][2] double
  static constexpr int S1 = NP >= 3 ? (N >> 8) : 1;                   // pass-1 group offsets
  static constexpr int OFF_TW1 = OFF_RED + ROWS * WPR * 2 * 8;        // [S1][16] float2
  static constexpr int OFF_SROW = (OFF_TW1 + S1 * 16 * 8 + 15) / 16 * 16;   // [ROWS][PHB]
  static constexpr int SMEM = OFF_SROW + ROWS * PHB * 16;
  static_assert(LOGN >= 8 && LOGN <= 12, "band-per-thread kernel covers 256..4096");
  // Three passes (N = 512..4096): pass 1 and the last pass (groups as in
  // f2_group) of the 16 threads of a band in a warp address positions
  // [256 a, 256 a + 256) of that band's buffer only, so the barriers between
  // them (either direction) are warp barriers
  static constexpr bool TAIL_WARP = NP >= 3;
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

template <int LOGN, int P>
__host__ __device__ __forceinline__ int f2_pos(int gi, int j) {
  using C = F2Cfg<LOGN>;
  constexpr int S = C::stride(P), L = C::len(P);
  return (gi / S) * L + (gi % S) + j * S;
}

// Group i of thread t in pass P.  WL (warp-local tail): the last pass's
// groups are taken as 16 G (t / 16) + 16 i + t mod 16 (G groups per thread)
// instead of t + i T, so that the 16 threads t = 16 a .. 16 a + 15 address
// positions [256 a, 256 a + 256) in the last pass as they do in pass 1
// (stride N / 256 <= 16): between pass 1 and the last pass only those 16
// threads exchange data, and a warp (one or two such groups) synchronizes
// with itself alone.  Both directions and every table lookup of the last
// pass must use the same choice.
template <int LOGN, int P, bool WL = false>
__host__ __device__ __forceinline__ int f2_group(int t, int i) {
  using C = F2Cfg<LOGN>;
  if constexpr (WL && P == C::NP - 1 && C::RL < 16)
    return (t >> 4) * (16 * C::groups(P)) + i * 16 + (t & 15);
  else
    return t + i * C::T;
}

// Table position of thread t's point k = i RL + j of the last pass, where
// the plan's propagator tables hold (P - 1)/N per band.  (The Forest-Ruth
// stage tables are kept in thread order instead: entry k T + t of a band.)
template <int LOGN>
__host__ __device__ __forceinline__ int f2_table_pos(int t, int k) {
  using C = F2Cfg<LOGN>;
  constexpr int P = C::NP - 1;
  return f2_pos<LOGN, P>(f2_group<LOGN, P, C::TAIL_WARP>(t, k / C::RL), k % C::RL);
}

template <int LOGN, int P, bool WL = false>
__device__ __forceinline__ void f2_store(float2* buf, const float2* v, int t) {
  using C = F2Cfg<LOGN>;
  constexpr int R = C::radix(P), G = C::groups(P);
#pragma unroll
  for (int i = 0; i < G; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j)
      buf[padi(f2_pos<LOGN, P>(f2_group<LOGN, P, WL>(t, i), j))] = v[i * R + j];
}

template <int LOGN, int P, bool WL = false>
__device__ __forceinline__ void f2_load(const float2* buf, float2* v, int t) {
  using C = F2Cfg<LOGN>;
  constexpr int R = C::radix(P), G = C::groups(P);
#pragma unroll
  for (int i = 0; i < G; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j)
      v[i * R + j] = buf[padi(f2_pos<LOGN, P>(f2_group<LOGN, P, WL>(t, i), j))];
}

template <int LOGN, int P, bool INV, bool EX, bool PACK = true>
__device__ __forceinline__ void f2_dft(float2* v) {
  using C = F2Cfg<LOGN>;
  constexpr int R = C::radix(P), G = C::groups(P);
#pragma unroll
  for (int i = 0; i < G; ++i) dft<R, INV, EX, PACK>(v + i * R);
}

// radix-16 twiddle pass with twiddles W^{o j} = w[j * STRIDE] (shared table)
template <bool INV, int STRIDE>
__device__ __forceinline__ void f2_twiddle_s(float2* v, const float2* w) {
#pragma unroll
  for (int j = 1; j < 16; ++j) {
    const float2 t = w[j * STRIDE];
    v[j] = INV ? cmul_f(v[j], t.x, -t.y) : cmul_f(v[j], t.x, t.y);
  }
}

// radix-16 twiddle pass with register twiddles w[j-1] = W^{o j}
template <bool INV>
__device__ __forceinline__ void f2_twiddle(float2* v, const float2* w) {
#pragma unroll
  for (int j = 1; j < 16; ++j) {
    const float2 t = w[j - 1];
    v[j] = INV ? cmul_f(v[j], t.x, -t.y) : cmul_f(v[j], t.x, t.y);
  }
}

// Coupling of this thread's 16 cells with the other band (lane ^ 16), the
// coefficients (a - 1, b) of the step (or of its half), e = the cells' strain
// phasors from the slice `ph` (separable slices: sr != null, ph the column
// phasors and sr the step's row head).
template <int T, bool SEP>
__device__ __forceinline__ void f2_couple_cells(float2* v, const float2* ph, const float4* sr,
                                                int t, int band, float2 am1, float2 bb) {
  SepHead sh{};
  if constexpr (SEP) {
    sh = sep_head(sr);
    bb = sep_b(bb, sh, band);
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const float2 q = make_float2(__shfl_xor_sync(0xffffffffu, v[j].x, 16),
                                 __shfl_xor_sync(0xffffffffu, v[j].y, 16));
    float2 e = SEP ? sep_cell(sh, ph[t + j * T], t + j * T) : ph[t + j * T];
    const bool inside = (e.x != 0.f) | (e.y != 0.f);
    if (band) e.y = -e.y;
    const float ax = inside ? am1.x : 0.f, ay = inside ? am1.y : 0.f;
    const float cx = fmaf(bb.x, e.x, -(bb.y * e.y)), cy = fmaf(bb.x, e.y, bb.y * e.x);
    const float2 p = v[j];
    float rx = fmaf(ax, p.x, p.x);
    rx = fmaf(-ay, p.y, rx);
    rx = fmaf(cx, q.x, rx);
    rx = fmaf(-cy, q.y, rx);
    float ry = fmaf(ax, p.y, p.y);
    ry = fmaf(ay, p.x, ry);
    ry = fmaf(cx, q.y, ry);
    ry = fmaf(cy, q.x, ry);
    v[j] = make_float2(rx, ry);
  }
}

template <int T>
__device__ __forceinline__ void f2_couple(float2* v, const float2* ph, const float4* sr, int t,
                                          int band, float2 am1, float2 bb) {
  if (sr) f2_couple_cells<T, true>(v, ph, sr, t, band, am1, bb);
  else f2_couple_cells<T, false>(v, ph, sr, t, band, am1, bb);
}

// Operator splitting of the step (Eq. split-op), SCH:
//   kSchFirst  the first-order step of Eq. fov10: propagate, then couple
//              with the step's coefficients (am1, b);
//   kSchVerlet the second-order (Verlet / Strang) step: couple with the
//              half-step coefficients (am1h, bh), propagate, couple with
//              them again;
//   kSchForestRuth the fourth-order step: couple (t/2), then three stages of
//              propagate + couple with the propagators of t dz, (1 - 2t) dz
//              and t dz and the couplings ((1 - t)/2, (1 - t)/2, t/2);
//              the row's table holds (P^t - 1)/N then (P^(1-2t) - 1)/N per
//              band, (am1, b) are the (1 - t)/2 coefficients and
//              (am1h, bh) the t/2 ones.
// Every coupling of step n uses the slice of step n.  The second- and
// fourth-order forms couple before the first propagation, so the slice of
// step n + 1 is fetched during step n into the other of two buffers.
constexpr int kSchFirst = 0, kSchVerlet = 1, kSchForestRuth = 2;

template <int LOGN, bool EX, int SCH = kSchFirst>
__global__ void __launch_bounds__(F2Cfg<LOGN>::THREADS, F2Cfg<LOGN>::THREADS >= 512 ? 1 : 2)
    fused2_march_kernel(const RowDescF32* __restrict__ rows, int n_rows, int steps,
                        const float4* __restrict__ tw, int* __restrict__ status) {
  constexpr bool HALF = SCH != kSchFirst;          // couples before propagating
  constexpr int STAGES = SCH == kSchForestRuth ? 3 : 1;
  using C = F2Cfg<LOGN, HALF ? 2 : 1>;
  constexpr int N = C::N, T = C::T, NP = C::NP, RL = C::RL;
  constexpr int WPB = T / 16;                  // warps per band-pair group
  // packed complex adds in the butterflies at every N (at N = 4096, with the
  // 128-register budget, measured 54.9-55.0 vs 55.0-55.9 ms for a 256-energy
  // batch against scalar adds)
  constexpr bool PK = true;
  extern __shared__ __align__(128) unsigned char smem[];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rl = warp / WPB;
  const int band = lane >> 4;
  const int t = (warp % WPB) * 16 + (lane & 15);
  const int row = blockIdx.x * C::ROWS + rl;
  const bool active = row < n_rows;
  const RowDescF32 d = rows[active ? row : 0];
  const bool lead = active && t == 0 && band == 0;

  float2* buf = reinterpret_cast<float2*>(smem + C::OFF_BUF) + (rl * 2 + band) * C::PADN;
  float2* org = reinterpret_cast<float2*>(smem + C::OFF_ORG) + (rl * 2 + band) * N;
  float2* ph0 = reinterpret_cast<float2*>(smem + C::OFF_PH) + rl * (HALF ? 2 : 1) * N;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + C::OFF_MBAR) + rl * (HALF ? 2 : 1);
  // the records' common phase, two slots by step parity: the lead writes a
  // record step's phase while a slower warp may still read the previous one
  float2* recph = reinterpret_cast<float2*>(smem + C::OFF_RECPH) + 2 * rl;
  double* red = reinterpret_cast<double*>(smem + C::OFF_RED) + rl * C::WPR * 2;
  float4* srow0 = reinterpret_cast<float4*>(smem + C::OFF_SROW) + rl * (HALF ? 2 : 1);
  const bool sep = d.srows != nullptr;

  if (t == 0 && band == 0) {
    mbar_init(bar);
    if constexpr (HALF) mbar_init(bar + 1);
  }
  fence_mbar_init();
  // separable slices: the column phasors stay in buffer 0 for the launch
  if (sep && active)
    for (int k = band * T + t; k < N; k += 2 * T) ph0[k] = __ldg(&d.scols[k]);

  // Twiddles: pass 0 (group o = t) in registers; pass 1 (o = t mod S1, only
  // S1 distinct groups) from a small shared table W_{N/16}^{o j}.
  float2 w0[15];
#pragma unroll
  for (int j = 1; j < 16; ++j) {
    const float4 a = __ldg(&tw[t * j]);
    w0[j - 1] = make_float2(a.x, a.y);
  }
  // table layout [j][o] (o fastest): lanes with consecutive o read
  // consecutive words
  float2* tw1 = reinterpret_cast<float2*>(smem + C::OFF_TW1);
  for (int k = threadIdx.x; k < C::S1 * 16; k += blockDim.x) {
    const int j = k / C::S1, o = k % C::S1;
    const float4 a = __ldg(&tw[(o * j) << 4]);
    tw1[k] = make_float2(a.x, a.y);
  }
  const float2* tw1o = tw1 + (t % C::S1);

  // this thread's slice of (P - 1)/N in the last pass (for the whole launch;
  // the fourth-order step reloads it per stage, see below, from its stage
  // tables in thread order, so that a warp's loads are coalesced)
  float2 pr[16];
  auto load_table = [&](const float2* tab) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int at = SCH == kSchForestRuth ? k * T + t : f2_table_pos<LOGN>(t, k);
      pr[k] = active ? __ldg(&tab[band * N + at]) : make_float2(0.f, 0.f);
    }
  };
  load_table(d.prop);
  float2 v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j)
    v[j] = active ? d.state[band * N + t + j * T] : make_float2(0.f, 0.f);
  __shared__ int s_abort;
  if (threadIdx.x == 0) s_abort = 0;
  __syncthreads();

  const uint32_t slice_bytes = uint32_t(N) * 8u;
  int pending_slot = -1;
  bool timed_out = false;
  // slice of step n into buffer `slot` (separable: the row head only)
  auto fetch = [&](int n, int slot) {
    if (sep) bulk_load(srow0 + slot, d.srows + n, kSepHeadBytes, bar + slot);
    else bulk_load(ph0 + slot * N, d.phasor + size_t(n) * N, slice_bytes, bar + slot);
  };
  if constexpr (HALF) {
    // the first step's slice; later ones are fetched a step ahead
    if (lead && steps > 0) fetch(d.n_begin, 0);
  }

  // Error path: a thread whose bounded wait expires skips this step's other
  // waits and raises s_abort; at the next step's first barrier (or after the
  // last step) the lead waits once more (again bounded) for its last slice
  // copy, so none is in flight when the CTA exits, and the CTA returns.
  const bool rec_on = active && d.record_every > 0 &&
                      (d.records != nullptr || d.powers != nullptr);
  RecSteps rsteps(d.record_every, d.n_begin);
  for (int it = 0; it < steps; ++it) {
    const int n = d.n_begin + it;
    const RecSteps::Step rs = rsteps.next();
    // the step's slice (separable: the column phasors and the row head)
    const float2* ph = ph0 + ((HALF && !sep) ? (it & 1) * N : 0);
    const float4* sr = sep ? srow0 + (HALF ? (it & 1) : 0) : nullptr;
    if constexpr (HALF) {
      // first half coupling, on this step's slice
      if (active && !timed_out && !mbar_wait(bar + (it & 1), uint32_t((it >> 1) & 1))) {
        timed_out = true;
        s_abort = 1;
      }
      f2_couple<T>(v, ph, sr, t, band, d.am1h, d.bh);
    }
    const bool rec = rec_on && rs.at;
    if (lead && rec) {
      double ang = fmod(double(n + 1 - d.n_phase0) * d.gphase, 6.283185307179586);
      double sa, ca;
      sincos(ang, &sa, &ca);
      recph[(n + 1) & 1] = make_float2(float(ca), float(sa));
    }
#pragma unroll 1
    for (int sg = 0; sg < STAGES; ++sg) {
    if constexpr (SCH == kSchForestRuth) {
      // the stage's table: (P^t - 1)/N for stages 0 and 2, (P^(1-2t) - 1)/N
      // for stage 1 (read from L2 while the forward passes run)
      if (sg > 0) load_table(d.prop + (sg == 1 ? 2 * N : 0));
    }
    // park the field of this stage; forward pass 0
#pragma unroll
    for (int j = 0; j < 16; ++j) org[t + j * T] = v[j];
    dft<16, false, EX, PK>(v);
    f2_twiddle<false>(v, w0);
    f2_store<LOGN, 0>(buf, v, t);
    __syncthreads();
    if (sg == 0 && s_abort) {   // the same value for every thread (read after the barrier)
      if (lead) {
        // slices up to it were issued (HALF), else up to it - 1
        if constexpr (HALF) mbar_wait(bar + (it & 1), uint32_t((it >> 1) & 1));
        else if (it > 0) mbar_wait(bar, uint32_t((it - 1) & 1));
      }
      if (threadIdx.x == 0) atomicOr(status, kStatusWaitTimeout);
      return;
    }
    if constexpr (HALF) {
      // every thread is past the couplings of step it - 1, which read the
      // other buffer: fetch step it + 1's slice into it
      if (lead && sg == 0 && it + 1 < steps) fetch(n + 1, (it + 1) & 1);
    } else {
      if (lead) fetch(n, 0);
    }
    if (lead && pending_slot >= 0) {
      double s0 = 0.0, s1 = 0.0;
      for (int w = 0; w < C::WPR; ++w) {
        s0 += red[2 * w];
        s1 += red[2 * w + 1];
      }
      d.powers[2 * pending_slot] = s0 * d.dx_um;
      d.powers[2 * pending_slot + 1] = s1 * d.dx_um;
      pending_slot = -1;
    }
    if constexpr (NP >= 3) {
      f2_load<LOGN, 1>(buf, v, t);
      dft<16, false, EX, PK>(v);
      f2_twiddle_s<false, C::S1>(v, tw1o);
      f2_store<LOGN, 1>(buf, v, t);
      tail_sync<C::TAIL_WARP>();
    }
    // last pass: forward DFT, (P - 1)/N, inverse DFT
    {
      constexpr int P = NP - 1;
      f2_load<LOGN, P, C::TAIL_WARP>(buf, v, t);
      f2_dft<LOGN, P, false, EX, PK>(v);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float2 dd = pr[k], x = v[k];
        v[k] = make_float2(fmaf(x.x, dd.x, -(x.y * dd.y)), fmaf(x.x, dd.y, x.y * dd.x));
      }
      f2_dft<LOGN, P, true, EX, PK>(v);
      f2_store<LOGN, P, C::TAIL_WARP>(buf, v, t);
      tail_sync<C::TAIL_WARP>();
    }
    if constexpr (NP >= 3) {
      f2_load<LOGN, 1>(buf, v, t);
      f2_twiddle_s<true, C::S1>(v, tw1o);
      dft<16, true, EX, PK>(v);
      f2_store<LOGN, 1>(buf, v, t);
      __syncthreads();
    }
    f2_load<LOGN, 0>(buf, v, t);
    f2_twiddle<true>(v, w0);
    dft<16, true, EX, PK>(v);
    // psi_p = psi + increment
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float2 o = org[t + j * T];
      v[j] = cadd<PK>(o, v[j]);
    }

    // ---- coupling with the other band (lane ^ 16) -------------------------
    if constexpr (SCH == kSchFirst) {
      if (active && !mbar_wait(bar, uint32_t(it & 1))) {
        timed_out = true;
        s_abort = 1;
      }
      f2_couple<T>(v, ph, sr, t, band, d.am1, d.b);
    } else if constexpr (SCH == kSchVerlet) {
      f2_couple<T>(v, ph, sr, t, band, d.am1h, d.bh);
    } else {
      const bool last = sg == STAGES - 1;
      f2_couple<T>(v, ph, sr, t, band, last ? d.am1h : d.am1, last ? d.bh : d.b);
    }
    }   // stages (the fourth-order step ends on the t dz table, which its
        // next step starts with)

    // ---- record ------------------------------------------------------------
    const bool want_pw = rec && d.powers != nullptr;
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
      if (want_pw) {
        double ds = s;
#pragma unroll
        for (int off = 8; off > 0; off >>= 1) ds += __shfl_xor_sync(0xffffffffu, ds, off);
        if ((lane & 15) == 0) red[2 * (warp % WPB) + band] = ds;
        if (lead) pending_slot = slot;
      }
    }
  }

  __syncthreads();
  if (s_abort && lead) {   // an expired wait in the last step: its slice copy
    const int last = steps - 1;
    if constexpr (HALF) mbar_wait(bar + (last & 1), uint32_t((last >> 1) & 1));
    else mbar_wait(bar, uint32_t(last & 1));
  }
  if (lead && pending_slot >= 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < C::WPR; ++w) {
      s0 += red[2 * w];
      s1 += red[2 * w + 1];
    }
    d.powers[2 * pending_slot] = s0 * d.dx_um;
    d.powers[2 * pending_slot + 1] = s1 * d.dx_um;
  }
  if (active) {
#pragma unroll
    for (int j = 0; j < 16; ++j) d.state[band * N + t + j * T] = v[j];
  }
  if (s_abort && threadIdx.x == 0) atomicOr(status, kStatusWaitTimeout);
}

}  // namespace bpm
