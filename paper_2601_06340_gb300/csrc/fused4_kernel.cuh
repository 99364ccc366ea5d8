// Split-band fused FP32 marches for N = 4096 P (P = 2 here, P = 4 in
// fused4t_kernel.cuh): one row per cluster of 2P CTAs, CTA rank c = b P + h
// advances band b on the samples x[P m + h] (m < 4096), i.e. one of the P
// interleaved sub-sequences of its band.
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

// N = 8192 (P = 2) with one spectral exchange per step.
//
// For P = 2 the forward combine, the propagator increment and the inverse
// combine above collapse, per local frequency k, into a 2x2
// circulant over the band's two halves:
//   H_h[k] = W_N^{-h k} (E_0[k] G_h[k] + E_1[k] G_{1-h}[k]),
//   E_0[k] = D[k] + D[k + 4096],   E_1[k] = D[k] - D[k + 4096],
// with G_h = W_N^{h k} F_h as before (E_0, E_1 are tabulated in FP64 and
// rounded once).  So each CTA only needs its peer's G: one exchange of 32 KB
// per CTA instead of two all-to-all rounds.  Both exchanges of the step (G
// within the band, psi_p across the bands) are asynchronous remote stores
// that complete on the receiver's mbarrier (see fused3_kernel.cuh), double
// buffered by step parity; no cluster-wide barrier runs inside the march.
// Buffer reuse: a half is rewritten two steps later, by a sender that has by
// then received values the receiver computed from that half.
struct F4ECfg {
  static constexpr int M = 4096;
  static constexpr int N = 2 * M;
  static constexpr int T = M / 16;
  static constexpr int PADM = M + (M >> 4);
  static constexpr int WARPS = T / 32;
  static constexpr int OFF_BUF = 0;                        // [PADM]
  static constexpr int OFF_G = OFF_BUF + PADM * 8;         // [2][M] peer's G
  static constexpr int OFF_C = OFF_G + 2 * M * 8;          // [2][M] other band's psi_p
  static constexpr int OFF_PH = OFF_C + 2 * M * 8;         // [M] strain slice
  static constexpr int OFF_E1 = OFF_PH + M * 8;            // [16][T] E_1 at this thread's k_j
  static constexpr int OFF_MBAR = OFF_E1 + M * 8;          // strain-slice barrier
  static constexpr int OFF_GBAR = OFF_MBAR + 8;            // [2] G barriers
  static constexpr int OFF_CBAR = OFF_GBAR + 16;           // [2] psi_p barriers
  static constexpr int OFF_PPEER = OFF_CBAR + 16;          // [2] peer's band-power part
  static constexpr int OFF_RECPH = OFF_PPEER + 16;
  static constexpr int OFF_RED = OFF_RECPH + 8;            // [WARPS] double
  static constexpr int OFF_PART = OFF_RED + WARPS * 8;
  static constexpr int SMEM = OFF_PART + 8;
  static_assert(SMEM <= 232448, "fits one SM");
};

__device__ __forceinline__ void st_async_f64(uint32_t raddr, double v, uint32_t rbar) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(raddr),
      "l"(__double_as_longlong(v)), "r"(rbar)
      : "memory");
}

template <bool EX>
__global__ void __cluster_dims__(4, 1, 1) __launch_bounds__(F4ECfg::T, 1)
    fused4e_march_kernel(const RowDescF32* __restrict__ rows, int n_rows, int steps,
                         const float4* __restrict__ tw, int* __restrict__ status) {
  namespace cg = cooperative_groups;
  using C = F4ECfg;
  using F = F2Cfg<12>;
  constexpr int L = 12, M = C::M, N = C::N, T = C::T, NP = F::NP;
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
  float2* recph = reinterpret_cast<float2*>(smem + C::OFF_RECPH);
  double* red = reinterpret_cast<double*>(smem + C::OFF_RED);
  double* part = reinterpret_cast<double*>(smem + C::OFF_PART);
  const uint32_t peer = uint32_t(c ^ 1);       // same band, other half of the samples
  const uint32_t partner = uint32_t(c ^ 2);    // other band, same samples
  const uint32_t g_peer = mapa_u32(smem_u32(gx), peer);
  const uint32_t gbar_peer = mapa_u32(smem_u32(gbar), peer);
  const uint32_t pp_peer = mapa_u32(smem_u32(ppeer), peer);
  const uint32_t c_part = mapa_u32(smem_u32(cb), partner);
  const uint32_t cbar_part = mapa_u32(smem_u32(cbar), partner);

  if (lead) {
    mbar_init(bar);
    mbar_init(&gbar[0]);
    mbar_init(&gbar[1]);
    mbar_init(&cbar[0]);
    mbar_init(&cbar[1]);
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
  // Last-pass slice: combine twiddle W_N^{h k_j}, E_0 in registers, E_1 in
  // shared memory (table [band][E_0 | E_1][position]).
  float2 cw[16], e0[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int pos = f2_pos<L, NP - 1>(t, j);
    const int k = (pos >> 8) + ((pos >> 4) & 15) * 16 + (pos & 15) * 256;
    const float4 a = __ldg(&tw[h * k]);
    cw[j] = make_float2(a.x, a.y);
    e0[j] = __ldg(&d.prop[(band * 2 + 0) * M + pos]);
    e1s[j * T + t] = __ldg(&d.prop[(band * 2 + 1) * M + pos]);
  }

  float2 v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = d.state[band * N + 2 * (t + j * T) + h];
  cluster.sync();   // every CTA's barriers initialised before any remote store

  const uint32_t slice_bytes = uint32_t(M) * 8u;
  bool timed_out = false;
  double my_part = 0.0;
  const float2 am1 = d.am1, bb = d.b;
  const bool pow_on = d.powers != nullptr && d.record_every > 0;

  for (int it = 0; it < steps; ++it) {
    const int n = d.n_begin + it;
    const int half = it & 1;
    const bool rec = d.record_every > 0 && ((n + 1) % d.record_every) == 0 &&
                     (d.records != nullptr || d.powers != nullptr);
    // the previous step was a record: its band-power part rides on this step's G
    const bool part_due = pow_on && it > 0 && (n % d.record_every) == 0;
    if (lead && rec) {
      double ang = fmod(double(n + 1 - d.n_phase0) * d.gphase, 6.283185307179586);
      double sa, ca;
      sincos(ang, &sa, &ca);
      *recph = make_float2(float(ca), float(sa));
    }
    float2 org[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) org[j] = v[j];
    dft<16, false, EX>(v);
    f2_twiddle<false>(v, w0);
    f2_store<L, 0>(buf, v, t);
    __syncthreads();
    if (lead) {
      bulk_load(ph, d.phasor + size_t(n) * N + size_t(h) * M, slice_bytes, bar);
      mbar_expect_tx(&gbar[half], uint32_t(M) * 8u + (part_due ? 8u : 0u));
      if (part_due) {
        double s = 0.0;
        for (int w = 0; w < C::WARPS; ++w) s += red[w];
        my_part = s;
        st_async_f64(pp_peer + uint32_t(half) * 8u, s, gbar_peer + uint32_t(half) * 8u);
      }
    }
    f2_load<L, 1>(buf, v, t);
    dft<16, false, EX>(v);
    f2_twiddle<false>(v, w1);
    f2_store<L, 1>(buf, v, t);
    __syncthreads();
    f2_load<L, NP - 1>(buf, v, t);
    dft<16, false, EX>(v);                       // v[j] = F_h[k_j]
    {
      const uint32_t go = g_peer + uint32_t(half * M) * 8u;
      const uint32_t gbo = gbar_peer + uint32_t(half) * 8u;
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = cmul_f(v[j], cw[j].x, cw[j].y);   // G_h[k_j]
#pragma unroll
      for (int pp = 0; pp < 8; ++pp)
        st_async_v4(go + uint32_t(xpair(pp, t, T)) * 8u, v[2 * pp], v[2 * pp + 1], gbo);
    }
    // (no barrier before the inverse pass rewrites buf: each thread's
    // last-pass positions are its own in both directions)
    if (!timed_out && !mbar_wait_cluster(&gbar[half], uint32_t((it >> 1) & 1))) timed_out = true;
    if (lead && part_due && h == 0)
      d.powers[2 * (n / d.record_every - 1) + band] = (my_part + ppeer[half]) * d.dx_um;
    {
      const float2* gi = gx + half * M;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float4 g2 = *reinterpret_cast<const float4*>(gi + xpair(j >> 1, t, T));
        const float2 gp = (j & 1) ? make_float2(g2.z, g2.w) : make_float2(g2.x, g2.y);
        const float2 e1 = e1s[j * T + t], a = e0[j], g = v[j];
        float sx = fmaf(a.x, g.x, -(a.y * g.y));
        float sy = fmaf(a.x, g.y, a.y * g.x);
        sx = fmaf(e1.x, gp.x, sx);
        sx = fmaf(-e1.y, gp.y, sx);
        sy = fmaf(e1.x, gp.y, sy);
        sy = fmaf(e1.y, gp.x, sy);
        v[j] = cmul_f(make_float2(sx, sy), cw[j].x, -cw[j].y);
      }
    }
    dft<16, true, EX>(v);
    f2_store<L, NP - 1>(buf, v, t);
    __syncthreads();
    f2_load<L, 1>(buf, v, t);
    f2_twiddle<true>(v, w1);
    dft<16, true, EX>(v);
    f2_store<L, 1>(buf, v, t);
    __syncthreads();
    f2_load<L, 0>(buf, v, t);
    f2_twiddle<true>(v, w0);
    dft<16, true, EX>(v);
    {
      if (lead) mbar_expect_tx(&cbar[half], uint32_t(M) * 8u);
      const uint32_t co = c_part + uint32_t(half * M) * 8u;
      const uint32_t cbo = cbar_part + uint32_t(half) * 8u;
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = cadd(org[j], v[j]);
#pragma unroll
      for (int pp = 0; pp < 8; ++pp)
        st_async_v4(co + uint32_t(xpair(pp, t, T)) * 8u, v[2 * pp], v[2 * pp + 1], cbo);
    }
    if (!timed_out && !mbar_wait_cluster(&cbar[half], uint32_t((it >> 1) & 1))) timed_out = true;
    if (!timed_out && !mbar_wait(bar, uint32_t(it & 1))) timed_out = true;
    const float2* ci = cb + half * M;
#pragma unroll
    for (int pp = 0; pp < 8; ++pp) {
      const float4 q2 = *reinterpret_cast<const float4*>(ci + xpair(pp, t, T));
      v[2 * pp] = couple_cell(v[2 * pp], make_float2(q2.x, q2.y), ph[t + 2 * pp * T], band, am1, bb);
      v[2 * pp + 1] =
          couple_cell(v[2 * pp + 1], make_float2(q2.z, q2.w), ph[t + (2 * pp + 1) * T], band, am1, bb);
    }

    if (rec) {
      const int slot = (n + 1) / d.record_every - 1;
      const float2 g = *recph;
      float s = 0.f;
      float2* r0 = d.records ? d.records + size_t(slot) * 2 * N + band * N : nullptr;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float2 p = v[j];
        s = fmaf(p.x, p.x, fmaf(p.y, p.y, s));
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
  if (timed_out && lead) atomicOr(status, kStatusWaitTimeout);
  cluster.sync();   // peers may still read our shared memory
}

}  // namespace bpm
