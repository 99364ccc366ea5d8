// Fused FP32 march for N = 16384: one row per cluster of 8 CTAs, CTA rank
// c = 4 band + h advances band b on the samples x[4 m + h] (m < 4096), with
// one all-to-all spectral exchange per step.
//
// With the band split over P = 4 interleaved sub-sequences, the forward
// recombination of the partial spectra G_h = W_N^{h k} F_h (F_h the local
// 4096-point spectrum), the propagator increment D = (P(q) - 1)/N and the
// inverse recombination collapse, per local frequency k, into a circulant
// over the four parts:
//   H_h[k] = W_N^{-h k} sum_{d=0..3} E_d[k] G_{(h+d) mod 4}[k]
//          = sum_d E_d[k] W_N^{(h'-h) k} F_{h'}[k],   h' = (h + d) mod 4,
//   E_d[k] = sum_r W_4^{d r} D[k + 4096 r].
// Part h keeps its own table set E_d W_N^{(h'-h) k}, tabulated in FP64 as
// double-float pairs hi + lo: E_d mixes D values of very different size, and
// one float would round the small ones far beyond their own size, an error
// that repeats every step.  Each CTA sends its F to the three other CTAs of
// its band and needs nothing else from them: one exchange of 3 x 32 KB per
// CTA replaces the two all-to-all rounds of the unfused form, and no
// twiddle multiply remains in the combine.
//
// Storage.  Shared memory holds the FFT scratch, the three received F, the
// other band's psi_p (double-buffered by step parity) and the strain slice:
// 226 KB.  The 64 complex table values of a thread (4 per owned frequency,
// hi and lo) live in tensor memory: written once per launch with
// tcgen05.st, read back one frequency (16 columns) at a time with
// tcgen05.ld each step, the next frequency's load in flight (all 512
// columns of the SM).
//
// Synchronisation, all point to point, no cluster-wide barrier in the march:
//   * F arrives by st.async on the receiver's mbarrier (expected bytes);
//   * a CTA that has read its three F slots arrives remotely on each sender's
//     "free" barrier; a sender waits for all three before writing the next
//     step's F (normally long satisfied: a whole inverse FFT lies between);
//   * psi_p goes to the other band as in the 2-CTA kernel (fused3_kernel.cuh).
// Band powers: the parts of CTAs h = 1..3 ride on the next step's F to h = 0,
// which sums the four in a fixed order.
#pragma once

#include <cooperative_groups.h>

#include "fused4_kernel.cuh"

namespace bpm {

struct F4TCfg {
  static constexpr int M = 4096;
  static constexpr int N = 4 * M;
  static constexpr int T = M / 16;
  static constexpr int PADM = M + (M >> 4);
  static constexpr int WARPS = T / 32;
  static constexpr int TMEM_COLS = 512;                    // 2 x 256 columns per lane
  static constexpr int OFF_BUF = 0;                        // [PADM]
  static constexpr int OFF_G = OFF_BUF + PADM * 8;         // [3][M] F of parts h+1, h+2, h+3
  static constexpr int OFF_C = OFF_G + 3 * M * 8;          // [2][M] other band's psi_p
  static constexpr int OFF_PH = OFF_C + 2 * M * 8;         // [M] strain slice
  static constexpr int OFF_MBAR = OFF_PH + M * 8;          // [2] strain-slice barriers
  static constexpr int OFF_GBAR = OFF_MBAR + 16;           // [WARPS] F arrival
  static constexpr int OFF_FREE = OFF_GBAR + 8 * WARPS;    // peers have read our F
  static constexpr int OFF_CBAR = OFF_FREE + 8;            // [2][WARPS] psi_p arrival
  static constexpr int OFF_PPEER = OFF_CBAR + 16 * WARPS;  // [3] band-power parts (h = 0)
  static constexpr int OFF_RECPH = OFF_PPEER + 24;
  static constexpr int OFF_RED = OFF_RECPH + 16;           // [WARPS] double
  static constexpr int OFF_PART = OFF_RED + WARPS * 8;
  static constexpr int OFF_TMEM = OFF_PART + 8;            // allocated TMEM address
  static constexpr int OFF_SROW = (OFF_TMEM + 8 + 15) / 16 * 16;   // [2] row heads
  static constexpr int SMEM = OFF_SROW + 2 * 16;
  static_assert(SMEM <= 232448, "fits one SM");
  // layout checks: fits one SM (227 KB); bulk-copy and 16-byte store
  // targets 16-byte aligned; mbarriers 8-byte aligned
  static_assert(OFF_G % 16 == 0 && OFF_C % 16 == 0 && OFF_PH % 16 == 0,
                "16-byte stores and bulk copy");
  static_assert(OFF_MBAR % 8 == 0 && OFF_GBAR % 8 == 0 && OFF_FREE % 8 == 0 &&
                    OFF_CBAR % 8 == 0 && OFF_PPEER % 8 == 0,
                "mbarrier and 8-byte store alignment");
};

__device__ __forceinline__ void mbar_init_count(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

// Arrive (release, cluster scope) on a barrier in another CTA's shared memory.
__device__ __forceinline__ void mbar_arrive_remote(uint32_t raddr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(raddr)
               : "memory");
}

// Tensor memory: allocation by one warp, per-thread loads/stores of
// consecutive columns of the thread's own lane (32x32b shape).
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tmem_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31, %32};" ::"r"(taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]),
      "f"(v[8]), "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]),
      "f"(v[15]), "f"(v[16]), "f"(v[17]), "f"(v[18]), "f"(v[19]), "f"(v[20]), "f"(v[21]),
      "f"(v[22]), "f"(v[23]), "f"(v[24]), "f"(v[25]), "f"(v[26]), "f"(v[27]), "f"(v[28]),
      "f"(v[29]), "f"(v[30]), "f"(v[31])
      : "memory");
}

// Issue a load of 16 columns; the registers are valid only after
// tmem_wait16 on the same array (the wait names them as operands, so the
// compiler cannot move their uses above it).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]),
        "=f"(v[7]), "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]),
        "=f"(v[14]), "=f"(v[15])
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ void tmem_wait16(float* v) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]),
                 "+f"(v[6]), "+f"(v[7]), "+f"(v[8]), "+f"(v[9]), "+f"(v[10]), "+f"(v[11]),
                 "+f"(v[12]), "+f"(v[13]), "+f"(v[14]), "+f"(v[15])
               :
               : "memory");
}

// HALF = true: the second-order (Verlet) step, as in fused4_kernel.cuh: the
// couplings of step n's second half (both bands) and of step n + 1's first
// half (own band) after the psi_p swap, the launch's first half-step on the
// other band read from global memory.  Step n + 1's slice is copied into the
// peer spectrum slot 0 once the combine has read it; the receiver's "free"
// arrival for that slot's sender waits until the couplings have used the
// slice (the sender needs it only before sending its step n + 1 spectrum).
template <bool EX, bool HALF = false>
__global__ void __cluster_dims__(8, 1, 1) __launch_bounds__(F4TCfg::T, 1)
    fused4t_march_kernel(const RowDescF32* __restrict__ rows, int n_rows, int steps,
                         const float4* __restrict__ tw, int* __restrict__ status) {
  namespace cg = cooperative_groups;
  using C = F4TCfg;
  using F = F2Cfg<12>;
  constexpr int L = 12, M = C::M, N = C::N, T = C::T, NP = F::NP;
  static_assert(T == 256, "the interval masks take T = 2^8");
  extern __shared__ __align__(128) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();

  const int c = int(cluster.block_rank());
  const int band = c >> 2, h = c & 3;
  const int row = blockIdx.x >> 3;
  const int t = threadIdx.x;
  const int lane = t & 31, warp = t >> 5;
  const RowDescF32 d = rows[row < n_rows ? row : 0];
  const bool lead = t == 0;

  float2* buf = reinterpret_cast<float2*>(smem + C::OFF_BUF);
  float2* gx = reinterpret_cast<float2*>(smem + C::OFF_G);
  float2* cb = reinterpret_cast<float2*>(smem + C::OFF_C);
  float2* ph = reinterpret_cast<float2*>(smem + C::OFF_PH);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + C::OFF_MBAR);
  uint64_t* gbar = reinterpret_cast<uint64_t*>(smem + C::OFF_GBAR);
  uint64_t* gfree = reinterpret_cast<uint64_t*>(smem + C::OFF_FREE);
  uint64_t* cbar = reinterpret_cast<uint64_t*>(smem + C::OFF_CBAR);
  double* ppeer = reinterpret_cast<double*>(smem + C::OFF_PPEER);
  // the records' common phase, two slots by step parity: the lead writes a
  // record step's phase while a slower warp may still read the previous one
  float2* recph = reinterpret_cast<float2*>(smem + C::OFF_RECPH);
  double* red = reinterpret_cast<double*>(smem + C::OFF_RED);
  double* part = reinterpret_cast<double*>(smem + C::OFF_PART);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::OFF_TMEM);

  // peer e (1..3) of the band is part (h + e) & 3; our F goes to its slot
  // 3 - e (the receiver indexes slots by d - 1, d = sender - receiver mod 4)
  // separable slices: the column phasors of the CTA's samples (column
  // 4m + h at position m, as in the stream) stay in the slice buffer; every
  // slice copy carries the step's row head instead (slot 1: the next step's)
  float4* srow0 = reinterpret_cast<float4*>(smem + C::OFF_SROW);
  const bool sep = d.srows != nullptr;
  uint32_t g_to[3], gbar_to[3], free_to[3];
#pragma unroll
  for (int e = 1; e <= 3; ++e) {
    const uint32_t r = uint32_t(band * 4 + ((h + e) & 3));
    g_to[e - 1] = mapa_u32(smem_u32(gx + (3 - e) * M), r);
    gbar_to[e - 1] = mapa_u32(smem_u32(gbar), r);
    free_to[e - 1] = mapa_u32(smem_u32(gfree), r);
  }
  const uint32_t pp_to = mapa_u32(smem_u32(ppeer + (h > 0 ? h - 1 : 0)), uint32_t(band * 4));
  const uint32_t partner = uint32_t(c ^ 4);
  const uint32_t c_part = mapa_u32(smem_u32(cb), partner);
  const uint32_t cbar_part = mapa_u32(smem_u32(cbar), partner);

  if (lead) {
    mbar_init(bar);
    if constexpr (HALF) mbar_init(bar + 1);   // the next-slice copies
    mbar_init_count(gfree, 3);
    for (int w = 0; w < C::WARPS; ++w) {
      mbar_init(&gbar[w]);
      mbar_init(&cbar[w]);
      mbar_init(&cbar[C::WARPS + w]);
    }
  }
  fence_mbar_init();
  if (warp == 0) tmem_alloc(tmem_slot, C::TMEM_COLS);
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  // this thread's 256 columns: lanes 32 (warp mod 4) + lane, columns from 0
  // (warps 0-3) or 256 (warps 4-7)
  const uint32_t tbase = *tmem_slot + (uint32_t(32 * (warp & 3)) << 16) +
                         uint32_t(warp >= 4 ? 256 : 0);

  float2 w0[15], w1[15];
#pragma unroll
  for (int j = 1; j < 16; ++j) {
    const float4 a = __ldg(&tw[4 * (t * j)]);
    w0[j - 1] = make_float2(a.x, a.y);
    const float4 bq = __ldg(&tw[4 * (((t % F::stride(1)) * j) << 4)]);
    w1[j - 1] = make_float2(bq.x, bq.y);
  }
  // this part's E_d W^{(h'-h) k_j} into tensor memory, frequency j at
  // columns 16 j + 4 d + {hi.re, hi.im, lo.re, lo.im}
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    float ev[32];
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
      const int j = 2 * q + jj;
      const int pos = f2_pos<L, NP - 1>(t, j);
#pragma unroll
      for (int dl = 0; dl < 4; ++dl) {
        const float4 e = __ldg(reinterpret_cast<const float4*>(d.prop) +
                               ((band * 4 + h) * 4 + dl) * M + pos);
        ev[jj * 16 + 4 * dl] = e.x;
        ev[jj * 16 + 4 * dl + 1] = e.y;
        ev[jj * 16 + 4 * dl + 2] = e.z;
        ev[jj * 16 + 4 * dl + 3] = e.w;
      }
    }
    tmem_st32(tbase + uint32_t(32 * q), ev);
  }
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");

  float2 v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = d.state[band * N + 4 * (t + j * T) + h];
  if (sep)
#pragma unroll
    for (int j = 0; j < 16; ++j) ph[t + j * T] = __ldg(&d.scols[h * M + t + j * T]);
  cluster.sync();   // every CTA's barriers initialised before any remote operation

  const uint32_t slice_bytes = uint32_t(M) * 8u;
  bool timed_out = false;
  double my_part = 0.0;
  const float2 am1 = HALF ? d.am1h : d.am1, bb = HALF ? d.bh : d.b;
  const bool pow_on = d.powers != nullptr && d.record_every > 0;
  // step n's slice (this part of it) into `dst`, separable: its row head
  // into row-head slot `slot`
  auto fetch = [&](int n, float2* dst, int slot, uint64_t* b) {
    if (sep) bulk_load(srow0 + slot, d.srows + n, kSepHeadBytes, b);
    else bulk_load(dst, d.phasor + size_t(n) * N + size_t(h) * M, slice_bytes, b);
  };
  if constexpr (HALF) {
    // the launch's first half-step on the slice of its first step (phase 0
    // of the slice barrier), the other band from global memory
    if (lead) fetch(d.n_begin, ph, 0, bar);
    float2 q[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) q[j] = d.state[(band ^ 1) * N + 4 * (t + j * T) + h];
    if (!mbar_wait(bar, 0u)) timed_out = true;
    const SepHead sh = sep ? sep_head(srow0) : SepHead{};
    auto first_half = [&](auto S) {
      constexpr bool SEP = decltype(S)::value;
      const uint32_t msk = SEP ? sep_mask<2, 8, 16>(sh, t, h) : 0u;   // T = 256
      const float2 bs = slice_b<SEP>(bb, sh, band);
#pragma unroll
      for (int j = 0; j < 16; ++j)
        v[j] = couple_at<SEP>(v[j], q[j], ph, t + j * T, msk, j, band, am1, bs);
    };
    if (sep) first_half(BoolC<true>{});
    else first_half(BoolC<false>{});
  }

  const bool rec_on = d.record_every > 0 && (d.records != nullptr || d.powers != nullptr);
  RecSteps rsteps(d.record_every, d.n_begin);
  for (int it = 0; it < steps; ++it) {
    const int n = d.n_begin + it;
    const int half = it & 1;
    const RecSteps::Step rs = rsteps.next();
    const bool rec = rec_on && rs.at;
    const bool part_due = pow_on && rs.prev;
    if (lead && rec) {
      double ang = fmod(double(n + 1 - d.n_phase0) * d.gphase, 6.283185307179586);
      double sa, ca;
      sincos(ang, &sa, &ca);
      recph[(n + 1) & 1] = make_float2(float(ca), float(sa));
    }
    float2 org[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) org[j] = v[j];
    dft<16, false, EX>(v);
    f2_twiddle<false>(v, w0);
    f2_store<L, 0>(buf, v, t);
    __syncthreads();
    if (lead) {
      // (second order: phase it + 1, the launch's first half-step took 0)
      fetch(n, ph, 0, bar);
      if (HALF && !sep && it + 1 < steps)
        bulk_prefetch_l2(d.phasor + size_t(n + 1) * N + size_t(h) * M, slice_bytes);
      if (part_due) {
        double s = 0.0;
        for (int w = 0; w < C::WARPS; ++w) s += red[w];
        my_part = s;
      }
    }
    // each warp's F barrier: its 32 threads' slots from the same warp of the
    // three peers (the band-power parts ride on warp 0's)
    if (lane == 0)
      mbar_expect_tx(&gbar[warp], 3u * 32u * 16u * 8u + ((lead && part_due && h == 0) ? 24u : 0u));
    f2_load<L, 1>(buf, v, t);
    dft<16, false, EX>(v);
    f2_twiddle<false>(v, w1);
    f2_store<L, 1>(buf, v, t);
    // (passes 1 and 2 of warp w address positions [512 w, 512 w + 512) only:
    // the barriers between them are the warp's)
    __syncwarp();
    f2_load<L, NP - 1>(buf, v, t);
    dft<16, false, EX>(v);                       // v[j] = F_h[k_j]
    // the peers have read our previous F before we overwrite their slots
    // the peers have read our previous F before we overwrite their slots
    if (it > 0 && !timed_out && !mbar_wait_cluster(gfree, uint32_t((it - 1) & 1))) timed_out = true;
#pragma unroll
    for (int pp = 0; pp < 8; ++pp)
#pragma unroll
      for (int e = 0; e < 3; ++e)
        st_async_v4(g_to[e] + uint32_t(xpair(pp, t, T)) * 8u, v[2 * pp], v[2 * pp + 1],
                    gbar_to[e] + uint32_t(warp) * 8u);
    if (lead && part_due && h > 0) st_async_f64(pp_to, my_part, gbar_to[3 - h]);
    if (!timed_out && !mbar_wait_cluster(&gbar[warp], uint32_t(it & 1))) timed_out = true;
    if (lead && part_due && h == 0)
      d.powers[2 * rs.pslot + band] =
          (((my_part + ppeer[0]) + ppeer[1]) + ppeer[2]) * d.dx_um;
    {
      // E of frequency j from tensor memory, the next frequency's load in
      // flight while this one is used; the lo products are summed first
      float ev[2][16];
      float2 odd[3];   // the odd frequency's half of the peers' 16-byte pairs
      tmem_ld16(tbase, ev[0]);
      tmem_wait16(ev[0]);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        if (j < 15) tmem_ld16(tbase + uint32_t(16 * (j + 1)), ev[(j + 1) & 1]);
        const float* e = ev[j & 1];
        float2 g[4];
        g[0] = v[j];
#pragma unroll
        for (int dl = 1; dl < 4; ++dl) {
          if ((j & 1) == 0) {
            const float4 q = *reinterpret_cast<const float4*>(gx + (dl - 1) * M + xpair(j >> 1, t, T));
            g[dl] = make_float2(q.x, q.y);
            odd[dl - 1] = make_float2(q.z, q.w);
          } else {
            g[dl] = odd[dl - 1];
          }
        }
        float sx = fmaf(e[2], g[0].x, -(e[3] * g[0].y));
        float sy = fmaf(e[2], g[0].y, e[3] * g[0].x);
#pragma unroll
        for (int dl = 1; dl < 4; ++dl) {
          sx = fmaf(e[4 * dl + 2], g[dl].x, sx);
          sx = fmaf(-e[4 * dl + 3], g[dl].y, sx);
          sy = fmaf(e[4 * dl + 2], g[dl].y, sy);
          sy = fmaf(e[4 * dl + 3], g[dl].x, sy);
        }
#pragma unroll
        for (int dl = 0; dl < 4; ++dl) {
          sx = fmaf(e[4 * dl], g[dl].x, sx);
          sx = fmaf(-e[4 * dl + 1], g[dl].y, sx);
          sy = fmaf(e[4 * dl], g[dl].y, sy);
          sy = fmaf(e[4 * dl + 1], g[dl].x, sy);
        }
        v[j] = make_float2(sx, sy);
        if (j < 15) tmem_wait16(ev[(j + 1) & 1]);
      }
    }
    // our F slots are read: release them to each sender (second order: slot
    // 0 holds step n + 1's slice until the couplings, so its sender is
    // released after them).  The release stays per CTA, after a CTA barrier:
    // per-warp releases (24 cluster-scope release arrivals per CTA and step
    // instead of 3) measured 3 % slower, while the F and psi_p arrival
    // barriers are per warp.
    __syncthreads();
    if (lead) {
#pragma unroll
      for (int e = HALF ? 1 : 0; e < 3; ++e) mbar_arrive_remote(free_to[e]);
    }
    if (HALF && lead && it + 1 < steps) fetch(n + 1, gx, 1, bar + 1);
    dft<16, true, EX>(v);
    f2_store<L, NP - 1>(buf, v, t);
    __syncwarp();
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
    // first order: the step's slice, and from its row head the interval mask
    // and the coupling coefficient, while the psi_p stores are in flight
    [[maybe_unused]] uint32_t msk1 = 0u;
    [[maybe_unused]] float2 bs1 = bb;
    if constexpr (!HALF) {
      if (!timed_out && !mbar_wait(bar, uint32_t(it & 1))) timed_out = true;
      if (sep) {
        const SepHead sh = sep_head(srow0);
        msk1 = sep_mask<2, 8, 16>(sh, t, h);
        bs1 = slice_b<true>(bb, sh, band);
      }
    }
    if (!timed_out && !mbar_wait_cluster(&cbar[half * C::WARPS + warp], uint32_t((it >> 1) & 1)))
      timed_out = true;
    if constexpr (HALF) {
      const bool next = it + 1 < steps;
      if (!timed_out && !mbar_wait(bar, uint32_t((it + 1) & 1))) timed_out = true;
      if (next && !timed_out && !mbar_wait(bar + 1, uint32_t(it & 1))) timed_out = true;
      const float2* ci = cb + half * M;
      const float2* phn = sep ? ph : gx;         // slot 0: step n + 1's slice
      const SepHead shc = sep ? sep_head(srow0) : SepHead{};
      const SepHead shn = (sep && next) ? sep_head(srow0 + 1) : SepHead{};
      const float2 g = rec ? recph[(n + 1) & 1] : make_float2(1.f, 0.f);
      const int slot = rec ? rs.slot : 0;
      float2* r0 = (rec && d.records) ? d.records + size_t(slot) * 2 * N + band * N : nullptr;
      double s = 0.0;
      // a loop over shared memory, as in fused4_kernel.cuh
      __syncthreads();
#pragma unroll
      for (int j = 0; j < 16; ++j) buf[t + j * T] = v[j];
      auto three_halves = [&](auto S) {
        constexpr bool SEP = decltype(S)::value;
        const float2 bc = slice_b<SEP>(bb, shc, band), bo = slice_b<SEP>(bb, shc, band ^ 1);
        const float2 bn = slice_b<SEP>(bb, shn, band);
        const uint32_t mc = SEP ? sep_mask<2, 8, 16>(shc, t, h) : 0u;
        const uint32_t mn = SEP ? sep_mask<2, 8, 16>(shn, t, h) : 0u;
#pragma unroll 1
        for (int pp = 0; pp < 8; ++pp) {
          const float4 q2 = *reinterpret_cast<const float4*>(ci + xpair(pp, t, T));
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const int j = 2 * pp + k;
            const int cell = t + j * T;
            const float2 p = buf[cell], q = k ? make_float2(q2.z, q2.w) : make_float2(q2.x, q2.y);
            // step it, second half (this band's and, below, the other band's)
            float2 cc = couple_at<SEP>(p, q, ph, cell, mc, j, band, am1, bc);
            if (rec) {
              s = pow_acc(s, cc);
              if (r0)   // records in natural order
                r0[4 * cell + h] =
                    make_float2(fmaf(cc.x, g.x, -(cc.y * g.y)), fmaf(cc.x, g.y, cc.y * g.x));
            }
            if (next) {   // step it + 1, first half, with the other band's value
              const float2 co = couple_at<SEP>(q, p, ph, cell, mc, j, band ^ 1, am1, bo);
              cc = couple_at<SEP>(cc, co, phn, cell, mn, j, band, am1, bn);
            }
            buf[cell] = cc;
          }
        }
      };
      if (sep) three_halves(BoolC<true>{});
      else three_halves(BoolC<false>{});
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = buf[t + j * T];
      __syncthreads();
      if (lead) mbar_arrive_remote(free_to[0]);   // slot 0 is free again
      if (rec && d.powers) {
        double ds = s;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) ds += __shfl_xor_sync(0xffffffffu, ds, off);
        if (lane == 0) red[warp] = ds;   // summed by the lead after the next barrier
      }
    } else {
    const float2* ci = cb + half * M;
    auto couple_all = [&](auto S) {
      constexpr bool SEP = decltype(S)::value;
      const float2 bs = SEP ? bs1 : bb;
      const uint32_t msk = SEP ? msk1 : 0u;
#pragma unroll
      for (int pp = 0; pp < 8; ++pp) {
        const float4 q2 = *reinterpret_cast<const float4*>(ci + xpair(pp, t, T));
        const int m0 = t + 2 * pp * T, m1 = t + (2 * pp + 1) * T;
        v[2 * pp] = couple_at<SEP>(v[2 * pp], make_float2(q2.x, q2.y), ph, m0, msk, 2 * pp, band,
                                   am1, bs);
        v[2 * pp + 1] = couple_at<SEP>(v[2 * pp + 1], make_float2(q2.z, q2.w), ph, m1, msk,
                                       2 * pp + 1, band, am1, bs);
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
          r0[4 * (t + j * T) + h] =
              make_float2(fmaf(p.x, g.x, -(p.y * g.y)), fmaf(p.x, g.y, p.y * g.x));
      }
      if (d.powers) {
        double ds = s;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) ds += __shfl_xor_sync(0xffffffffu, ds, off);
        if (lane == 0) red[warp] = ds;   // summed by the lead after the next barrier
      }
    }
    }   // first-order coupling
  }

  __syncthreads();
  const bool last_due = pow_on && steps > 0 && ((d.n_begin + steps) % d.record_every) == 0;
  if (lead && last_due) {
    double s = 0.0;
    for (int w = 0; w < C::WARPS; ++w) s += red[w];
    *part = s;
  }
  cluster.sync();
  if (lead && last_due && h == 0) {
    double s = *part;
    for (int r = 1; r < 4; ++r) s += *cluster.map_shared_rank(part, band * 4 + r);
    d.powers[2 * ((d.n_begin + steps) / d.record_every - 1) + band] = s * d.dx_um;
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) d.state[band * N + 4 * (t + j * T) + h] = v[j];
  // Error path: after an expired wait a thread skips its later waits and the
  // march runs on to the end of the launch; the lead still issues one slice
  // copy per step on its barrier, so waiting (again bounded) for the last
  // step's phase leaves no copy of its own in flight when the CTA exits.
  if (timed_out) {
    if constexpr (HALF) {
      // phase `steps` of the slice barrier (phase 0 was the launch's first
      // half-step) and phase steps - 2 of the next-slice barrier
      if (lead && steps >= 2) mbar_wait(bar + 1, uint32_t(steps & 1));
      give_up_after_march(bar, uint32_t(steps & 1), lead, status);
    } else {
      give_up_after_march(bar, uint32_t((steps - 1) & 1), lead, status);
    }
  }
  tmem_fence_before();
  cluster.sync();   // peers may still read our shared memory
  tmem_fence_after();
  if (warp == 0) tmem_dealloc(*tmem_slot, C::TMEM_COLS);
}

}  // namespace bpm
