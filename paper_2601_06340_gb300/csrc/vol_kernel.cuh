// FP32 march with both transverse coordinates (x, y): Eq. fov4 in 3D with
// the two-beam envelopes of Eq. fov10, each band propagated by
// exp(i dz^ sqrt(1 - (qx +- s)^2 - qy^2)) and coupled pointwise.
//
// One z-step is two kernels over an L2-resident working set (the x-spectra
// of both bands, [B][2][Ny][Nx] c64, and the field of the step's start):
//   column kernel: for every x-frequency column of every band, the forward
//     FFT along y, the increment (P(qx, qy) - 1)/(Nx Ny) and the inverse FFT
//     along y -- the x-spectrum of the step's increment;
//   row kernel: for every line y (both bands in one group of threads), the
//     inverse FFT along x, psi_p = psi + increment (the real-space increment
//     form of fused2_kernel.cuh), the coupling with the strain/mask slice,
//     records, and the forward FFT along x of the new field for the next
//     step.
// Both kernels use the radix-16 pass machinery of the band-per-thread kernel
// (16 points per thread, padded shared memory, digit-reversed spectra): the
// row kernel keeps x-spectra in the x-FFT's output order and the column
// kernel's propagator table is laid out in the y-FFT's output order, so no
// bit reversal is ever done.
#pragma once

#include "fused3_kernel.cuh"

namespace bpm {

struct VolParams {
  float2* org;             // [B][2][Ny][Nx] field at the step's start (natural order)
  float2* spec;            // [B][2][Ny][Nx] x-spectra (x-FFT output order)
  const float2* phasor;    // [nz][Ny][Nx] exp(i h u_x), (0,0) outside
  const float2* prop;      // [B][2][Ny][Nx] (P - 1)/(Nx Ny) in (y-output, x-output) order
  float2* records;         // [B][n_rec][2][Ny][Nx] or null
  double* pwpart;          // [B][n_rec][2][Ny] line sums of |psi|^2 or null
  const float4* twx;       // [Nx] hi/lo twiddles
  const float4* twy;       // [Ny]
  const float2* coup;      // [B][2]: (a - 1, b) per row
  const float2* coup_half; // [B][2]: the same for half a step (second-order splitting)
  const double* gphase;    // [B]
  int nb, nx, ny;
  int n;                   // absolute step of this launch
  int n_phase0;            // absolute step at which `org` carries phase 0
  int record_every, n_rec;
  int mode;                // row kernel: 0 forward FFT only, 1 full step, 2 full step without the forward FFT
};

// ---------------------------------------------------------------------------
// Row kernel: one x-line (both bands) per 2T threads, T = Nx/16.
template <int LOGN>
struct VolRowCfg {
  using F = F2Cfg<LOGN>;
  static constexpr int N = F::N, T = F::T, NP = F::NP;
  static constexpr int THREADS = 2 * T;
  static constexpr int WARPS = THREADS / 32;
  static constexpr int PADN = N + (N >> 4);
  static constexpr int S1 = F::S1;
  static constexpr int OFF_BUF = 0;                               // [2][PADN]
  static constexpr int OFF_TW1 = OFF_BUF + 2 * PADN * 8;          // [S1][16]
  static constexpr int OFF_RED = OFF_TW1 + S1 * 16 * 8;           // [WARPS][2] double
  static constexpr int SMEM = OFF_RED + WARPS * 2 * 8;
  static_assert(SMEM <= 232448, "fits one SM");
};

// HALF = true: the second-order (Verlet) step of Eq. split-op.  The CTA
// holds both bands of its line, so the launch's first step starts with a
// half-step coupling (mode 0) and every step ends with its second half and,
// unless it is the launch's last, the next step's first half; records are
// taken after the second half.
template <int LOGN, bool EX, bool HALF = false>
__global__ void __launch_bounds__(VolRowCfg<LOGN>::THREADS)
    vol_row_kernel(VolParams p) {
  using C = VolRowCfg<LOGN>;
  constexpr int N = C::N, T = C::T, NP = C::NP;
  extern __shared__ __align__(128) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int band = lane >> 4;
  const int t = warp * 16 + (lane & 15);
  const int line = blockIdx.x;                 // r * Ny + y
  const int r = line / p.ny, y = line % p.ny;
  const size_t plane = size_t(p.ny) * N;
  const size_t off = (size_t(r) * 2 + band) * plane + size_t(y) * N;
  float2* buf = reinterpret_cast<float2*>(smem + C::OFF_BUF) + band * C::PADN;
  double* red = reinterpret_cast<double*>(smem + C::OFF_RED);

  float2 w0[15];
#pragma unroll
  for (int j = 1; j < 16; ++j) {
    const float4 a = __ldg(&p.twx[t * j]);
    w0[j - 1] = make_float2(a.x, a.y);
  }
  float2* tw1 = reinterpret_cast<float2*>(smem + C::OFF_TW1);
  for (int k = threadIdx.x; k < C::S1 * 16; k += blockDim.x) {
    const int j = k / C::S1, o = k % C::S1;
    const float4 a = __ldg(&p.twx[(o * j) << 4]);
    tw1[k] = make_float2(a.x, a.y);
  }
  const float2* tw1o = tw1 + (t % C::S1);
  __syncthreads();

  float2 v[16];
  if (p.mode == 0) {
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = p.org[off + t + j * T];
    if constexpr (HALF) {   // the launch's first half-step, on the slice of its first step
      const float2* ph = p.phasor + size_t(p.n) * plane + size_t(y) * N;
      const float2 am1 = p.coup_half[2 * r], bb = p.coup_half[2 * r + 1];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float2 q = make_float2(__shfl_xor_sync(0xffffffffu, v[j].x, 16),
                                     __shfl_xor_sync(0xffffffffu, v[j].y, 16));
        v[j] = couple_cell(v[j], q, __ldg(&ph[t + j * T]), band, am1, bb);
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) p.org[off + t + j * T] = v[j];
    }
  } else {
    // every global read of the step is issued here, so their latencies
    // overlap (a line is too little work to hide three in a row)
    const float2* ph = p.phasor + size_t(p.n) * plane + size_t(y) * N;
    float2 org[16], phv[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      org[j] = p.org[off + t + j * T];
      phv[j] = __ldg(&ph[t + j * T]);
    }
    [[maybe_unused]] float2 phn[16];   // second order: the next step's slice
    if constexpr (HALF) {
      if (p.mode == 1) {
#pragma unroll
        for (int j = 0; j < 16; ++j) phn[j] = __ldg(&ph[plane + t + j * T]);
      }
    }
    // inverse FFT along x of the increment's x-spectrum
    constexpr int P = NP - 1;
    constexpr int R = F2Cfg<LOGN>::radix(P), G = F2Cfg<LOGN>::groups(P);
#pragma unroll
    for (int i = 0; i < G; ++i)
#pragma unroll
      for (int j = 0; j < R; ++j) v[i * R + j] = p.spec[off + f2_pos<LOGN, P>(t + i * T, j)];
    f2_dft<LOGN, P, true, EX>(v);
    f2_store<LOGN, P>(buf, v, t);
    __syncthreads();
    if constexpr (NP >= 3) {
      f2_load<LOGN, 1>(buf, v, t);
      f2_twiddle_s<true, C::S1>(v, tw1o);
      dft<16, true, EX>(v);
      f2_store<LOGN, 1>(buf, v, t);
      __syncthreads();
    }
    f2_load<LOGN, 0>(buf, v, t);
    f2_twiddle<true>(v, w0);
    dft<16, true, EX>(v);
    // psi_p = psi + increment, then the coupling with the other band (lane ^ 16)
    const float2 am1 = HALF ? p.coup_half[2 * r] : p.coup[2 * r];
    const float2 bb = HALF ? p.coup_half[2 * r + 1] : p.coup[2 * r + 1];
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = cadd<false>(org[j], v[j]);   // scalar: measured faster here
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float2 q = make_float2(__shfl_xor_sync(0xffffffffu, v[j].x, 16),
                                   __shfl_xor_sync(0xffffffffu, v[j].y, 16));
      v[j] = couple_cell(v[j], q, phv[j], band, am1, bb);
    }
    const int n1 = p.n + 1;
    if (p.record_every > 0 && (n1 % p.record_every) == 0 && (p.records || p.pwpart)) {
      const int slot = n1 / p.record_every - 1;
      double ang = fmod(double(n1 - p.n_phase0) * p.gphase[r], 6.283185307179586);
      double sa, ca;
      sincos(ang, &sa, &ca);
      const float2 g = make_float2(float(ca), float(sa));
      double s = 0.0;
      float2* r0 = p.records ? p.records + ((size_t(r) * p.n_rec + slot) * 2 + band) * plane +
                                   size_t(y) * N
                             : nullptr;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float2 q = v[j];
        s = pow_acc(s, q);
        if (r0) r0[t + j * T] = make_float2(fmaf(q.x, g.x, -(q.y * g.y)), fmaf(q.x, g.y, q.y * g.x));
      }
      if (p.pwpart) {
        double ds = s;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) ds += __shfl_xor_sync(0xffffffffu, ds, o);
        if ((lane & 15) == 0) red[2 * warp + band] = ds;
        __syncthreads();
        if (threadIdx.x < 2) {
          double tot = 0.0;
          for (int w = 0; w < C::WARPS; ++w) tot += red[2 * w + threadIdx.x];
          p.pwpart[((size_t(r) * p.n_rec + slot) * 2 + threadIdx.x) * p.ny + y] = tot;
        }
      }
    }
    if constexpr (HALF) {
      if (p.mode == 1) {   // the next step's first half, on its slice
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float2 q = make_float2(__shfl_xor_sync(0xffffffffu, v[j].x, 16),
                                       __shfl_xor_sync(0xffffffffu, v[j].y, 16));
          v[j] = couple_cell(v[j], q, phn[j], band, am1, bb);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) p.org[off + t + j * T] = v[j];
    if (p.mode == 2) return;
  }
  // forward FFT along x of the new field (the next step's x-spectrum)
  dft<16, false, EX>(v);
  f2_twiddle<false>(v, w0);
  f2_store<LOGN, 0>(buf, v, t);
  __syncthreads();
  if constexpr (NP >= 3) {
    f2_load<LOGN, 1>(buf, v, t);
    dft<16, false, EX>(v);
    f2_twiddle_s<false, C::S1>(v, tw1o);
    f2_store<LOGN, 1>(buf, v, t);
    __syncthreads();
  }
  {
    constexpr int P = NP - 1;
    constexpr int R = F2Cfg<LOGN>::radix(P), G = F2Cfg<LOGN>::groups(P);
    f2_load<LOGN, P>(buf, v, t);
    f2_dft<LOGN, P, false, EX>(v);
#pragma unroll
    for (int i = 0; i < G; ++i)
#pragma unroll
      for (int j = 0; j < R; ++j) p.spec[off + f2_pos<LOGN, P>(t + i * T, j)] = v[i * R + j];
  }
}

// ---------------------------------------------------------------------------
// Column kernel: COLS = 4 x-frequency columns of one band per CTA (many
// small CTAs, so a single solve spreads over the GPU), T = Ny/16 threads
// per column; lane = column fastest, so table reads and the tile copies move
// whole 32-byte sectors.
template <int LOGN>
struct VolColCfg {
  using F = F2Cfg<LOGN>;
  static constexpr int N = F::N, T = F::T, NP = F::NP;
  static constexpr int COLS = 4;
  static constexpr int THREADS = COLS * T;
  // column stride = 4 mod 16 in 8-byte words: 8-byte accesses are served
  // per half-warp (4 rows x 4 columns here), and the 4 columns land on
  // 4 different quarters of the 16 bank pairs, so the tile copies and the
  // radix-16 passes take 2 wavefronts per warp access, the minimum for 256
  // bytes (a stride of 8 mod 16 put columns 0/2 and 1/3 on the same banks:
  // 4 wavefronts, half of them conflicts in the profile)
  static constexpr int PADC = N + (N >> 4) + 4;
  static constexpr int S1 = F::S1;
  static constexpr int OFF_BUF = 0;                               // [COLS][PADC]
  static constexpr int OFF_TW1 = OFF_BUF + COLS * PADC * 8;       // [S1][16]
  static constexpr int SMEM = OFF_TW1 + S1 * 16 * 8;
  static_assert(THREADS >= 64 && THREADS <= 256, "Ny in [256, 1024]");
  static_assert(SMEM <= 232448, "fits one SM");
};

template <int LOGN, bool EX>
__global__ void __launch_bounds__(VolColCfg<LOGN>::THREADS)
    vol_col_kernel(VolParams p) {
  using C = VolColCfg<LOGN>;
  constexpr int N = C::N, T = C::T, NP = C::NP, COLS = C::COLS;
  extern __shared__ __align__(128) unsigned char smem[];
  const int c = threadIdx.x % COLS, tt = threadIdx.x / COLS;
  const int tiles = p.nx / COLS;
  const int tile = blockIdx.x % tiles;
  const int rb = blockIdx.x / tiles;           // r * 2 + band
  const int band = rb & 1;
  const int col = tile * COLS + c;
  const size_t plane = size_t(N) * p.nx;
  float2* spec = p.spec + size_t(rb) * plane;
  const float2* prop = p.prop + size_t(rb) * plane;
  float2* buf = reinterpret_cast<float2*>(smem + C::OFF_BUF) + c * C::PADC;
  (void)band;

  // this thread's slice of the increment table, issued before the FFT
  float2 pr[16];
  {
    constexpr int P = NP - 1;
    constexpr int R = F2Cfg<LOGN>::radix(P), G = F2Cfg<LOGN>::groups(P);
#pragma unroll
    for (int i = 0; i < G; ++i)
#pragma unroll
      for (int j = 0; j < R; ++j)
        pr[i * R + j] = __ldg(&prop[size_t(f2_pos<LOGN, P>(tt + i * T, j)) * p.nx + col]);
  }
  float2 w0[15];
#pragma unroll
  for (int j = 1; j < 16; ++j) {
    const float4 a = __ldg(&p.twy[tt * j]);
    w0[j - 1] = make_float2(a.x, a.y);
  }
  float2* tw1 = reinterpret_cast<float2*>(smem + C::OFF_TW1);
  for (int k = threadIdx.x; k < C::S1 * 16; k += blockDim.x) {
    const int j = k / C::S1, o = k % C::S1;
    const float4 a = __ldg(&p.twy[(o * j) << 4]);
    tw1[k] = make_float2(a.x, a.y);
  }
  const float2* tw1o = tw1 + (tt % C::S1);

  // tile in: rows y, columns tile*COLS .. +COLS (contiguous per row); all
  // N * COLS / THREADS = 16 loads of a thread issued before the first store
  {
    static_assert(N * COLS == 16 * C::THREADS, "16 tile values per thread");
    float2 tv[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int k = threadIdx.x + i * C::THREADS;
      tv[i] = spec[size_t(k / COLS) * p.nx + tile * COLS + k % COLS];
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int k = threadIdx.x + i * C::THREADS;
      reinterpret_cast<float2*>(smem + C::OFF_BUF)[(k % COLS) * C::PADC + padi(k / COLS)] = tv[i];
    }
  }
  __syncthreads();

  float2 v[16];
  f2_load<LOGN, 0>(buf, v, tt);
  dft<16, false, EX>(v);
  f2_twiddle<false>(v, w0);
  f2_store<LOGN, 0>(buf, v, tt);
  __syncthreads();
  if constexpr (NP >= 3) {
    f2_load<LOGN, 1>(buf, v, tt);
    dft<16, false, EX>(v);
    f2_twiddle_s<false, C::S1>(v, tw1o);
    f2_store<LOGN, 1>(buf, v, tt);
    __syncthreads();
  }
  {
    constexpr int P = NP - 1;
    f2_load<LOGN, P>(buf, v, tt);
    f2_dft<LOGN, P, false, EX>(v);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float2 dd = pr[k], x = v[k];
      v[k] = make_float2(fmaf(x.x, dd.x, -(x.y * dd.y)), fmaf(x.x, dd.y, x.y * dd.x));
    }
    f2_dft<LOGN, P, true, EX>(v);
    f2_store<LOGN, P>(buf, v, tt);
    __syncthreads();
  }
  if constexpr (NP >= 3) {
    f2_load<LOGN, 1>(buf, v, tt);
    f2_twiddle_s<true, C::S1>(v, tw1o);
    dft<16, true, EX>(v);
    f2_store<LOGN, 1>(buf, v, tt);
    __syncthreads();
  }
  f2_load<LOGN, 0>(buf, v, tt);
  f2_twiddle<true>(v, w0);
  dft<16, true, EX>(v);
  f2_store<LOGN, 0>(buf, v, tt);
  __syncthreads();
  // tile out
  for (int k = threadIdx.x; k < N * COLS; k += blockDim.x) {
    const int yy = k / COLS, cc = k % COLS;
    spec[size_t(yy) * p.nx + tile * COLS + cc] =
        reinterpret_cast<const float2*>(smem + C::OFF_BUF)[cc * C::PADC + padi(yy)];
  }
}

}  // namespace bpm
