// Input conversion, output finishing (common phase, final powers) and the
// energy -> time synthesis of a batch of exit fields.
#include <algorithm>
#include <cstring>

#include "bpm_internal.h"

namespace bpm {

namespace {

__global__ void convert_in_kernel(const double2* __restrict__ src, float2* __restrict__ dst,
                                  size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x)
    dst[i] = make_float2(float(src[i].x), float(src[i].y));
}

// One block per (row, band): out = state * g_row (FP64 product), power of
// the line in FP64 (fixed summation order).
template <typename TIn>
__global__ void finish_kernel(const TIn* __restrict__ state, double2* __restrict__ out128,
                              float2* __restrict__ out64, const double2* __restrict__ g,
                              int nx, double dx, double* __restrict__ pw, int pw_stride) {
  __shared__ double part[32];
  const int row = blockIdx.x >> 1, band = blockIdx.x & 1;
  const size_t base = (size_t(row) * 2 + band) * nx;
  const double2 gr = g[row];
  double s = 0.0;
  for (int j = threadIdx.x; j < nx; j += blockDim.x) {
    const double vx = double(state[base + j].x), vy = double(state[base + j].y);
    s += vx * vx + vy * vy;
    const double ox = vx * gr.x - vy * gr.y, oy = vx * gr.y + vy * gr.x;
    if (out128) out128[base + j] = make_double2(ox, oy);
    if (out64) out64[base + j] = make_float2(float(ox), float(oy));
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0 && pw) {
    double tot = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) tot += part[w];
    pw[size_t(row) * pw_stride + band] = tot * dx;
  }
}

// Energy -> time: for each (band, x) line, out[band][x][m] =
// sum_j in[j][band][x] exp(-2 pi i j m / B) -- the superposition of the
// monochromatic solutions, each with time dependence exp(-i omega_j t)
// (Eq. fov4 advances a forward wave by exp(+i k dz)) -- by a radix-2
// Stockham transform in shared memory.  A block handles `tx` consecutive x
// of one band.
template <typename C, typename R>
__global__ void omega_to_t_kernel(const C* __restrict__ in, C* __restrict__ out, int nb,
                                  int logb, int nx, int tx) {
  extern __shared__ __align__(16) unsigned char sm[];
  C* a = reinterpret_cast<C*>(sm);
  C* b = a + size_t(tx) * nb;
  const int band = blockIdx.y;
  const int x0 = blockIdx.x * tx;
  // load [nb][tx] -> a[xi][j]
  for (int c = threadIdx.x; c < nb * tx; c += blockDim.x) {
    const int j = c / tx, xi = c % tx;
    a[xi * nb + j] = in[(size_t(j) * 2 + band) * nx + x0 + xi];
  }
  __syncthreads();
  const int half = nb >> 1;
  for (int ns = 1; ns < nb; ns <<= 1) {
    for (int c = threadIdx.x; c < half * tx; c += blockDim.x) {
      const int xi = c / half, j = c % half;
      const int k = j % ns;
      const C u = a[xi * nb + j];
      C v = a[xi * nb + j + half];
      // w = exp(-i pi k / ns)
      R sw, cw;
      if constexpr (sizeof(R) == 8) sincospi(double(k) / double(ns), &sw, &cw);
      else sincospif(float(k) / float(ns), &sw, &cw);
      v = C{v.x * cw + v.y * sw, v.y * cw - v.x * sw};
      const int base = (j / ns) * ns * 2 + k;
      b[xi * nb + base] = C{u.x + v.x, u.y + v.y};
      b[xi * nb + base + ns] = C{u.x - v.x, u.y - v.y};
    }
    __syncthreads();
    C* t = a;
    a = b;
    b = t;
  }
  for (int c = threadIdx.x; c < nb * tx; c += blockDim.x) {
    const int xi = c / nb, m = c % nb;
    out[(size_t(band) * nx + x0 + xi) * nb + m] = a[xi * nb + m];
  }
}

// The coupling of Eq. fov10 alone, for a step of the coefficients (am1h,
// bh) of each row: psi_+ <- psi_+ + (a-1) psi_+ + b e psi_-, psi_- <- psi_- +
// (a-1) psi_- + b conj(e) psi_+ (old values on the right) inside the crystal
// (e != 0), e the slice of step n.  One thread per cell; split plans
// (nx >= 8192) store the slice per part: column x = P m + h at h (nx/P) + m
// (the column phasors of separable slices likewise).
__global__ void couple_only_kernel(const RowDescF32* __restrict__ rows, int nb, int nx, int n,
                                   int log_parts) {
  const int row = blockIdx.y;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= nb || x >= nx) return;
  const RowDescF32 d = rows[row];
  const int m_len = nx >> log_parts;
  const int h = x & ((1 << log_parts) - 1), m = x >> log_parts;
  const float2 am1 = d.am1h;
  float2 e, b0 = d.bh, b1 = d.bh;   // b e = b0 e, b conj(e) = b1 conj(e)
  if (d.srows) {
    // separable slices: e the column phasor inside [lo0, hi0), the row
    // phasor folded into b (b row, b conj(row)) as in the fused kernels
    const SepRow* r = d.srows + n;
    if (x < r->lo0 || x >= r->hi0) return;
    e = d.scols[size_t(h) * m_len + m];
    const float2 rp = r->ph, bb = d.bh;
    b0 = make_float2(fmaf(bb.x, rp.x, -(bb.y * rp.y)), fmaf(bb.x, rp.y, bb.y * rp.x));
    b1 = make_float2(fmaf(bb.x, rp.x, bb.y * rp.y), fmaf(bb.x, -rp.y, bb.y * rp.x));
  } else {
    e = d.phasor[size_t(n) * nx + size_t(h) * m_len + m];
  }
  if (e.x == 0.f && e.y == 0.f) return;
  const float2 p = d.state[x], q = d.state[nx + x];
  const float cx = fmaf(b0.x, e.x, -(b0.y * e.y)), cy = fmaf(b0.x, e.y, b0.y * e.x);   // b e
  const float dx = fmaf(b1.x, e.x, b1.y * e.y), dy = fmaf(b1.y, e.x, -(b1.x * e.y));   // b conj(e)
  float rx = fmaf(am1.x, p.x, p.x);
  rx = fmaf(-am1.y, p.y, rx);
  rx = fmaf(cx, q.x, rx);
  rx = fmaf(-cy, q.y, rx);
  float ry = fmaf(am1.x, p.y, p.y);
  ry = fmaf(am1.y, p.x, ry);
  ry = fmaf(cx, q.y, ry);
  ry = fmaf(cy, q.x, ry);
  float sx = fmaf(am1.x, q.x, q.x);
  sx = fmaf(-am1.y, q.y, sx);
  sx = fmaf(dx, p.x, sx);
  sx = fmaf(-dy, p.y, sx);
  float sy = fmaf(am1.x, q.y, q.y);
  sy = fmaf(am1.y, q.x, sy);
  sy = fmaf(dx, p.y, sy);
  sy = fmaf(dy, p.x, sy);
  d.state[x] = make_float2(rx, ry);
  d.state[nx + x] = make_float2(sx, sy);
}

}  // namespace

int launch_couple_only(const RowDescF32* d_rows, int nb, int nx, int n, cudaStream_t st) {
  int log_parts = 0;
  while ((4096 << log_parts) < nx) ++log_parts;   // parts of 4096 columns (nx >= 8192)
  if (nx < 8192) log_parts = 0;
  const int threads = 256;
  dim3 grid((nx + threads - 1) / threads, nb);
  couple_only_kernel<<<grid, threads, 0, st>>>(d_rows, nb, nx, n, log_parts);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BPM_OK : cuda_fail(e, "coupling launch");
}

int launch_convert_in(const double2* src, float2* dst, size_t n, cudaStream_t st) {
  const int threads = 256;
  size_t blocks = (n + threads - 1) / threads;
  if (blocks > 65536) blocks = 65536;
  convert_in_kernel<<<int(blocks), threads, 0, st>>>(src, dst, n);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BPM_OK : cuda_fail(e, "convert input");
}

int launch_finish_f32(const float2* state, double2* out_c128, float2* out_c64,
                      const double* g, int n_rows, int nx, int /*steps*/, double dx,
                      double* final_powers, int power_stride, cudaStream_t st) {
  finish_kernel<float2><<<2 * n_rows, 256, 0, st>>>(state, out_c128, out_c64,
                                                    reinterpret_cast<const double2*>(g), nx, dx,
                                                    final_powers, power_stride);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BPM_OK : cuda_fail(e, "finish (fp32)");
}

int launch_finish_f64(const double2* state, double2* out, const double* g, int n_rows, int nx,
                      int /*steps*/, double dx, double* final_powers, int power_stride,
                      cudaStream_t st) {
  finish_kernel<double2><<<2 * n_rows, 256, 0, st>>>(state, out, nullptr,
                                                     reinterpret_cast<const double2*>(g), nx, dx,
                                                     final_powers, power_stride);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BPM_OK : cuda_fail(e, "finish (fp64)");
}

int launch_omega_to_t(const void* d_in, void* d_out, int nb, int nx, int precision,
                      cudaStream_t st) {
  int logb = 0;
  while ((1 << logb) < nb) ++logb;
  const size_t csize = precision == BPM_FP32_FUSED ? 8 : 16;
  int tx = 1;
  while (tx < 16 && size_t(tx) * 2 * nb * 2 * csize <= 96 * 1024 && (nx % (tx * 2)) == 0) tx *= 2;
  const size_t smem = size_t(tx) * nb * 2 * csize;
  dim3 grid(nx / tx, 2);
  cudaError_t e;
  if (precision == BPM_FP32_FUSED) {
    auto k = omega_to_t_kernel<float2, float>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e == cudaSuccess) {
      k<<<grid, 256, smem, st>>>(static_cast<const float2*>(d_in), static_cast<float2*>(d_out),
                                 nb, logb, nx, tx);
      e = cudaGetLastError();
    }
  } else {
    auto k = omega_to_t_kernel<double2, double>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e == cudaSuccess) {
      k<<<grid, 256, smem, st>>>(static_cast<const double2*>(d_in), static_cast<double2*>(d_out),
                                 nb, logb, nx, tx);
      e = cudaGetLastError();
    }
  }
  return e == cudaSuccess ? BPM_OK : cuda_fail(e, "omega_to_t");
}

namespace {

// Host bytes carried to the device as a kernel parameter: a launch captured
// into a CUDA graph keeps its parameters, so the graph replays the data it
// was captured with (a captured copy from host memory would read that
// memory again at every replay).  3840 bytes keep a launch's parameters
// (chunk, pointer, count) within the 4 KB parameter space.
struct ParamChunk {
  unsigned char b[3840];
};

__global__ void param_copy_kernel(unsigned char* dst, ParamChunk c, int bytes) {
  for (int i = threadIdx.x; i < bytes; i += blockDim.x) dst[i] = c.b[i];
}

}  // namespace

int upload_by_params(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  const unsigned char* from = static_cast<const unsigned char*>(src);
  unsigned char* to = static_cast<unsigned char*>(dst);
  for (size_t off = 0; off < bytes; off += sizeof(ParamChunk)) {
    ParamChunk c;
    const size_t n = std::min(bytes - off, sizeof(ParamChunk));
    std::memcpy(c.b, from + off, n);
    param_copy_kernel<<<1, 256, 0, st>>>(to + off, c, int(n));
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BPM_OK : cuda_fail(e, "upload by kernel parameters");
}

}  // namespace bpm
