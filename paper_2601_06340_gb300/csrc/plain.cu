// Plain per-step FP64 march: the same step as the fused path (Eq. fov10 of
// arXiv 2601.06340), written the straightforward way with complex128 fields
// in global memory and one kernel launch per FFT pass and per pointwise
// operation:
//   forward Stockham passes (radix 4, plus one radix-2 pass for odd log2 N)
//   -> propagator multiply P(q)/N (natural order) -> inverse passes
//   -> real-space coupling with the strain phasor and mask -> [record].
// It is the FP64 reference form on the GPU and the baseline the fused FP32
// kernel is measured against.
#include <mutex>
#include <string>
#include <vector>

#include "bpm_internal.h"

namespace bpm {

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double2 csub(double2 a, double2 b) {
  return make_double2(a.x - b.x, a.y - b.y);
}

// One Stockham autosort pass of radix R over `lines` independent transforms
// of length n: sub-transforms of length ns are combined into length ns*R.
template <int R, bool INV>
__global__ void stockham_pass(const double2* __restrict__ in, double2* __restrict__ out,
                              int n, int ns, int lines, const double2* __restrict__ tw) {
  const int per_line = n / R;
  const long total = long(lines) * per_line;
  for (long g = blockIdx.x * long(blockDim.x) + threadIdx.x; g < total;
       g += long(gridDim.x) * blockDim.x) {
    const int line = int(g / per_line), j = int(g % per_line);
    const double2* src = in + size_t(line) * n;
    double2* dst = out + size_t(line) * n;
    const int k = j % ns;
    double2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[j + r * per_line];
    // twiddle W_{ns R}^{r k} = table[r k n / (ns R)]
    const int step = n / (ns * R);
#pragma unroll
    for (int r = 1; r < R; ++r) {
      double2 w = tw[r * k * step];
      if (INV) w.y = -w.y;
      v[r] = cmul(v[r], w);
    }
    if (R == 2) {
      double2 a = v[0], b = v[1];
      v[0] = cadd(a, b);
      v[1] = csub(a, b);
    } else {
      double2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
      double2 t2 = cadd(v[1], v[3]), t3 = csub(v[1], v[3]);
      t3 = INV ? make_double2(-t3.y, t3.x) : make_double2(t3.y, -t3.x);
      v[0] = cadd(t0, t2);
      v[2] = csub(t0, t2);
      v[1] = cadd(t1, t3);
      v[3] = csub(t1, t3);
    }
    const int base = (j / ns) * ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[base + r * ns] = v[r];
  }
}

// x[row][band][m] *= P_band(q_m) / N
__global__ void prop_kernel(double2* __restrict__ x, const RowDescF64* __restrict__ rows,
                            int n, int nb) {
  const long total = long(nb) * 2 * n;
  for (long c = blockIdx.x * long(blockDim.x) + threadIdx.x; c < total;
       c += long(gridDim.x) * blockDim.x) {
    const int row = int(c / (2 * n));
    const int rem = int(c % (2 * n));   // band * n + m
    x[c] = cmul(x[c], rows[row].prop[rem]);
  }
}

// Coupling of Eq. fov10 inside the crystal (phasor != 0).
__global__ void couple_kernel(double2* __restrict__ x, const RowDescF64* __restrict__ rows,
                              const double2* __restrict__ phasor_row, int n, int nb) {
  const long total = long(nb) * n;
  for (long c = blockIdx.x * long(blockDim.x) + threadIdx.x; c < total;
       c += long(gridDim.x) * blockDim.x) {
    const int row = int(c / n), j = int(c % n);
    const double2 e = phasor_row[j];
    if (e.x == 0.0 && e.y == 0.0) continue;
    double2* xr = x + size_t(row) * 2 * n;
    const double2 p = xr[j], m = xr[n + j];
    const double2 a = rows[row].a, b = rows[row].b;
    const double2 be = cmul(b, e), bc = cmul(b, make_double2(e.x, -e.y));
    xr[j] = cadd(cmul(a, p), cmul(be, m));
    xr[n + j] = cadd(cmul(a, m), cmul(bc, p));
  }
}

// Block-wide FP64 sum of |x|^2 over one (row, band) line, fixed order.
__device__ double line_power(const double2* x, int n) {
  __shared__ double part[32];
  double s = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) s += x[j].x * x[j].x + x[j].y * x[j].y;
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < int(blockDim.x >> 5); ++w) tot += part[w];
  }
  __syncthreads();
  return tot;
}

// Record slot `slot`: records[row][slot][band][:] = x * g^k, powers.
__global__ void record_kernel(const double2* __restrict__ x, double2* __restrict__ rec,
                              double* __restrict__ pw, const double2* __restrict__ gk,
                              int n, int n_rec, int slot, double dx) {
  const int row = blockIdx.x >> 1, band = blockIdx.x & 1;
  const double2* src = x + (size_t(row) * 2 + band) * n;
  const double2 g = gk[row];
  if (rec) {
    double2* dst = rec + ((size_t(row) * n_rec + slot) * 2 + band) * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) dst[j] = cmul(src[j], g);
  }
  if (pw) {
    double tot = line_power(src, n);
    if (threadIdx.x == 0) pw[(size_t(row) * (n_rec + 1) + slot) * 2 + band] = tot * dx;
  }
}

int grid_for(long work, int threads) {
  long b = (work + threads - 1) / threads;
  return int(b < 32768 ? (b > 0 ? b : 1) : 32768);
}

}  // namespace

// x: current buffer (state), y: scratch; returns the buffer holding the result.
static double2* fft_lines(double2* x, double2* y, int logn, int lines, const double2* tw,
                          bool inv, cudaStream_t st) {
  const int n = 1 << logn;
  int ns = 1;
  const int threads = 256;
  if (logn & 1) {
    const int g = grid_for(long(lines) * n / 2, threads);
    if (inv) stockham_pass<2, true><<<g, threads, 0, st>>>(x, y, n, ns, lines, tw);
    else stockham_pass<2, false><<<g, threads, 0, st>>>(x, y, n, ns, lines, tw);
    std::swap(x, y);
    ns *= 2;
  }
  while (ns < n) {
    const int g = grid_for(long(lines) * n / 4, threads);
    if (inv) stockham_pass<4, true><<<g, threads, 0, st>>>(x, y, n, ns, lines, tw);
    else stockham_pass<4, false><<<g, threads, 0, st>>>(x, y, n, ns, lines, tw);
    std::swap(x, y);
    ns *= 4;
  }
  return x;
}

// March the plan's state (d_state, c128 [B][2][N]) from n_begin to n_end.
// d_records: c128 [B][n_rec][2][N] or null; d_powers: [B][n_rec+1][2] or null.
// Records carry the common phase g^k with k = steps since n_phase0 (the step
// at which the state had phase 0);
// the returned state in d_state is raw (caller applies g^(n_end-n_begin)).
int plain_march(bpm_plan_s* plan, int n_begin, int n_end, int n_phase0, void* d_records,
                double* d_powers, cudaStream_t st) {
  const int n = plan->nx, nb = plan->nb, logn = plan->logn;
  const int lines = 2 * nb;
  const double2* tw = static_cast<const double2*>(plan->d_tw);
  const RowDescF64* rows = static_cast<const RowDescF64*>(plan->d_rows);
  double2* x = static_cast<double2*>(plan->d_state);
  double2* y = static_cast<double2*>(plan->d_state2);
  const double2* phasor = static_cast<const double2*>(plan->d_phasor);
  const int threads = 256;

  // Per-record common phases g^k (host FP64, uploaded once per record slot).
  std::vector<double2> gk(nb);
  double2* d_gk = nullptr;
  const bool any_rec = plan->record_every > 0 && (d_records || d_powers);
  if (any_rec) {
    cudaError_t e = cudaMallocAsync(&d_gk, sizeof(double2) * nb * 2, st);
    if (e != cudaSuccess) return cuda_fail(e, "plain march: phase buffer");
  }
  int slot_toggle = 0;
  // stages of one step: (propagates?, descriptors); first order = one stage
  std::vector<std::pair<bool, const RowDescF64*>> stages;
  if (plan->split == BPM_SPLIT_FIRST_ORDER || plan->n_stages == 0) {
    stages.push_back({true, rows});
  } else {
    const RowDescF64* sr = static_cast<const RowDescF64*>(plan->d_stage_rows);
    for (int i = 0; i < plan->n_stages; ++i)
      stages.push_back({plan->stage_has_prop[i] != 0, sr + size_t(i) * nb});
  }
  for (int s = n_begin; s < n_end; ++s) {
    for (const auto& stage : stages) {
      if (stage.first) {
        double2* r = fft_lines(x, y, logn, lines, tw, false, st);
        if (r != x) std::swap(x, y);
        prop_kernel<<<grid_for(long(lines) * n, threads), threads, 0, st>>>(x, stage.second, n, nb);
        r = fft_lines(x, y, logn, lines, tw, true, st);
        if (r != x) std::swap(x, y);
      }
      couple_kernel<<<grid_for(long(nb) * n, threads), threads, 0, st>>>(
          x, stage.second, phasor + size_t(s) * n, n, nb);
    }
    if (any_rec && (s + 1) % plan->record_every == 0) {
      const int slot = (s + 1) / plan->record_every - 1;
      for (int row = 0; row < nb; ++row) {
        double ang = std::fmod(double(s + 1 - n_phase0) * plan->ec[row].gphase, kTwoPi);
        gk[row] = make_double2(std::cos(ang), std::sin(ang));
      }
      double2* dg = d_gk + slot_toggle * nb;   // two halves so the async copy never races a reader
      slot_toggle ^= 1;
      cudaMemcpyAsync(dg, gk.data(), sizeof(double2) * nb, cudaMemcpyHostToDevice, st);
      record_kernel<<<2 * nb, 256, 0, st>>>(x, static_cast<double2*>(d_records), d_powers, dg,
                                            n, plan->n_rec, slot, plan->dx_um);
    }
  }
  cudaError_t e = cudaGetLastError();
  if (d_gk) cudaFreeAsync(d_gk, st);
  if (e != cudaSuccess) return cuda_fail(e, "plain march launch");
  if (x != static_cast<double2*>(plan->d_state)) {
    // the result ended in the scratch buffer: swap ownership
    std::swap(plan->d_state, plan->d_state2);
  }
  return BPM_OK;
}

}  // namespace bpm

// ---------------------------------------------------------------------------
// Allocation-free variant of the plain FP64 march.
//
// For callers that cannot allocate device memory (for example code that runs
// where cudaMalloc is not allowed, such as inside a host callback, under an
// allocator that must not grow, or in a process whose device memory is owned
// by someone else): it marches caller-owned buffers and keeps its own working
// memory -- the Stockham ping-pong buffer, the twiddle table and the row
// descriptors -- in the file-scope device arrays below, which every GPU that
// loads this library holds until the process exits.  Limits: at most
// kNoAllocMaxRows rows and n_rows * 2 * nx <= kNoAllocMaxComplex complex
// values (16 MiB of scratch).  All calls share these arrays, so calls that
// overlap on the GPU (on different streams or from different threads) race;
// each call rewrites the twiddles and descriptors it reads before using them,
// and the ping-pong buffer needs no clearing because every pass overwrites
// what it later reads.
namespace bpm {
namespace {

constexpr size_t kNoAllocMaxComplex = size_t(1) << 20;
constexpr int kNoAllocMaxRows = 1024;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double2 g_noalloc_scratch[kNoAllocMaxComplex];
constexpr int kNoAllocMaxLogN = 13;
static __device__ __align__(256) double2 g_noalloc_twiddles[1 << kNoAllocMaxLogN];
static __device__ __align__(256) RowDescF64 g_noalloc_rows[kNoAllocMaxRows];

struct NoAllocSymbols {
  bool ready = false;
  double2* scratch = nullptr;
  double2* twiddles = nullptr;
  RowDescF64* rows = nullptr;
};
std::mutex g_noalloc_mu;
NoAllocSymbols g_noalloc_sym[kNoAllocMaxDevices];

// W_n^m = exp(-2 pi i m / n), exact on the axes.
__global__ void noalloc_twiddle_kernel(double2* tw, int n) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * double(m) / double(n), &s, &c);
    if ((4 * m) % n == 0) {
      const int q = ((4 * m) / n) & 3;
      c = (q == 0) ? 1.0 : (q == 2) ? -1.0 : 0.0;
      s = (q == 1) ? 1.0 : (q == 3) ? -1.0 : 0.0;
    }
    tw[m] = make_double2(c, -s);
  }
}

__global__ void noalloc_rows_kernel(RowDescF64* rows, const double2* prop, const double2* ab,
                                    int nx, int n_rows) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n_rows; r += gridDim.x * blockDim.x) {
    rows[r].prop = prop + size_t(r) * 2 * nx;
    rows[r].a = ab[2 * r];
    rows[r].b = ab[2 * r + 1];
    rows[r].gphase = 0.0;
  }
}

}  // namespace

}  // namespace bpm

extern "C" int bpm_march_f64_noalloc(void* d_psi, int32_t nx, int32_t n_rows,
                                     const void* d_prop, const void* d_coupling,
                                     const void* d_phasor, int32_t n_begin, int32_t n_end,
                                     void* stream) {
  using namespace bpm;
  if (!d_psi || !d_prop || !d_coupling || !d_phasor)
    return fail(BPM_ERR_INVALID, "noalloc march: a buffer is NULL");
  if (nx < 8 || nx > (1 << kNoAllocMaxLogN) || (nx & (nx - 1)))
    return fail(BPM_ERR_INVALID, "noalloc march: nx must be a power of two in [8, " +
                                     std::to_string(1 << kNoAllocMaxLogN) + "]");
  if (n_rows < 1 || n_rows > kNoAllocMaxRows)
    return fail(BPM_ERR_INVALID, "noalloc march: n_rows must be in [1, " +
                                     std::to_string(kNoAllocMaxRows) + "]");
  if (size_t(n_rows) * 2 * size_t(nx) > kNoAllocMaxComplex)
    return fail(BPM_ERR_INVALID, "noalloc march: n_rows * 2 * nx exceeds the " +
                                     std::to_string(kNoAllocMaxComplex) +
                                     " complex values of static scratch");
  if (n_begin < 0 || n_end <= n_begin)
    return fail(BPM_ERR_INVALID, "noalloc march: need 0 <= n_begin < n_end");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "noalloc march: no device");
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    return fail(BPM_ERR_INVALID, "noalloc march: device index out of range");
  NoAllocSymbols sym;
  {
    // Once per device, with that device current: device addresses of the
    // static arrays (their host-side names are not device addresses).
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoAllocSymbols& s = g_noalloc_sym[dev];
    if (!s.ready) {
      e = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.scratch), g_noalloc_scratch);
      if (e == cudaSuccess)
        e = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.twiddles), g_noalloc_twiddles);
      if (e == cudaSuccess)
        e = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.rows), g_noalloc_rows);
      if (e != cudaSuccess) return cuda_fail(e, "noalloc march: cudaGetSymbolAddress");
      s.ready = true;
    }
    sym = s;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int logn = 0;
  while ((1 << logn) < nx) ++logn;
  const int lines = 2 * n_rows;
  // An error left pending by earlier, unrelated work is not this call's:
  // clear it so the checks below see only this call's launches.
  cudaGetLastError();
  noalloc_twiddle_kernel<<<(nx + 255) / 256, 256, 0, st>>>(sym.twiddles, nx);
  noalloc_rows_kernel<<<(n_rows + 127) / 128, 128, 0, st>>>(
      sym.rows, static_cast<const double2*>(d_prop), static_cast<const double2*>(d_coupling), nx,
      n_rows);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "noalloc march: table set-up launch");
  double2* user = static_cast<double2*>(d_psi);
  double2* x = user;
  double2* y = sym.scratch;
  const double2* phasor = static_cast<const double2*>(d_phasor);
  const int threads = 256;
  for (int s = n_begin; s < n_end; ++s) {
    double2* r = fft_lines(x, y, logn, lines, sym.twiddles, false, st);
    if (r != x) std::swap(x, y);
    prop_kernel<<<grid_for(long(lines) * nx, threads), threads, 0, st>>>(x, sym.rows, nx, n_rows);
    r = fft_lines(x, y, logn, lines, sym.twiddles, true, st);
    if (r != x) std::swap(x, y);
    couple_kernel<<<grid_for(long(n_rows) * nx, threads), threads, 0, st>>>(
        x, sym.rows, phasor + size_t(s) * nx, nx, n_rows);
  }
  if (x != user)
    e = cudaMemcpyAsync(user, x, size_t(lines) * nx * sizeof(double2), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "noalloc march");
  return BPM_OK;
}
