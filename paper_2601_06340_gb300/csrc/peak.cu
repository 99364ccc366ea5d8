// Measured arithmetic peak of the device (bpm_fp_peak): the denominator of
// the march kernels' roofline fractions.
//
// Every thread runs eight independent multiply-add chains (x <- x * b + c)
// for `iters` x 16 rounds; the grid fills every SM (eight 256-thread CTAs per
// SM), so the FMA pipes, not latency, set the rate.  Kinds: FP32 FFMA, FP32
// packed FFMA2 (two lanes per instruction) and FP64 DFMA.  One FMA counts as
// two flops.  The chains' sum is stored only when it equals a value it cannot
// reach, which keeps the compiler from removing them.
#include "bpm_internal.h"

namespace bpm {

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;
constexpr int kCtasPerSm = 8;

__global__ void __launch_bounds__(kThreads) ffma_peak_kernel(float* sink, int iters, float seed) {
  float x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = seed + float(threadIdx.x + i);
  const float b = 0.99999994f, c = 1.0e-7f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], b, c);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == -1.0f) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) ffma2_peak_kernel(float* sink, int iters, float seed) {
  float2 x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i)
    x[i] = make_float2(seed + float(threadIdx.x + i), seed - float(threadIdx.x + i));
  const float2 b = make_float2(0.99999994f, 0.99999994f), c = make_float2(1.0e-7f, 1.0e-7f);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) x[i] = __ffma2_rn(x[i], b, c);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i].x + x[i].y;
  if (s == -1.0f) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) dfma_peak_kernel(double* sink, int iters, double seed) {
  double x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = seed + double(threadIdx.x + i);
  const double b = 0.9999999999999999, c = 1.0e-15;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], b, c);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == -1.0) sink[blockIdx.x] = s;
}

}  // namespace

}  // namespace bpm

extern "C" int bpm_fp_peak(int32_t kind, int32_t iters, double* flops_per_s, double* seconds) {
  using namespace bpm;
  if (!flops_per_s || !seconds) return fail(BPM_ERR_INVALID, "flops_per_s / seconds is NULL");
  if (kind < BPM_PEAK_FP64_DFMA || kind > BPM_PEAK_FP32_FFMA2)
    return fail(BPM_ERR_INVALID, "kind must be BPM_PEAK_FP64_DFMA, _FP32_FFMA or _FP32_FFMA2");
  if (iters < 1 || iters > (1 << 22)) return fail(BPM_ERR_INVALID, "iters must be in [1, 2^22]");
  *flops_per_s = 0.0;
  *seconds = 0.0;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess || sms <= 0) return cuda_fail(e, "fp peak: device attributes");
  const int ctas = sms * kCtasPerSm;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  void* sink = nullptr;
  e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaMalloc(&sink, size_t(ctas) * sizeof(double));
  auto launch = [&](int n) {
    if (kind == BPM_PEAK_FP32_FFMA)
      ffma_peak_kernel<<<ctas, kThreads, 0, st>>>(static_cast<float*>(sink), n, 1.0f);
    else if (kind == BPM_PEAK_FP32_FFMA2)
      ffma2_peak_kernel<<<ctas, kThreads, 0, st>>>(static_cast<float*>(sink), n, 1.0f);
    else
      dfma_peak_kernel<<<ctas, kThreads, 0, st>>>(static_cast<double*>(sink), n, 1.0);
    return cudaGetLastError();
  };
  // a short warm-up launch, then the timed one
  if (e == cudaSuccess) e = launch(iters / 8 > 0 ? iters / 8 : 1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) e = launch(iters);
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (sink) cudaFree(sink);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (e != cudaSuccess) return cuda_fail(e, "fp peak kernel");
  const double lanes = kind == BPM_PEAK_FP32_FFMA2 ? 2.0 : 1.0;
  const double flops = 2.0 * lanes * double(kChains) * kUnroll * double(iters) *
                       double(ctas) * kThreads;
  *seconds = double(ms) * 1e-3;
  *flops_per_s = *seconds > 0 ? flops / *seconds : 0.0;
  return BPM_OK;
}
