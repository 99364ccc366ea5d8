// Self-test of the bounded device wait (bpm_selftest_wait_expiry).
//
// Every march kernel waits on mbarriers (strain-slice bulk copies, peer data)
// through mbar_wait, which gives up after a fixed number of try_wait polls.
// This kernel arms a barrier for 16 bytes that no copy will deliver, so the
// wait runs to its limit without any fault; the kernel then sets the status
// bit the march kernels set and returns.  Nothing asynchronous is issued, so
// nothing is in flight when the CTA exits.
#include "bpm_internal.h"
#include "fused_kernel.cuh"

namespace bpm {

namespace {

__global__ void wait_expiry_kernel(int* status, unsigned long long* cycles) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0)
    asm volatile(
        "{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(
            smem_u32(&bar)),
        "r"(16u)
        : "memory");
  __syncthreads();
  const long long t0 = clock64();
  const bool ok = mbar_wait(&bar, 0u);
  const long long t1 = clock64();
  if (!ok) atomicOr(status, kStatusWaitTimeout);
  if (threadIdx.x == 0) *cycles = static_cast<unsigned long long>(t1 - t0);
}

}  // namespace

}  // namespace bpm

extern "C" int bpm_selftest_wait_expiry(int32_t* status, double* seconds) {
  using namespace bpm;
  if (!status || !seconds) return fail(BPM_ERR_INVALID, "status / seconds is NULL");
  *status = 0;
  *seconds = 0.0;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int* d_status = nullptr;
  unsigned long long* d_cycles = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaMalloc(&d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&d_cycles, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) {
    wait_expiry_kernel<<<1, 32, 0, st>>>(d_status, d_cycles);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  int h_status = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&h_status, d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (d_status) cudaFree(d_status);
  if (d_cycles) cudaFree(d_cycles);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (e != cudaSuccess) return cuda_fail(e, "wait-expiry self-test");
  *status = h_status;
  *seconds = double(ms) * 1e-3;
  return BPM_OK;
}
