// Launcher template for the fused march (instantiated per transform size in
// separate translation units so they compile in parallel).
#pragma once

#include "fused_kernel.cuh"

namespace bpm {

template <int LOGN>
int fused_launch_impl(const RowDescF32* d_rows, int n_rows, int steps,
                      const float4* d_tw, int* d_status, cudaStream_t st) {
  using C = FusedCfg<LOGN>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(fused_march_kernel<LOGN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         C::SMEM);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(fused)");
    configured = true;
  }
  const int grid = (n_rows + C::ROWS - 1) / C::ROWS;
  fused_march_kernel<LOGN><<<grid, C::THREADS, C::SMEM, st>>>(d_rows, n_rows, steps,
                                                              d_tw, d_status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "fused march launch");
  return BPM_OK;
}

}  // namespace bpm

#define BPM_INSTANTIATE_FUSED(L)                                                  \
  namespace bpm {                                                                 \
  int fused_launch_##L(const RowDescF32* r, int n, int s, const float4* tw,      \
                       int* status, cudaStream_t st) {                            \
    return fused_launch_impl<L>(r, n, s, tw, status, st);                         \
  }                                                                               \
  }
