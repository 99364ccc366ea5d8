// Launcher template for the fused march (instantiated per transform size in
// separate translation units so they compile in parallel).
#pragma once

#include <atomic>
#include <cstdlib>

#include "fused_kernel.cuh"
#include "fused2_kernel.cuh"
#include "fused3_kernel.cuh"
#include "fused4_kernel.cuh"
#include "fused4t_kernel.cuh"
#include "fused4s_kernel.cuh"

namespace bpm {

// Butterfly-constant policy: hi+lo constants (default) unless BPM_FUSED_EXACT=0.
inline bool fused_exact_constants() {
  static std::atomic<int> cached{-1};
  int v = cached.load(std::memory_order_relaxed);
  if (v < 0) {
    const char* e = std::getenv("BPM_FUSED_EXACT");
    v = (e && e[0] == '0') ? 0 : 1;
    cached.store(v, std::memory_order_relaxed);
  }
  return v == 1;
}

// Both-bands-per-thread kernel (N <= 128); SCH the operator splitting.
template <int LOGN, int SCH = 0>
int fused_launch_impl(const RowDescF32* d_rows, int n_rows, int steps,
                      const float4* d_tw, int* d_status, cudaStream_t st) {
  using C = FusedCfg<LOGN, SCH != 0 ? 2 : 1>;
  static std::atomic<bool> configured{false};
  if (!configured.load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(fused_march_kernel<LOGN, SCH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         C::SMEM);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(fused)");
    configured.store(true, std::memory_order_release);
  }
  const int grid = (n_rows + C::ROWS - 1) / C::ROWS;
  fused_march_kernel<LOGN, SCH><<<grid, C::THREADS, C::SMEM, st>>>(d_rows, n_rows, steps,
                                                                   d_tw, d_status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "fused march launch");
  return BPM_OK;
}

// Band-per-thread kernel (256 <= N <= 4096); EX selects hi+lo butterfly
// constants, SCH the operator splitting (first order, Verlet, Forest-Ruth).
template <int LOGN, bool EX, int SCH = kSchFirst>
int fused2_launch_impl(const RowDescF32* d_rows, int n_rows, int steps, const float4* d_tw,
                       int* d_status, cudaStream_t st) {
  using C = F2Cfg<LOGN, SCH != kSchFirst ? 2 : 1>;
  static std::atomic<bool> configured{false};
  if (!configured.load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(fused2_march_kernel<LOGN, EX, SCH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(fused2)");
    configured.store(true, std::memory_order_release);
  }
  const int grid = (n_rows + C::ROWS - 1) / C::ROWS;
  fused2_march_kernel<LOGN, EX, SCH><<<grid, C::THREADS, C::SMEM, st>>>(d_rows, n_rows, steps,
                                                                       d_tw, d_status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "fused2 march launch");
  return BPM_OK;
}

// N = 4096 as a half-band split: one row per 4-CTA cluster, each CTA a
// 2048-point half of one band (fused4_kernel.cuh with M = 2048).
template <bool EX, bool HALF = false>
int fused4h_launch_impl(const RowDescF32* d_rows, int n_rows, int steps, const float4* d_tw,
                        int* d_status, cudaStream_t st) {
  constexpr int SCH = HALF ? kSchVerlet : kSchFirst;
  using C = F4ECfg<11, HALF ? 2 : 1>;
  static std::atomic<bool> configured{false};
  if (!configured.load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(fused4e_march_kernel<11, EX, SCH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(fused4h)");
    configured.store(true, std::memory_order_release);
  }
  fused4e_march_kernel<11, EX, SCH><<<4 * n_rows, C::T, C::SMEM, st>>>(d_rows, n_rows, steps,
                                                                       d_tw, d_status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "fused4h march launch");
  return BPM_OK;
}

// N = 4096 as a half-band split with 8 points per thread (fused4s_kernel.cuh);
// SCH the operator splitting.
template <bool EX, int SCH = kSchFirst>
int fused4s_launch_impl(const RowDescF32* d_rows, int n_rows, int steps, const float4* d_tw,
                        int* d_status, cudaStream_t st) {
  using C = F4SCfg<SCH != kSchFirst ? 2 : 1>;
  static std::atomic<bool> configured{false};
  if (!configured.load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(fused4s_march_kernel<EX, SCH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(fused4s)");
    configured.store(true, std::memory_order_release);
  }
  fused4s_march_kernel<EX, SCH><<<4 * n_rows, C::T, C::SMEM, st>>>(d_rows, n_rows, steps, d_tw,
                                                                   d_status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "fused4s march launch");
  return BPM_OK;
}

// Resident CTAs per SM of a kernel with its launch shape.
template <typename K>
int blocks_per_sm(K kernel, int threads, int smem) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n > 0 ? n : 1;
}

// Clusters of a kernel with compile-time cluster dimensions that the GPU
// keeps resident at once (cluster-occupancy query; 1 if it fails).
template <typename K>
int clusters_resident(K kernel, int cluster, int threads, int smem) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster * 64);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (void*)kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n > 0 ? n : 1;
}

// 2-CTA cluster kernel (one row per cluster, one band per CTA); SCH the
// operator splitting.
template <int LOGN, bool EX, int SCH = kSchFirst>
int fused3_launch_impl(const RowDescF32* d_rows, int n_rows, int steps, const float4* d_tw,
                       int* d_status, cudaStream_t st) {
  using C = F3Cfg<LOGN, SCH != kSchFirst ? 2 : 1>;
  static std::atomic<bool> configured{false};
  if (!configured.load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(fused3_march_kernel<LOGN, EX, SCH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(fused3)");
    configured.store(true, std::memory_order_release);
  }
  fused3_march_kernel<LOGN, EX, SCH><<<2 * n_rows, C::T, C::SMEM, st>>>(d_rows, n_rows, steps,
                                                                       d_tw, d_status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "fused3 march launch");
  return BPM_OK;
}

// Split-band cluster kernels for N = 4096 P (cluster of 2P CTAs per row):
// both run the one-exchange form (P = 4 with its tables in tensor memory).
// SCH: the operator splitting (Forest-Ruth: P = 2 only).
template <int P, bool EX, int SCH = kSchFirst>
int fused4_launch_impl(const RowDescF32* d_rows, int n_rows, int steps, const float4* d_tw,
                       int* d_status, cudaStream_t st) {
  static_assert(P == 2 || P == 4, "N = 8192 or 16384");
  static_assert(P == 2 || SCH != kSchForestRuth, "fourth-order split band: N = 8192");
  auto kern = [] {
    if constexpr (P == 2) return fused4e_march_kernel<12, EX, SCH>;
    else return fused4t_march_kernel<EX, SCH != kSchFirst>;
  }();
  constexpr int smem = P == 2 ? F4ECfg<12>::SMEM : F4TCfg::SMEM;
  constexpr int threads = P == 2 ? F4ECfg<12>::T : F4TCfg::T;
  static std::atomic<bool> configured{false};
  if (!configured.load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(fused4)");
    configured.store(true, std::memory_order_release);
  }
  kern<<<2 * P * n_rows, threads, smem, st>>>(d_rows, n_rows, steps, d_tw, d_status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "fused4 march launch");
  return BPM_OK;
}

}  // namespace bpm

#define BPM_INSTANTIATE_FUSED4(P, L)                                              \
  namespace bpm {                                                                 \
  int fused4_rows_resident_##L() {                                                \
    if constexpr (P == 2)                                                         \
      return clusters_resident(fused4e_march_kernel<12, true>, 4, F4ECfg<12>::T,  \
                               F4ECfg<12>::SMEM);                                 \
    else                                                                          \
      return clusters_resident(fused4t_march_kernel<true>, 8, F4TCfg::T,          \
                               F4TCfg::SMEM);                                     \
  }                                                                               \
  int fused4_launch_##L(const RowDescF32* r, int n, int s, const float4* tw,     \
                        int* status, cudaStream_t st) {                           \
    return fused_exact_constants()                                                \
               ? fused4_launch_impl<P, true>(r, n, s, tw, status, st)             \
               : fused4_launch_impl<P, false>(r, n, s, tw, status, st);           \
  }                                                                               \
  int fused4v_launch_##L(const RowDescF32* r, int n, int s, const float4* tw,    \
                         int* status, cudaStream_t st) {                          \
    return fused_exact_constants()                                                \
               ? fused4_launch_impl<P, true, kSchVerlet>(r, n, s, tw, status, st) \
               : fused4_launch_impl<P, false, kSchVerlet>(r, n, s, tw, status, st); \
  }                                                                               \
  }

// fourth-order (Forest-Ruth) form of the N = 8192 split band
#define BPM_INSTANTIATE_FUSED4F                                                   \
  namespace bpm {                                                                 \
  int fused4f_rows_resident_13() {                                                \
    return clusters_resident(fused4e_march_kernel<12, true, kSchForestRuth>, 4,  \
                             F4ECfg<12>::T, F4ECfg<12>::SMEM);                    \
  }                                                                               \
  int fused4f_launch_13(const RowDescF32* r, int n, int s, const float4* tw,     \
                        int* status, cudaStream_t st) {                           \
    return fused_exact_constants()                                                \
               ? fused4_launch_impl<2, true, kSchForestRuth>(r, n, s, tw, status, st) \
               : fused4_launch_impl<2, false, kSchForestRuth>(r, n, s, tw, status, st); \
  }                                                                               \
  }

#define BPM_INSTANTIATE_FUSED3(L)                                                 \
  namespace bpm {                                                                 \
  int fused3_rows_resident_##L() {                                                \
    return clusters_resident(fused3_march_kernel<L, true>, 2, F3Cfg<L>::T,        \
                             F3Cfg<L>::SMEM);                                     \
  }                                                                               \
  int fused3_launch_##L(const RowDescF32* r, int n, int s, const float4* tw,     \
                        int* status, cudaStream_t st) {                           \
    return fused_exact_constants()                                                \
               ? fused3_launch_impl<L, true>(r, n, s, tw, status, st)             \
               : fused3_launch_impl<L, false>(r, n, s, tw, status, st);           \
  }                                                                               \
  }

// second-order (Verlet) form of the 2-CTA cluster kernel
#define BPM_INSTANTIATE_FUSED3H(L)                                                \
  namespace bpm {                                                                 \
  int fused3h_rows_resident_##L() {                                               \
    return clusters_resident(fused3_march_kernel<L, true, kSchVerlet>, 2,         \
                             F3Cfg<L, 2>::T, F3Cfg<L, 2>::SMEM);                  \
  }                                                                               \
  int fused3h_launch_##L(const RowDescF32* r, int n, int s, const float4* tw,    \
                         int* status, cudaStream_t st) {                          \
    return fused_exact_constants()                                                \
               ? fused3_launch_impl<L, true, kSchVerlet>(r, n, s, tw, status, st) \
               : fused3_launch_impl<L, false, kSchVerlet>(r, n, s, tw, status, st); \
  }                                                                               \
  }

// fourth-order (Forest-Ruth) form of the 2-CTA cluster kernel
#define BPM_INSTANTIATE_FUSED3F(L)                                                \
  namespace bpm {                                                                 \
  int fused3f_rows_resident_##L() {                                               \
    return clusters_resident(fused3_march_kernel<L, true, kSchForestRuth>, 2,     \
                             F3Cfg<L, 2>::T, F3Cfg<L, 2>::SMEM);                  \
  }                                                                               \
  int fused3f_launch_##L(const RowDescF32* r, int n, int s, const float4* tw,    \
                         int* status, cudaStream_t st) {                          \
    return fused_exact_constants()                                                \
               ? fused3_launch_impl<L, true, kSchForestRuth>(r, n, s, tw, status, st) \
               : fused3_launch_impl<L, false, kSchForestRuth>(r, n, s, tw, status, st); \
  }                                                                               \
  }

#define BPM_INSTANTIATE_FUSED2(L)                                                 \
  namespace bpm {                                                                 \
  int fused2_rows_resident_##L() {                                                \
    using C = F2Cfg<L>;                                                           \
    return blocks_per_sm(fused2_march_kernel<L, true>, C::THREADS, C::SMEM) *     \
           C::ROWS;                                                               \
  }                                                                               \
  int fused2_launch_##L(const RowDescF32* r, int n, int s, const float4* tw,     \
                        int* status, cudaStream_t st) {                           \
    return fused_exact_constants()                                                \
               ? fused2_launch_impl<L, true>(r, n, s, tw, status, st)             \
               : fused2_launch_impl<L, false>(r, n, s, tw, status, st);           \
  }                                                                               \
  int fused2h_rows_resident_##L() {                                               \
    using C = F2Cfg<L, 2>;                                                        \
    return blocks_per_sm(fused2_march_kernel<L, true, kSchVerlet>, C::THREADS,    \
                         C::SMEM) * C::ROWS;                                      \
  }                                                                               \
  int fused2h_launch_##L(const RowDescF32* r, int n, int s, const float4* tw,    \
                         int* status, cudaStream_t st) {                          \
    return fused_exact_constants()                                                \
               ? fused2_launch_impl<L, true, kSchVerlet>(r, n, s, tw, status, st) \
               : fused2_launch_impl<L, false, kSchVerlet>(r, n, s, tw, status, st); \
  }                                                                               \
  int fused2f_rows_resident_##L() {                                               \
    using C = F2Cfg<L, 2>;                                                        \
    return blocks_per_sm(fused2_march_kernel<L, true, kSchForestRuth>, C::THREADS, \
                         C::SMEM) * C::ROWS;                                      \
  }                                                                               \
  int fused2f_launch_##L(const RowDescF32* r, int n, int s, const float4* tw,    \
                         int* status, cudaStream_t st) {                          \
    return fused_exact_constants()                                                \
               ? fused2_launch_impl<L, true, kSchForestRuth>(r, n, s, tw, status, st) \
               : fused2_launch_impl<L, false, kSchForestRuth>(r, n, s, tw, status, st); \
  }                                                                               \
  }

#define BPM_INSTANTIATE_FUSED(L)                                                  \
  namespace bpm {                                                                 \
  int fused_rows_resident_##L() {                                                 \
    using C = FusedCfg<L>;                                                        \
    return blocks_per_sm(fused_march_kernel<L>, C::THREADS, C::SMEM) * C::ROWS;   \
  }                                                                               \
  int fused_launch_##L(const RowDescF32* r, int n, int s, const float4* tw,      \
                       int* status, cudaStream_t st) {                            \
    return fused_launch_impl<L>(r, n, s, tw, status, st);                         \
  }                                                                               \
  int fusedh_rows_resident_##L() {                                                \
    using C = FusedCfg<L, 2>;                                                     \
    return blocks_per_sm(fused_march_kernel<L, 1>, C::THREADS, C::SMEM) * C::ROWS; \
  }                                                                               \
  int fusedh_launch_##L(const RowDescF32* r, int n, int s, const float4* tw,     \
                        int* status, cudaStream_t st) {                           \
    return fused_launch_impl<L, 1>(r, n, s, tw, status, st);                      \
  }                                                                               \
  int fusedf_rows_resident_##L() {                                                \
    using C = FusedCfg<L, 2>;                                                     \
    return blocks_per_sm(fused_march_kernel<L, 2>, C::THREADS, C::SMEM) * C::ROWS; \
  }                                                                               \
  int fusedf_launch_##L(const RowDescF32* r, int n, int s, const float4* tw,     \
                        int* status, cudaStream_t st) {                           \
    return fused_launch_impl<L, 2>(r, n, s, tw, status, st);                      \
  }                                                                               \
  }

#define BPM_INSTANTIATE_FUSED4H                                                   \
  namespace bpm {                                                                 \
  int fused4h_launch_12(const RowDescF32* r, int n, int s, const float4* tw,     \
                        int* status, cudaStream_t st) {                           \
    return fused_exact_constants()                                                \
               ? fused4h_launch_impl<true>(r, n, s, tw, status, st)               \
               : fused4h_launch_impl<false>(r, n, s, tw, status, st);             \
  }                                                                               \
  }

// second-order (Verlet) form of the N = 4096 half-band split
#define BPM_INSTANTIATE_FUSED4HH                                                  \
  namespace bpm {                                                                 \
  int fused4hh_rows_resident_12() {                                               \
    return clusters_resident(fused4e_march_kernel<11, true, kSchVerlet>, 4,       \
                             F4ECfg<11, 2>::T, F4ECfg<11, 2>::SMEM);              \
  }                                                                               \
  int fused4hh_launch_12(const RowDescF32* r, int n, int s, const float4* tw,    \
                         int* status, cudaStream_t st) {                          \
    return fused_exact_constants()                                                \
               ? fused4h_launch_impl<true, true>(r, n, s, tw, status, st)         \
               : fused4h_launch_impl<false, true>(r, n, s, tw, status, st);       \
  }                                                                               \
  }

// 8-points-per-thread form of the N = 4096 half-band split
#define BPM_INSTANTIATE_FUSED4S                                                   \
  namespace bpm {                                                                 \
  int fused4s_rows_resident_12() {                                                \
    return clusters_resident(fused4s_march_kernel<true>, 4, F4SCfg<1>::T,         \
                             F4SCfg<1>::SMEM);                                    \
  }                                                                               \
  int fused4s_launch_12(const RowDescF32* r, int n, int s, const float4* tw,     \
                        int* status, cudaStream_t st) {                           \
    return fused_exact_constants()                                                \
               ? fused4s_launch_impl<true>(r, n, s, tw, status, st)               \
               : fused4s_launch_impl<false>(r, n, s, tw, status, st);             \
  }                                                                               \
  int fused4sh_rows_resident_12() {                                               \
    return clusters_resident(fused4s_march_kernel<true, kSchVerlet>, 4,           \
                             F4SCfg<2>::T, F4SCfg<2>::SMEM);                      \
  }                                                                               \
  int fused4sh_launch_12(const RowDescF32* r, int n, int s, const float4* tw,    \
                         int* status, cudaStream_t st) {                          \
    return fused_exact_constants()                                                \
               ? fused4s_launch_impl<true, kSchVerlet>(r, n, s, tw, status, st)   \
               : fused4s_launch_impl<false, kSchVerlet>(r, n, s, tw, status, st); \
  }                                                                               \
  int fused4sf_rows_resident_12() {                                               \
    return clusters_resident(fused4s_march_kernel<true, kSchForestRuth>, 4,       \
                             F4SCfg<2>::T, F4SCfg<2>::SMEM);                      \
  }                                                                               \
  int fused4sf_launch_12(const RowDescF32* r, int n, int s, const float4* tw,    \
                         int* status, cudaStream_t st) {                          \
    return fused_exact_constants()                                                \
               ? fused4s_launch_impl<true, kSchForestRuth>(r, n, s, tw, status, st) \
               : fused4s_launch_impl<false, kSchForestRuth>(r, n, s, tw, status, st); \
  }                                                                               \
  }
