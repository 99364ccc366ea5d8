// Launchers and host loop of the 3D march (kernels in vol_kernel.cuh).
#include <atomic>
#include <string>

#include "fused_launch.cuh"
#include "vol_kernel.cuh"

namespace bpm {

namespace {

template <typename K>
int set_smem(K kernel, int bytes, std::atomic<bool>* done, const char* what) {
  if (done->load(std::memory_order_acquire)) return BPM_OK;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return cuda_fail(e, what);
  done->store(true, std::memory_order_release);
  return BPM_OK;
}

// (shared-memory attributes are set by prepare_kernels before any launch)
template <int LX, bool EX, bool HALF>
int row_launch(const VolParams& p, cudaStream_t st) {
  using C = VolRowCfg<LX>;
  vol_row_kernel<LX, EX, HALF><<<p.nb * p.ny, C::THREADS, C::SMEM, st>>>(p);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BPM_OK : cuda_fail(e, "vol row kernel");
}

template <int LY, bool EX>
int col_launch(const VolParams& p, cudaStream_t st) {
  using C = VolColCfg<LY>;
  vol_col_kernel<LY, EX><<<p.nb * 2 * (p.nx / C::COLS), C::THREADS, C::SMEM, st>>>(p);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BPM_OK : cuda_fail(e, "vol column kernel");
}

// Shared-memory attributes of the kernels a plan uses, set before any
// capture (the first launch would set them too, but not inside a capture).
template <bool EX>
int prepare_kernels(int lognx, int logny) {
  static std::atomic<bool> done[3][16] = {};   // callers' and server threads
  auto row = [&](auto kern, int bytes) { return set_smem(kern, bytes, &done[0][lognx], "vol row"); };
  auto rowh = [&](auto kern, int bytes) { return set_smem(kern, bytes, &done[2][lognx], "vol row"); };
  auto col = [&](auto kern, int bytes) { return set_smem(kern, bytes, &done[1][logny], "vol col"); };
  int rc = BPM_OK;
  switch (lognx) {
    case 8: rc = row(vol_row_kernel<8, EX>, VolRowCfg<8>::SMEM); break;
    case 9: rc = row(vol_row_kernel<9, EX>, VolRowCfg<9>::SMEM); break;
    case 10: rc = row(vol_row_kernel<10, EX>, VolRowCfg<10>::SMEM); break;
    case 11: rc = row(vol_row_kernel<11, EX>, VolRowCfg<11>::SMEM); break;
    case 12: rc = row(vol_row_kernel<12, EX>, VolRowCfg<12>::SMEM); break;
    default: return fail(BPM_ERR_INVALID, "3D: unsupported nx");
  }
  if (rc != BPM_OK) return rc;
  switch (lognx) {   // the second-order form of the row kernel
    case 8: rc = rowh(vol_row_kernel<8, EX, true>, VolRowCfg<8>::SMEM); break;
    case 9: rc = rowh(vol_row_kernel<9, EX, true>, VolRowCfg<9>::SMEM); break;
    case 10: rc = rowh(vol_row_kernel<10, EX, true>, VolRowCfg<10>::SMEM); break;
    case 11: rc = rowh(vol_row_kernel<11, EX, true>, VolRowCfg<11>::SMEM); break;
    default: rc = rowh(vol_row_kernel<12, EX, true>, VolRowCfg<12>::SMEM); break;
  }
  if (rc != BPM_OK) return rc;
  switch (logny) {
    case 8: return col(vol_col_kernel<8, EX>, VolColCfg<8>::SMEM);
    case 9: return col(vol_col_kernel<9, EX>, VolColCfg<9>::SMEM);
    case 10: return col(vol_col_kernel<10, EX>, VolColCfg<10>::SMEM);
    default: return fail(BPM_ERR_INVALID, "3D: unsupported ny");
  }
}

template <bool EX>
int row_dispatch(int lognx, const VolParams& p, cudaStream_t st, bool half) {
  if (half) {
    switch (lognx) {
      case 8: return row_launch<8, EX, true>(p, st);
      case 9: return row_launch<9, EX, true>(p, st);
      case 10: return row_launch<10, EX, true>(p, st);
      case 11: return row_launch<11, EX, true>(p, st);
      case 12: return row_launch<12, EX, true>(p, st);
      default: return fail(BPM_ERR_INVALID, "3D: unsupported nx");
    }
  }
  switch (lognx) {
    case 8: return row_launch<8, EX, false>(p, st);
    case 9: return row_launch<9, EX, false>(p, st);
    case 10: return row_launch<10, EX, false>(p, st);
    case 11: return row_launch<11, EX, false>(p, st);
    case 12: return row_launch<12, EX, false>(p, st);
    default: return fail(BPM_ERR_INVALID, "3D: unsupported nx");
  }
}

template <bool EX>
int col_dispatch(int logny, const VolParams& p, cudaStream_t st) {
  switch (logny) {
    case 8: return col_launch<8, EX>(p, st);
    case 9: return col_launch<9, EX>(p, st);
    case 10: return col_launch<10, EX>(p, st);
    default: return fail(BPM_ERR_INVALID, "3D: unsupported ny");
  }
}

// powers[r][slot][band] = dx dy * sum over lines y (in order) of the line sums
__global__ void vol_reduce_powers(const double* __restrict__ part, double* __restrict__ pw,
                                  int nb, int n_rec, int ny, int s0, int s1, double dxdy) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int nslot = s1 - s0;
  if (i >= nb * nslot * 2) return;
  const int band = i & 1, rs = i >> 1;
  const int r = rs / nslot, slot = s0 + rs % nslot;
  const double* src = part + ((size_t(r) * n_rec + slot) * 2 + band) * ny;
  double s = 0.0;
  for (int y = 0; y < ny; ++y) s += src[y];
  pw[(size_t(r) * (n_rec + 1) + slot) * 2 + band] = s * dxdy;
}

// A march captured as a CUDA graph (two launches per step) on a private
// stream and launched on the caller's; reused while the same call repeats.
struct VolGraph {
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  const void* state = nullptr;
  const void* rec = nullptr;
  const void* pw = nullptr;
  int n_begin = -1, n_end = -1;
  bool half = false;   // second-order splitting
};

}  // namespace

void vol_release(bpm_plan_s* plan) {
  auto* g = static_cast<VolGraph*>(plan->vol_graph);
  if (g) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->cap) cudaStreamDestroy(g->cap);
    delete g;
  }
  plan->vol_graph = nullptr;
}

int vol_march(bpm_plan_s* plan, float2* state, float2* d_rec, double* d_pw, int n_begin,
              int n_end, cudaStream_t st) {
  const int k = plan->record_every;
  const bool want = (d_rec || d_pw) && k > 0 && plan->n_rec > 0;
  if (want && d_pw) {
    const size_t bytes = size_t(plan->nb) * plan->n_rec * 2 * plan->ny * sizeof(double);
    if (plan->pwpart_bytes < bytes) {
      if (plan->d_pwpart) cudaFree(plan->d_pwpart);
      plan->d_pwpart = nullptr;
      plan->pwpart_bytes = 0;
      cudaError_t e = cudaMalloc(&plan->d_pwpart, bytes);
      if (e != cudaSuccess) {
        plan->d_pwpart = nullptr;
        cudaGetLastError();
        return fail(BPM_ERR_OOM, "3D line power buffer");
      }
      plan->pwpart_bytes = bytes;
    }
  }
  VolParams p{};
  p.org = state;
  p.spec = static_cast<float2*>(plan->d_spec);
  p.phasor = static_cast<const float2*>(plan->d_phasor);
  p.prop = static_cast<const float2*>(plan->d_prop);
  p.records = want ? d_rec : nullptr;
  p.pwpart = (want && d_pw) ? plan->d_pwpart : nullptr;
  p.twx = static_cast<const float4*>(plan->d_tw);
  p.twy = static_cast<const float4*>(plan->d_twy);
  p.coup = static_cast<const float2*>(plan->d_rows);
  p.gphase = reinterpret_cast<const double*>(static_cast<const float2*>(plan->d_rows) + 2 * plan->nb);
  p.coup_half = static_cast<const float2*>(plan->d_rows) + 3 * plan->nb;
  p.nb = plan->nb;
  p.nx = plan->nx;
  p.ny = plan->ny;
  p.n_phase0 = n_begin;
  p.record_every = want ? k : 0;
  p.n_rec = plan->n_rec;
  const bool ex = fused_exact_constants();
  cudaStream_t lst = st;   // the stream the kernels are enqueued on
  const bool half = plan->split == BPM_SPLIT_VERLET;
  auto row = [&]() {
    return ex ? row_dispatch<true>(plan->logn, p, lst, half)
              : row_dispatch<false>(plan->logn, p, lst, half);
  };
  auto col = [&]() { return ex ? col_dispatch<true>(plan->logny, p, lst) : col_dispatch<false>(plan->logny, p, lst); };
  auto enqueue = [&]() {
    p.mode = 0;
    p.n = n_begin;
    int r = row();
    for (int n = n_begin; n < n_end && r == BPM_OK; ++n) {
      p.n = n;
      r = col();
      if (r != BPM_OK) break;
      p.mode = (n + 1 == n_end) ? 2 : 1;
      r = row();
    }
    return r;
  };
  // Unless the caller's stream is itself being captured, the march runs as a
  // CUDA graph: captured on a private stream, launched on the caller's, and
  // re-captured only when the buffers or the step range change.
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    cs = cudaStreamCaptureStatusActive;
  }
  int rc = ex ? prepare_kernels<true>(plan->logn, plan->logny)
              : prepare_kernels<false>(plan->logn, plan->logny);
  if (rc != BPM_OK) return rc;
  if (cs != cudaStreamCaptureStatusNone) {
    rc = enqueue();
    if (rc != BPM_OK) return rc;
  } else {
    auto* g = static_cast<VolGraph*>(plan->vol_graph);
    if (!g) {
      g = new VolGraph();
      plan->vol_graph = g;
      cudaError_t e = cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking);
      if (e != cudaSuccess) {
        g->cap = nullptr;
        return cuda_fail(e, "3D capture stream");
      }
    }
    const bool hit = g->exec && g->state == state && g->rec == p.records && g->pw == p.pwpart &&
                     g->n_begin == n_begin && g->n_end == n_end && g->half == half;
    if (!hit) {
      cudaGraph_t graph = nullptr;
      lst = g->cap;
      cudaError_t e = cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_fail(e, "3D march capture");
      rc = enqueue();
      e = cudaStreamEndCapture(g->cap, &graph);
      lst = st;
      if (rc != BPM_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return rc != BPM_OK ? rc : cuda_fail(e, "3D march capture");
      }
      if (g->exec) cudaGraphExecDestroy(g->exec);
      g->exec = nullptr;
      e = cudaGraphInstantiate(&g->exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        g->exec = nullptr;
        return cuda_fail(e, "3D march graph instantiate");
      }
      g->state = state;
      g->rec = p.records;
      g->pw = p.pwpart;
      g->n_begin = n_begin;
      g->n_end = n_end;
      g->half = half;
    }
    cudaError_t e = cudaGraphLaunch(g->exec, st);
    if (e != cudaSuccess) return cuda_fail(e, "3D march graph launch");
  }
  if (p.pwpart) {
    const int s0 = n_begin / k, s1 = n_end / k;
    if (s1 > s0) {
      const int items = plan->nb * (s1 - s0) * 2;
      vol_reduce_powers<<<(items + 127) / 128, 128, 0, st>>>(
          plan->d_pwpart, d_pw, plan->nb, plan->n_rec, plan->ny, s0, s1,
          plan->dx_um * plan->dy_um);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(e, "3D power reduction");
    }
  }
  return BPM_OK;
}

}  // namespace bpm
