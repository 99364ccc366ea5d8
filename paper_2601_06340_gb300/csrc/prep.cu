// Slice preparation: the crystal mask Pi(x_j, z_n) and the strain phasor
// exp(i h u_x(x_j, z_n)) for every cell, computed once per set_crystal /
// set_strain on the device -- the phase h u_x and its reduction modulo 2 pi
// in FP64, the unit phasor in the precision it is stored in -- as c64
// (fused path) or c128 (plain path), with (0, 0) marking cells outside the
// crystal.
//
// Mask decisions (slab faces, polygon edges) use the IEEE operations
// __dadd_rn / __dmul_rn / __ddiv_rn explicitly so that no multiply-add is
// contracted and the result is the one the documented formula gives in
// FP64: x_j = x0 + j*dx, z_n = n*dz, depth = nx*(x - xs) + nz*(z - zs),
// crossing = (x2 - x1)*(z - z1)/(z2 - z1) + x1.
#include <cmath>
#include <string>
#include <vector>

#include "bpm_internal.h"

namespace bpm {

namespace {

struct PrepParams {
  int nx, nz;
  double x0, dx, dz;
  int crystal_kind;
  double ncx, ncz, thick, sx, sz;
  const uint8_t* mask;
  const double* poly;
  int nv;
  int strain_kind;
  const double* ux;
  double p0, p1, p2, p3;
  double h;
  float2* out32;
  double2* out64;
  int parts;     // > 1: out32 row layout [parts][nx/parts], column j at (j % parts, j / parts)
};

__device__ bool inside_cell(const PrepParams& p, int n, int j, double x, double z) {
  const int k = p.crystal_kind;
  if (k == BPM_CRYSTAL_VACUUM) return false;
  if (k == BPM_CRYSTAL_BULK) return true;
  if (k == BPM_CRYSTAL_MASK) return p.mask[size_t(n) * p.nx + j] != 0;
  const double depth = __dadd_rn(__dmul_rn(p.ncx, __dsub_rn(x, p.sx)),
                                 __dmul_rn(p.ncz, __dsub_rn(z, p.sz)));
  bool in = (depth >= 0.0) && (depth <= p.thick);
  if (k == BPM_CRYSTAL_SLAB_AND_MASK) in = in && (p.mask[size_t(n) * p.nx + j] != 0);
  if (k == BPM_CRYSTAL_SLAB_AND_POLYGON) {
    bool odd = false;
    for (int i = 0; i < p.nv; ++i) {
      const int i2 = (i + 1 == p.nv) ? 0 : i + 1;
      const double x1 = p.poly[2 * i], z1 = p.poly[2 * i + 1];
      const double x2 = p.poly[2 * i2], z2 = p.poly[2 * i2 + 1];
      if ((z1 > z) != (z2 > z)) {
        const double xc = __dadd_rn(
            __ddiv_rn(__dmul_rn(__dsub_rn(x2, x1), __dsub_rn(z, z1)), __dsub_rn(z2, z1)), x1);
        if (x < xc) odd = !odd;
      }
    }
    in = in && odd;
  }
  return in;
}

__device__ double strain_ux(const PrepParams& p, int n, int j, double x, double z) {
  switch (p.strain_kind) {
    case BPM_STRAIN_ARRAY:
      return p.ux[size_t(n) * p.nx + j];
    case BPM_STRAIN_BENT: {   // (x'^2 + nu z'^2) / (2R), Eq. fov110 (configured form)
      const double xp = x - p.p2, zp = z - p.p3;
      return (xp * xp + p.p1 * (zp * zp)) / (2.0 * p.p0);
    }
    case BPM_STRAIN_EDGE_DISLOCATION: {   // Eq. fov120, b along x
      const double xp = x - p.p2, zp = z - p.p3;
      const double r2 = xp * xp + zp * zp;
      if (r2 == 0.0) return 0.0;
      return p.p0 / 6.283185307179586 *
             (atan2(zp, xp) + xp * zp / (2.0 * (1.0 - p.p1) * r2));
    }
    default:
      return 0.0;
  }
}

__global__ void prep_kernel(PrepParams p) {
  const size_t total = size_t(p.nx) * p.nz;
  for (size_t c = blockIdx.x * size_t(blockDim.x) + threadIdx.x; c < total;
       c += size_t(gridDim.x) * blockDim.x) {
    const int n = int(c / p.nx), j = int(c % p.nx);
    const double x = __dadd_rn(p.x0, __dmul_rn(double(j), p.dx));
    const double z = __dmul_rn(double(n), p.dz);
    double re = 0.0, im = 0.0;
    if (inside_cell(p, n, j, x, z)) {
      // h u_x in FP64, reduced to [-pi, pi] in FP64; the unit phasor is
      // evaluated in the precision it is stored in (FP64 plans: FP64,
      // FP32 plans: FP32 of the reduced angle).
      const double theta = p.h * strain_ux(p, n, j, x, z);
      const double t = theta - 6.283185307179586 * rint(theta * 0.15915494309189535);
      if (p.out64) {
        sincos(t, &im, &re);
      } else {
        float sf, cf;
        sincosf(float(t), &sf, &cf);
        re = cf;
        im = sf;
      }
    }
    if (p.out32) {
      size_t o = c;
      if (p.parts > 1) {
        const int m = p.nx / p.parts;
        o = size_t(n) * p.nx + size_t(j % p.parts) * m + j / p.parts;
      }
      p.out32[o] = make_float2(float(re), float(im));
    }
    if (p.out64) p.out64[c] = make_double2(re, im);
  }
}

}  // namespace

int prepare_slices(bpm_plan_s* plan, cudaStream_t st, bool sync) {
  const size_t phasor_bytes = size_t(plan->nx) * plan->nz *
                              (plan->precision == BPM_FP32_FUSED ? 8 : 16);
  if (!plan->d_phasor) {
    cudaError_t ea = cudaMalloc(&plan->d_phasor, phasor_bytes);
    if (ea != cudaSuccess) {
      plan->d_phasor = nullptr;
      cudaGetLastError();
      return fail(ea == cudaErrorMemoryAllocation ? BPM_ERR_OOM : BPM_ERR_CUDA,
                  "cudaMalloc(strain phasor): " + std::string(cudaGetErrorString(ea)));
    }
  }
  PrepParams p{};
  p.nx = plan->nx;
  p.nz = plan->nz;
  p.x0 = plan->x0_um;
  p.dx = plan->dx_um;
  p.dz = plan->dz_um;
  p.crystal_kind = plan->crystal_kind;
  double cx = std::cos(plan->asym), sz = std::sin(plan->asym);
  if (std::fabs(cx) < 1e-12) { cx = 0.0; sz = std::copysign(1.0, sz); }
  else if (std::fabs(sz) < 1e-12) { sz = 0.0; cx = std::copysign(1.0, cx); }
  p.ncx = cx;
  p.ncz = sz;
  p.thick = plan->thick;
  p.sx = plan->surf_x;
  p.sz = plan->surf_z;
  p.strain_kind = plan->strain_kind;
  p.p0 = plan->sparams[0];
  p.p1 = plan->sparams[1];
  p.p2 = plan->sparams[2];
  p.p3 = plan->sparams[3];
  p.h = plan->h_per_um;
  p.parts = 1;
  if (plan->precision == BPM_FP32_FUSED && plan->logn >= kSplitLogN) p.parts = plan->nx >> 12;
  if (plan->precision == BPM_FP32_FUSED) p.out32 = static_cast<float2*>(plan->d_phasor);
  else p.out64 = static_cast<double2*>(plan->d_phasor);

  uint8_t* d_mask = nullptr;
  double* d_poly = nullptr;
  double* d_ux = nullptr;
  int rc = BPM_OK;
  cudaError_t e = cudaSuccess;
  const size_t cells = size_t(plan->nx) * plan->nz;
  if (!plan->mask.empty()) {
    e = cudaMalloc(&d_mask, cells);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_mask, plan->mask.data(), cells, cudaMemcpyHostToDevice, st);
    p.mask = d_mask;
  }
  if (e == cudaSuccess && !plan->poly.empty()) {
    e = cudaMalloc(&d_poly, plan->poly.size() * sizeof(double));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_poly, plan->poly.data(), plan->poly.size() * sizeof(double),
                          cudaMemcpyHostToDevice, st);
    p.poly = d_poly;
    p.nv = int(plan->poly.size() / 2);
  }
  if (e == cudaSuccess && plan->strain_kind == BPM_STRAIN_ARRAY) {
    e = cudaMalloc(&d_ux, cells * sizeof(double));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_ux, plan->ux.data(), cells * sizeof(double), cudaMemcpyHostToDevice, st);
    p.ux = d_ux;
  }
  if (e == cudaSuccess) {
    const int threads = 256;
    const size_t want = (cells + threads - 1) / threads;
    const int blocks = int(want < 65536 ? want : 65536);
    prep_kernel<<<blocks, threads, 0, st>>>(p);
    e = cudaGetLastError();
  }
  const bool temporaries = d_mask || d_poly || d_ux;
  if (e == cudaSuccess && (sync || temporaries)) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) rc = (e == cudaErrorMemoryAllocation) ? fail(BPM_ERR_OOM, "slice preparation: out of device memory")
                                                             : cuda_fail(e, "slice preparation");
  if (d_mask) cudaFree(d_mask);
  if (d_poly) cudaFree(d_poly);
  if (d_ux) cudaFree(d_ux);
  if (rc == BPM_OK) plan->slices_dirty = false;
  return rc;
}

}  // namespace bpm
