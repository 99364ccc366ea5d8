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
//
// FP32 plans with an analytic crystal (vacuum, bulk, slab, slab AND polygon
// of at most kMaxPolyV vertices) and an analytic strain (none, bent, edge
// dislocation) take a faster route that gives the same mask and the phasor
// to FP32 accuracy, with FP64 arithmetic only per row and per column:
//   * mask: x_j is non-decreasing in j, so each face test and each polygon
//     crossing test is monotone in j and splits a row at one column.  One
//     thread per row finds those columns by bisection, evaluating exactly the
//     FP64 expressions above, and stores the row's inside set as at most
//     kMaxIv intervals -- the decisions are those of the per-cell test;
//   * bent crystal: h u = h x'^2/(2R) + h nu z'^2/(2R) is a column term plus
//     a row term; each is reduced modulo 2 pi in FP64 and turned into a unit
//     phasor, and a cell's phasor is the FP32 product of its column's and its
//     row's (error a few 1e-7);
//   * edge dislocation: h u = (h b / 2 pi) (atan2(z', x') + x' z' / (2 (1 -
//     nu) r^2)) is O(h b) in size (a few radians for a unit dislocation), so
//     it is evaluated in FP32 from x' and z' rounded from FP64 (absolute
//     error about |h b / 2 pi| x 1e-6 rad).
// This removes the per-cell FP64 work, which on this GPU costs far more than
// the march of the same cells.
//
// Separable form: a vacuum, bulk or slab crystal (one inside interval per
// step) with no strain or the bent-crystal strain needs no per-cell data at
// all.  Such FP32 2D plans keep the rows of fast_rows_kernel (the interval
// and the row phasor, SepRow) and the column phasors (in the stream's
// order), and the fused kernels form each cell as they couple -- the same
// FP32 product and the same decision as sep_cells_kernel, which writes the
// stream of the same crystal bit for bit (for bpm_fetch_slices).  A bent
// 16384 x 20000 request then holds 2 MB of slices instead of 2.6 GB.
#include <cmath>
#include <cstdlib>
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

// 3D plans: cell (n, i, j) at (x_j, y_i, z_n); the 2D kinds hold at every
// y, masks and u_x arrays are [nz][ny][nx], the box is tested in FP64.
struct Prep3D {
  int ny;
  double y0, dy;
  double box[6];
};

__global__ void prep3d_kernel(PrepParams p, Prep3D q) {
  const size_t plane = size_t(p.nx) * q.ny;
  const size_t total = plane * p.nz;
  for (size_t c = blockIdx.x * size_t(blockDim.x) + threadIdx.x; c < total;
       c += size_t(gridDim.x) * blockDim.x) {
    const int n = int(c / plane);
    const size_t rem = c % plane;
    const int i = int(rem / p.nx), j = int(rem % p.nx);
    const double x = __dadd_rn(p.x0, __dmul_rn(double(j), p.dx));
    const double y = __dadd_rn(q.y0, __dmul_rn(double(i), q.dy));
    const double z = __dmul_rn(double(n), p.dz);
    bool in;
    if (p.crystal_kind == BPM_CRYSTAL_BOX) {
      in = x >= q.box[0] && x <= q.box[1] && y >= q.box[2] && y <= q.box[3] &&
           z >= q.box[4] && z <= q.box[5];
    } else if (p.crystal_kind == BPM_CRYSTAL_MASK) {
      in = p.mask[c] != 0;
    } else if (p.crystal_kind == BPM_CRYSTAL_SLAB_AND_MASK) {
      PrepParams slab = p;
      slab.crystal_kind = BPM_CRYSTAL_SLAB;
      in = inside_cell(slab, n, j, x, z) && p.mask[c] != 0;
    } else {
      in = inside_cell(p, n, j, x, z);
    }
    float2 v = make_float2(0.f, 0.f);
    if (in) {
      const double u = p.strain_kind == BPM_STRAIN_ARRAY ? p.ux[c] : strain_ux(p, n, j, x, z);
      const double theta = p.h * u;
      const double t = theta - 6.283185307179586 * rint(theta * 0.15915494309189535);
      float sf, cf;
      sincosf(float(t), &sf, &cf);
      v = make_float2(cf, sf);
    }
    p.out32[c] = v;
  }
}

constexpr int kMaxPolyV = 16;
static_assert(kMaxIv == kMaxPolyV / 2 + 1, "intervals of a row cut by the polygon");

struct FastParams {
  int nx, nz, parts;
  double x0, dx, dz;
  int crystal_kind;
  double ncx, ncz, thick, sx, sz;
  int nv;
  double poly[2 * kMaxPolyV];
  int strain_kind;
  double p0, p1, p2, p3, h;
};

struct ColInfo {      // one column
  float2 ph;                    // bent: exp(i h x'^2 / (2R)), reduced in FP64
  float xp;                     // dislocation: x - x_core
  float pad;
};

__device__ __forceinline__ double x_of(const FastParams& p, int j) {
  return __dadd_rn(p.x0, __dmul_rn(double(j), p.dx));
}

__device__ __forceinline__ double depth_of(const FastParams& p, double x, double z) {
  return __dadd_rn(__dmul_rn(p.ncx, __dsub_rn(x, p.sx)), __dmul_rn(p.ncz, __dsub_rn(z, p.sz)));
}

// Smallest j in [0, nx] with pred(j) true, for pred monotone false -> true.
template <typename Pred>
__device__ int first_true(int nx, Pred pred) {
  int lo = 0, hi = nx;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (pred(mid)) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

__device__ double unit_phase(double a) {   // a reduced to [-pi, pi] in FP64
  return a - 6.283185307179586 * rint(a * 0.15915494309189535);
}

// One thread per z-step: the row's inside intervals (the union of [lo, hi))
// and its phase term.
__global__ void fast_rows_kernel(FastParams p, SepRow* rows) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= p.nz) return;
  const double z = __dmul_rn(double(n), p.dz);
  SepRow r{};
  r.ph = make_float2(1.f, 0.f);
  int slo = 0, shi = 0;   // slab (or whole-row) interval
  if (p.crystal_kind == BPM_CRYSTAL_BULK) {
    shi = p.nx;
  } else if (p.crystal_kind == BPM_CRYSTAL_SLAB || p.crystal_kind == BPM_CRYSTAL_SLAB_AND_POLYGON) {
    if (p.ncx >= 0.0) {   // depth non-decreasing in j
      slo = first_true(p.nx, [&](int j) { return depth_of(p, x_of(p, j), z) >= 0.0; });
      shi = first_true(p.nx, [&](int j) { return depth_of(p, x_of(p, j), z) > p.thick; });
    } else {              // depth non-increasing in j
      slo = first_true(p.nx, [&](int j) { return depth_of(p, x_of(p, j), z) <= p.thick; });
      shi = first_true(p.nx, [&](int j) { return depth_of(p, x_of(p, j), z) < 0.0; });
    }
  }
  if (p.crystal_kind == BPM_CRYSTAL_SLAB_AND_POLYGON && shi > slo) {
    // even-odd rule: cell j is inside when an odd number of crossings lie
    // right of it; crossing i covers the prefix j < c_i
    int c[kMaxPolyV];
    int m = 0;
    for (int i = 0; i < p.nv; ++i) {
      const int i2 = (i + 1 == p.nv) ? 0 : i + 1;
      const double x1 = p.poly[2 * i], z1 = p.poly[2 * i + 1];
      const double x2 = p.poly[2 * i2], z2 = p.poly[2 * i2 + 1];
      if ((z1 > z) != (z2 > z)) {
        const double xc = __dadd_rn(
            __ddiv_rn(__dmul_rn(__dsub_rn(x2, x1), __dsub_rn(z, z1)), __dsub_rn(z2, z1)), x1);
        const int ci = first_true(p.nx, [&](int j) { return !(x_of(p, j) < xc); });
        int k = m++;
        while (k > 0 && c[k - 1] > ci) {   // insertion sort
          c[k] = c[k - 1];
          --k;
        }
        c[k] = ci;
      }
    }
    // with c sorted, the columns of [c_{k-1}, c_k) lie left of crossings
    // k..m-1 only: m - k of them
    int start = 0;
    for (int k = 0; k <= m; ++k) {
      const int end = k < m ? c[k] : p.nx;
      if (((m - k) & 1) && end > start) {
        const int a = max(start, slo), b = min(end, shi);
        if (b > a && r.nint < kMaxIv) {
          r.lo[r.nint] = a;
          r.hi[r.nint] = b;
          ++r.nint;
        }
      }
      start = end;
    }
  } else if (shi > slo) {
    r.nint = 1;
    r.lo[0] = slo;
    r.hi[0] = shi;
  }
  if (r.nint > 0) {
    r.lo0 = r.lo[0];
    r.hi0 = r.hi[0];
  }
  if (p.strain_kind == BPM_STRAIN_BENT) {
    const double zp = z - p.p3;
    const double b = unit_phase(p.h * (p.p1 * (zp * zp) / (2.0 * p.p0)));
    double sb, cb;
    sincos(b, &sb, &cb);
    r.ph = make_float2(float(cb), float(sb));
  } else if (p.strain_kind == BPM_STRAIN_EDGE_DISLOCATION) {
    r.zp = float(z - p.p3);
  }
  rows[n] = r;
}

// One thread per column: its phase term (cols, natural order) and, for the
// separable form, the column phasor at the stream's position of column j,
// (j mod parts) m + j div parts (scols).  Either output may be null.
__global__ void fast_cols_kernel(FastParams p, ColInfo* cols, float2* scols) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= p.nx) return;
  const double x = x_of(p, j);
  ColInfo c{};
  c.ph = make_float2(1.f, 0.f);
  if (p.strain_kind == BPM_STRAIN_BENT) {
    const double xp = x - p.p2;
    const double a = unit_phase(p.h * ((xp * xp) / (2.0 * p.p0)));
    double sa, ca;
    sincos(a, &sa, &ca);
    c.ph = make_float2(float(ca), float(sa));
  } else if (p.strain_kind == BPM_STRAIN_EDGE_DISLOCATION) {
    c.xp = float(x - p.p2);
  }
  if (cols) cols[j] = c;
  if (scols) {
    const int m = p.nx / p.parts;
    scols[(j % p.parts) * m + j / p.parts] = c.ph;
  }
}

// The per-cell stream of the separable form: position o of row n holds
// column j = (o mod m) parts + o div m; its phasor col[j] row[n] inside the
// row's intervals, (0, 0) outside -- the product and the decisions the fused
// kernels form from the same tables, and the values fast_cells_kernel
// writes for a bent or unstrained crystal.
__global__ void __launch_bounds__(256)
    sep_cells_kernel(const SepRow* __restrict__ rows, const float2* __restrict__ scols, int nx,
                     int nz, int parts, float2* __restrict__ out) {
  const int m = nx / parts;
  for (int n = blockIdx.y; n < nz; n += gridDim.y) {
    const SepRow* r = rows + n;
    const int nint = __ldg(&r->nint);
    const float2 rp = __ldg(&r->ph);
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < nx; o += gridDim.x * blockDim.x) {
      const int j = (o % m) * parts + o / m;
      bool in = false;
      for (int k = 0; k < nint; ++k) in |= (j >= __ldg(&r->lo[k])) & (j < __ldg(&r->hi[k]));
      const float2 a = __ldg(&scols[o]);
      out[size_t(n) * nx + o] =
          in ? make_float2(fmaf(a.x, rp.x, -(a.y * rp.y)), fmaf(a.x, rp.y, a.y * rp.x))
             : make_float2(0.f, 0.f);
    }
  }
}

// Every thread writes 4 consecutive outputs of a row (two 16-byte stores);
// blocks stride over the rows.  The row's intervals and phase are read from
// global memory with the same address in every lane (broadcast loads that
// stay in L1).  Output position o of a row holds column
// j = (o mod m) parts + o div m, m = nx / parts (a power of two).
template <int STRAIN>
__global__ void __launch_bounds__(256)
    fast_cells_kernel(FastParams p, const SepRow* __restrict__ rows,
                      const ColInfo* __restrict__ cols, float k_disl, float q_disl, int log_m,
                      float2* __restrict__ out) {
  const int m_mask = (1 << log_m) - 1;
  const int o0 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (o0 >= p.nx) return;
  for (int n = blockIdx.y; n < p.nz; n += gridDim.y) {
    const SepRow* r = rows + n;
    const int nint = __ldg(&r->nint);
    float2 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int o = o0 + u;
      const int j = (o & m_mask) * p.parts + (o >> log_m);
      bool in = false;
      for (int k = 0; k < nint; ++k) in |= (j >= __ldg(&r->lo[k])) & (j < __ldg(&r->hi[k]));
      v[u] = make_float2(0.f, 0.f);
      if (in) {
        if constexpr (STRAIN == BPM_STRAIN_BENT) {
          const float2 a = __ldg(&cols[j].ph), b = __ldg(&r->ph);
          v[u] = make_float2(fmaf(a.x, b.x, -(a.y * b.y)), fmaf(a.x, b.y, a.y * b.x));
        } else if constexpr (STRAIN == BPM_STRAIN_EDGE_DISLOCATION) {
          const float xp = __ldg(&cols[j].xp), zp = __ldg(&r->zp);
          const float r2 = fmaf(xp, xp, zp * zp);
          float th = 0.f;
          if (r2 != 0.f) th = k_disl * (atan2f(zp, xp) + (xp * zp) * q_disl / r2);
          float sn, cs;
          sincosf(th, &sn, &cs);
          v[u] = make_float2(cs, sn);
        } else {
          v[u] = make_float2(1.f, 0.f);
        }
      }
    }
    float4* dst = reinterpret_cast<float4*>(out + size_t(n) * p.nx + o0);
    dst[0] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    dst[1] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
  }
}

bool fast_path_applies(const bpm_plan_s* plan) {
  if (plan->precision != BPM_FP32_FUSED) return false;
  const int k = plan->crystal_kind;
  const bool crystal_ok = k == BPM_CRYSTAL_VACUUM || k == BPM_CRYSTAL_BULK ||
                          k == BPM_CRYSTAL_SLAB ||
                          (k == BPM_CRYSTAL_SLAB_AND_POLYGON &&
                           plan->poly.size() <= size_t(2 * kMaxPolyV));
  const int sk = plan->strain_kind;
  return crystal_ok && (sk == BPM_STRAIN_NONE || sk == BPM_STRAIN_BENT ||
                        sk == BPM_STRAIN_EDGE_DISLOCATION);
}

// sep: write the separable form (rows and column phasors) to plan->d_sep
// instead of the per-cell stream.
int prepare_fast(bpm_plan_s* plan, const PrepParams& q, cudaStream_t st, bool sync, bool sep) {
  FastParams p{};
  p.nx = q.nx;
  p.nz = q.nz;
  p.parts = q.parts;
  p.x0 = q.x0;
  p.dx = q.dx;
  p.dz = q.dz;
  p.crystal_kind = q.crystal_kind;
  p.ncx = q.ncx;
  p.ncz = q.ncz;
  p.thick = q.thick;
  p.sx = q.sx;
  p.sz = q.sz;
  p.nv = int(plan->poly.size() / 2);
  for (size_t i = 0; i < plan->poly.size(); ++i) p.poly[i] = plan->poly[i];
  p.strain_kind = q.strain_kind;
  p.p0 = q.p0;
  p.p1 = q.p1;
  p.p2 = q.p2;
  p.p3 = q.p3;
  p.h = q.h;
  SepRow* d_rows = nullptr;
  ColInfo* d_cols = nullptr;
  cudaError_t e = cudaSuccess;
  if (sep) {
    d_rows = static_cast<SepRow*>(plan->d_sep);
    float2* d_scols = reinterpret_cast<float2*>(d_rows + p.nz);
    fast_rows_kernel<<<(p.nz + 127) / 128, 128, 0, st>>>(p, d_rows);
    fast_cols_kernel<<<(p.nx + 255) / 256, 256, 0, st>>>(p, nullptr, d_scols);
    e = cudaGetLastError();
    if (e == cudaSuccess && sync) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "slice preparation (separable form)");
    plan->slices_dirty = false;
    return BPM_OK;
  }
  e = cudaMallocAsync(&d_rows, size_t(p.nz) * sizeof(SepRow), st);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_cols, size_t(p.nx) * sizeof(ColInfo), st);
  if (e == cudaSuccess) {
    fast_rows_kernel<<<(p.nz + 127) / 128, 128, 0, st>>>(p, d_rows);
    fast_cols_kernel<<<(p.nx + 255) / 256, 256, 0, st>>>(p, d_cols, nullptr);
    const float k_disl = float(p.h * p.p0 / 6.283185307179586);
    const float q_disl = float(1.0 / (2.0 * (1.0 - p.p1)));
    const int threads = 256;
    int log_m = 0;
    while ((1 << log_m) < p.nx / p.parts) ++log_m;
    dim3 grid((p.nx + 4 * threads - 1) / (4 * threads), p.nz < 65535 ? p.nz : 65535);
    if (p.strain_kind == BPM_STRAIN_BENT)
      fast_cells_kernel<BPM_STRAIN_BENT><<<grid, threads, 0, st>>>(p, d_rows, d_cols, k_disl,
                                                                  q_disl, log_m, q.out32);
    else if (p.strain_kind == BPM_STRAIN_EDGE_DISLOCATION)
      fast_cells_kernel<BPM_STRAIN_EDGE_DISLOCATION><<<grid, threads, 0, st>>>(
          p, d_rows, d_cols, k_disl, q_disl, log_m, q.out32);
    else
      fast_cells_kernel<BPM_STRAIN_NONE><<<grid, threads, 0, st>>>(p, d_rows, d_cols, k_disl,
                                                                  q_disl, log_m, q.out32);
    e = cudaGetLastError();
  }
  if (d_rows) cudaFreeAsync(d_rows, st);
  if (d_cols) cudaFreeAsync(d_cols, st);
  if (e == cudaSuccess && sync) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    return e == cudaErrorMemoryAllocation ? fail(BPM_ERR_OOM, "slice preparation: out of device memory")
                                          : cuda_fail(e, "slice preparation");
  }
  plan->slices_dirty = false;
  return BPM_OK;
}

}  // namespace

bool sep_slices_apply(const bpm_plan_s* plan) {
  if (plan->precision != BPM_FP32_FUSED || plan->ny > 1) return false;
  // one inside interval per step at most (the kernels test [lo0, hi0))
  const int k = plan->crystal_kind;
  if (k != BPM_CRYSTAL_VACUUM && k != BPM_CRYSTAL_BULK && k != BPM_CRYSTAL_SLAB) return false;
  if (plan->strain_kind != BPM_STRAIN_NONE && plan->strain_kind != BPM_STRAIN_BENT) return false;
  const char* e = std::getenv("BPM_SLICE_STREAM");
  if (e && e[0] == '1') return false;
  if (e && e[0] == '0') return true;
  // Where the separable form is taken (same GPU, back to back, 8000-step
  // bent solves): N = 4096 rows that each get the 4-SM half-band split run
  // the 8-point kernel, which reads its column phasors without the stream's
  // stride-2 bank conflicts: 22.8 ms against 23.4 ms with the stream (its
  // Verlet form, with three couplings per step, 27.0 against 26.2 ms: the
  // stream there).  At
  // N >= 8192 the two forms are within 1-3 % and the stream would take
  // 8 B x N x Nz (2.6 GB for a 16384 x 20000 request).  Elsewhere the
  // per-cell interval test costs more than the stream's read: 7-11 % at
  // N = 1024 and 2048 (a 2048 x 20000 stream is 328 MB), 8 % on batches
  // that fill the GPU (which share one stream among all rows): they keep
  // the stream.
  static int sms = 0;
  if (sms == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    sms = v > 0 ? v : 1;
  }
  if (plan->logn == 12) return plan->split == BPM_SPLIT_FIRST_ORDER && 4 * plan->nb <= sms;
  return plan->logn >= kSplitLogN && 2 * plan->nb <= sms;
}

size_t slice_data_bytes(const bpm_plan_s* plan) {
  if (sep_slices_apply(plan)) return sep_bytes(plan);
  return plane_of(plan) * plan->nz * (plan->precision == BPM_FP32_FUSED ? 8 : 16);
}

int expand_sep_slices(const bpm_plan_s* plan, float2* out, cudaStream_t st) {
  if (!plan->sep_slices || !plan->d_sep) return fail(BPM_ERR_INVALID, "no separable slices");
  const int parts = plan->logn >= kSplitLogN ? plan->nx >> 12 : 1;
  const SepRow* rows = static_cast<const SepRow*>(plan->d_sep);
  const float2* scols = reinterpret_cast<const float2*>(rows + plan->nz);
  dim3 grid((plan->nx + 255) / 256, plan->nz < 65535 ? plan->nz : 65535);
  sep_cells_kernel<<<grid, 256, 0, st>>>(rows, scols, plan->nx, plan->nz, parts, out);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BPM_OK : cuda_fail(e, "sep_cells_kernel");
}

int prepare_slices(bpm_plan_s* plan, cudaStream_t st, bool sync) {
  NvtxRange nvtx("bpm_prepare_slices");
  const bool sep = sep_slices_apply(plan);
  void** dst = sep ? &plan->d_sep : &plan->d_phasor;
  if (!*dst) {
    cudaError_t ea = cudaMalloc(dst, slice_data_bytes(plan));
    if (ea != cudaSuccess) {
      *dst = nullptr;
      cudaGetLastError();
      return fail(ea == cudaErrorMemoryAllocation ? BPM_ERR_OOM : BPM_ERR_CUDA,
                  "cudaMalloc(strain phasor): " + std::string(cudaGetErrorString(ea)));
    }
  }
  plan->sep_slices = false;   // set again once the separable form is written
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
  if (sep) {
    const int rc = prepare_fast(plan, p, st, sync, true);
    plan->sep_slices = rc == BPM_OK;
    return rc;
  }
  if (plan->ny <= 1 && fast_path_applies(plan)) return prepare_fast(plan, p, st, sync, false);

  uint8_t* d_mask = nullptr;
  double* d_poly = nullptr;
  double* d_ux = nullptr;
  int rc = BPM_OK;
  cudaError_t e = cudaSuccess;
  const size_t cells = plane_of(plan) * plan->nz;
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
    if (plan->ny > 1) {
      Prep3D q{};
      q.ny = plan->ny;
      q.y0 = plan->y0_um;
      q.dy = plan->dy_um;
      for (int i = 0; i < 6; ++i) q.box[i] = plan->box[i];
      prep3d_kernel<<<blocks, threads, 0, st>>>(p, q);
    } else {
      prep_kernel<<<blocks, threads, 0, st>>>(p);
    }
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
