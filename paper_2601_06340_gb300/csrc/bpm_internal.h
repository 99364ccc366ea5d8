// Internal types shared by the host runtime and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/bpm.h"

namespace bpm {

// NVTX range over a host-side phase (plan, slice preparation, march,
// launch-shape trials, server admission / batches / retirement), seen by
// Nsight tools (e.g. ncu --nvtx --nvtx-include "bpm_propagate/"); a no-op
// without a tool attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr int kMinLogN = 3;
constexpr int kMaxLogN = 14;          // nx <= 16384
// N >= 2^kSplitLogN: each band is split over a cluster of N/4096 CTAs
// (interleaved samples), and the strain stream / propagator tables of FP32
// plans are stored per part (see fused4_kernel.cuh).
constexpr int kSplitLogN = 13;
constexpr double kTwoPi = 6.283185307179586;
constexpr double kHcEvAngstrom = 12398.419843320026;

// Device status word bits (per launch).
enum : int { kStatusWaitTimeout = 1 };

// Inside intervals of one z-step of an analytic crystal (slab, or slab cut
// by a polygon with up to 16 vertices: at most 9 runs of inside columns).
constexpr int kMaxIv = 9;

// One z-step of the separable slice form.  For a bent or unstrained crystal
// whose mask is a union of column intervals per step, the strain phasor of
// cell (j, n) is col[j] * ph_n inside and (0, 0) outside (h u = h x'^2/(2R)
// + h nu z'^2/(2R), each term reduced in FP64): the kernels form it from
// this row and a per-column table instead of reading a per-cell stream.
// The first 16 bytes hold everything a row with one interval needs.
struct alignas(16) SepRow {
  float2 ph;                // exp(i h nu z'^2/(2R)) (bent), (1, 0) unstrained
  int lo0, hi0;             // first inside interval [lo0, hi0) (0, 0: none)
  int nint;                 // number of intervals
  int lo[kMaxIv], hi[kMaxIv];   // all intervals, natural column indices
  float zp;                 // dislocation core offset z - z_core (slice preparation)
};
static_assert(sizeof(SepRow) == 96, "bulk-copied rows: a multiple of 16 bytes");

// One batch row of a fused FP32 launch.  Everything the kernel needs for a
// row is here, so rows of different plans (different energies, strain
// streams, step ranges) can share one launch.
struct RowDescF32 {
  float2* state;            // [2][N] raw envelopes (common phase removed)
  const float2* prop;       // [2][N] (P(q)-1)/N in the FFT's output order
  const float2* prop_split; // N = 4096 rows on a 4-CTA cluster: [2][3][N/2] circulant
                            // tables of the half-band split, else null
  const float2* phasor;     // [nz][N] exp(i h u_x), (0,0) outside the crystal; null in
                            // the separable form
  const SepRow* srows;      // separable form: [nz] rows, else null
  const float2* scols;      // separable form: [N] column phasors in the stream's order
  float2* records;          // [n_rec][2][N] or null
  double* powers;           // [n_rec+1][2] or null
  float2 am1;               // Delta_eps_0 - 1 inside the crystal
  float2 b;                 // Delta_eps_{+-1} inside the crystal
  float2 am1h, bh;          // the same for half a step (second-order splitting)
  double gphase;            // common per-step phase (dz^ cos alpha) mod 2 pi
  double dx_um;
  int32_t n_begin;          // first step of this launch (absolute)
  int32_t n_end;            // one past the last step this row may take
  int32_t n_phase0;         // absolute step at which `state` carries phase 0
  int32_t record_every;     // 0 = no records
};

// One batch row of the FP64 plain path (all rows of a plan share N).
struct RowDescF64 {
  const double2* prop;      // [2][N] P(q)/N in natural FFT order
  double2 a;                // Delta_eps_0
  double2 b;                // Delta_eps_{+-1}
  double gphase;
};

// Per-plan runtime buffers of the march entry points (capi.cpp): the plan's
// stream, the host-API record / power buffers, the common phase factors and
// the rotated launch schedule.
struct PlanAux {
  cudaStream_t stream = nullptr;
  void* d_rec = nullptr;      // host-API record buffer
  size_t rec_bytes = 0;
  double* d_pow = nullptr;    // host-API powers buffer
  size_t pow_bytes = 0;
  double2* d_g = nullptr;     // [B] common phase factors
  RowDescF32* d_sched = nullptr;  // rotated launch schedule
  size_t sched_cap = 0;
};

// FP64 constants of one photon energy (Eqs. fov4-fov12).
struct EnergyConsts {
  double e_ev, k_um, s, c, dzh, dxh;
  std::complex<double> w, phi0, a, b, am1;
  double gphase;            // fmod(dzh * c, 2 pi)
};

}  // namespace bpm

struct bpm_plan_s {
  std::mutex mu;
  // problem
  int32_t nx = 0, nz = 0, logn = 0, nb = 0, record_every = 0, precision = 0;
  double dx_um = 0, dz_um = 0, x0_um = 0, e_ref_ev = 0, theta_b_ref = 0;
  // second transverse coordinate (3D plans: ny > 1; fields are [ny][nx])
  int32_t ny = 1, logny = 0;
  double dy_um = 0, y0_um = 0;
  std::complex<double> chi0, chih;
  std::vector<double> energies;
  std::vector<bpm::EnergyConsts> ec;
  int32_t n_rec = 0;
  double d_um = 0, h_per_um = 0;
  // crystal and strain descriptions (host copies)
  int32_t crystal_kind = BPM_CRYSTAL_VACUUM;
  double asym = 0, thick = 0, surf_x = 0, surf_z = 0;
  double box[6] = {0, 0, 0, 0, 0, 0};   // BPM_CRYSTAL_BOX: x0, x1, y0, y1, z0, z1
  std::vector<uint8_t> mask;
  std::vector<double> poly;
  int32_t strain_kind = BPM_STRAIN_NONE;
  std::vector<double> ux;
  double sparams[4] = {0, 0, 0, 0};
  bool slices_dirty = true;
  // device
  int device = 0;
  void* d_phasor = nullptr;       // [nz][nx] c64 (FP32) or c128 (FP64)
  // separable slice form (FP32 plans, bent or unstrained analytic crystals):
  // [nz] SepRow then [nx] float2 column phasors, in place of d_phasor
  void* d_sep = nullptr;
  bool sep_slices = false;        // the last prepared slices are separable
  void* d_prop = nullptr;         // [B][2][nx] c64 (delta form) or c128
  void* d_prop_split = nullptr;   // [B][2][3][nx/2] c64: N = 4096 half-band split tables
  void* d_tw = nullptr;           // FP32: float4 [nx] hi/lo; FP64: double2 [nx]
  void* d_state = nullptr;        // [B][2][nx] c64 / c128
  void* d_state2 = nullptr;       // FP64 ping-pong buffer
  void* d_rows = nullptr;         // RowDescF32[B] or RowDescF64[B]
  void* d_io = nullptr;           // [B][2][nx] c128 host-transfer staging
  int* d_status = nullptr;        // device status word
  void* d_spec = nullptr;         // 3D: [B][2][ny][nx] c64 x-spectra
  void* d_twy = nullptr;          // 3D: float4 [ny] twiddles along y
  double* d_pwpart = nullptr;     // 3D: [B][n_rec][2][ny] line power sums
  size_t pwpart_bytes = 0;
  void* vol_graph = nullptr;      // 3D: captured march (vol.cu)
  // operator splitting (FP64 plans): stages of one step
  int32_t split = BPM_SPLIT_FIRST_ORDER;
  int32_t n_stages = 0;
  std::vector<int> stage_has_prop;   // [n_stages]: stage propagates (a_i != 0)
  void* d_stage_rows = nullptr;      // RowDescF64 [n_stages][B]
  void* d_stage_prop = nullptr;      // FP64: double2 [tables][B][2][nx]; FP32 Forest-Ruth:
                                     // float2 [B][2 tables][2][nx] (t dz, (1 - 2t) dz)
  void* d_stage_prop_split = nullptr;   // FP32 Forest-Ruth on the split kernels (nx = 4096
                                        // half-band split, nx = 8192 split band): float2
                                        // [B][2 tables][split table in thread order]
  size_t device_bytes = 0;
  int pending = 0;                // tickets not yet finished
  // launch shape of the last fused march: layout 1 cluster / 0 CTA / -1 rule,
  // rotation chunk (0: one launch)
  int shape_layout = -1, shape_chunk = 0;
  bpm::PlanAux aux;
};

namespace bpm {

// Points of one band's transverse field (nx, or nx * ny for 3D plans).
inline size_t plane_of(const bpm_plan_s* p) { return size_t(p->nx) * size_t(p->ny); }

// Thread-local error reporting (capi.cpp).
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

// Plan math (plan.cpp).
int validate_problem(const bpm_problem* p, std::string* why);
void compute_energy_consts(bpm_plan_s* plan);
void fused_prop_table(const bpm_plan_s* plan, int row, std::vector<float2>* out);
// (P^frac - 1)/N per band in the fused FFT's output order (nx <= 4096): the
// propagator increment of a stage of frac * dz
void fused_prop_table_frac(const bpm_plan_s* plan, int row, double frac,
                           std::vector<float2>* out);
// 3D: (P(qx, qy) - 1)/(nx ny) per band, [band][y position][x position] in the
// output orders of the radix-16 FFTs along y and x.
void vol_prop_table(const bpm_plan_s* plan, int row, std::vector<float2>* out);
int validate_problem3d(const bpm_problem* p, int ny, double dy_um, double y0_um,
                       std::string* why);
void plain_prop_table(const bpm_plan_s* plan, int row, std::vector<double2>* out);
// exp(i frac dz^ delta_+-(q)) / nx: the propagator of a stage of frac * dz
void plain_prop_table_frac(const bpm_plan_s* plan, int row, double frac,
                           std::vector<double2>* out);
// (Delta_eps_0, Delta_eps_+-1) of a coupling stage of frac * dz
void coupling_frac(const bpm_plan_s* plan, int row, double frac, std::complex<double>* a,
                   std::complex<double>* b);
// stage coefficients (a_i, b_i) of a splitting method
std::vector<std::pair<double, double>> split_stages(int method);
void twiddle_table_f32(int n, std::vector<float4>* out);
void twiddle_table_f64(int n, std::vector<double2>* out);
std::vector<int> fft_output_order(int logn);   // position -> frequency index

// Kernels (launchers in *.cu).
// Prepare mask + strain phasor on `st`; with sync = false the call returns
// once the work is enqueued (temporaries, if any, still force a wait).
int prepare_slices(bpm_plan_s* plan, cudaStream_t st, bool sync = true);
// Whether the plan's slices take the separable form (FP32 2D plans of a
// vacuum, bulk or slab crystal with bent or no strain, at nx = 4096 for the
// first-order step while 4 x rows <= the SM count and at nx >= 8192 while
// 2 x rows <= it;
// BPM_SLICE_STREAM=1 / 0 forces the stream / separable form), and the
// device bytes of either form.
bool sep_slices_apply(const bpm_plan_s* plan);
size_t slice_data_bytes(const bpm_plan_s* plan);
inline size_t sep_bytes(const bpm_plan_s* p) {
  return size_t(p->nz) * sizeof(SepRow) + size_t(p->nx) * 8;
}
// Write the per-cell stream of separable slices (the values the stream
// form would hold, bit for bit) to out [nz][nx] c64 in the stream's order.
int expand_sep_slices(const bpm_plan_s* plan, float2* out, cudaStream_t st);
int launch_fused(int logn, const RowDescF32* d_rows, int n_rows, int steps,
                 const float4* d_tw, int* d_status, cudaStream_t st);
// layout: -1 automatic, 0 one CTA per row, 1 two-CTA cluster per row (only
// for 1024 <= N <= 4096; larger N always use the split-band cluster).
int launch_fused_layout(int logn, const RowDescF32* d_rows, int n_rows, int steps,
                        const float4* d_tw, int* d_status, cudaStream_t st, int layout);
// SMs one row occupies in its cluster layout (0 if the size has none).
int fused_cluster_sms(int logn);
// 3D march of all rows on `st` (state: [B][2][ny][nx] c64, the field after
// n_begin steps, replaced by the field after n_end steps without the common
// phase); records / powers as for the 2D fused path.
int vol_march(bpm_plan_s* plan, float2* state, float2* d_rec, double* d_pw, int n_begin,
              int n_end, cudaStream_t st);
void vol_release(bpm_plan_s* plan);   // the captured march, if any
int plain_march(bpm_plan_s* plan, int n_begin, int n_end, int n_phase0, void* d_records,
                double* d_powers, cudaStream_t st);
int launch_convert_in(const double2* src, float2* dst, size_t n, cudaStream_t st);
// Upload `bytes` of host memory to `dst` through kernel parameters (used
// while the stream is being captured into a graph).
int upload_by_params(void* dst, const void* src, size_t bytes, cudaStream_t st);
int launch_finish_f32(const float2* state, double2* out_c128, float2* out_c64,
                      const double* gphase, int n_rows, int nx, int steps,
                      double dx, double* final_powers, int power_stride,
                      cudaStream_t st);
int launch_finish_f64(const double2* state, double2* out, const double* gphase,
                      int n_rows, int nx, int steps, double dx,
                      double* final_powers, int power_stride, cudaStream_t st);
int launch_omega_to_t(const void* d_in, void* d_out, int nb, int nx,
                      int precision, cudaStream_t st);
int fused_smem_bytes(int logn);
int fused_rows_resident(int logn, int n_rows);
// Tables of the split-band form with local length 2^logm (N = 2^logm P).
void split_prop_table(const bpm_plan_s* plan, int row, int logm, std::vector<float2>* out);
// the same tables for a propagation of frac * dz (a stage of Eq. split-op)
void split_prop_table_frac(const bpm_plan_s* plan, int row, int logm, double frac,
                           std::vector<float2>* out);
int split_table_stride(const bpm_plan_s* plan, int logm);   // float2 per row
// Layout codes of launch_fused_layout: -1 rule, 0 CTA per row, 1 2-CTA
// cluster per row, 2 4-CTA cluster per row (N = 4096, half-band split, 8
// points per thread).
constexpr int kLayoutSplit4 = 2;
// one CTA per row, second-order (Verlet) step, N <= 4096
constexpr int kLayoutCtaHalf = 3;
// one 2-CTA cluster per row, second-order (Verlet) step, N = 512..4096
constexpr int kLayoutClusterHalf = 4;
// one 4-CTA cluster per row (N = 4096 half-band split), second-order step
constexpr int kLayoutSplit4Half = 5;
// one CTA per row, fourth-order (Forest-Ruth) step, N <= 4096
constexpr int kLayoutCtaFR = 6;
// the fourth-order step stage by stage (N = 16384; N = 8192 when
// BPM_FUSED_LAYOUT=staged): a coupling launch and three one-step launches
// of the split-band kernels per step
constexpr int kLayoutStagedFR = 7;
// one 4-CTA cluster per row (N = 4096 half-band split) with 16 points per
// thread (fused4e_march_kernel<11>); layout 2 runs the 8-point form
// (fused4s_kernel.cuh), measured 5 % faster
constexpr int kLayoutSplit4S = 8;
// fourth-order (Forest-Ruth) step on one 4-CTA cluster per row: the N = 4096
// half-band split (8 points per thread) or the N = 8192 split band
constexpr int kLayoutSplit4FR = 9;
// one 2-CTA cluster per row, fourth-order (Forest-Ruth) step, N = 512..4096
constexpr int kLayoutClusterFR = 10;
// Coupling alone (the leading coupling of a step), on rows[0..nb): each row's
// state [2][nx], the slice of step n of its stream (stored per part for
// nx >= 8192), coefficients (am1h, bh).
int launch_couple_only(const RowDescF32* d_rows, int nb, int nx, int n, cudaStream_t st);
int fused_launch_capacity(int logn, bool cluster);
int fused_split4_capacity();
int fused_half_capacity(int logn);   // logn <= 12
int fused_fr_capacity(int logn);     // logn <= 12
int fused_cluster_half_capacity(int logn);   // 9 <= logn <= 12
int fused_cluster_fr_capacity(int logn);     // 9 <= logn <= 12
int fused_split4_half_capacity();            // N = 4096
int fused_split4_fr_capacity();              // N = 4096
// Positions of the Forest-Ruth stage tables in the split kernels' thread
// order (logn 12: the half-band split, 13: the split band), M per band table.
int fr_split_table_order(int logn, std::vector<int>* pos);
// ... and of the one-CTA kernels (thread order for 256 <= nx <= 4096,
// position order below), nx per band table.
int fr_cta_table_order(int logn, std::vector<int>* pos);
int fused_rows_per_cta(int logn);
int fused_threads(int logn);

}  // namespace bpm
