/*
 * bpm.h -- C ABI of the GB300 (sm_103a) two-beam FFT beam-propagation march.
 *
 * Method: Krzywinski & Halavanau, arXiv 2601.06340, Section 2.  Two slowly
 * varying envelopes psi_+ (transmitted) and psi_- (reflected) (Eqs. fov6-7)
 * are advanced in z by the first-order split step of Eq. fov10: each band is
 * propagated through its own angular-spectrum operator exp(i dz^ sqrt(1 -
 * kx^2)) centred on its carrier (forward FFT, multiply, inverse FFT), then
 * the two are coupled in real space through chi_0, chi_h (Eqs. fov8,
 * fov11-12), the strain phase h*u_x (Eq. Authier) and the crystal mask Pi.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Units: lengths in micrometres, angles in radians, energies in eV.
 * Grid: x_j = x0 + j*dx (j < nx), z_n = n*dz; the mask and strain of step n
 *   are sampled at z_n (start of the step).
 * Complex numbers are interleaved (re, im).  "c128" = 2 doubles, "c64" = 2
 *   floats.
 * Field layout: [B][2][nx], B = number of photon energies (batch rows), band
 *   0 = psi_+, band 1 = psi_-.  Records: [B][n_rec][2][nx] with
 *   n_rec = nz / record_every (0 when record_every = 0); record i is the
 *   state after step (i+1)*record_every.  Powers: [B][n_rec+1][2] doubles,
 *   P = dx * sum_j |psi_j|^2 per band, at each record and (last entry) for
 *   the returned state.
 * Precision: BPM_FP64_PLAIN marches complex128 with one kernel launch per
 *   FFT pass and per pointwise step; BPM_FP32_FUSED marches complex64 in a
 *   persistent kernel that keeps each row on chip for many steps, with every
 *   phase argument (propagator, strain phase, common phase) formed in FP64
 *   and rounded once.  FP32 plans return c64 records; FP64 plans c128.
 * Errors: every call returns a bpm_status; negative values are errors and
 *   bpm_last_error() (thread-local) describes the last one.  Nothing aborts
 *   the process.  Arguments are validated on the host before any device
 *   work, so an invalid call leaves the plan unchanged.
 * Ownership: the caller owns every pointer it passes.  bpm_plan and
 *   bpm_set_* copy what they need before returning.  The plan owns all
 *   device memory it allocates and frees it in bpm_destroy.
 * Threading: calls on one plan are serialised by the plan's lock; distinct
 *   plans may be used from different threads.
 */
#ifndef BPM_H
#define BPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bpm_plan_s* bpm_plan_t;
typedef uint64_t bpm_ticket_t;

enum bpm_status {
  BPM_OK = 0,
  BPM_NOT_READY = 1,     /* bpm_poll: ticket still running (not an error) */
  BPM_ERR_INVALID = -1,  /* bad argument; nothing was changed              */
  BPM_ERR_OOM = -2,      /* device allocation failed or over the budget   */
  BPM_ERR_CUDA = -3,     /* a CUDA call failed (message in last_error)    */
  BPM_ERR_BUSY = -4,     /* plan has pending tickets, or queue is full    */
  BPM_ERR_TIMEOUT = -5,  /* a bounded device wait gave up                 */
  BPM_ERR_NUMERIC = -6   /* a non-finite power appeared in the result     */
};

enum bpm_precision { BPM_FP64_PLAIN = 0, BPM_FP32_FUSED = 1 };

/* Crystal shape Pi(x, z) (Eqs. fov11-12: 1 inside, 0 outside; Section 4
 * for the slab and its asymmetry angle, Section 7 for arbitrary shapes). */
enum bpm_crystal_kind {
  BPM_CRYSTAL_VACUUM = 0,          /* Pi = 0 everywhere (free space)        */
  BPM_CRYSTAL_BULK = 1,            /* Pi = 1 everywhere                     */
  BPM_CRYSTAL_SLAB = 2,            /* slab of thickness T, see set_crystal  */
  BPM_CRYSTAL_MASK = 3,            /* user map [nz][nx], nonzero = inside   */
  BPM_CRYSTAL_SLAB_AND_MASK = 4,   /* slab AND user map                     */
  BPM_CRYSTAL_SLAB_AND_POLYGON = 5, /* slab AND polygon (even-odd rule)     */
  BPM_CRYSTAL_BOX = 6              /* 3D plans: box, see set_crystal_box    */
};

/* Displacement u_x(x, z) entering as exp(+-i h u_x) (Eq. Authier). */
enum bpm_strain_kind {
  BPM_STRAIN_NONE = 0,
  BPM_STRAIN_ARRAY = 1,            /* u_x[nz][nx] in um                       */
  BPM_STRAIN_BENT = 2,             /* Eq. fov110, configured form, see below  */
  BPM_STRAIN_EDGE_DISLOCATION = 3  /* Eq. fov120 with b along x, see below    */
};

typedef struct {
  int32_t nx;              /* transverse points: power of two in [8, 16384]    */
  int32_t nz;              /* z steps in the plan's march: >= 1                */
  double dx_um;            /* > 0                                              */
  double dz_um;            /* > 0                                              */
  double x0_um;            /* x of the first cell                              */
  int32_t n_energy;        /* B >= 1 batch rows (photon energies)              */
  const double* energy_ev; /* [B] photon energies (copied)                     */
  double e_ref_ev;         /* energy at which theta_b_ref_rad is the Bragg     */
  double theta_b_ref_rad;  /*   angle; fixes d = lambda(E_ref) / (2 sin theta) */
  double chi0_re, chi0_im; /* chi_0 (Eq. fov8)                                 */
  double chih_re, chih_im; /* chi_h (Eq. fov8), used as given (no sign fix-up) */
  int32_t record_every;    /* zsep: record every k steps; 0 = no records       */
  int32_t precision;       /* enum bpm_precision                               */
} bpm_problem;

/* Create a plan: per-energy constants of Eqs. fov4-fov12 in FP64 (wave
 * number, s = sin theta_B(E) = lambda/2d, cos(alpha) = sqrt(1 - s^2), dz^,
 * the Jacobi-Anger coefficients J0(w)e^{i phi0}, i J1(w)e^{i phi0} with
 * w = dz^ chi_h / cos(alpha), phi0 = dz^ chi_0 / (2 cos(alpha)), each band's
 * propagator table) and the device buffers.  The crystal starts as VACUUM
 * and the strain as NONE.  Returns BPM_ERR_INVALID for a bad problem
 * (including an evanescent band, 1 - (|q| + s)^2 <= 0), BPM_ERR_OOM if
 * device memory runs out, BPM_ERR_CUDA without a usable device. */
int bpm_plan(const bpm_problem* problem, bpm_plan_t* out);

/* Set the crystal shape.  Slab: unit normal n = (cos a, sin a) in (x, z)
 * (a = asym_angle_rad: 0 = Bragg, pi/2 = Laue, between = asymmetric;
 * components below 1e-12 in magnitude are set to 0), surface point
 * r_s = (surf_x_um, surf_z_um), inside = {0 <= n.(r - r_s) <= thickness}.
 * mask: uint8 [nz][nx] (row n = z_n), nonzero = inside, for MASK and
 * SLAB_AND_MASK, else ignored (may be NULL).  poly_xz_um: nv vertices
 * (x, z) in order, nv >= 3, for SLAB_AND_POLYGON, else ignored.  A cell is
 * inside when its centre is (even-odd rule; an edge is crossed when exactly
 * one end lies above z and x is left of its crossing point).  The decision
 * is taken in FP64 with the operations in the documented order and no
 * fused multiply-add. */
int bpm_set_crystal(bpm_plan_t plan, int32_t kind, double asym_angle_rad,
                    double thickness_um, double surf_x_um, double surf_z_um,
                    const uint8_t* mask, const double* poly_xz_um, int32_t nv);

/* Set the displacement.  ux_um: [nz][nx] doubles for ARRAY, else ignored.
 * params (n_params values) for the parametric kinds:
 *   BENT:  {R_um, nu, x_ref_um, z_ref_um}:
 *          u_x = ((x - x_ref)^2 + nu (z - z_ref)^2) / (2 R)
 *   EDGE_DISLOCATION: {b_um, nu, x_core_um, z_core_um}: with x' = x - x_core,
 *          z' = z - z_core, u_x = b/(2 pi) [atan2(z', x')
 *                              + x' z' / (2 (1 - nu) (x'^2 + z'^2))],
 *          u_x = 0 at the core itself.
 * The strain phase h u_x (h = 2 pi / d, d from bpm_problem) is formed in
 * FP64, reduced modulo 2 pi, and turned into exp(i h u_x) once, on the
 * device; the march streams that phasor (c64 or c128 per cell). */
int bpm_set_strain(bpm_plan_t plan, int32_t kind, const double* ux_um,
                   const double* params, int32_t n_params);

/* Operator splitting of Eq. split-op: the step applies
 * A(a_1 dz) B(b_1 dz) A(a_2 dz) B(b_2 dz) ... in that order (A: the
 * angular-spectrum propagation of each band, B: the coupling of Eqs.
 * fov11-fov12 formed for a step of b_i dz), every stage of step n with the
 * mask and strain of z_n.
 *   BPM_SPLIT_FIRST_ORDER: a = (1), b = (1), Eq. fov10 (the default);
 *   BPM_SPLIT_VERLET:      a = (0, 1), b = (1/2, 1/2);
 *   BPM_SPLIT_FOREST_RUTH: a = (0, t, 1-2t, t), b = (t/2, (1-t)/2, (1-t)/2,
 *                          t/2), t = 1/(2 - 2^(1/3)).
 * FP64 plans take every method.  FP32 (fused) plans take the first-order
 * step, and for nx <= 4096 Verlet (half-step couplings on either side of
 * the full-step propagation; at nx = 4096 one 4-CTA half-band split per
 * solve while every solve gets four SMs, else one 2-CTA cluster per solve
 * while every solve gets two SMs and 512 <= nx != 2048, else one CTA per
 * solve) and Forest-Ruth (the leading coupling, then three
 * propagate-and-couple stages with the propagator increments of t dz and
 * (1 - 2t) dz, tabulated here once; at nx = 4096 one 4-CTA half-band split
 * per solve while every solve gets four SMs, for 512 <= nx <= 4096 one
 * 2-CTA cluster per solve while every solve gets two SMs, else one CTA per
 * solve), for
 * nx = 8192 Verlet and Forest-Ruth on one split-band cluster per solve, and
 * for nx = 16384 Verlet (one split-band cluster per solve) and Forest-Ruth
 * stage by stage (per step a coupling launch and three one-step launches
 * of the first-order split-band kernel with the stage's tables; several
 * times slower, and refused under stream capture; BPM_FUSED_LAYOUT=staged
 * takes it at nx = 8192 too); 3D plans take the first-order step
 * and Verlet (the row kernel, which holds both bands of a line, applies the
 * half-step couplings); other combinations return BPM_ERR_INVALID.
 * bpm_submit takes FP32 plans set to Verlet or Forest-Ruth: their rows
 * march in their own launch groups, one CTA per row for nx <= 4096 and one
 * split-band cluster per row for nx = 8192 (and 16384, Verlet); Forest-Ruth
 * plans of nx = 16384 are refused there (BPM_ERR_INVALID).
 * BPM_ERR_BUSY while tickets are pending. */
enum bpm_splitting {
  BPM_SPLIT_FIRST_ORDER = 0,
  BPM_SPLIT_VERLET = 1,
  BPM_SPLIT_FOREST_RUTH = 2
};
int bpm_set_splitting(bpm_plan_t plan, int32_t method);

/* 3D plans: the march of Eq. fov4 with both transverse coordinates (x, y)
 * and the two-beam envelopes of Eqs. fov6-fov10 (the Bragg shift k_d/2 is
 * along x only): each band goes through exp(i dz^ sqrt(1 - (qx +- s)^2 -
 * qy^2)), qy = 2 pi fftfreq(ny, dy^), and the coupling is pointwise in (x, y)
 * (Sec. 2; the paper's 3D cases, Sec. 7).  `problem` as for bpm_plan with
 * precision BPM_FP32_FUSED and nx a power of two in [256, 4096]; ny a power
 * of two in [256, 1024], dy_um > 0, y0_um the y of the first cell.  Every
 * field of the other calls then carries [ny][nx] per band: psi [B][2][ny][nx],
 * records [B][n_rec][2][ny][nx], mask and u_x arrays [nz][ny][nx]; band
 * powers are dx dy sum |psi|^2.  The 2D crystal kinds and strain fields apply
 * at every y.  bpm_submit does not take 3D plans (BPM_ERR_INVALID). */
int bpm_plan3d(const bpm_problem* problem, int32_t ny, double dy_um, double y0_um,
               bpm_plan_t* out);

/* 3D plans: a box crystal, inside = {x0 <= x <= x1, y0 <= y <= y1,
 * z0 <= z <= z1} at the cell centres (x_j, y_i, z_n), box_um = {x0, x1, y0,
 * y1, z0, z1} (FP64 comparisons).  BPM_ERR_INVALID for a 2D plan or
 * non-finite bounds. */
int bpm_set_crystal_box(bpm_plan_t plan, const double* box_um);

/* March rows [0, B) from the state after n_begin steps to the state after
 * n_end steps (0 <= n_begin < n_end <= nz) and copy results to the host.
 * psi_in / psi_out: host c128 [B][2][nx] (may alias).  records: host buffer
 * laid out [B][n_rec][2][nx] (c64 for FP32 plans, c128 for FP64 plans) or
 * NULL; only records with index in [n_begin/k, n_end/k) are written.
 * powers: host double [B][n_rec+1][2] or NULL (same slots as records; the
 * last slot is the returned state).  Synchronous.  BPM_ERR_NUMERIC if a
 * power is not finite (outputs are still written). */
int bpm_propagate(bpm_plan_t plan, const double* psi_in, double* psi_out,
                  void* records, double* powers, int32_t n_begin,
                  int32_t n_end);

/* Same march on device buffers, asynchronous on `stream` (a cudaStream_t;
 * NULL = legacy default stream).  d_psi_in / d_psi_out: [B][2][nx], c64 for
 * FP32 plans and c128 for FP64 plans (may alias).  d_records: device
 * buffer as in bpm_propagate or NULL.  d_powers: device double
 * [B][n_rec+1][2] or NULL.  The call returns after enqueueing; the caller
 * synchronises the stream before reading outputs or freeing inputs.
 * Marches of one plan share its device scratch (row descriptors, phase
 * factors, the FP64 state): enqueue them on one stream, or order the
 * streams.  An expired bounded wait inside a march is reported by
 * bpm_device_status (or by the plan's next bpm_propagate).  Graph capture:
 * FP32 plans (2D and 3D) may be captured into a CUDA graph once they have
 * marched outside a capture (strain slices prepared, schedule buffers
 * sized); the march's per-call uploads then travel as kernel parameters,
 * so a replay repeats the captured march (same buffers, steps and launch
 * shape -- the fixed rule's).  While `stream` is capturing, FP64 plans,
 * Forest-Ruth plans that march stage by stage (nx = 16384, or 8192 with
 * BPM_FUSED_LAYOUT=staged) and plans not yet marched return BPM_ERR_INVALID
 * and enqueue nothing. */
int bpm_propagate_device(bpm_plan_t plan, const void* d_psi_in,
                         void* d_psi_out, void* d_records, void* d_powers,
                         int32_t n_begin, int32_t n_end, void* stream);

/* Status of the plan's device marches so far: reads the plan's status word
 * on `stream` (after the work enqueued there), waits for it and clears it.
 * BPM_ERR_TIMEOUT if a bounded device wait (strain-slice copy or peer-CTA
 * data) expired in one of them, else BPM_OK; BPM_ERR_INVALID for a NULL
 * plan, BPM_ERR_CUDA if the stream failed.  Blocks the host. */
int bpm_device_status(bpm_plan_t plan, void* stream);

/* Energy -> time synthesis of a batch of exit fields (Section
 * "Time-Dependent Simulation"): out[b][x][m] = sum_j in[j][b][x]
 * exp(-2 pi i j m / B) over the B rows (energies E_j = E_0 + j dE,
 * ascending), i.e. the superposition of the monochromatic solutions with
 * time dependence exp(-i omega_j t) (Eq. fov4: a forward wave advances by
 * exp(+i k dz)) relative to the carrier exp(-i omega_0 t), sampled at
 * t_m = m h / (B dE).  B a power of two in [2, 4096].  Device buffers, c64
 * if precision == BPM_FP32_FUSED else c128; in: [B][2][nx], out:
 * [2][nx][B].  Asynchronous on stream. */
int bpm_omega_to_t_device(const void* d_in, void* d_out, int32_t n_energy,
                          int32_t nx, int32_t precision, void* stream);

/* Continuous-batching server.  bpm_submit enqueues a full march (steps
 * [0, nz)) of the plan's B rows with input psi_in (host c128 [B][2][nx],
 * copied before return); outputs as in bpm_propagate and must stay valid
 * until bpm_poll returns BPM_OK or an error.  Requests are admitted as
 * device memory (within the configured budget) and launch slots free up;
 * admitted requests advance together in epochs of fused launches, grouped by
 * transverse size.  A plan carries at most one request at a time.
 * BPM_ERR_BUSY if the queue is full or the plan already has a request in
 * flight; BPM_ERR_OOM if the request alone exceeds the memory budget.
 * bpm_poll waits up
 * to timeout_ms (0 = just test, <0 = wait forever) and returns BPM_OK once
 * (outputs written), BPM_NOT_READY, or the request's error. */
int bpm_submit(bpm_plan_t plan, const double* psi_in, double* psi_out,
               void* records, double* powers, bpm_ticket_t* out);
int bpm_poll(bpm_ticket_t ticket, int32_t timeout_ms);

/* Server settings (call before the first submit or when idle):
 * mem_fraction of the device's free memory usable for admitted requests
 * (0 < f <= 0.9), max_active admitted requests, epoch_steps z steps per
 * epoch launch, max_queue pending requests.  Values <= 0 keep defaults
 * (0.6, 256, 256, 100000). */
int bpm_server_configure(double mem_fraction, int32_t max_active,
                         int32_t epoch_steps, int32_t max_queue);

/* Test hook (no counterpart in the paper): the next `count` batch launches of
 * FP32 requests with transform size nx fail on the host with BPM_ERR_CUDA
 * instead of launching, as a failed kernel launch would.  The requests of
 * that size in those batches (and the others sharing their bucket at that
 * moment) then end with BPM_ERR_CUDA; requests of other sizes are not
 * affected and the server takes new requests of the size afterwards.
 * count = 0 clears it.  BPM_ERR_INVALID for a bad nx or count < 0. */
int bpm_server_inject_launch_failure(int32_t nx, int32_t count);

/* Timestamps (seconds, steady clock) of a finished or running ticket:
 * submit, admission to the device, completion (0 while not reached). */
int bpm_ticket_times(bpm_ticket_t ticket, double* t_submit, double* t_admit,
                     double* t_done);

/* Copy the plan's prepared slices to the host: mask uint8 [nz][nx] (1 =
 * inside) and/or the strain phasor exp(i h u_x) as c128 [nz][nx] (0 outside
 * the crystal).  Either pointer may be NULL.  For inspection and tests. */
int bpm_fetch_slices(bpm_plan_t plan, uint8_t* mask, double* phasor);

/* Form of the plan's prepared slices (the crystal mask Pi and the strain
 * phasor of Eq. fov10 per step).  *form = 1: separable -- FP32 2D plans of a
 * vacuum, bulk or slab crystal with no strain or the bent-crystal strain,
 * whose phase h u = h x'^2/(2R) + h nu z'^2/(2R) is a column term plus a row
 * term: the plan keeps one row per z-step (the inside interval and the row
 * phasor, 96 bytes) and one phasor per column, and the fused kernels form
 * each cell's phasor (column x row inside the interval, 0 outside) as they
 * couple; 0: the per-cell stream (c64 per cell for FP32 plans, c128 for
 * FP64 plans); -1: not prepared yet (slices are prepared at the first march
 * after bpm_set_crystal / bpm_set_strain).  Eligible plans take the
 * separable form where it pays: nx = 4096 first-order plans while 4 x rows
 * <= the GPU's SM count (the half-band split), nx >= 8192 while 2 x rows <=
 * the SM count
 * (a stream of 8 B per cell: 2.6 GB for 16384 x 20000); smaller nx and
 * batches that fill the GPU keep the stream (faster there; a batch shares
 * it among its rows).  BPM_SLICE_STREAM=1 (0) in the environment when the
 * slices are prepared forces the stream (the separable) form of eligible
 * plans.  The
 * two forms hold the same cells bit for bit (bpm_fetch_slices); the kernels
 * fold the row phasor into the coupling coefficient, so marches agree to
 * FP32 rounding.  *bytes = the device bytes of the slice data.  Either
 * pointer may be NULL.  BPM_ERR_INVALID for a NULL plan. */
int bpm_slice_form(bpm_plan_t plan, int32_t* form, int64_t* bytes);

/* Allocation-free FP64 march.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory -- code that
 * runs where cudaMalloc is not allowed or not wanted (a host callback, a
 * process whose device memory is owned by another allocator or budget, an
 * embedding that must not grow its footprint after start-up).  It advances
 * caller-owned device buffers with the plain FP64 step of bpm_propagate
 * (one launch per Stockham pass, propagator and coupling) and calls no
 * cudaMalloc, cudaFree or allocating library routine: its working memory
 * (16 MiB ping-pong buffer, 8192-entry twiddle table, 1024 row descriptors)
 * lives in static device arrays that every GPU loading this library holds
 * until the process exits.
 *   d_psi      [n_rows][2][nx] c128, in/out: the state after n_begin steps
 *              becomes the state after n_end steps WITHOUT the common phase
 *              exp(i dz^ cos(alpha)) per step (bpm_propagate_device includes
 *              it: multiply by exp(i (n_end-n_begin) dz^ cos(alpha)) to
 *              compare);
 *   d_prop     [n_rows][2][nx] c128: exp(i dz^ delta_+-(q_m)) / nx per band,
 *              natural FFT order, q_m = 2 pi fftfreq(nx, dx^) (band 0 uses
 *              q + s, band 1 q - s);
 *   d_coupling [n_rows][2] c128: (Delta_eps_0, Delta_eps_{+-1}) inside Pi;
 *   d_phasor   [>= n_end][nx] c128: exp(i h u_x) per cell, (0,0) outside.
 * Limits: nx a power of two in [8, 8192], 1 <= n_rows <= 1024 and
 * n_rows * 2 * nx <= 2^20; other sizes return BPM_ERR_INVALID before any
 * device work.  Asynchronous on `stream`.  The first call on a device looks
 * up the arrays' device addresses (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  All calls share
 * the arrays, and each rewrites what it reads, so calls that overlap on the
 * GPU race. */
int bpm_march_f64_noalloc(void* d_psi, int32_t nx, int32_t n_rows, const void* d_prop,
                          const void* d_coupling, const void* d_phasor, int32_t n_begin,
                          int32_t n_end, void* stream);

/* Launch shape of the plan's last FP32 march (the fused kernels of the
 * step of Eq. fov10): *layout = 10 the Forest-Ruth step on one 2-CTA
 * cluster per row (512 <= nx <= 4096, while every row gets two SMs), 9 the
 * Forest-Ruth step on one 4-CTA
 * cluster per row (nx = 4096 half-band split, while every row gets four
 * SMs; nx = 8192 split band), 8 the nx = 4096 half-band split with 16
 * points per thread (forced by BPM_FUSED_LAYOUT=split16), 7 the Forest-Ruth
 * step stage by stage (nx = 16384, or nx = 8192 with
 * BPM_FUSED_LAYOUT=staged), 6 one CTA per row with the Forest-Ruth step (plans set to
 * BPM_SPLIT_FOREST_RUTH), 5 one split-band cluster per row with
 * the Verlet step (nx = 4096, 8192, 16384), 4 one 2-CTA cluster per row with the Verlet
 * step, 3 one CTA per row with the Verlet step (plans set to
 * BPM_SPLIT_VERLET), 2 one 4-CTA cluster per row (nx = 4096 as
 * two half-band parts per band; the rule while every row gets four SMs),
 * 1 one 2-CTA cluster per row, 0 one CTA per row, -1 chosen by the fixed
 * rule (2-CTA cluster while every row gets two SMs, else one CTA per row);
 * *chunk = steps per launch of the rotation schedule (more rows than one
 * launch keeps resident), 0 for a single launch.  A batch march with a
 * choice of shapes (the layouts above for up to one row per two SMs at
 * 512 <= nx <= 4096, or rotation chunks of 64..512 steps) times each on a
 * short march of a scratch copy of the state the first time a given
 * (nx, rows) is marched, blocking the host for those trials, and keeps the
 * fastest for the process; BPM_AUTOTUNE=0 in the environment or a single
 * row leaves the fixed rule in charge.  Either
 * pointer may be NULL.  BPM_ERR_INVALID for a NULL plan. */
int bpm_launch_shape(bpm_plan_t plan, int32_t* layout, int32_t* chunk);

/* Release the plan and its device memory.  BPM_ERR_BUSY while tickets of
 * the plan are pending. */
int bpm_destroy(bpm_plan_t plan);

/* Message for the calling thread's last error ("" if none). */
const char* bpm_last_error(void);

/* Library version string. */
const char* bpm_version(void);

/* Self-test of the bounded device wait that every march kernel uses on its
 * mbarriers (strain-slice copies, peer data).  No counterpart in the paper.
 * One CTA arms a barrier for bytes that no copy delivers and waits with the
 * march kernels' bounded loop, which gives up without any fault; the kernel
 * then sets the status bit that a march would report as BPM_ERR_TIMEOUT.
 * *status receives that word (1: the wait expired and the kernel returned),
 * *seconds the kernel's duration (the wait limit).  Blocks the host until
 * the kernel ends.  BPM_ERR_INVALID for NULL pointers, BPM_ERR_CUDA if the
 * launch failed. */
int bpm_selftest_wait_expiry(int32_t* status, double* seconds);

/* Measured arithmetic peak of the current device: the denominator of the
 * march kernels' roofline fractions (the march is bound by FP32 ALU work;
 * FP64 explains the plain path).  No counterpart in the paper.  Every SM
 * runs eight 256-thread CTAs whose threads each carry eight independent
 * multiply-add chains for iters x 16 rounds; one FMA is two flops (a packed
 * FFMA2 four).  *flops_per_s receives the rate of the timed launch (after a
 * warm-up launch of iters / 8 rounds), *seconds its CUDA-event duration, at
 * whatever clock the GPU runs.  Blocks the host.  BPM_ERR_INVALID for NULL
 * pointers, an unknown kind or iters outside [1, 2^22]; BPM_ERR_CUDA if a
 * launch failed. */
enum bpm_peak_kind {
  BPM_PEAK_FP64_DFMA = 0,
  BPM_PEAK_FP32_FFMA = 1,
  BPM_PEAK_FP32_FFMA2 = 2
};
int bpm_fp_peak(int32_t kind, int32_t iters, double* flops_per_s, double* seconds);

#ifdef __cplusplus
}
#endif

#endif /* BPM_H */
