// C ABI: plan lifetime, crystal/strain description, synchronous and
// stream-ordered marches.  See include/bpm.h for the contract.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "bpm_internal.h"

namespace bpm {

static thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();  // clear a sticky-free error so later calls start clean
  return e == cudaErrorMemoryAllocation ? BPM_ERR_OOM : BPM_ERR_CUDA;
}

namespace {

struct DevAlloc {
  std::vector<void**> owned;
};

int dev_alloc(bpm_plan_s* plan, void** p, size_t bytes, const char* what) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? BPM_ERR_OOM : BPM_ERR_CUDA,
                std::string("cudaMalloc(") + what + ", " + std::to_string(bytes) +
                    " bytes): " + cudaGetErrorString(e));
  }
  plan->device_bytes += bytes;
  return BPM_OK;
}

void free_plan_memory(bpm_plan_s* plan) {
  vol_release(plan);
  void** ptrs[] = {&plan->d_phasor, &plan->d_sep, &plan->d_prop, &plan->d_prop_split, &plan->d_tw, &plan->d_state,
                   &plan->d_state2, &plan->d_rows, &plan->d_io, &plan->d_spec,
                   &plan->d_twy, reinterpret_cast<void**>(&plan->d_pwpart),
                   &plan->d_stage_rows, &plan->d_stage_prop, &plan->d_stage_prop_split};
  for (void** p : ptrs) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  if (plan->d_status) cudaFree(plan->d_status);
  plan->d_status = nullptr;
}

size_t csize(const bpm_plan_s* plan) { return plan->precision == BPM_FP32_FUSED ? 8 : 16; }

// float2 per row of the fused propagator tables (the split form of
// N = 8192 carries a third table per band)
size_t prop_stride(const bpm_plan_s* plan) {
  if (plan->precision == BPM_FP32_FUSED && plan->ny <= 1 && plan->logn >= kSplitLogN)
    return size_t(split_table_stride(plan, 12));
  return 2 * size_t(plan->nx) * (plan->ny > 1 ? plan->ny : 1);
}

int device_sm_count() {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

}  // namespace

inline PlanAux* aux_of(bpm_plan_s* plan) { return &plan->aux; }

// float2 per Forest-Ruth stage table of one row: (P^a - 1)/N per band in the
// fused FFT's output order, or the split-band tables for nx >= 8192
size_t fr_table_stride(const bpm_plan_s* plan) {
  return plan->logn >= kSplitLogN ? size_t(split_table_stride(plan, 12)) : 2 * size_t(plan->nx);
}

// Build the fused row descriptors for rows [0, B) of `plan`.
void fused_rows(bpm_plan_s* plan, float2* state, float2* rec, double* pw, int n_begin,
                int n_end, std::vector<RowDescF32>* out) {
  out->resize(plan->nb);
  const size_t n = plan->nx;
  for (int r = 0; r < plan->nb; ++r) {
    RowDescF32& d = (*out)[r];
    d.state = state + size_t(r) * 2 * n;
    d.prop = static_cast<const float2*>(plan->d_prop) + size_t(r) * prop_stride(plan);
    if (plan->split == BPM_SPLIT_FOREST_RUTH)   // [2 tables][table] per row: t dz, (1-2t) dz
      d.prop = static_cast<const float2*>(plan->d_stage_prop) + size_t(r) * 2 * fr_table_stride(plan);
    d.prop_split = plan->d_prop_split ? static_cast<const float2*>(plan->d_prop_split) +
                                            size_t(r) * split_table_stride(plan, 11)
                                      : nullptr;
    if (plan->split == BPM_SPLIT_FOREST_RUTH && plan->d_stage_prop_split)
      // [2 tables][split table in thread order] per row: t dz, (1 - 2t) dz
      d.prop_split = static_cast<const float2*>(plan->d_stage_prop_split) +
                     size_t(r) * 2 * split_table_stride(plan, plan->logn == kSplitLogN ? 12 : 11);
    if (plan->sep_slices) {
      d.phasor = nullptr;
      d.srows = static_cast<const SepRow*>(plan->d_sep);
      d.scols = reinterpret_cast<const float2*>(d.srows + plan->nz);
    } else {
      d.phasor = static_cast<const float2*>(plan->d_phasor);
      d.srows = nullptr;
      d.scols = nullptr;
    }
    d.records = rec ? rec + size_t(r) * plan->n_rec * 2 * n : nullptr;
    d.powers = pw ? pw + size_t(r) * (plan->n_rec + 1) * 2 : nullptr;
    const EnergyConsts& c = plan->ec[r];
    d.am1 = make_float2(float(c.am1.real()), float(c.am1.imag()));
    d.b = make_float2(float(c.b.real()), float(c.b.imag()));
    if (plan->split == BPM_SPLIT_VERLET || plan->split == BPM_SPLIT_FOREST_RUTH) {
      // Verlet: (am1h, bh) for half a step.  Forest-Ruth: (am1h, bh) for the
      // outer couplings (t/2), (am1, b) for the two inner ones ((1 - t)/2).
      const auto stg = split_stages(plan->split);
      std::complex<double> ah, bh;
      coupling_frac(plan, r, stg.front().second, &ah, &bh);
      d.am1h = make_float2(float((ah - 1.0).real()), float((ah - 1.0).imag()));
      d.bh = make_float2(float(bh.real()), float(bh.imag()));
      if (plan->split == BPM_SPLIT_FOREST_RUTH) {
        coupling_frac(plan, r, stg[1].second, &ah, &bh);
        d.am1 = make_float2(float((ah - 1.0).real()), float((ah - 1.0).imag()));
        d.b = make_float2(float(bh.real()), float(bh.imag()));
      }
    } else {
      d.am1h = d.am1;
      d.bh = d.b;
    }
    d.gphase = c.gphase;
    d.dx_um = plan->dx_um;
    d.n_begin = n_begin;
    d.n_end = n_end;
    d.n_phase0 = n_begin;
    d.record_every = (rec || pw) ? plan->record_every : 0;
  }
}

// Common phase g^(steps) per row in FP64.
void phase_factors(const bpm_plan_s* plan, int steps, std::vector<double2>* out) {
  out->resize(plan->nb);
  for (int r = 0; r < plan->nb; ++r) {
    double ang = std::fmod(double(steps) * plan->ec[r].gphase, kTwoPi);
    (*out)[r] = make_double2(std::cos(ang), std::sin(ang));
  }
}

// More rows than the GPU keeps resident: split the march into equal chunks
// and issue launches of exactly `resident` (row, chunk) items taken in
// round-robin order (item i = row i mod B, chunk i div B).  Every launch is
// full, each row's chunks run in order (item i + B lands in a later launch),
// no row appears twice in a launch, and rows sweeping the same z-range share
// their strain slices in L2.  A remainder shorter than a chunk runs as a
// second round of the same kind.
// Host-to-device upload on the march's stream: a plain async copy, or, while
// the stream is being captured into a graph, kernel parameters (which the
// graph keeps; a captured copy would re-read the host memory at replay).
static bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return cs != cudaStreamCaptureStatusNone;
}

static int upload(void* dst, const void* src, size_t bytes, cudaStream_t st, bool captured,
                  const char* what) {
  if (captured) return upload_by_params(dst, src, bytes, st);
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
  return e == cudaSuccess ? BPM_OK : cuda_fail(e, what);
}

static int launch_rotated(bpm_plan_s* plan, PlanAux* aux, const std::vector<RowDescF32>& rows,
                          int n_begin, int steps, int resident, cudaStream_t st, int chunk = 0,
                          int layout = -1) {
  const int nb = plan->nb;
  if (chunk <= 0) chunk = std::max(std::min(steps, 64), steps / 24);
  chunk = std::min(chunk, steps);
  const int full = steps / chunk, rem = steps - full * chunk;
  std::vector<RowDescF32> sched;
  struct Launch { size_t off; int count; int steps; };
  std::vector<Launch> launches;
  auto round = [&](int c0, int c1, int len) {
    const long items = long(nb) * (c1 - c0);
    for (long i = 0; i < items; i += resident) {
      const int cnt = int(std::min<long>(resident, items - i));
      launches.push_back({sched.size(), cnt, len});
      for (int k = 0; k < cnt; ++k) {
        const long it = i + k;
        RowDescF32 d = rows[it % nb];
        d.n_begin = n_begin + int(c0 + it / nb) * chunk;
        d.n_end = d.n_begin + len;
        sched.push_back(d);
      }
    }
  };
  round(0, full, chunk);
  if (rem > 0) round(full, full + 1, rem);
  const bool captured = capturing(st);
  if (aux->sched_cap < sched.size()) {
    if (captured)
      return fail(BPM_ERR_INVALID,
                  "march the plan once outside the graph capture first (launch schedule)");
    if (aux->d_sched) cudaFree(aux->d_sched);
    aux->d_sched = nullptr;
    aux->sched_cap = 0;
    int rc = dev_alloc(plan, reinterpret_cast<void**>(&aux->d_sched),
                       sched.size() * sizeof(RowDescF32), "launch schedule");
    if (rc != BPM_OK) return rc;
    aux->sched_cap = sched.size();
  }
  int urc = upload(aux->d_sched, sched.data(), sched.size() * sizeof(RowDescF32), st, captured,
                   "upload launch schedule");
  if (urc != BPM_OK) return urc;
  for (const Launch& l : launches) {
    int rc = launch_fused_layout(plan->logn, aux->d_sched + l.off, l.count, l.steps,
                                 static_cast<const float4*>(plan->d_tw), plan->d_status, st,
                                 layout);
    if (rc != BPM_OK) return rc;
  }
  return BPM_OK;
}

// ---- launch-shape autotuning ---------------------------------------------
// A batch march of N <= 4096 can run in more than one launch shape with the
// same per-row arithmetic: while every row can have two SMs, one 2-CTA
// cluster per row or one CTA per row; with more rows than one CTA-per-row
// launch keeps resident, the rotation's chunk length (64..512 steps).  The
// first march of a shape (N, rows) times each candidate on a short march of
// a scratch copy of the state on the march's stream (CUDA events, best of
// two) and keeps the fastest in a process-wide table that later marches of
// the shape reuse.  Layout candidates differ in kernel (results agree within
// the FP32 tolerance); chunk candidates give identical bits.  No search runs
// while the stream is being captured into a graph, for single rows (the
// cluster is the latency choice) or when BPM_AUTOTUNE=0: the fixed rule
// decides.
struct LaunchShape {
  int layout = -1;   // 1: cluster per row, 0: CTA per row, -1: the rule
  int chunk = 0;     // rotation chunk (CTA layout, more rows than resident)
  bool rotated = false;
};

static std::mutex g_tune_mu;
static std::map<std::pair<int, int>, LaunchShape> g_tune;   // (logn, rows) -> shape

static bool autotune_enabled() {
  const char* v = std::getenv("BPM_AUTOTUNE");
  return !(v && v[0] == '0');
}

// Milliseconds of one trial march (best of two), or a large value on error.
static double time_trial(bpm_plan_s* plan, PlanAux* aux, const LaunchShape& sh, void* scratch,
                         int n_begin, int steps, cudaStream_t st) {
  std::vector<RowDescF32> rows;
  fused_rows(plan, static_cast<float2*>(scratch), nullptr, nullptr, n_begin, n_begin + steps,
             &rows);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 1e30;
  for (int rep = 0; rep < 2; ++rep) {
    cudaEventRecord(e0, st);
    int rc;
    if (sh.rotated) {
      rc = launch_rotated(plan, aux, rows, n_begin, steps, fused_launch_capacity(plan->logn, false),
                          st, sh.chunk);
    } else {
      cudaMemcpyAsync(plan->d_rows, rows.data(), sizeof(RowDescF32) * rows.size(),
                      cudaMemcpyHostToDevice, st);
      rc = launch_fused_layout(plan->logn, static_cast<const RowDescF32*>(plan->d_rows), plan->nb,
                               steps, static_cast<const float4*>(plan->d_tw), plan->d_status, st,
                               sh.layout);
    }
    cudaEventRecord(e1, st);
    if (rc != BPM_OK || cudaEventSynchronize(e1) != cudaSuccess) {
      cudaGetLastError();
      best = 1e30;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, double(ms));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

// Forest-Ruth plans that march stage by stage: N = 16384, and N = 8192 when
// BPM_FUSED_LAYOUT=staged (N = 8192 otherwise runs the split band's fused
// fourth-order form).
static bool fr_staged(const bpm_plan_s* plan) {
  if (plan->precision != BPM_FP32_FUSED || plan->split != BPM_SPLIT_FOREST_RUTH ||
      plan->logn < kSplitLogN)
    return false;
  if (plan->logn > kSplitLogN || plan->d_stage_prop_split == nullptr) return true;
  const char* fv = std::getenv("BPM_FUSED_LAYOUT");
  return fv && std::strcmp(fv, "staged") == 0;
}

static LaunchShape choose_shape(bpm_plan_s* plan, PlanAux* aux, const void* state, int n_begin,
                                int steps, cudaStream_t st) {
  NvtxRange nvtx("bpm_launch_shape_search");
  LaunchShape rule;
  const int nb = plan->nb, logn = plan->logn;
  if (plan->split == BPM_SPLIT_FOREST_RUTH) {
    // the fourth-order form: N = 4096 rows that each get four SMs on the
    // half-band split (three propagations per step; the 8000-step bent solve
    // measured 70.0 ms against 140 ms on one CTA), rows of 512 <= N <= 4096
    // that each get two SMs on the 2-CTA cluster (per step against one CTA:
    // N = 512 6.5 / 10.7 us, 1024 7.0 / 11.4, 2048 7.7 / 10.5, 4096 12.0 /
    // 17.5), else one CTA per row; BPM_FUSED_LAYOUT=cta|cluster forces
    // either
    int sms = 1, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (logn == kSplitLogN) {   // N = 8192 (staged plans do not get here)
      rule.layout = kLayoutSplit4FR;
      return rule;
    }
    const char* fv = std::getenv("BPM_FUSED_LAYOUT");
    const bool cta = fv && std::strcmp(fv, "cta") == 0;
    const bool cl = fv && std::strcmp(fv, "cluster") == 0;
    if (!cta && !cl && logn == 12 && plan->d_stage_prop_split != nullptr && 4 * nb <= sms &&
        nb <= fused_split4_fr_capacity()) {
      rule.layout = kLayoutSplit4FR;
      return rule;
    }
    if (!cta && logn >= 9 && logn <= 12 && 2 * nb <= sms &&
        nb <= fused_cluster_fr_capacity(logn)) {
      rule.layout = kLayoutClusterFR;
      return rule;
    }
    rule.layout = kLayoutCtaFR;
    rule.rotated = nb > fused_fr_capacity(logn);
    return rule;
  }
  if (plan->split == BPM_SPLIT_VERLET && logn >= kSplitLogN) {
    // N = 8192, 16384: the split-band clusters with the second-order step
    rule.layout = kLayoutSplit4Half;
    return rule;
  }
  if (plan->split == BPM_SPLIT_VERLET) {
    // the second-order forms: a 2-CTA cluster per row while every row gets
    // two SMs, else one CTA per row; measured per 8000-step single solve,
    // cluster against one CTA: N = 512 23.5 / 28.3 ms, 1024 25.9 / 29.1,
    // 2048 29.8 / 28.7 (one CTA kept there), 4096 42.6 / 50.6;
    // BPM_FUSED_LAYOUT=cluster|cta forces either
    int sms = 1, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const char* fv = std::getenv("BPM_FUSED_LAYOUT");
    const bool cta = fv && std::strcmp(fv, "cta") == 0;
    const bool cl = fv && std::strcmp(fv, "cluster") == 0;
    // N = 4096 rows that each get four SMs: the half-band split
    if (!cta && !cl && logn == 12 && plan->d_prop_split != nullptr && 4 * nb <= sms &&
        nb <= fused_split4_half_capacity()) {
      rule.layout = kLayoutSplit4Half;
      return rule;
    }
    if (!cta && (cl || logn != 11) && logn >= 9 && 2 * nb <= sms &&
        nb <= fused_cluster_half_capacity(logn)) {
      rule.layout = kLayoutClusterHalf;
      return rule;
    }
    rule.layout = kLayoutCtaHalf;
    rule.rotated = nb > fused_half_capacity(logn);
    return rule;
  }
  const int resident = fused_rows_resident(logn, nb);   // 0 when the rule picks clusters
  rule.rotated = resident > 0 && nb > resident;
  // N = 4096 rows that each get four SMs march fastest as half-band splits
  // (their tables exist exactly then)
  const bool split_ok = logn == 12 && plan->d_prop_split != nullptr;
  const char* fv = std::getenv("BPM_FUSED_LAYOUT");
  if (fv && (std::strcmp(fv, "cluster") == 0 || std::strcmp(fv, "cta") == 0)) return rule;
  if (split_ok) {
    rule.layout = kLayoutSplit4;
    rule.rotated = false;
    if (fv && std::strcmp(fv, "split") == 0) return rule;
    if (fv && std::strcmp(fv, "split16") == 0) {
      rule.layout = kLayoutSplit4S;
      return rule;
    }
  }
  if (logn >= kSplitLogN || nb < 2 || !autotune_enabled()) return rule;
  int sms = 1, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // candidates, the rule's own shape first
  std::vector<LaunchShape> cands;
  const int cta_cap = fused_launch_capacity(logn, false);
  if (logn >= 9 && 2 * nb <= sms) {
    LaunchShape c;
    if (split_ok) {
      c.layout = kLayoutSplit4;
      cands.push_back(c);
    }
    c.layout = 1;
    cands.push_back(c);
    c.layout = 0;
    cands.push_back(c);   // nb <= sms / 2 rows always fit one CTA-per-row launch
  } else if (nb > cta_cap) {
    const int rule_chunk = std::max(std::min(steps, 64), steps / 24);
    for (int ch : {rule_chunk, 64, 128, 256, 512}) {
      if (ch != rule_chunk && (ch == cands.front().chunk || ch >= 2 * steps)) continue;
      LaunchShape c;
      c.layout = 0;
      c.rotated = true;
      c.chunk = ch;
      cands.push_back(c);
    }
  }
  if (cands.size() < 2) return rule;
  const std::pair<int, int> key(logn, nb);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return rule;
  }
  // trial length: a few chunks for the rotation, a short march for the layout
  const int trial = std::min(steps, cands.front().rotated ? 1024 : 128);
  const size_t bytes = size_t(nb) * 2 * plan->nx * sizeof(float2);
  void* scratch = nullptr;
  if (cudaMallocAsync(&scratch, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return rule;
  }
  cudaMemcpyAsync(scratch, state, bytes, cudaMemcpyDeviceToDevice, st);
  // another shape replaces the rule's only if it is at least 2% faster
  // (run-to-run noise of the trials is below 1%)
  LaunchShape best = cands.front();
  const double rule_ms = time_trial(plan, aux, cands.front(), scratch, n_begin, trial, st);
  double best_ms = rule_ms;
  for (size_t i = 1; i < cands.size(); ++i) {
    const double ms = time_trial(plan, aux, cands[i], scratch, n_begin, trial, st);
    if (ms < best_ms && ms < 0.98 * rule_ms) {
      best_ms = ms;
      best = cands[i];
    }
  }
  cudaFreeAsync(scratch, st);
  if (rule_ms >= 1e30) return rule;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best;
  return best;
}

// Forest-Ruth at nx >= 8192, stage by stage: per step a coupling launch (t/2
// on the step's slice) and three one-step launches of the first-order
// split-band kernel, with the propagator tables of t dz, (1 - 2t) dz, t dz and
// the couplings (1 - t)/2, (1 - t)/2, t/2, all on the step's slice; records
// and powers in the third.  The row descriptors of every (step, stage) are
// built once and uploaded as one schedule.
static int march_staged_fr(bpm_plan_s* plan, PlanAux* aux, void* state, void* d_rec,
                           double* d_pw, int n_begin, int n_end, bool captured, cudaStream_t st) {
  if (captured)
    return fail(BPM_ERR_INVALID,
                "Forest-Ruth plans with nx >= 8192 march stage by stage; not under capture");
  const int nb = plan->nb, steps = n_end - n_begin;
  std::vector<RowDescF32> rows;
  fused_rows(plan, static_cast<float2*>(state), static_cast<float2*>(d_rec), d_pw, n_begin,
             n_end, &rows);
  const size_t ts = fr_table_stride(plan);
  // the schedule of up to `chunk` steps at a time (stream order keeps a
  // chunk's launches ahead of the next upload into the same buffer)
  const int chunk = std::min(steps, 1024);
  const size_t cap = size_t(chunk) * 3 * nb;
  if (aux->sched_cap < cap) {
    if (aux->d_sched) cudaFree(aux->d_sched);
    aux->d_sched = nullptr;
    aux->sched_cap = 0;
    int rc = dev_alloc(plan, reinterpret_cast<void**>(&aux->d_sched), cap * sizeof(RowDescF32),
                       "launch schedule");
    if (rc != BPM_OK) return rc;
    aux->sched_cap = cap;
  }
  plan->shape_layout = kLayoutStagedFR;
  plan->shape_chunk = 0;
  const float4* tw = static_cast<const float4*>(plan->d_tw);
  std::vector<RowDescF32> sched(cap);
  int rc = BPM_OK;
  for (int i0 = 0; i0 < steps && rc == BPM_OK; i0 += chunk) {
    const int len = std::min(chunk, steps - i0);
    for (int k = 0; k < len; ++k)
      for (int sg = 0; sg < 3; ++sg)
        for (int r = 0; r < nb; ++r) {
          RowDescF32 d = rows[r];
          d.n_begin = n_begin + i0 + k;
          d.n_end = d.n_begin + 1;
          d.n_phase0 = n_begin;
          if (sg == 1) d.prop = rows[r].prop + ts;       // (1 - 2t) dz
          if (sg == 2) {                                  // the outer coupling t/2
            d.am1 = rows[r].am1h;
            d.b = rows[r].bh;
          } else {
            d.record_every = 0;                           // records after the last stage
          }
          sched[(size_t(k) * 3 + sg) * nb + r] = d;
        }
    rc = upload(aux->d_sched, sched.data(), size_t(len) * 3 * nb * sizeof(RowDescF32), st, false,
                "upload launch schedule");
    for (int k = 0; k < len && rc == BPM_OK; ++k) {
      const RowDescF32* base = aux->d_sched + size_t(k) * 3 * nb;
      rc = launch_couple_only(base, nb, plan->nx, n_begin + i0 + k, st);
      for (int sg = 0; sg < 3 && rc == BPM_OK; ++sg)
        rc = launch_fused_layout(plan->logn, base + size_t(sg) * nb, nb, 1, tw, plan->d_status,
                                 st, -1);
    }
  }
  return rc;
}

// Enqueue the march of all rows on `st`.  state: the buffer holding the
// state at n_begin (c64 for FP32, the plan's d_state for FP64); outputs as
// documented for bpm_propagate_device.
static int enqueue_march(bpm_plan_s* plan, PlanAux* aux, void* state, void* d_rec, double* d_pw,
                         int n_begin, int n_end, void* out, bool out_c128, cudaStream_t st) {
  const int steps = n_end - n_begin;
  const bool captured = capturing(st);
  std::vector<double2> g;
  phase_factors(plan, steps, &g);
  int urc = upload(aux->d_g, g.data(), sizeof(double2) * plan->nb, st, captured,
                   "upload phase factors");
  if (urc != BPM_OK) return urc;
  double* final_pw = d_pw ? d_pw + 2 * plan->n_rec : nullptr;
  const int pw_stride = 2 * (plan->n_rec + 1);
  if (plan->ny > 1) {
    int rc = vol_march(plan, static_cast<float2*>(state), static_cast<float2*>(d_rec), d_pw,
                       n_begin, n_end, st);
    if (rc != BPM_OK) return rc;
    return launch_finish_f32(static_cast<const float2*>(state),
                             out_c128 ? static_cast<double2*>(out) : nullptr,
                             out_c128 ? nullptr : static_cast<float2*>(out),
                             reinterpret_cast<const double*>(aux->d_g), plan->nb,
                             int(plane_of(plan)), steps, plan->dx_um * plan->dy_um, final_pw,
                             pw_stride, st);
  }
  if (fr_staged(plan)) {
    int rc = march_staged_fr(plan, aux, state, d_rec, d_pw, n_begin, n_end, captured, st);
    if (rc != BPM_OK) return rc;
    return launch_finish_f32(static_cast<const float2*>(state),
                             out_c128 ? static_cast<double2*>(out) : nullptr,
                             out_c128 ? nullptr : static_cast<float2*>(out),
                             reinterpret_cast<const double*>(aux->d_g), plan->nb, plan->nx, steps,
                             plan->dx_um, final_pw, pw_stride, st);
  }
  if (plan->precision == BPM_FP32_FUSED) {
    std::vector<RowDescF32> rows;
    fused_rows(plan, static_cast<float2*>(state), static_cast<float2*>(d_rec), d_pw, n_begin,
               n_end, &rows);
    const LaunchShape sh = choose_shape(plan, aux, state, n_begin, steps, st);
    plan->shape_layout = sh.layout;
    plan->shape_chunk =
        sh.rotated ? std::min(steps, sh.chunk > 0 ? sh.chunk
                                                  : std::max(std::min(steps, 64), steps / 24))
                   : 0;
    int rc = BPM_OK;
    if (!sh.rotated) {
      rc = upload(plan->d_rows, rows.data(), sizeof(RowDescF32) * rows.size(), st, captured,
                  "upload row descriptors");
      if (rc != BPM_OK) return rc;
      rc = launch_fused_layout(plan->logn, static_cast<const RowDescF32*>(plan->d_rows), plan->nb,
                               steps, static_cast<const float4*>(plan->d_tw), plan->d_status, st,
                               sh.layout);
    } else {
      const int cap = sh.layout == kLayoutCtaHalf ? fused_half_capacity(plan->logn)
                      : sh.layout == kLayoutCtaFR ? fused_fr_capacity(plan->logn)
                                                  : fused_launch_capacity(plan->logn, false);
      rc = launch_rotated(plan, aux, rows, n_begin, steps, cap, st, sh.chunk, sh.layout);
    }
    if (rc != BPM_OK) return rc;
    return launch_finish_f32(static_cast<const float2*>(state),
                             out_c128 ? static_cast<double2*>(out) : nullptr,
                             out_c128 ? nullptr : static_cast<float2*>(out),
                             reinterpret_cast<const double*>(aux->d_g), plan->nb, plan->nx, steps,
                             plan->dx_um, final_pw, pw_stride, st);
  }
  int rc = plain_march(plan, n_begin, n_end, n_begin, d_rec, d_pw, st);
  if (rc != BPM_OK) return rc;
  return launch_finish_f64(static_cast<const double2*>(plan->d_state), static_cast<double2*>(out),
                           reinterpret_cast<const double*>(aux->d_g), plan->nb, plan->nx, steps,
                           plan->dx_um, final_pw, pw_stride, st);
}

}  // namespace bpm

using namespace bpm;

extern "C" {

const char* bpm_last_error(void) { return g_last_error.c_str(); }

const char* bpm_version(void) { return "bpm-gb300 0.1 (sm_103a)"; }

}  // extern "C"

// Plan creation shared by 2D (ny = 1) and 3D plans; `p` already validated.
static int make_plan(const bpm_problem* p, int ny, double dy_um, double y0_um,
                     bpm_plan_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "no usable CUDA device");

  auto plan = std::make_unique<bpm_plan_s>();
  plan->device = dev;
  plan->nx = p->nx;
  plan->nz = p->nz;
  plan->logn = 0;
  while ((1 << plan->logn) < p->nx) ++plan->logn;
  plan->ny = ny;
  plan->logny = 0;
  while ((1 << plan->logny) < ny) ++plan->logny;
  plan->dy_um = dy_um;
  plan->y0_um = y0_um;
  plan->nb = p->n_energy;
  plan->record_every = p->record_every;
  plan->precision = p->precision;
  plan->dx_um = p->dx_um;
  plan->dz_um = p->dz_um;
  plan->x0_um = p->x0_um;
  plan->e_ref_ev = p->e_ref_ev;
  plan->theta_b_ref = p->theta_b_ref_rad;
  plan->chi0 = std::complex<double>(p->chi0_re, p->chi0_im);
  plan->chih = std::complex<double>(p->chih_re, p->chih_im);
  plan->energies.assign(p->energy_ev, p->energy_ev + p->n_energy);
  plan->n_rec = p->record_every > 0 ? p->nz / p->record_every : 0;
  double lam_ref_um = kHcEvAngstrom / p->e_ref_ev * 1e-4;
  plan->d_um = lam_ref_um / (2.0 * std::sin(p->theta_b_ref_rad));
  plan->h_per_um = kTwoPi / plan->d_um;
  compute_energy_consts(plan.get());

  bpm_plan_s* pl = plan.get();
  const size_t n = plane_of(pl), nb = pl->nb, cs = csize(pl);
  const bool vol = pl->ny > 1;
  int rc = BPM_OK;
  auto A = [&](void** ptr, size_t bytes, const char* what) {
    if (rc == BPM_OK) rc = dev_alloc(pl, ptr, bytes, what);
  };
  A(&pl->d_prop, nb * std::max(prop_stride(pl) * cs, 2 * n * cs), "propagator tables");
  // N = 4096 rows can also march as half-band splits on 4-CTA clusters
  // while every row gets four SMs: their tables too
  const bool half_split = !vol && pl->precision == BPM_FP32_FUSED && pl->logn == 12 &&
                          4 * int(nb) <= device_sm_count();
  if (half_split)
    A(&pl->d_prop_split, nb * size_t(split_table_stride(pl, 11)) * cs, "split propagator tables");
  A(&pl->d_tw, size_t(pl->nx) * 16, "twiddles");
  if (vol) {
    A(&pl->d_twy, size_t(pl->ny) * 16, "twiddles along y");
    A(&pl->d_spec, nb * 2 * n * cs, "x-spectra");
  }
  A(&pl->d_state, nb * 2 * n * cs, "state");
  if (pl->precision == BPM_FP64_PLAIN) A(&pl->d_state2, nb * 2 * n * cs, "state scratch");
  A(&pl->d_rows, nb * std::max(sizeof(RowDescF32), sizeof(RowDescF64)), "row descriptors");
  A(&pl->d_io, nb * 2 * n * 16, "host staging");
  A(reinterpret_cast<void**>(&pl->d_status), sizeof(int), "status");
  PlanAux* aux = aux_of(pl);
  A(reinterpret_cast<void**>(&aux->d_g), nb * sizeof(double2), "phase factors");
  if (rc == BPM_OK) {
    e = cudaStreamCreateWithFlags(&aux->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) rc = cuda_fail(e, "stream");
  }
  if (rc == BPM_OK) {
    cudaStream_t st = aux->stream;
    if (vol) {
      std::vector<float4> tw, twy;
      twiddle_table_f32(pl->nx, &tw);
      twiddle_table_f32(pl->ny, &twy);
      e = cudaMemcpyAsync(pl->d_tw, tw.data(), tw.size() * 16, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(pl->d_twy, twy.data(), twy.size() * 16, cudaMemcpyHostToDevice, st);
      // per row: (a - 1, b) as float2 pairs, then the common phases as doubles
      std::vector<float2> coup(2 * size_t(pl->nb));
      std::vector<double> gph(pl->nb);
      for (int r = 0; r < pl->nb; ++r) {
        const EnergyConsts& c = pl->ec[r];
        coup[2 * r] = make_float2(float(c.am1.real()), float(c.am1.imag()));
        coup[2 * r + 1] = make_float2(float(c.b.real()), float(c.b.imag()));
        gph[r] = c.gphase;
      }
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(pl->d_rows, coup.data(), coup.size() * sizeof(float2),
                            cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(static_cast<float2*>(pl->d_rows) + coup.size(), gph.data(),
                            gph.size() * sizeof(double), cudaMemcpyHostToDevice, st);
      // then (a - 1, b) of a half step, for the second-order splitting
      std::vector<float2> coup_half(2 * size_t(pl->nb));
      for (int r = 0; r < pl->nb; ++r) {
        std::complex<double> ah, bh;
        coupling_frac(pl, r, 0.5, &ah, &bh);
        coup_half[2 * r] = make_float2(float((ah - 1.0).real()), float((ah - 1.0).imag()));
        coup_half[2 * r + 1] = make_float2(float(bh.real()), float(bh.imag()));
      }
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(static_cast<float2*>(pl->d_rows) + 3 * size_t(pl->nb),
                            coup_half.data(), coup_half.size() * sizeof(float2),
                            cudaMemcpyHostToDevice, st);
      for (int r = 0; r < pl->nb && e == cudaSuccess; ++r) {
        std::vector<float2> t;
        vol_prop_table(pl, r, &t);
        e = cudaMemcpyAsync(static_cast<float2*>(pl->d_prop) + size_t(r) * 2 * n, t.data(),
                            t.size() * sizeof(float2), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // t is reused
      }
    } else if (pl->precision == BPM_FP32_FUSED) {
      std::vector<float4> tw;
      twiddle_table_f32(pl->nx, &tw);
      e = cudaMemcpyAsync(pl->d_tw, tw.data(), n * 16, cudaMemcpyHostToDevice, st);
      for (int r = 0; r < pl->nb && e == cudaSuccess; ++r) {
        std::vector<float2> t;
        fused_prop_table(pl, r, &t);
        e = cudaMemcpyAsync(static_cast<float2*>(pl->d_prop) + size_t(r) * prop_stride(pl),
                            t.data(), t.size() * sizeof(float2), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && pl->d_prop_split) {
          split_prop_table(pl, r, 11, &t);
          e = cudaMemcpyAsync(static_cast<float2*>(pl->d_prop_split) +
                                  size_t(r) * split_table_stride(pl, 11),
                              t.data(), t.size() * sizeof(float2), cudaMemcpyHostToDevice, st);
        }
      }
    } else {
      std::vector<double2> tw;
      twiddle_table_f64(pl->nx, &tw);
      e = cudaMemcpyAsync(pl->d_tw, tw.data(), n * 16, cudaMemcpyHostToDevice, st);
      std::vector<RowDescF64> rows(pl->nb);
      for (int r = 0; r < pl->nb && e == cudaSuccess; ++r) {
        std::vector<double2> t;
        plain_prop_table(pl, r, &t);
        e = cudaMemcpyAsync(static_cast<double2*>(pl->d_prop) + size_t(r) * 2 * n, t.data(),
                            t.size() * sizeof(double2), cudaMemcpyHostToDevice, st);
        rows[r].prop = static_cast<const double2*>(pl->d_prop) + size_t(r) * 2 * n;
        rows[r].a = make_double2(pl->ec[r].a.real(), pl->ec[r].a.imag());
        rows[r].b = make_double2(pl->ec[r].b.real(), pl->ec[r].b.imag());
        rows[r].gphase = pl->ec[r].gphase;
      }
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(pl->d_rows, rows.data(), rows.size() * sizeof(RowDescF64),
                            cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(pl->d_status, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "plan upload");
  }
  if (rc != BPM_OK) {
    if (aux->stream) cudaStreamDestroy(aux->stream);
    if (aux->d_g) cudaFree(aux->d_g);
    free_plan_memory(pl);
    return rc;
  }
  *out = plan.release();
  return BPM_OK;
}

extern "C" {

int bpm_plan(const bpm_problem* p, bpm_plan_t* out) {
  NvtxRange nvtx("bpm_plan");
  if (!out) return fail(BPM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  std::string why;
  if (validate_problem(p, &why) != BPM_OK) return fail(BPM_ERR_INVALID, why);
  return make_plan(p, 1, 0.0, 0.0, out);
}

int bpm_plan3d(const bpm_problem* p, int32_t ny, double dy_um, double y0_um, bpm_plan_t* out) {
  NvtxRange nvtx("bpm_plan3d");
  if (!out) return fail(BPM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  std::string why;
  if (validate_problem3d(p, ny, dy_um, y0_um, &why) != BPM_OK) return fail(BPM_ERR_INVALID, why);
  return make_plan(p, ny, dy_um, y0_um, out);
}

int bpm_set_splitting(bpm_plan_t plan, int32_t method) {
  if (!plan) return fail(BPM_ERR_INVALID, "plan is NULL");
  std::lock_guard<std::mutex> lk(plan->mu);
  if (plan->pending) return fail(BPM_ERR_BUSY, "plan has pending tickets");
  if (method < BPM_SPLIT_FIRST_ORDER || method > BPM_SPLIT_FOREST_RUTH)
    return fail(BPM_ERR_INVALID, "unknown splitting method");
  if (method == BPM_SPLIT_FOREST_RUTH && plan->ny > 1)
    return fail(BPM_ERR_INVALID, "3D plans march first order or Verlet");
  for (void** p : {&plan->d_stage_rows, &plan->d_stage_prop, &plan->d_stage_prop_split}) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  plan->split = BPM_SPLIT_FIRST_ORDER;
  plan->n_stages = 0;
  plan->stage_has_prop.clear();
  const auto stages = split_stages(method);
  const size_t n = plan->nx, nb = plan->nb;
  if (plan->precision == BPM_FP32_FUSED) {
    // the fused kernels take the coupling coefficients from the row
    // descriptors, built at each march; Forest-Ruth also needs the
    // propagator increments of its t dz and (1 - 2t) dz stages
    if (method == BPM_SPLIT_FOREST_RUTH) {
      const size_t ts = fr_table_stride(plan);
      // nx <= 4096: [band][nx] in the one-CTA kernels' thread order
      std::vector<int> cpos;
      int rc = plan->logn < kSplitLogN ? fr_cta_table_order(plan->logn, &cpos) : BPM_OK;
      if (rc != BPM_OK) return rc;
      rc = dev_alloc(plan, &plan->d_stage_prop, nb * 2 * ts * sizeof(float2),
                     "splitting propagators");
      if (rc != BPM_OK) return rc;
      std::vector<float2> host(nb * 2 * ts);
      for (size_t r = 0; r < nb; ++r)
        for (int k = 0; k < 2; ++k) {
          std::vector<float2> tab;
          float2* dst = host.data() + (r * 2 + k) * ts;
          if (plan->logn >= kSplitLogN) {
            split_prop_table_frac(plan, int(r), 12, stages[1 + k].first, &tab);
            std::copy(tab.begin(), tab.end(), dst);
          } else {
            fused_prop_table_frac(plan, int(r), stages[1 + k].first, &tab);
            for (size_t b = 0; b < 2; ++b)
              for (size_t i = 0; i < n; ++i) dst[b * n + i] = tab[b * n + size_t(cpos[i])];
          }
        }
      cudaStream_t st = aux_of(plan)->stream;
      cudaError_t e = cudaMemcpyAsync(plan->d_stage_prop, host.data(),
                                      host.size() * sizeof(float2), cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail(e, "splitting tables");
      if (plan->d_prop_split || plan->logn == kSplitLogN) {
        // the split kernels' fused forms (nx = 4096 rows that get four SMs,
        // nx = 8192): the tables of the t dz and (1 - 2t) dz propagations,
        // [band][D(k) | D(k + M)] in the kernels' thread order
        const int slog = plan->logn == kSplitLogN ? 12 : 11;
        std::vector<int> pos;
        rc = fr_split_table_order(plan->logn, &pos);
        if (rc != BPM_OK) return rc;
        const size_t hs = size_t(split_table_stride(plan, slog)), m = pos.size();
        if (hs != 4 * m) return fail(BPM_ERR_INVALID, "split table layout");
        rc = dev_alloc(plan, &plan->d_stage_prop_split, nb * 2 * hs * sizeof(float2),
                       "splitting propagators (split kernels)");
        if (rc != BPM_OK) return rc;
        std::vector<float2> hh(nb * 2 * hs);
        for (size_t r = 0; r < nb; ++r)
          for (int k = 0; k < 2; ++k) {
            std::vector<float2> tab;
            split_prop_table_frac(plan, int(r), slog, stages[1 + k].first, &tab);
            float2* dst = hh.data() + (r * 2 + k) * hs;
            for (size_t q = 0; q < 4; ++q)
              for (size_t i = 0; i < m; ++i) dst[q * m + i] = tab[q * m + size_t(pos[i])];
          }
        e = cudaMemcpyAsync(plan->d_stage_prop_split, hh.data(), hh.size() * sizeof(float2),
                            cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "splitting tables");
      }
    }
    plan->split = method;
    // the slice form depends on the step form (nx = 4096): prepare again if
    // it changes
    if (!plan->slices_dirty && plan->sep_slices != sep_slices_apply(plan))
      plan->slices_dirty = true;
    return BPM_OK;
  }
  plan->split = method;
  if (method == BPM_SPLIT_FIRST_ORDER) return BPM_OK;
  // one table per distinct nonzero a_i
  std::vector<double> fracs;
  for (auto& st : stages)
    if (st.first != 0.0 && std::find(fracs.begin(), fracs.end(), st.first) == fracs.end())
      fracs.push_back(st.first);
  int rc = dev_alloc(plan, &plan->d_stage_prop, fracs.size() * nb * 2 * n * sizeof(double2),
                     "splitting propagators");
  if (rc == BPM_OK)
    rc = dev_alloc(plan, &plan->d_stage_rows, stages.size() * nb * sizeof(RowDescF64),
                   "splitting stages");
  if (rc != BPM_OK) return rc;
  double2* tables = static_cast<double2*>(plan->d_stage_prop);
  std::vector<RowDescF64> rows(stages.size() * nb);
  // Uploads are ordered on the plan's stream and waited for: a plain
  // cudaMemcpy from pageable memory may return before its DMA has landed,
  // and the marches run on non-blocking streams.
  cudaStream_t st = aux_of(plan)->stream;
  std::vector<double2> host(fracs.size() * nb * 2 * n);
  for (size_t f = 0; f < fracs.size(); ++f)
    for (size_t r = 0; r < nb; ++r) {
      std::vector<double2> t;
      plain_prop_table_frac(plan, int(r), fracs[f], &t);
      std::copy(t.begin(), t.end(), host.begin() + long((f * nb + r) * 2 * n));
    }
  cudaError_t e = cudaMemcpyAsync(tables, host.data(), host.size() * sizeof(double2),
                                  cudaMemcpyHostToDevice, st);
  for (size_t s = 0; s < stages.size(); ++s) {
    const size_t f = std::find(fracs.begin(), fracs.end(), stages[s].first) - fracs.begin();
    plan->stage_has_prop.push_back(stages[s].first != 0.0 ? 1 : 0);
    for (size_t r = 0; r < nb; ++r) {
      RowDescF64& d = rows[s * nb + r];
      d.prop = stages[s].first != 0.0 ? tables + (f * nb + r) * 2 * n : nullptr;
      std::complex<double> a, b;
      coupling_frac(plan, int(r), stages[s].second, &a, &b);
      d.a = make_double2(a.real(), a.imag());
      d.b = make_double2(b.real(), b.imag());
      d.gphase = plan->ec[r].gphase;
    }
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(plan->d_stage_rows, rows.data(), rows.size() * sizeof(RowDescF64),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "splitting tables");
  plan->n_stages = int(stages.size());
  return BPM_OK;
}

int bpm_set_crystal_box(bpm_plan_t plan, const double* box_um) {
  if (!plan || !box_um) return fail(BPM_ERR_INVALID, "plan / box_um is NULL");
  std::lock_guard<std::mutex> lk(plan->mu);
  if (plan->pending) return fail(BPM_ERR_BUSY, "plan has pending tickets");
  if (plan->ny <= 1) return fail(BPM_ERR_INVALID, "box crystals need a 3D plan");
  for (int i = 0; i < 6; ++i)
    if (!std::isfinite(box_um[i])) return fail(BPM_ERR_INVALID, "box bounds must be finite");
  plan->crystal_kind = BPM_CRYSTAL_BOX;
  for (int i = 0; i < 6; ++i) plan->box[i] = box_um[i];
  plan->mask.clear();
  plan->poly.clear();
  plan->slices_dirty = true;
  return BPM_OK;
}

int bpm_set_crystal(bpm_plan_t plan, int32_t kind, double asym_angle_rad, double thickness_um,
                    double surf_x_um, double surf_z_um, const uint8_t* mask,
                    const double* poly_xz_um, int32_t nv) {
  if (!plan) return fail(BPM_ERR_INVALID, "plan is NULL");
  std::lock_guard<std::mutex> lk(plan->mu);
  if (plan->pending) return fail(BPM_ERR_BUSY, "plan has pending tickets");
  if (kind < BPM_CRYSTAL_VACUUM || kind > BPM_CRYSTAL_SLAB_AND_POLYGON)
    return fail(BPM_ERR_INVALID, "unknown crystal kind");
  const bool slab = kind == BPM_CRYSTAL_SLAB || kind == BPM_CRYSTAL_SLAB_AND_MASK ||
                    kind == BPM_CRYSTAL_SLAB_AND_POLYGON;
  if (slab && (!std::isfinite(asym_angle_rad) || !(thickness_um >= 0) ||
               !std::isfinite(thickness_um) || !std::isfinite(surf_x_um) ||
               !std::isfinite(surf_z_um)))
    return fail(BPM_ERR_INVALID, "slab parameters must be finite, thickness >= 0");
  const bool needs_mask = kind == BPM_CRYSTAL_MASK || kind == BPM_CRYSTAL_SLAB_AND_MASK;
  if (needs_mask && !mask) return fail(BPM_ERR_INVALID, "mask is NULL");
  if (kind == BPM_CRYSTAL_SLAB_AND_POLYGON) {
    if (!poly_xz_um || nv < 3) return fail(BPM_ERR_INVALID, "polygon needs nv >= 3 vertices");
    for (int i = 0; i < 2 * nv; ++i)
      if (!std::isfinite(poly_xz_um[i])) return fail(BPM_ERR_INVALID, "polygon not finite");
  }
  plan->crystal_kind = kind;
  plan->asym = asym_angle_rad;
  plan->thick = thickness_um;
  plan->surf_x = surf_x_um;
  plan->surf_z = surf_z_um;
  if (needs_mask) plan->mask.assign(mask, mask + plane_of(plan) * plan->nz);
  else plan->mask.clear();
  if (kind == BPM_CRYSTAL_SLAB_AND_POLYGON) plan->poly.assign(poly_xz_um, poly_xz_um + 2 * nv);
  else plan->poly.clear();
  plan->slices_dirty = true;
  return BPM_OK;
}

int bpm_set_strain(bpm_plan_t plan, int32_t kind, const double* ux_um, const double* params,
                   int32_t n_params) {
  if (!plan) return fail(BPM_ERR_INVALID, "plan is NULL");
  std::lock_guard<std::mutex> lk(plan->mu);
  if (plan->pending) return fail(BPM_ERR_BUSY, "plan has pending tickets");
  if (kind < BPM_STRAIN_NONE || kind > BPM_STRAIN_EDGE_DISLOCATION)
    return fail(BPM_ERR_INVALID, "unknown strain kind");
  const size_t cells = plane_of(plan) * plan->nz;
  if (kind == BPM_STRAIN_ARRAY) {
    if (!ux_um) return fail(BPM_ERR_INVALID, "ux_um is NULL");
    for (size_t i = 0; i < cells; ++i)
      if (!std::isfinite(ux_um[i])) return fail(BPM_ERR_INVALID, "ux_um not finite");
  }
  if (kind == BPM_STRAIN_BENT || kind == BPM_STRAIN_EDGE_DISLOCATION) {
    if (!params || n_params < 4) return fail(BPM_ERR_INVALID, "need 4 strain parameters");
    for (int i = 0; i < 4; ++i)
      if (!std::isfinite(params[i])) return fail(BPM_ERR_INVALID, "strain parameters not finite");
    if (kind == BPM_STRAIN_BENT && params[0] == 0.0)
      return fail(BPM_ERR_INVALID, "bend radius must be nonzero");
    if (kind == BPM_STRAIN_EDGE_DISLOCATION && params[1] == 1.0)
      return fail(BPM_ERR_INVALID, "Poisson ratio must differ from 1");
  }
  plan->strain_kind = kind;
  if (kind == BPM_STRAIN_ARRAY) plan->ux.assign(ux_um, ux_um + cells);
  else plan->ux.clear();
  for (int i = 0; i < 4; ++i)
    plan->sparams[i] = (params && i < n_params) ? params[i] : 0.0;
  plan->slices_dirty = true;
  return BPM_OK;
}

static int check_range(bpm_plan_s* plan, int32_t n_begin, int32_t n_end) {
  if (n_begin < 0 || n_end > plan->nz || n_begin >= n_end)
    return fail(BPM_ERR_INVALID, "need 0 <= n_begin < n_end <= nz");
  return BPM_OK;
}

static int finish_status(bpm_plan_s* plan, cudaStream_t st) {
  int status = 0;
  cudaError_t e = cudaMemcpyAsync(&status, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "march");
  if (status & kStatusWaitTimeout) {
    cudaMemsetAsync(plan->d_status, 0, sizeof(int), st);
    cudaStreamSynchronize(st);
    return fail(BPM_ERR_TIMEOUT, "a bounded wait (strain slice or peer data) expired on the device");
  }
  return BPM_OK;
}

int bpm_propagate(bpm_plan_t plan, const double* psi_in, double* psi_out, void* records,
                  double* powers, int32_t n_begin, int32_t n_end) {
  NvtxRange nvtx("bpm_propagate");
  if (!plan) return fail(BPM_ERR_INVALID, "plan is NULL");
  if (!psi_in || !psi_out) return fail(BPM_ERR_INVALID, "psi_in / psi_out is NULL");
  std::lock_guard<std::mutex> lk(plan->mu);
  if (plan->pending) return fail(BPM_ERR_BUSY, "plan has pending tickets");
  int rc = check_range(plan, n_begin, n_end);
  if (rc != BPM_OK) return rc;
  PlanAux* aux = aux_of(plan);
  cudaStream_t st = aux->stream;
  if (plan->slices_dirty && (rc = prepare_slices(plan, st)) != BPM_OK) return rc;

  const size_t n = plane_of(plan), nb = plan->nb, cs = csize(plan);
  const int nrec = plan->n_rec;
  const bool want_rec = records && nrec > 0;
  const bool want_pw = powers != nullptr;
  size_t rec_bytes = nb * size_t(nrec) * 2 * n * cs;
  size_t pow_bytes = nb * size_t(nrec + 1) * 2 * sizeof(double);
  if (want_rec && aux->rec_bytes < rec_bytes) {
    if (aux->d_rec) cudaFree(aux->d_rec);
    aux->d_rec = nullptr;
    aux->rec_bytes = 0;
    if ((rc = dev_alloc(plan, &aux->d_rec, rec_bytes, "records")) != BPM_OK) return rc;
    aux->rec_bytes = rec_bytes;
  }
  if (want_pw && aux->pow_bytes < pow_bytes) {
    if (aux->d_pow) cudaFree(aux->d_pow);
    aux->d_pow = nullptr;
    aux->pow_bytes = 0;
    if ((rc = dev_alloc(plan, reinterpret_cast<void**>(&aux->d_pow), pow_bytes, "powers")) != BPM_OK)
      return rc;
    aux->pow_bytes = pow_bytes;
  }
  const size_t io_bytes = nb * 2 * n * 16;
  cudaError_t e = cudaMemcpyAsync(plan->d_io, psi_in, io_bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "copy psi_in");
  void* state = plan->d_state;
  if (plan->precision == BPM_FP32_FUSED) {
    rc = launch_convert_in(static_cast<const double2*>(plan->d_io), static_cast<float2*>(state),
                           nb * 2 * n, st);
  } else {
    e = cudaMemcpyAsync(state, plan->d_io, io_bytes, cudaMemcpyDeviceToDevice, st);
    rc = e == cudaSuccess ? BPM_OK : cuda_fail(e, "stage psi_in");
  }
  if (rc != BPM_OK) return rc;
  rc = enqueue_march(plan, aux, state, want_rec ? aux->d_rec : nullptr,
                     want_pw ? aux->d_pow : nullptr, n_begin, n_end, plan->d_io, true, st);
  if (rc != BPM_OK) return rc;
  e = cudaMemcpyAsync(psi_out, plan->d_io, io_bytes, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e, "copy psi_out");
  if (want_rec || want_pw) {
    const int k = plan->record_every;
    const int s0 = k > 0 ? n_begin / k : 0, s1 = k > 0 ? n_end / k : 0;
    for (size_t r = 0; r < nb && e == cudaSuccess; ++r) {
      if (want_rec && s1 > s0) {
        const size_t off = (r * nrec + s0) * 2 * n * cs;
        e = cudaMemcpyAsync(static_cast<char*>(records) + off, static_cast<char*>(aux->d_rec) + off,
                            size_t(s1 - s0) * 2 * n * cs, cudaMemcpyDeviceToHost, st);
      }
      if (want_pw && e == cudaSuccess) {
        if (s1 > s0) {
          const size_t off = (r * (nrec + 1) + s0) * 2;
          e = cudaMemcpyAsync(powers + off, aux->d_pow + off, size_t(s1 - s0) * 2 * sizeof(double),
                              cudaMemcpyDeviceToHost, st);
        }
        const size_t fin = (r * (nrec + 1) + nrec) * 2;
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(powers + fin, aux->d_pow + fin, 2 * sizeof(double),
                              cudaMemcpyDeviceToHost, st);
      }
    }
    if (e != cudaSuccess) return cuda_fail(e, "copy records / powers");
  }
  rc = finish_status(plan, st);
  if (rc != BPM_OK) return rc;
  if (want_pw) {
    for (size_t r = 0; r < nb; ++r)
      for (int i = 0; i < 2 * (nrec + 1); ++i) {
        double v = powers[r * 2 * (nrec + 1) + i];
        if (!std::isfinite(v)) return fail(BPM_ERR_NUMERIC, "non-finite band power");
      }
  }
  return BPM_OK;
}

int bpm_propagate_device(bpm_plan_t plan, const void* d_psi_in, void* d_psi_out, void* d_records,
                         void* d_powers, int32_t n_begin, int32_t n_end, void* stream) {
  NvtxRange nvtx("bpm_propagate_device");
  if (!plan) return fail(BPM_ERR_INVALID, "plan is NULL");
  if (!d_psi_in || !d_psi_out) return fail(BPM_ERR_INVALID, "d_psi_in / d_psi_out is NULL");
  std::lock_guard<std::mutex> lk(plan->mu);
  if (plan->pending) return fail(BPM_ERR_BUSY, "plan has pending tickets");
  int rc = check_range(plan, n_begin, n_end);
  if (rc != BPM_OK) return rc;
  PlanAux* aux = aux_of(plan);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // Under graph capture the march's per-call uploads go through kernel
  // parameters (see upload); what cannot be captured is refused before
  // anything is enqueued: FP64 plans (their march uploads per-record phase
  // factors and swaps buffers on the host), Forest-Ruth plans that march
  // stage by stage (their schedule is uploaded in chunks from the host) and
  // plans whose strain slices still have to be prepared (allocation and a
  // host wait).
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t ce = cudaStreamIsCapturing(st, &cs);
  if (ce != cudaSuccess) return cuda_fail(ce, "stream capture status");
  if (cs != cudaStreamCaptureStatusNone) {
    if (plan->precision != BPM_FP32_FUSED)
      return fail(BPM_ERR_INVALID, "FP64 plans cannot be captured into a CUDA graph");
    if (fr_staged(plan))
      return fail(BPM_ERR_INVALID,
                  "Forest-Ruth plans that march stage by stage cannot be captured");
    if (plan->slices_dirty)
      return fail(BPM_ERR_INVALID, "march the plan once outside the graph capture first");
  }
  if (plan->slices_dirty && (rc = prepare_slices(plan, aux->stream)) != BPM_OK) return rc;
  const size_t bytes = size_t(plan->nb) * 2 * plane_of(plan) * csize(plan);
  void* rec = plan->n_rec > 0 ? d_records : nullptr;
  if (plan->precision == BPM_FP32_FUSED) {
    if (d_psi_out != d_psi_in) {
      cudaError_t e = cudaMemcpyAsync(d_psi_out, d_psi_in, bytes, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return cuda_fail(e, "copy input");
    }
    return enqueue_march(plan, aux, d_psi_out, rec, static_cast<double*>(d_powers), n_begin, n_end,
                         d_psi_out, false, st);
  }
  cudaError_t e = cudaMemcpyAsync(plan->d_state, d_psi_in, bytes, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "copy input");
  return enqueue_march(plan, aux, plan->d_state, rec, static_cast<double*>(d_powers), n_begin,
                       n_end, d_psi_out, true, st);
}

int bpm_device_status(bpm_plan_t plan, void* stream) {
  if (!plan) return fail(BPM_ERR_INVALID, "plan is NULL");
  std::lock_guard<std::mutex> lk(plan->mu);
  return finish_status(plan, static_cast<cudaStream_t>(stream));
}

int bpm_omega_to_t_device(const void* d_in, void* d_out, int32_t n_energy, int32_t nx,
                          int32_t precision, void* stream) {
  if (!d_in || !d_out) return fail(BPM_ERR_INVALID, "buffer is NULL");
  if (n_energy < 2 || n_energy > 4096 || (n_energy & (n_energy - 1)))
    return fail(BPM_ERR_INVALID, "n_energy must be a power of two in [2, 4096]");
  if (nx < 1) return fail(BPM_ERR_INVALID, "nx must be >= 1");
  if (precision != BPM_FP32_FUSED && precision != BPM_FP64_PLAIN)
    return fail(BPM_ERR_INVALID, "bad precision");
  return launch_omega_to_t(d_in, d_out, n_energy, nx, precision, static_cast<cudaStream_t>(stream));
}

int bpm_fetch_slices(bpm_plan_t plan, uint8_t* mask, double* phasor) {
  if (!plan) return fail(BPM_ERR_INVALID, "plan is NULL");
  std::lock_guard<std::mutex> lk(plan->mu);
  PlanAux* aux = aux_of(plan);
  int rc = BPM_OK;
  if (plan->slices_dirty && (rc = prepare_slices(plan, aux->stream)) != BPM_OK) return rc;
  const size_t cells = plane_of(plan) * plan->nz;
  std::vector<double> buf;
  if (plan->precision == BPM_FP32_FUSED) {
    std::vector<float> f(2 * cells);
    const void* src = plan->d_phasor;
    float2* d_tmp = nullptr;
    if (plan->sep_slices) {   // the cells the kernels form from the separable tables
      cudaError_t e = cudaMalloc(&d_tmp, cells * 8);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(e, "fetch slices");
      }
      rc = expand_sep_slices(plan, d_tmp, aux->stream);
      if (rc == BPM_OK) {
        e = cudaStreamSynchronize(aux->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "fetch slices");
      }
      if (rc != BPM_OK) {
        cudaFree(d_tmp);
        return rc;
      }
      src = d_tmp;
    }
    cudaError_t e = cudaMemcpy(f.data(), src, cells * 8, cudaMemcpyDeviceToHost);
    if (d_tmp) cudaFree(d_tmp);
    if (e != cudaSuccess) return cuda_fail(e, "fetch slices");
    buf.assign(f.begin(), f.end());
  } else {
    buf.resize(2 * cells);
    cudaError_t e = cudaMemcpy(buf.data(), plan->d_phasor, cells * 16, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "fetch slices");
  }
  const int parts =
      (plan->ny <= 1 && plan->precision == BPM_FP32_FUSED && plan->logn >= kSplitLogN)
          ? (plan->nx >> 12) : 1;
  const size_t nx = plan->nx, m = nx / parts;
  for (size_t c = 0; c < cells; ++c) {
    size_t src = c;
    if (parts > 1) {
      const size_t n = c / nx, j = c % nx;
      src = n * nx + (j % parts) * m + j / parts;
    }
    if (mask) mask[c] = (buf[2 * src] != 0.0 || buf[2 * src + 1] != 0.0) ? 1 : 0;
    if (phasor) {
      phasor[2 * c] = buf[2 * src];
      phasor[2 * c + 1] = buf[2 * src + 1];
    }
  }
  return BPM_OK;
}

int bpm_slice_form(bpm_plan_t plan, int32_t* form, int64_t* bytes) {
  if (!plan) return fail(BPM_ERR_INVALID, "plan is NULL");
  std::lock_guard<std::mutex> lk(plan->mu);
  const bool ready = !plan->slices_dirty;
  if (form) *form = !ready ? -1 : plan->sep_slices ? 1 : 0;
  if (bytes) {
    *bytes = !ready ? 0
             : plan->sep_slices
                 ? int64_t(sep_bytes(plan))
                 : int64_t(plane_of(plan) * plan->nz * (plan->precision == BPM_FP32_FUSED ? 8 : 16));
  }
  return BPM_OK;
}

int bpm_launch_shape(bpm_plan_t plan, int32_t* layout, int32_t* chunk) {
  if (!plan) return fail(BPM_ERR_INVALID, "plan is NULL");
  std::lock_guard<std::mutex> lk(plan->mu);
  if (layout) *layout = plan->shape_layout;
  if (chunk) *chunk = plan->shape_chunk;
  return BPM_OK;
}

int bpm_destroy(bpm_plan_t plan) {
  if (!plan) return fail(BPM_ERR_INVALID, "plan is NULL");
  {
    std::lock_guard<std::mutex> lk(plan->mu);
    if (plan->pending) return fail(BPM_ERR_BUSY, "plan has pending tickets");
  }
  PlanAux* aux = aux_of(plan);
  if (aux->stream) {
    cudaStreamSynchronize(aux->stream);
    cudaStreamDestroy(aux->stream);
  }
  if (aux->d_rec) cudaFree(aux->d_rec);
  if (aux->d_pow) cudaFree(aux->d_pow);
  if (aux->d_g) cudaFree(aux->d_g);
  if (aux->d_sched) cudaFree(aux->d_sched);
  free_plan_memory(plan);
  delete plan;
  return BPM_OK;
}

}  // extern "C"
