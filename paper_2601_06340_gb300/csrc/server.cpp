// Continuous-batching request server (bpm_submit / bpm_poll).
//
// A worker thread owns the device side.  Requests wait in arrival order and
// are admitted while the number of active requests and their device
// footprint (state, staging, records, powers and, if the plan has none yet,
// its slice memory: the strain-phasor stream, or the separable rows and
// column phasors of a bent or unstrained analytic crystal) stay within the
// configured limits.  Active
// requests are grouped into buckets by transform size (FP32) -- FP64
// requests get a bucket each -- and every bucket runs its own pipeline on
// its own stream.  A bucket advances its members in batches: a batch takes
// the next members in round-robin order, at most as many rows as one launch
// of that size keeps resident on the GPU, and advances each by one chunk
// (`epoch_steps` steps, or what is left); rows of a batch with the same
// chunk length share one fused launch.  Two batches are kept in flight per
// bucket, so the next one is already queued on the stream when the current
// one ends, and a launch never holds more rows than run at once (no partial
// last wave).  A member's chunks run in order because its batches share the
// stream.  Requests that arrive while others run join the rotation at the
// next batch of their size, and sizes do not wait for each other.  Device
// memory of requests is allocated and released stream-ordered
// (cudaMallocAsync / cudaFreeAsync), so retiring a request never stalls
// other buckets; a request is retired only once every batch holding it has
// completed.
//
// A request's arithmetic does not depend on which other requests share its
// launches (rows are independent and each row runs the same code for the
// same shape and layout), so a result is the same alone and in the mix.
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bpm_internal.h"

namespace bpm {

// from capi.cpp
void fused_rows(bpm_plan_s* plan, float2* state, float2* rec, double* pw, int n_begin, int n_end,
                std::vector<RowDescF32>* out);
void phase_factors(const bpm_plan_s* plan, int steps, std::vector<double2>* out);

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  bpm_ticket_t id = 0;
  bpm_plan_s* plan = nullptr;
  std::vector<double> psi_in;
  double* psi_out = nullptr;
  void* records = nullptr;
  double* powers = nullptr;
  int status = BPM_NOT_READY;
  std::string error;
  double t_submit = 0, t_admit = 0, t_done = 0;
  // device side
  size_t footprint = 0;
  void** owned_slices = nullptr;   // the plan's slice memory this request allocated
  void* d_state = nullptr;     // c64 (FP32); FP64 requests march in their plan's state
  void* d_rec = nullptr;
  double* d_pow = nullptr;
  double2* d_g = nullptr;
  double2* d_out = nullptr;    // c128 staging
  cudaEvent_t ready = nullptr; // staged and prepared on io_stream
  cudaEvent_t out_ev = nullptr;   // results copied to the pinned staging
  void* h_stage = nullptr;        // pinned staging: psi c128, records, powers
  size_t h_stage_bytes = 0;
  int n_sched = 0;             // steps enqueued on the bucket's stream
  int n_done = 0;              // steps of batches that have completed
  int failed = BPM_OK;         // error of a completed batch that held it
};
using ReqPtr = std::shared_ptr<Request>;

// One launch group in flight: its rows, completion event and status word.
struct Batch {
  cudaEvent_t ev = nullptr;
  int* h_status = nullptr;      // pinned copy of the batch's status word
  int* d_status = nullptr;
  std::vector<std::pair<ReqPtr, int>> items;   // (request, steps)
  int err = BPM_OK;             // a launch of the batch failed on the host
};

struct Bucket {
  cudaStream_t st = nullptr;
  std::vector<ReqPtr> members;
  std::deque<Batch> inflight;   // oldest first
  std::vector<Batch> free;      // recycled batches (event, status words)
  size_t rr = 0;                // round-robin cursor into members
  RowDescF32* d_rows = nullptr; // descriptors of the batch being uploaded
  size_t cap = 0;               // (stream order keeps one buffer safe)
};

constexpr size_t kBatchesInFlight = 2;

struct Server {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<ReqPtr> queue;
  int n_active = 0;
  std::unordered_map<bpm_ticket_t, ReqPtr> tickets;
  std::map<bpm_ticket_t, std::array<double, 3>> times;
  bpm_ticket_t next_id = 1;
  double mem_fraction = 0.6;
  int max_active = 256, epoch_steps = 256, max_queue = 100000;
  size_t budget = 0, used = 0;
  bool started = false;
  std::thread worker;
  // worker-owned
  std::map<long, Bucket> buckets;   // key: logn (FP32) or -(ticket id) (FP64)
  std::vector<ReqPtr> retiring;     // results on their way to the caller
  std::vector<Bucket> spare;        // recycled per-request buckets
  std::map<size_t, std::vector<void*>> pinned_pool;   // pinned staging by size
  cudaStream_t io_stream = nullptr;    // admission: staging and strain preparation
  cudaStream_t out_stream = nullptr;   // retirement: finishing and copies out
  int sm_count = 1;
  bool per_request = false;  // true: one launch stream per request (else one per size)
  float4* d_tw[kMaxLogN + 1] = {};
  // test hook: launches of FP32 batches of transform size 2^logn still to
  // fail on the host, as if the launch had returned a CUDA error
  std::atomic<int> inject_fail[kMaxLogN + 1] = {};
};

Server& srv() {
  static Server* s = new Server();   // never destroyed: the worker may outlive main()
  return *s;
}

size_t csize_of(const bpm_plan_s* p) { return p->precision == BPM_FP32_FUSED ? 8 : 16; }

// The plan holds device memory for its slices in the form it will prepare
// (the per-cell stream, or the separable rows and columns).
bool slices_resident(const bpm_plan_s* p) {
  return sep_slices_apply(p) ? p->d_sep != nullptr : p->d_phasor != nullptr;
}

size_t footprint_of(const bpm_plan_s* p, bool need_rec) {
  const size_t n = p->nx, nb = p->nb, cs = csize_of(p);
  size_t b = nb * 2 * n * cs                       // state
             + nb * 2 * n * 16                     // c128 output staging
             + nb * size_t(p->n_rec + 1) * 2 * 8   // powers
             + nb * 16;                            // phase factors
  if (need_rec) b += nb * size_t(p->n_rec) * 2 * n * cs;
  if (!slices_resident(p)) b += slice_data_bytes(p);
  return b;
}

void* pinned_get(Server& s, size_t bytes) {
  auto& v = s.pinned_pool[bytes];
  if (!v.empty()) {
    void* p = v.back();
    v.pop_back();
    return p;
  }
  void* p = nullptr;
  if (cudaHostAlloc(&p, bytes, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void pinned_put(Server& s, void* p, size_t bytes) {
  if (p) s.pinned_pool[bytes].push_back(p);
}

// Pinned staging of a request: [psi c128][records][powers].
size_t stage_bytes(const bpm_plan_s* p, bool rec) {
  const size_t n = p->nx, nb = p->nb, cs = csize_of(p);
  return nb * 2 * n * 16 + (rec ? nb * size_t(p->n_rec) * 2 * n * cs : 0) +
         nb * size_t(p->n_rec + 1) * 2 * 8;
}

void release(Server& s, Request& r) {
  if (r.out_ev) {
    cudaEventDestroy(r.out_ev);
    r.out_ev = nullptr;
  }
  pinned_put(s, r.h_stage, r.h_stage_bytes);
  r.h_stage = nullptr;
  if (r.ready) {
    cudaEventDestroy(r.ready);
    r.ready = nullptr;
  }
  void* ptrs[] = {r.d_state, r.d_rec, r.d_pow, r.d_g, r.d_out};
  for (void* p : ptrs)
    if (p) cudaFreeAsync(p, s.io_stream);
  r.d_state = r.d_rec = nullptr;
  r.d_pow = nullptr;
  r.d_g = r.d_out = nullptr;
}

// Allocate and stage a request (stream-ordered on io_stream).
int admit_device(Server& s, Request& r) {
  NvtxRange nvtx("bpm_server_admit");
  bpm_plan_s* p = r.plan;
  const size_t n = p->nx, nb = p->nb, cs = csize_of(p);
  cudaStream_t st = s.io_stream;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMallocAsync(ptr, bytes, st);
  };
  {
    std::lock_guard<std::mutex> lk(p->mu);
    if (!slices_resident(p)) {
      void** dst = sep_slices_apply(p) ? &p->d_sep : &p->d_phasor;
      A(dst, slice_data_bytes(p));
      if (e == cudaSuccess) r.owned_slices = dst;
      p->slices_dirty = true;
    }
    if (e == cudaSuccess && p->slices_dirty) {
      int rc = prepare_slices(p, st, false);
      if (rc != BPM_OK) return rc;
    }
  }
  if (p->precision == BPM_FP32_FUSED) A(&r.d_state, nb * 2 * n * cs);
  if (r.records && p->n_rec > 0) A(&r.d_rec, nb * size_t(p->n_rec) * 2 * n * cs);
  A(reinterpret_cast<void**>(&r.d_pow), nb * size_t(p->n_rec + 1) * 2 * 8);
  A(reinterpret_cast<void**>(&r.d_g), nb * 16);
  A(reinterpret_cast<void**>(&r.d_out), nb * 2 * n * 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? BPM_ERR_OOM : BPM_ERR_CUDA;
  }
  r.h_stage_bytes = stage_bytes(p, r.d_rec != nullptr);
  r.h_stage = pinned_get(s, r.h_stage_bytes);
  if (!r.h_stage) return BPM_ERR_OOM;
  std::memcpy(r.h_stage, r.psi_in.data(), nb * 2 * n * 16);
  e = cudaMemcpyAsync(r.d_out, r.h_stage, nb * 2 * n * 16, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return BPM_ERR_CUDA;
  if (p->precision == BPM_FP32_FUSED) {
    int rc = launch_convert_in(r.d_out, static_cast<float2*>(r.d_state), nb * 2 * n, st);
    if (rc != BPM_OK) return rc;
  } else {
    e = cudaMemcpyAsync(p->d_state, r.d_out, nb * 2 * n * 16, cudaMemcpyDeviceToDevice, st);
  }
  // No wait here: the request's first epoch waits on this event instead, so
  // preparing a large strain stream never stalls the other buckets.
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r.ready, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(r.ready, st);
  return e == cudaSuccess ? BPM_OK : BPM_ERR_CUDA;
}

// Enqueue the end of a request on out_stream: common phase, conversion to
// c128, final powers, copies into the pinned staging; completion is an event.
int retire_enqueue(Server& s, Request& r) {
  NvtxRange nvtx("bpm_server_retire");
  bpm_plan_s* p = r.plan;
  const size_t n = p->nx, nb = p->nb, cs = csize_of(p);
  std::vector<double2> g;
  phase_factors(p, p->nz, &g);
  cudaStream_t st = s.out_stream;
  double2* hg = reinterpret_cast<double2*>(
      static_cast<char*>(r.h_stage) + r.h_stage_bytes - nb * size_t(p->n_rec + 1) * 2 * 8);
  // phase factors go through the (not yet used) powers area of the staging
  std::memcpy(hg, g.data(), nb * 16);
  cudaError_t e = cudaMemcpyAsync(r.d_g, hg, nb * 16, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return BPM_ERR_CUDA;
  const int pw_stride = 2 * (p->n_rec + 1);
  int rc;
  if (p->precision == BPM_FP32_FUSED)
    rc = launch_finish_f32(static_cast<const float2*>(r.d_state), r.d_out, nullptr,
                           reinterpret_cast<const double*>(r.d_g), p->nb, p->nx, p->nz, p->dx_um,
                           r.d_pow + 2 * p->n_rec, pw_stride, st);
  else
    rc = launch_finish_f64(static_cast<const double2*>(p->d_state), r.d_out,
                           reinterpret_cast<const double*>(r.d_g), p->nb, p->nx, p->nz, p->dx_um,
                           r.d_pow + 2 * p->n_rec, pw_stride, st);
  if (rc != BPM_OK) return rc;
  char* h = static_cast<char*>(r.h_stage);
  e = cudaMemcpyAsync(h, r.d_out, nb * 2 * n * 16, cudaMemcpyDeviceToHost, st);
  h += nb * 2 * n * 16;
  if (e == cudaSuccess && r.d_rec) {
    e = cudaMemcpyAsync(h, r.d_rec, nb * size_t(p->n_rec) * 2 * n * cs, cudaMemcpyDeviceToHost, st);
    h += nb * size_t(p->n_rec) * 2 * n * cs;
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h, r.d_pow, nb * size_t(p->n_rec + 1) * 2 * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r.out_ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(r.out_ev, st);
  return e == cudaSuccess ? BPM_OK : BPM_ERR_CUDA;
}

// Copy a finished request's staged results to the caller's buffers.
int retire_complete(Request& r) {
  bpm_plan_s* p = r.plan;
  const size_t n = p->nx, nb = p->nb, cs = csize_of(p);
  const char* h = static_cast<const char*>(r.h_stage);
  std::memcpy(r.psi_out, h, nb * 2 * n * 16);
  h += nb * 2 * n * 16;
  if (r.d_rec) {
    std::memcpy(r.records, h, nb * size_t(p->n_rec) * 2 * n * cs);
    h += nb * size_t(p->n_rec) * 2 * n * cs;
  }
  const double* pw = reinterpret_cast<const double*>(h);
  const size_t npw = nb * size_t(p->n_rec + 1) * 2;
  if (r.powers) std::memcpy(r.powers, pw, npw * 8);
  for (size_t i = 0; i < npw; ++i)
    if (!std::isfinite(pw[i])) return BPM_ERR_NUMERIC;
  return BPM_OK;
}

void finish_request(Server& s, const ReqPtr& r, int status, const std::string& msg) {
  release(s, *r);
  {
    std::lock_guard<std::mutex> lk(r->plan->mu);
    if (r->owned_slices) {
      cudaFreeAsync(*r->owned_slices, s.io_stream);
      *r->owned_slices = nullptr;
      r->plan->slices_dirty = true;
    }
    r->plan->pending -= 1;
  }
  std::lock_guard<std::mutex> lk(s.mu);
  s.used -= r->footprint;
  s.n_active -= 1;
  r->status = status;
  r->error = msg;
  r->t_done = now_s();
  s.times[r->id] = {r->t_submit, r->t_admit, r->t_done};
  s.cv_done.notify_all();
}

Bucket& bucket_for(Server& s, long key) {
  auto it = s.buckets.find(key);
  if (it != s.buckets.end()) return it->second;
  if (!s.spare.empty()) {
    Bucket& b = s.buckets[key];
    b = std::move(s.spare.back());
    s.spare.pop_back();
    b.members.clear();
    b.rr = 0;
    return b;
  }
  Bucket& b = s.buckets[key];
  cudaStreamCreateWithFlags(&b.st, cudaStreamNonBlocking);
  return b;
}

Batch take_batch(Bucket& b) {
  if (!b.free.empty()) {
    Batch bt = std::move(b.free.back());
    b.free.pop_back();
    bt.items.clear();
    bt.err = BPM_OK;
    return bt;
  }
  Batch bt;
  cudaEventCreateWithFlags(&bt.ev, cudaEventDisableTiming);
  cudaMalloc(&bt.d_status, sizeof(int));
  cudaHostAlloc(reinterpret_cast<void**>(&bt.h_status), sizeof(int), cudaHostAllocDefault);
  *bt.h_status = 0;
  return bt;
}

bool has_unscheduled(const Bucket& b) {
  for (auto& r : b.members)
    if (r->failed == BPM_OK && r->n_sched < r->plan->nz) return true;
  return false;
}

// SMs the active FP32 rows would occupy in their cluster layouts.
int cluster_demand(Server& s) {
  int d = 0;
  for (auto& kv : s.buckets)
    for (auto& r : kv.second.members)
      if (r->plan->precision == BPM_FP32_FUSED) d += fused_cluster_sms(r->plan->logn);
  return d;
}

// Launch the next batch of a bucket.  Layout by load: when every active row
// can have the SMs of its cluster layout the launch is latency-first (a
// 2-CTA cluster per row for N <= 4096, a 4-CTA half-band split for N = 4096
// while two more SMs per row are free); once that demand would exceed the
// GPU, rows of N <= 4096 go one CTA per row (several rows per SM for small N),
// which does more cell-updates per SM.  The batch takes at most as many
// rows as that layout keeps resident, in round-robin order over the members
// that still have steps to enqueue.
int launch_batch(Server& s, Bucket& b) {
  NvtxRange nvtx("bpm_server_batch");
  Batch bt = take_batch(b);
  const bool fp32 = b.members.front()->plan->precision == BPM_FP32_FUSED;
  const int logn = b.members.front()->plan->logn;   // one size per bucket
  const int demand = cluster_demand(s);
  int layout = fp32 && demand <= s.sm_count ? -1 : 0;
  // N = 4096 rows go as half-band splits (four SMs each, as bpm_propagate
  // marches them alone) while the GPU has the two extra SMs per row
  if (fp32 && logn == 12 && demand + 2 * int(b.members.size()) <= s.sm_count) {
    bool tables = true;
    for (auto& r : b.members) tables = tables && r->plan->d_prop_split != nullptr;
    if (tables) layout = kLayoutSplit4;
  }
  size_t limit = b.members.size();
  if (fp32) {
    const bool cluster = layout < 0 && 2 * int(b.members.size()) <= s.sm_count;
    limit = size_t(std::max(1, layout == kLayoutSplit4 ? fused_split4_capacity()
                                                       : fused_launch_capacity(logn, cluster)));
    // rows of the splitting forms march on their own kernels (N <= 4096: one
    // CTA per row, on the half-step or the fourth-order form; N = 8192,
    // 16384: the split-band cluster forms); a batch holding any stays
    // within the one-CTA forms' residency
    if (logn < kSplitLogN)
      for (auto& r : b.members) {
        if (r->plan->split == BPM_SPLIT_VERLET)
          limit = std::min(limit, size_t(std::max(1, fused_half_capacity(logn))));
        if (r->plan->split == BPM_SPLIT_FOREST_RUTH)
          limit = std::min(limit, size_t(std::max(1, fused_fr_capacity(logn))));
      }
  }
  // FP32 rows by (step count, splitting): key 3 * steps + bpm_split (0 first
  // order, 1 Verlet, 2 Forest-Ruth)
  std::map<int, std::vector<RowDescF32>> groups;
  std::vector<RowDescF32> rows;
  cudaMemsetAsync(bt.d_status, 0, sizeof(int), b.st);
  const size_t nm = b.members.size();
  for (size_t k = 0; k < nm && bt.items.size() < limit; ++k) {
    ReqPtr r = b.members[(b.rr + k) % nm];
    bpm_plan_s* p = r->plan;
    if (r->failed != BPM_OK || r->n_sched >= p->nz) continue;
    if (r->ready) {   // first batch of this request: wait for its staging
      cudaStreamWaitEvent(b.st, r->ready, 0);
      cudaEventDestroy(r->ready);
      r->ready = nullptr;
    }
    const int steps = std::min(s.epoch_steps, p->nz - r->n_sched);
    const int n0 = r->n_sched;
    bt.items.push_back({r, steps});
    r->n_sched += steps;
    if (!fp32) {
      bt.err = plain_march(p, n0, n0 + steps, 0, r->d_rec, r->d_pow, b.st);
      if (bt.err != BPM_OK) break;
      continue;
    }
    fused_rows(p, static_cast<float2*>(r->d_state), static_cast<float2*>(r->d_rec), r->d_pow,
               n0, n0 + steps, &rows);
    for (auto& d : rows) d.n_phase0 = 0;
    auto& g = groups[3 * steps + p->split];
    g.insert(g.end(), rows.begin(), rows.end());
  }
  b.rr = nm ? (b.rr + bt.items.size()) % nm : 0;
  if (bt.err == BPM_OK && !groups.empty()) {
    size_t total = 0;
    for (auto& kv : groups) total += kv.second.size();
    if (total > b.cap) {
      if (b.d_rows) cudaFreeAsync(b.d_rows, b.st);
      b.cap = std::max<size_t>(2 * total, 64);
      if (cudaMallocAsync(&b.d_rows, b.cap * sizeof(RowDescF32), b.st) != cudaSuccess) {
        b.d_rows = nullptr;
        b.cap = 0;
        cudaGetLastError();
        bt.err = BPM_ERR_OOM;
      }
    }
    if (!s.d_tw[logn]) {
      std::vector<float4> tw;
      twiddle_table_f32(1 << logn, &tw);
      // ordered on the launch stream and waited for (a plain cudaMemcpy from
      // pageable memory may return before its DMA lands, and the launches
      // of every size run on non-blocking streams)
      cudaMalloc(&s.d_tw[logn], tw.size() * sizeof(float4));
      cudaMemcpyAsync(s.d_tw[logn], tw.data(), tw.size() * sizeof(float4),
                      cudaMemcpyHostToDevice, b.st);
      cudaStreamSynchronize(b.st);
    }
    size_t off = 0;
    for (auto& kv : groups) {
      if (bt.err != BPM_OK) break;
      cudaMemcpyAsync(b.d_rows + off, kv.second.data(), kv.second.size() * sizeof(RowDescF32),
                      cudaMemcpyHostToDevice, b.st);
      int pending = s.inject_fail[logn].load();
      while (pending > 0 && !s.inject_fail[logn].compare_exchange_weak(pending, pending - 1)) {
      }
      if (pending > 0) {
        bt.err = fail(BPM_ERR_CUDA, "injected launch failure");
        break;
      }
      const int split = kv.first % 3;
      const int lay = split == BPM_SPLIT_VERLET
                          ? (logn >= kSplitLogN ? kLayoutSplit4Half : kLayoutCtaHalf)
                      : split == BPM_SPLIT_FOREST_RUTH
                          ? (logn >= kSplitLogN ? kLayoutSplit4FR : kLayoutCtaFR)
                          : layout;
      bt.err = launch_fused_layout(logn, b.d_rows + off, int(kv.second.size()), kv.first / 3,
                                   s.d_tw[logn], bt.d_status, b.st, lay);
      off += kv.second.size();
    }
  }
  // Even a batch whose launch failed part-way goes in flight: what was
  // enqueued may still use its requests' memory, so they retire (failed)
  // only after its event.
  cudaMemcpyAsync(bt.h_status, bt.d_status, sizeof(int), cudaMemcpyDeviceToHost, b.st);
  cudaEventRecord(bt.ev, b.st);
  const int err = bt.err;
  b.inflight.push_back(std::move(bt));
  return err;
}

// Hand a request whose every scheduled batch has completed to retirement.
void retire_or_fail(Server& s, const ReqPtr& r) {
  const int rc = r->failed != BPM_OK ? r->failed : retire_enqueue(s, *r);
  if (rc == BPM_OK) s.retiring.push_back(r);
  else finish_request(s, r, rc, "request failed on the device");
}

void worker_loop() {
  Server& s = srv();
  for (;;) {
    // ---- admission (arrival order, memory budget, active cap)
    std::vector<ReqPtr> admitted;
    {
      std::unique_lock<std::mutex> lk(s.mu);
      bool any_work = false;
      for (auto& kv : s.buckets)
        any_work = any_work || !kv.second.inflight.empty() || !kv.second.members.empty();
      any_work = any_work || !s.retiring.empty();
      if (s.queue.empty() && !any_work)
        s.cv_work.wait(lk, [&] { return !s.queue.empty(); });
      while (!s.queue.empty() && s.n_active < s.max_active) {
        auto r = s.queue.front();
        if (s.used + r->footprint > s.budget) break;
        s.queue.pop_front();
        s.used += r->footprint;
        s.n_active += 1;
        admitted.push_back(r);
      }
    }
    for (auto& r : admitted) {
      r->t_admit = now_s();
      int rc = admit_device(s, *r);
      if (rc != BPM_OK) {
        finish_request(s, r, rc, "admission failed on the device");
        continue;
      }
      const long key = s.per_request ? -long(r->id)
                       : (r->plan->precision == BPM_FP32_FUSED ? long(r->plan->logn) : -long(r->id));
      bucket_for(s, key).members.push_back(r);
    }

    // ---- hand finished results to their callers
    bool progressed = !admitted.empty();
    for (size_t i = 0; i < s.retiring.size();) {
      ReqPtr r = s.retiring[i];
      cudaError_t q = cudaEventQuery(r->out_ev);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      s.retiring.erase(s.retiring.begin() + long(i));
      progressed = true;
      const int rc = q == cudaSuccess ? retire_complete(*r) : BPM_ERR_CUDA;
      finish_request(s, r, rc, rc == BPM_OK ? "" : "request failed on the device");
    }

    // ---- progress every bucket independently
    for (auto it = s.buckets.begin(); it != s.buckets.end();) {
      Bucket& b = it->second;
      // completed batches, oldest first
      while (!b.inflight.empty()) {
        Batch& bt = b.inflight.front();
        cudaError_t q = cudaEventQuery(bt.ev);
        if (q == cudaErrorNotReady) break;
        progressed = true;
        int err = q == cudaSuccess ? BPM_OK : BPM_ERR_CUDA;
        if (*bt.h_status) {
          *bt.h_status = 0;
          err = BPM_ERR_TIMEOUT;
        }
        if (bt.err != BPM_OK) err = bt.err;
        std::vector<ReqPtr> done;
        for (auto& rs : bt.items) {
          Request& r = *rs.first;
          r.n_done += rs.second;
          if (err != BPM_OK && r.failed == BPM_OK) r.failed = err;
          // retire once nothing of it is left on the stream
          if (r.n_done == r.n_sched && (r.failed != BPM_OK || r.n_done >= r.plan->nz))
            done.push_back(rs.first);
        }
        bt.items.clear();
        b.free.push_back(std::move(bt));
        b.inflight.pop_front();
        for (auto& r : done) {
          b.members.erase(std::remove(b.members.begin(), b.members.end(), r), b.members.end());
          retire_or_fail(s, r);
        }
      }
      while (b.inflight.size() < kBatchesInFlight && has_unscheduled(b)) {
        const int err = launch_batch(s, b);
        progressed = true;
        if (err != BPM_OK) {
          // stop scheduling; members with batches in flight (the failed one
          // included) retire, failed, when those complete
          std::vector<ReqPtr> idle;
          for (auto& r : b.members) {
            if (r->failed == BPM_OK) r->failed = err;
            if (r->n_done == r->n_sched) idle.push_back(r);
          }
          for (auto& r : idle) {
            b.members.erase(std::remove(b.members.begin(), b.members.end(), r), b.members.end());
            finish_request(s, r, err, "batch launch failed");
          }
          break;
        }
      }
      if (b.inflight.empty() && b.members.empty() && it->first < 0) {
        // keep the stream, events and buffers for the next request (freeing
        // them would synchronise the device)
        s.spare.push_back(std::move(b));
        it = s.buckets.erase(it);
        continue;
      }
      ++it;
    }
    if (!progressed) {
      std::unique_lock<std::mutex> lk(s.mu);
      s.cv_work.wait_for(lk, std::chrono::microseconds(50));
    }
  }
}

void ensure_started(Server& s) {
  if (s.started) return;
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  s.budget = size_t(double(free_b) * s.mem_fraction);
  cudaStreamCreateWithFlags(&s.io_stream, cudaStreamNonBlocking);
  cudaStreamCreateWithFlags(&s.out_stream, cudaStreamNonBlocking);
  s.started = true;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&s.sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (s.sm_count <= 0) s.sm_count = 1;
  s.worker = std::thread([dev] {
    cudaSetDevice(dev);
    worker_loop();
  });
  s.worker.detach();
}

}  // namespace
}  // namespace bpm

using namespace bpm;

extern "C" {

int bpm_server_configure(double mem_fraction, int32_t max_active, int32_t epoch_steps,
                         int32_t max_queue) {
  Server& s = srv();
  std::lock_guard<std::mutex> lk(s.mu);
  if (!s.queue.empty() || s.n_active > 0)
    return fail(BPM_ERR_BUSY, "server has requests in flight");
  if (mem_fraction > 0.9) return fail(BPM_ERR_INVALID, "mem_fraction must be <= 0.9");
  s.mem_fraction = mem_fraction > 0 ? mem_fraction : 0.6;
  s.max_active = max_active > 0 ? max_active : 256;
  s.epoch_steps = epoch_steps > 0 ? epoch_steps : 256;
  s.max_queue = max_queue > 0 ? max_queue : 100000;
  if (s.started) {
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    s.budget = size_t(double(free_b) * s.mem_fraction);
  }
  return BPM_OK;
}

int bpm_server_inject_launch_failure(int32_t nx, int32_t count) {
  int logn = 0;
  while (logn <= kMaxLogN && (1 << logn) < nx) ++logn;
  if (nx < 8 || logn > kMaxLogN || (1 << logn) != nx || count < 0)
    return fail(BPM_ERR_INVALID, "nx must be a power of two in [8, 16384], count >= 0");
  srv().inject_fail[logn].store(count);
  return BPM_OK;
}

int bpm_submit(bpm_plan_t plan, const double* psi_in, double* psi_out, void* records,
               double* powers, bpm_ticket_t* out) {
  if (!plan || !psi_in || !psi_out || !out)
    return fail(BPM_ERR_INVALID, "plan, psi_in, psi_out and out must be non-NULL");
  *out = 0;
  if (plan->ny > 1) return fail(BPM_ERR_INVALID, "the server takes 2D plans only");
  // (Forest-Ruth at nx = 16384 marches stage by stage: not in a shared launch)
  if (plan->precision == BPM_FP32_FUSED && plan->split == BPM_SPLIT_FOREST_RUTH &&
      plan->logn > kSplitLogN)
    return fail(BPM_ERR_INVALID, "the server marches FP32 Forest-Ruth plans up to nx = 8192");
  Server& s = srv();
  auto r = std::make_shared<Request>();
  r->plan = plan;
  const size_t count = size_t(plan->nb) * 2 * plan->nx * 2;
  r->psi_in.assign(psi_in, psi_in + count);
  r->psi_out = psi_out;
  r->records = records;
  r->powers = powers;
  {
    // The check and the reservation are one critical section: of two
    // threads submitting on the same plan, exactly one gets the plan.
    std::lock_guard<std::mutex> lk(plan->mu);
    if (plan->pending > 0)
      return fail(BPM_ERR_BUSY, "the plan already has a request in flight");
    plan->pending += 1;
    r->footprint = footprint_of(plan, records != nullptr && plan->n_rec > 0);
  }
  auto release = [plan](int code, const char* why) {
    std::lock_guard<std::mutex> pk(plan->mu);
    plan->pending -= 1;
    return fail(code, why);
  };
  std::lock_guard<std::mutex> lk(s.mu);
  ensure_started(s);
  if (r->footprint > s.budget)
    return release(BPM_ERR_OOM, "request needs more device memory than the server budget");
  if (int(s.queue.size()) >= s.max_queue) return release(BPM_ERR_BUSY, "server queue is full");
  r->id = s.next_id++;
  r->t_submit = now_s();
  s.tickets[r->id] = r;
  s.queue.push_back(r);
  s.cv_work.notify_one();
  *out = r->id;
  return BPM_OK;
}

int bpm_poll(bpm_ticket_t ticket, int32_t timeout_ms) {
  Server& s = srv();
  std::unique_lock<std::mutex> lk(s.mu);
  auto it = s.tickets.find(ticket);
  if (it == s.tickets.end()) return fail(BPM_ERR_INVALID, "unknown or already collected ticket");
  auto r = it->second;
  auto ready = [&] { return r->status != BPM_NOT_READY; };
  if (timeout_ms < 0) s.cv_done.wait(lk, ready);
  else if (timeout_ms > 0) s.cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
  if (!ready()) return BPM_NOT_READY;
  s.tickets.erase(ticket);
  if (r->status != BPM_OK) return fail(r->status, r->error);
  return BPM_OK;
}

int bpm_ticket_times(bpm_ticket_t ticket, double* t_submit, double* t_admit, double* t_done) {
  Server& s = srv();
  std::lock_guard<std::mutex> lk(s.mu);
  auto it = s.tickets.find(ticket);
  double a = 0, b = 0, c = 0;
  if (it != s.tickets.end()) {
    a = it->second->t_submit;
    b = it->second->t_admit;
    c = it->second->t_done;
  } else {
    auto jt = s.times.find(ticket);
    if (jt == s.times.end()) return fail(BPM_ERR_INVALID, "unknown ticket");
    a = jt->second[0];
    b = jt->second[1];
    c = jt->second[2];
  }
  if (t_submit) *t_submit = a;
  if (t_admit) *t_admit = b;
  if (t_done) *t_done = c;
  return BPM_OK;
}

}  // extern "C"
