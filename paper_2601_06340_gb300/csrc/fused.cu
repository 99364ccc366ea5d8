// Dispatch of the fused FP32 march by transform size.
#include <atomic>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <vector>

#include "fused_kernel.cuh"
#include "fused2_kernel.cuh"
#include "fused4_kernel.cuh"
#include "fused4t_kernel.cuh"
#include "fused4s_kernel.cuh"

namespace bpm {

#define BPM_DECLARE_FUSED(L)                                                     \
  int fused_launch_##L(const RowDescF32*, int, int, const float4*, int*,         \
                       cudaStream_t);                                            \
  int fusedh_launch_##L(const RowDescF32*, int, int, const float4*, int*,        \
                        cudaStream_t);                                           \
  int fusedf_launch_##L(const RowDescF32*, int, int, const float4*, int*,        \
                        cudaStream_t);                                           \
  int fusedh_rows_resident_##L();                                                \
  int fusedf_rows_resident_##L();
#define BPM_DECLARE_FUSED2(L)                                                    \
  int fused2_launch_##L(const RowDescF32*, int, int, const float4*, int*,        \
                        cudaStream_t);                                           \
  int fused2h_launch_##L(const RowDescF32*, int, int, const float4*, int*,       \
                         cudaStream_t);                                          \
  int fused2h_rows_resident_##L();                                               \
  int fused2f_launch_##L(const RowDescF32*, int, int, const float4*, int*,       \
                         cudaStream_t);                                          \
  int fused2f_rows_resident_##L();
#define BPM_DECLARE_FUSED3H(L)                                                   \
  int fused3h_launch_##L(const RowDescF32*, int, int, const float4*, int*,       \
                         cudaStream_t);                                          \
  int fused3h_rows_resident_##L();
BPM_DECLARE_FUSED3H(9) BPM_DECLARE_FUSED3H(10) BPM_DECLARE_FUSED3H(11) BPM_DECLARE_FUSED3H(12)
#define BPM_DECLARE_FUSED3F(L)                                                   \
  int fused3f_launch_##L(const RowDescF32*, int, int, const float4*, int*,       \
                         cudaStream_t);                                          \
  int fused3f_rows_resident_##L();
BPM_DECLARE_FUSED3F(9) BPM_DECLARE_FUSED3F(10) BPM_DECLARE_FUSED3F(11) BPM_DECLARE_FUSED3F(12)
BPM_DECLARE_FUSED(3) BPM_DECLARE_FUSED(4) BPM_DECLARE_FUSED(5)
BPM_DECLARE_FUSED(6) BPM_DECLARE_FUSED(7) BPM_DECLARE_FUSED2(8)
BPM_DECLARE_FUSED2(9) BPM_DECLARE_FUSED2(10) BPM_DECLARE_FUSED2(11)
BPM_DECLARE_FUSED2(12)
int fused4_launch_13(const RowDescF32*, int, int, const float4*, int*, cudaStream_t);
int fused4h_launch_12(const RowDescF32*, int, int, const float4*, int*, cudaStream_t);
int fused4s_launch_12(const RowDescF32*, int, int, const float4*, int*, cudaStream_t);
int fused4s_rows_resident_12();
int fused4hh_launch_12(const RowDescF32*, int, int, const float4*, int*, cudaStream_t);
int fused4hh_rows_resident_12();
int fused4sh_launch_12(const RowDescF32*, int, int, const float4*, int*, cudaStream_t);
int fused4sh_rows_resident_12();
int fused4sf_launch_12(const RowDescF32*, int, int, const float4*, int*, cudaStream_t);
int fused4sf_rows_resident_12();
int fused4f_launch_13(const RowDescF32*, int, int, const float4*, int*, cudaStream_t);
int fused4_launch_14(const RowDescF32*, int, int, const float4*, int*, cudaStream_t);
int fused4v_launch_13(const RowDescF32*, int, int, const float4*, int*, cudaStream_t);
int fused4v_launch_14(const RowDescF32*, int, int, const float4*, int*, cudaStream_t);
#define BPM_DECLARE_FUSED3(L)                                                    \
  int fused3_launch_##L(const RowDescF32*, int, int, const float4*, int*,        \
                        cudaStream_t);
BPM_DECLARE_FUSED3(9) BPM_DECLARE_FUSED3(10) BPM_DECLARE_FUSED3(11) BPM_DECLARE_FUSED3(12)
int fused3_rows_resident_9(); int fused3_rows_resident_10(); int fused3_rows_resident_11();
int fused3_rows_resident_12();
int fused4_rows_resident_13(); int fused4_rows_resident_14();
int fused_rows_resident_3(); int fused_rows_resident_4(); int fused_rows_resident_5();
int fused_rows_resident_6(); int fused_rows_resident_7(); int fused2_rows_resident_8();
int fused2_rows_resident_9(); int fused2_rows_resident_10(); int fused2_rows_resident_11();
int fused2_rows_resident_12();

// Layout choice: a 2-CTA cluster per row (a whole SM per band) when every
// row of the launch gets its own pair of SMs, else one CTA per row.  The
// environment variable BPM_FUSED_LAYOUT=cta|cluster forces one of them
// (read at every launch).
static int sm_count();

static int forced_layout() {
  const char* v = std::getenv("BPM_FUSED_LAYOUT");
  if (!v) return -1;
  if (std::strcmp(v, "cluster") == 0) return 1;
  if (std::strcmp(v, "cta") == 0) return 0;
  return -1;
}

// BPM_FUSED_LAYOUT=split16: the N = 4096 half-band split with 16 points per
// thread (fused4e_march_kernel<11>) instead of 8.
static bool split16_forced() {
  const char* v = std::getenv("BPM_FUSED_LAYOUT");
  return v && std::strcmp(v, "split16") == 0;
}

static bool use_cluster_layout(int logn, int n_rows) {
  if (logn < 9 || logn > 12) return false;
  const int forced = forced_layout();
  if (forced == 0 || forced == 1) return forced == 1;
  return 2 * n_rows <= sm_count();
}

int launch_fused(int logn, const RowDescF32* d_rows, int n_rows, int steps,
                 const float4* d_tw, int* d_status, cudaStream_t st) {
  return launch_fused_layout(logn, d_rows, n_rows, steps, d_tw, d_status, st, -1);
}

int fused_cluster_sms(int logn) {
  if (logn >= kSplitLogN) return 2 << (logn - 12);
  return (logn >= 9 && logn <= 12) ? 2 : 0;
}

int launch_fused_layout(int logn, const RowDescF32* d_rows, int n_rows, int steps,
                        const float4* d_tw, int* d_status, cudaStream_t st, int layout) {
  if (n_rows <= 0 || steps <= 0) return BPM_OK;
  // (only for rows that carry the split tables: the caller checks)
  // the half-band split: 8 points per thread (the rule), or the 16-point
  // form of fused4e_march_kernel<11> when forced
  if (logn == 12 && layout == kLayoutSplit4)
    return fused4s_launch_12(d_rows, n_rows, steps, d_tw, d_status, st);
  if (logn == 12 && layout == kLayoutSplit4S)
    return fused4h_launch_12(d_rows, n_rows, steps, d_tw, d_status, st);
  if (layout == kLayoutSplit4FR) {
    switch (logn) {
      case 12: return fused4sf_launch_12(d_rows, n_rows, steps, d_tw, d_status, st);
      case 13: return fused4f_launch_13(d_rows, n_rows, steps, d_tw, d_status, st);
      default:
        return fail(BPM_ERR_INVALID, "fourth-order split layout needs nx = 4096 or 8192");
    }
  }
  if (layout == kLayoutSplit4Half) {
    switch (logn) {
      case 12:   // 8 points per thread unless the 16-point form is forced
        return split16_forced() ? fused4hh_launch_12(d_rows, n_rows, steps, d_tw, d_status, st)
                                : fused4sh_launch_12(d_rows, n_rows, steps, d_tw, d_status, st);
      case 13: return fused4v_launch_13(d_rows, n_rows, steps, d_tw, d_status, st);
      case 14: return fused4v_launch_14(d_rows, n_rows, steps, d_tw, d_status, st);
      default:
        return fail(BPM_ERR_INVALID, "second-order split layout needs nx = 4096, 8192 or 16384");
    }
  }
  if (layout == kLayoutClusterHalf) {
    switch (logn) {
      case 9: return fused3h_launch_9(d_rows, n_rows, steps, d_tw, d_status, st);
      case 10: return fused3h_launch_10(d_rows, n_rows, steps, d_tw, d_status, st);
      case 11: return fused3h_launch_11(d_rows, n_rows, steps, d_tw, d_status, st);
      case 12: return fused3h_launch_12(d_rows, n_rows, steps, d_tw, d_status, st);
      default: return fail(BPM_ERR_INVALID, "second-order cluster layout needs 512 <= nx <= 4096");
    }
  }
  if (layout == kLayoutClusterFR) {
    switch (logn) {
      case 9: return fused3f_launch_9(d_rows, n_rows, steps, d_tw, d_status, st);
      case 10: return fused3f_launch_10(d_rows, n_rows, steps, d_tw, d_status, st);
      case 11: return fused3f_launch_11(d_rows, n_rows, steps, d_tw, d_status, st);
      case 12: return fused3f_launch_12(d_rows, n_rows, steps, d_tw, d_status, st);
      default: return fail(BPM_ERR_INVALID, "fourth-order cluster layout needs 512 <= nx <= 4096");
    }
  }
  if (layout == kLayoutCtaFR) {
    switch (logn) {
      case 3: return fusedf_launch_3(d_rows, n_rows, steps, d_tw, d_status, st);
      case 4: return fusedf_launch_4(d_rows, n_rows, steps, d_tw, d_status, st);
      case 5: return fusedf_launch_5(d_rows, n_rows, steps, d_tw, d_status, st);
      case 6: return fusedf_launch_6(d_rows, n_rows, steps, d_tw, d_status, st);
      case 7: return fusedf_launch_7(d_rows, n_rows, steps, d_tw, d_status, st);
      case 8: return fused2f_launch_8(d_rows, n_rows, steps, d_tw, d_status, st);
      case 9: return fused2f_launch_9(d_rows, n_rows, steps, d_tw, d_status, st);
      case 10: return fused2f_launch_10(d_rows, n_rows, steps, d_tw, d_status, st);
      case 11: return fused2f_launch_11(d_rows, n_rows, steps, d_tw, d_status, st);
      case 12: return fused2f_launch_12(d_rows, n_rows, steps, d_tw, d_status, st);
      default: return fail(BPM_ERR_INVALID, "fourth-order splitting needs nx <= 4096");
    }
  }
  if (layout == kLayoutCtaHalf) {
    switch (logn) {
      case 3: return fusedh_launch_3(d_rows, n_rows, steps, d_tw, d_status, st);
      case 4: return fusedh_launch_4(d_rows, n_rows, steps, d_tw, d_status, st);
      case 5: return fusedh_launch_5(d_rows, n_rows, steps, d_tw, d_status, st);
      case 6: return fusedh_launch_6(d_rows, n_rows, steps, d_tw, d_status, st);
      case 7: return fusedh_launch_7(d_rows, n_rows, steps, d_tw, d_status, st);
      case 8: return fused2h_launch_8(d_rows, n_rows, steps, d_tw, d_status, st);
      case 9: return fused2h_launch_9(d_rows, n_rows, steps, d_tw, d_status, st);
      case 10: return fused2h_launch_10(d_rows, n_rows, steps, d_tw, d_status, st);
      case 11: return fused2h_launch_11(d_rows, n_rows, steps, d_tw, d_status, st);
      case 12: return fused2h_launch_12(d_rows, n_rows, steps, d_tw, d_status, st);
      default: return fail(BPM_ERR_INVALID, "second-order splitting needs nx <= 4096");
    }
  }
  const bool cluster = logn >= 9 && logn <= 12 &&
                       (layout == 1 || (layout < 0 && use_cluster_layout(logn, n_rows)));
  if (cluster) {
    switch (logn) {
      case 9: return fused3_launch_9(d_rows, n_rows, steps, d_tw, d_status, st);
      case 10: return fused3_launch_10(d_rows, n_rows, steps, d_tw, d_status, st);
      case 11: return fused3_launch_11(d_rows, n_rows, steps, d_tw, d_status, st);
      default: return fused3_launch_12(d_rows, n_rows, steps, d_tw, d_status, st);
    }
  }
  switch (logn) {
    case 3: return fused_launch_3(d_rows, n_rows, steps, d_tw, d_status, st);
    case 4: return fused_launch_4(d_rows, n_rows, steps, d_tw, d_status, st);
    case 5: return fused_launch_5(d_rows, n_rows, steps, d_tw, d_status, st);
    case 6: return fused_launch_6(d_rows, n_rows, steps, d_tw, d_status, st);
    case 7: return fused_launch_7(d_rows, n_rows, steps, d_tw, d_status, st);
    case 8: return fused2_launch_8(d_rows, n_rows, steps, d_tw, d_status, st);
    case 9: return fused2_launch_9(d_rows, n_rows, steps, d_tw, d_status, st);
    case 10: return fused2_launch_10(d_rows, n_rows, steps, d_tw, d_status, st);
    case 11: return fused2_launch_11(d_rows, n_rows, steps, d_tw, d_status, st);
    case 12: return fused2_launch_12(d_rows, n_rows, steps, d_tw, d_status, st);
    case 13: return fused4_launch_13(d_rows, n_rows, steps, d_tw, d_status, st);
    case 14: return fused4_launch_14(d_rows, n_rows, steps, d_tw, d_status, st);
    default: return fail(BPM_ERR_INVALID, "unsupported transform size");
  }
}

template <typename Cfg>
static void cfg4_of(int* smem, int* rows, int* threads) {
  *smem = Cfg::SMEM;
  *rows = 1;
  *threads = Cfg::T;
}

template <int L>
static void cfg_of(int* smem, int* rows, int* threads) {
  *smem = FusedCfg<L>::SMEM;
  *rows = FusedCfg<L>::ROWS;
  *threads = FusedCfg<L>::THREADS;
}

template <int L>
static void cfg2_of(int* smem, int* rows, int* threads) {
  *smem = F2Cfg<L>::SMEM;
  *rows = F2Cfg<L>::ROWS;
  *threads = F2Cfg<L>::THREADS;
}

static void fused_cfg(int logn, int* smem, int* rows, int* threads) {
  switch (logn) {
    case 3: cfg_of<3>(smem, rows, threads); break;
    case 4: cfg_of<4>(smem, rows, threads); break;
    case 5: cfg_of<5>(smem, rows, threads); break;
    case 6: cfg_of<6>(smem, rows, threads); break;
    case 7: cfg_of<7>(smem, rows, threads); break;
    case 8: cfg2_of<8>(smem, rows, threads); break;
    case 9: cfg2_of<9>(smem, rows, threads); break;
    case 10: cfg2_of<10>(smem, rows, threads); break;
    case 11: cfg2_of<11>(smem, rows, threads); break;
    case 12: cfg2_of<12>(smem, rows, threads); break;
    case 13: cfg4_of<F4ECfg<12>>(smem, rows, threads); break;
    default: cfg4_of<F4TCfg>(smem, rows, threads); break;
  }
}

// The lazily filled caches below are atomics: the request server's worker
// thread and callers' threads reach them concurrently (every writer stores
// the same value).
static int sm_count() {
  static std::atomic<int> cached{0};
  int sms = cached.load(std::memory_order_relaxed);
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    cached.store(sms, std::memory_order_relaxed);
  }
  return sms;
}

// Rows of size 2^logn that one launch keeps resident on the whole GPU (one
// CTA per row layout).  0 when a launch of n_rows would use the cluster
// layout, where every row already has its own SMs.
int fused_rows_resident(int logn, int n_rows) {
  if (logn >= kSplitLogN || use_cluster_layout(logn, n_rows)) return 0;
  static std::atomic<int> cache[kMaxLogN + 1] = {};
  int c = cache[logn].load(std::memory_order_relaxed);
  if (c == 0) {
    int r = 1;
    switch (logn) {
      case 3: r = fused_rows_resident_3(); break;
      case 4: r = fused_rows_resident_4(); break;
      case 5: r = fused_rows_resident_5(); break;
      case 6: r = fused_rows_resident_6(); break;
      case 7: r = fused_rows_resident_7(); break;
      case 8: r = fused2_rows_resident_8(); break;
      case 9: r = fused2_rows_resident_9(); break;
      case 10: r = fused2_rows_resident_10(); break;
      case 11: r = fused2_rows_resident_11(); break;
      default: r = fused2_rows_resident_12(); break;
    }
    c = r * sm_count();
    cache[logn].store(c, std::memory_order_relaxed);
  }
  return c;
}

// Rows one launch of the given layout keeps resident on the whole GPU:
// clusters for the cluster kernels (N >= 8192 always, 512..4096 when
// `cluster`), else CTA rows per SM times the SMs.
int fused_launch_capacity(int logn, bool cluster) {
  static std::atomic<int> cache[2][kMaxLogN + 1] = {};
  const bool cl = logn >= kSplitLogN || (cluster && logn >= 9 && logn <= 12);
  std::atomic<int>& slot = cache[cl ? 1 : 0][logn];
  int c = slot.load(std::memory_order_relaxed);
  if (c == 0) {
    if (cl) {
      switch (logn) {
        case 9: c = fused3_rows_resident_9(); break;
        case 10: c = fused3_rows_resident_10(); break;
        case 11: c = fused3_rows_resident_11(); break;
        case 12: c = fused3_rows_resident_12(); break;
        case 13: c = fused4_rows_resident_13(); break;
        default: c = fused4_rows_resident_14(); break;
      }
    } else {
      int r = 1;
      switch (logn) {
        case 3: r = fused_rows_resident_3(); break;
        case 4: r = fused_rows_resident_4(); break;
        case 5: r = fused_rows_resident_5(); break;
        case 6: r = fused_rows_resident_6(); break;
        case 7: r = fused_rows_resident_7(); break;
        case 8: r = fused2_rows_resident_8(); break;
        case 9: r = fused2_rows_resident_9(); break;
        case 10: r = fused2_rows_resident_10(); break;
        case 11: r = fused2_rows_resident_11(); break;
        default: r = fused2_rows_resident_12(); break;
      }
      c = r * sm_count();
    }
    slot.store(c, std::memory_order_relaxed);
  }
  return c;
}

// Rows one launch of the second-order (Verlet) CTA kernel keeps resident.
int fused_fr_capacity(int logn) {
  static std::atomic<int> cache[kMaxLogN + 1] = {};
  int c = cache[logn].load(std::memory_order_relaxed);
  if (c == 0) {
    int r = 1;
    switch (logn) {
      case 3: r = fusedf_rows_resident_3(); break;
      case 4: r = fusedf_rows_resident_4(); break;
      case 5: r = fusedf_rows_resident_5(); break;
      case 6: r = fusedf_rows_resident_6(); break;
      case 7: r = fusedf_rows_resident_7(); break;
      case 8: r = fused2f_rows_resident_8(); break;
      case 9: r = fused2f_rows_resident_9(); break;
      case 10: r = fused2f_rows_resident_10(); break;
      case 11: r = fused2f_rows_resident_11(); break;
      default: r = fused2f_rows_resident_12(); break;
    }
    c = r * sm_count();
    cache[logn].store(c, std::memory_order_relaxed);
  }
  return c;
}

int fused_half_capacity(int logn) {
  static std::atomic<int> cache[kMaxLogN + 1] = {};
  int c = cache[logn].load(std::memory_order_relaxed);
  if (c == 0) {
    int r = 1;
    switch (logn) {
      case 3: r = fusedh_rows_resident_3(); break;
      case 4: r = fusedh_rows_resident_4(); break;
      case 5: r = fusedh_rows_resident_5(); break;
      case 6: r = fusedh_rows_resident_6(); break;
      case 7: r = fusedh_rows_resident_7(); break;
      case 8: r = fused2h_rows_resident_8(); break;
      case 9: r = fused2h_rows_resident_9(); break;
      case 10: r = fused2h_rows_resident_10(); break;
      case 11: r = fused2h_rows_resident_11(); break;
      default: r = fused2h_rows_resident_12(); break;
    }
    c = r * sm_count();
    cache[logn].store(c, std::memory_order_relaxed);
  }
  return c;
}

// Rows one launch of the second-order (Verlet) 2-CTA cluster kernel keeps
// resident (clusters).
int fused_cluster_half_capacity(int logn) {
  static std::atomic<int> cache[kMaxLogN + 1] = {};
  int c = cache[logn].load(std::memory_order_relaxed);
  if (c == 0) {
    switch (logn) {
      case 9: c = fused3h_rows_resident_9(); break;
      case 10: c = fused3h_rows_resident_10(); break;
      case 11: c = fused3h_rows_resident_11(); break;
      default: c = fused3h_rows_resident_12(); break;
    }
    cache[logn].store(c, std::memory_order_relaxed);
  }
  return c;
}

// Rows one launch of the fourth-order (Forest-Ruth) 2-CTA cluster kernel
// keeps resident (clusters).
int fused_cluster_fr_capacity(int logn) {
  static std::atomic<int> cache[kMaxLogN + 1] = {};
  int c = cache[logn].load(std::memory_order_relaxed);
  if (c == 0) {
    switch (logn) {
      case 9: c = fused3f_rows_resident_9(); break;
      case 10: c = fused3f_rows_resident_10(); break;
      case 11: c = fused3f_rows_resident_11(); break;
      default: c = fused3f_rows_resident_12(); break;
    }
    cache[logn].store(c, std::memory_order_relaxed);
  }
  return c;
}

// Rows of N = 4096 one second-order half-band-split launch keeps resident.
int fused_split4_half_capacity() {
  static std::atomic<int> cached{0};
  int c = cached.load(std::memory_order_relaxed);
  if (c == 0) {
    c = std::min(fused4sh_rows_resident_12(), fused4hh_rows_resident_12());
    cached.store(c, std::memory_order_relaxed);
  }
  return c;
}

// Positions of the Forest-Ruth stage tables in the split kernels' thread
// order: entry j T + t of a band's D(k) or D(k + M) table (M entries) holds
// the position that thread t reads as its point j of the last pass, in the
// N = 4096 half-band split (8 points per thread) or the N = 8192 split band
// (16), computed by the kernels' own mapping.
int fr_split_table_order(int logn, std::vector<int>* pos) {
  if (logn == 12) {
    using C = F4SCfg<>;
    pos->assign(C::M, 0);
    for (int j = 0; j < C::M / C::T; ++j)
      for (int t = 0; t < C::T; ++t) (*pos)[j * C::T + t] = s4_table_pos(t, j);
    return BPM_OK;
  }
  if (logn == 13) {
    using C = F4ECfg<12>;
    pos->assign(C::M, 0);
    for (int j = 0; j < C::M / C::T; ++j)
      for (int t = 0; t < C::T; ++t) (*pos)[j * C::T + t] = f4e_table_pos<12>(t, j);
    return BPM_OK;
  }
  return fail(BPM_ERR_INVALID, "thread-order tables exist for nx = 4096 and 8192 only");
}

template <int LOGN>
static void f2_table_order(std::vector<int>* pos) {
  using C = F2Cfg<LOGN>;
  pos->assign(C::N, 0);
  for (int k = 0; k < C::E; ++k)
    for (int t = 0; t < C::T; ++t) (*pos)[k * C::T + t] = f2_table_pos<LOGN>(t, k);
}

// Positions of the Forest-Ruth stage tables of the one-CTA kernels: for
// 256 <= N <= 4096 the band-per-thread kernel's thread order (entry k T + t
// of a band's table holds the position of thread t's point k of the last
// pass), for N <= 128 the position order itself.
int fr_cta_table_order(int logn, std::vector<int>* pos) {
  switch (logn) {
    case 8: f2_table_order<8>(pos); return BPM_OK;
    case 9: f2_table_order<9>(pos); return BPM_OK;
    case 10: f2_table_order<10>(pos); return BPM_OK;
    case 11: f2_table_order<11>(pos); return BPM_OK;
    case 12: f2_table_order<12>(pos); return BPM_OK;
    default: break;
  }
  if (logn < 3 || logn > 7) return fail(BPM_ERR_INVALID, "one-CTA tables exist for nx <= 4096");
  pos->resize(size_t(1) << logn);
  for (size_t i = 0; i < pos->size(); ++i) (*pos)[i] = int(i);
  return BPM_OK;
}

// Rows of N = 4096 one fourth-order half-band-split launch keeps resident.
int fused_split4_fr_capacity() {
  static std::atomic<int> cached{0};
  int c = cached.load(std::memory_order_relaxed);
  if (c == 0) {
    c = fused4sf_rows_resident_12();
    cached.store(c, std::memory_order_relaxed);
  }
  return c;
}

// Rows of N = 4096 one half-band-split launch keeps resident (4-CTA clusters).
int fused_split4_capacity() {
  static std::atomic<int> cached{0};
  int c = cached.load(std::memory_order_relaxed);
  if (c == 0) {
    c = fused4s_rows_resident_12();
    cached.store(c, std::memory_order_relaxed);
  }
  return c;
}

int fused_smem_bytes(int logn) { int a, b, c; fused_cfg(logn, &a, &b, &c); return a; }
int fused_rows_per_cta(int logn) { int a, b, c; fused_cfg(logn, &a, &b, &c); return b; }
int fused_threads(int logn) { int a, b, c; fused_cfg(logn, &a, &b, &c); return c; }

}  // namespace bpm
