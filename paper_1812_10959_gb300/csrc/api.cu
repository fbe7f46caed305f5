// C ABI of the DIC library (include/dic.h): database loading, the host side
// of ParallelDIC's stop loop (Algorithm 2), results and errors.
//
// The loop itself runs on the device: every stop is the kernel sequence
//   count (Algorithm 3) -> promote/prune (Algorithm 4) -> box-set insert ->
//   generate (MAKECANDIDATES) -> finish (Algorithm 5, trace, loop test)
// and all loop state lives in a device-resident Ctrl record, so the host
// enqueues several stops at a time and only reads Ctrl back between groups
// (to stop when DASHED is empty, or to grow a buffer a kernel found short).
#include <algorithm>
#include <atomic>
#include <cstddef>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/dic.h"
#include "dic_internal.cuh"

using namespace dic;

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error;

static dic_status fail(dic_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

void dic::set_last_error(const char *msg) { g_last_error = msg ? msg : ""; }

bool &dic::pdl_enabled() {
  static thread_local bool on = false;
  return on;
}

#define CU(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      return fail(e_ == cudaErrorMemoryAllocation ? DIC_ENOMEM : DIC_ECUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                   \
    }                                                                                   \
  } while (0)

#define TRY(expr)                      \
  do {                                 \
    dic_status st_ = (expr);           \
    if (st_ != DIC_OK) return st_;     \
  } while (0)

// ---------------------------------------------------------------- objects
struct dic_db {
  uint64_t *words = nullptr;  // device, n*W
  uint64_t n = 0;
  uint32_t m = 0, W = 0;
  int device = 0;
  std::atomic<int> busy{0};
};

struct dic_result {
  uint32_t W = 0;
  std::vector<uint64_t> masks;  // count*W
  std::vector<uint32_t> k, supp;
  std::vector<uint64_t> trace;  // rows*TRACE_COLS
  dic_stats stats{};
};

// Page-locked host blocks are kept for reuse by later calls: allocating and
// releasing them (cudaMallocHost / cudaFreeHost) costs far more than a mine's
// own device work at small sizes. Blocks are reused by size class (powers of
// two from 256 bytes) and live until the process exits.
namespace {
std::mutex g_pinned_mu;
std::unordered_map<size_t, std::vector<void *>> g_pinned_free;
size_t pinned_class(size_t bytes) {
  size_t c = 256;
  while (c < bytes) c <<= 1;
  return c;
}
}  // namespace

static cudaError_t pinned_alloc(void **p, size_t bytes) {
  const size_t c = pinned_class(bytes);
  {
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    auto it = g_pinned_free.find(c);
    if (it != g_pinned_free.end() && !it->second.empty()) {
      *p = it->second.back();
      it->second.pop_back();
      return cudaSuccess;
    }
  }
  return cudaMallocHost(p, c);
}

static void pinned_free(void *p, size_t bytes) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pinned_mu);
  g_pinned_free[pinned_class(bytes)].push_back(p);
}

// Allocation-failure injection (dic_debug_fail_device_alloc): the calling
// thread's next `after` working-buffer allocations succeed, the one after
// them fails as if the device were out of memory, later ones succeed.
static thread_local int64_t g_fail_alloc_after = -1;
static bool injected_alloc_failure() {
  if (g_fail_alloc_after < 0) return false;
  if (g_fail_alloc_after == 0) {
    g_fail_alloc_after = -1;
    return true;
  }
  --g_fail_alloc_after;
  return false;
}

// Graphs and events of finished mines are destroyed by a later call, after
// it has started its first-pass kernel (the destruction then overlaps device
// work instead of delaying the finished mine's result).
namespace {
std::mutex g_retire_mu;
std::vector<std::pair<cudaGraphExec_t, cudaGraph_t>> g_retired_graphs;
std::vector<cudaEvent_t> g_retired_events;
// Streams of finished calls, for reuse (one call at a time per stream).
std::mutex g_stream_mu;
std::vector<std::pair<int, cudaStream_t>> g_free_streams;
}  // namespace

static void retire_graph(cudaGraphExec_t e, cudaGraph_t g) {
  std::lock_guard<std::mutex> lk(g_retire_mu);
  g_retired_graphs.push_back({e, g});
}
static void retire_event(cudaEvent_t e) {
  std::lock_guard<std::mutex> lk(g_retire_mu);
  g_retired_events.push_back(e);
}
static void drain_retired() {
  std::vector<std::pair<cudaGraphExec_t, cudaGraph_t>> gs;
  std::vector<cudaEvent_t> es;
  {
    std::lock_guard<std::mutex> lk(g_retire_mu);
    gs.swap(g_retired_graphs);
    es.swap(g_retired_events);
  }
  for (auto &p : gs) {
    if (p.first) cudaGraphExecDestroy(p.first);
    if (p.second) cudaGraphDestroy(p.second);
  }
  for (cudaEvent_t e : es) cudaEventDestroy(e);
}
static cudaError_t take_stream(int dev, cudaStream_t *s) {
  {
    std::lock_guard<std::mutex> lk(g_stream_mu);
    for (size_t i = 0; i < g_free_streams.size(); ++i)
      if (g_free_streams[i].first == dev) {
        *s = g_free_streams[i].second;
        g_free_streams.erase(g_free_streams.begin() + i);
        return cudaSuccess;
      }
  }
  return cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
}
static void give_stream(int dev, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_stream_mu);
  g_free_streams.push_back({dev, s});
}

// A page-locked host staging buffer from the reuse cache above.
template <class T>
struct PinnedBuf {
  T *p = nullptr;
  size_t bytes = 0;
  cudaError_t get(size_t count) {
    bytes = std::max<size_t>(count * sizeof(T), 16);
    return pinned_alloc((void **)&p, bytes);
  }
  ~PinnedBuf() { pinned_free(p, bytes); }
};

// Itemset mask arrays of freed results, reused by later results (a fresh
// array of this size would page-fault on every page as it is first written).
namespace {
std::mutex g_mask_pool_mu;
std::vector<std::vector<uint64_t>> g_mask_pool;
}  // namespace

static std::vector<uint64_t> take_mask_array(size_t words) {
  std::vector<uint64_t> v;
  {
    std::lock_guard<std::mutex> lk(g_mask_pool_mu);
    size_t best = g_mask_pool.size();
    for (size_t i = 0; i < g_mask_pool.size(); ++i)
      if (g_mask_pool[i].capacity() >= words &&
          (best == g_mask_pool.size() || g_mask_pool[i].capacity() < g_mask_pool[best].capacity()))
        best = i;
    if (best < g_mask_pool.size()) {
      v = std::move(g_mask_pool[best]);
      g_mask_pool.erase(g_mask_pool.begin() + best);
    }
  }
  v.assign(words, 0);
  return v;
}

static void give_mask_array(std::vector<uint64_t> &&v) {
  if (v.capacity() < (1u << 12)) return;
  std::lock_guard<std::mutex> lk(g_mask_pool_mu);
  if (g_mask_pool.size() < 8) g_mask_pool.push_back(std::move(v));
}

static void init_pool(int dev) {
  static std::atomic<uint64_t> done_mask{0};
  if (dev < 64 && (done_mask.load() >> dev) & 1) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  if (dev < 64) done_mask.fetch_or(1ull << dev);
}

// Free device memory for the prestaging rule, refreshed at most every
// 50 ms per device (the query costs tens of microseconds; the rule only
// needs its order of magnitude).
static size_t free_device_memory() {
  static std::mutex mu;
  static std::map<int, std::pair<std::chrono::steady_clock::time_point, size_t>> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  const auto now = std::chrono::steady_clock::now();
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(dev);
  if (it != cache.end() && now - it->second.first < std::chrono::milliseconds(50))
    return it->second.second;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    free_b = 0;
  }
  cache[dev] = {now, free_b};
  return free_b;
}

static int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

// ----------------------------------------------------------------- loading
static dic_status new_db(uint64_t n, uint32_t m, dic_db **out) {
  if (m == 0) return fail(DIC_EINVAL, "m must be > 0");
  if (n >= (1ull << 31)) return fail(DIC_EINVAL, "n must be < 2^31 (got %llu)", (unsigned long long)n);
  dic_db *db = new (std::nothrow) dic_db();
  if (!db) return fail(DIC_ENOMEM, "host allocation");
  db->n = n;
  db->m = m;
  db->W = (m + 63) / 64;
  cudaGetDevice(&db->device);
  init_pool(db->device);
  if (n) {
    cudaError_t e = cudaMalloc(&db->words, (size_t)n * db->W * 8);
    if (e != cudaSuccess) {
      delete db;
      return fail(DIC_ENOMEM, "device allocation of %llu bytes: %s",
                  (unsigned long long)(n * db->W * 8), cudaGetErrorString(e));
    }
  }
  *out = db;
  return DIC_OK;
}

extern "C" dic_status dic_load_db(const uint64_t *words, uint64_t n, uint32_t m, dic_db **out) {
  if (!out) return fail(DIC_EINVAL, "out is NULL");
  *out = nullptr;
  if (n && !words) return fail(DIC_EINVAL, "words is NULL");
  if (m == 0) return fail(DIC_EINVAL, "m must be > 0");
  const uint32_t W = (m + 63) / 64;
  if (m % 64) {
    const uint64_t pad = ~((1ull << (m % 64)) - 1);
    for (uint64_t t = 0; t < n; ++t)
      if (words[t * W + W - 1] & pad)
        return fail(DIC_EINVAL, "row %llu has a bit set at an item >= m", (unsigned long long)t);
  }
  dic_db *db = nullptr;
  TRY(new_db(n, m, &db));
  if (n) {
    cudaError_t e = cudaMemcpy(db->words, words, (size_t)n * W * 8, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(db->words);
      delete db;
      return fail(DIC_ECUDA, "copy to device: %s", cudaGetErrorString(e));
    }
  }
  *out = db;
  return DIC_OK;
}

extern "C" dic_status dic_load_db_csr(const uint64_t *row_ptr, const uint32_t *items, uint64_t n,
                                      uint32_t m, dic_db **out) {
  if (!out) return fail(DIC_EINVAL, "out is NULL");
  *out = nullptr;
  if (!row_ptr) return fail(DIC_EINVAL, "row_ptr is NULL");
  if (row_ptr[0] != 0) return fail(DIC_EINVAL, "row_ptr[0] must be 0");
  for (uint64_t t = 0; t < n; ++t)
    if (row_ptr[t + 1] < row_ptr[t])
      return fail(DIC_EINVAL, "row_ptr decreases at row %llu", (unsigned long long)t);
  const uint64_t nnz = row_ptr[n];
  if (nnz && !items) return fail(DIC_EINVAL, "items is NULL");
  dic_db *db = nullptr;
  TRY(new_db(n, m, &db));
  if (n == 0) { *out = db; return DIC_OK; }
  cudaStream_t s;
  uint64_t *d_rp = nullptr;
  uint32_t *d_it = nullptr, *d_bad = nullptr;
  uint32_t bad = 0;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_rp, (n + 1) * 8, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_it, (nnz ? nnz : 1) * 4, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_bad, 4, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_rp, row_ptr, (n + 1) * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(d_it, items, nnz * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(db->words, 0, (size_t)n * db->W * 8, s);
  if (e == cudaSuccess) e = launch_pack_csr(d_rp, d_it, n, m, db->W, db->words, d_bad, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFreeAsync(d_rp, s);
  cudaFreeAsync(d_it, s);
  cudaFreeAsync(d_bad, s);
  cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  if (e != cudaSuccess || bad) {
    cudaFree(db->words);
    delete db;
    if (e != cudaSuccess) return fail(DIC_ECUDA, "csr load: %s", cudaGetErrorString(e));
    return fail(DIC_EINVAL, "an item id is >= m");
  }
  *out = db;
  return DIC_OK;
}

extern "C" dic_status dic_load_db_device(const uint64_t *dev_words, uint64_t n, uint32_t m,
                                         void *stream, dic_db **out) {
  if (!out) return fail(DIC_EINVAL, "out is NULL");
  *out = nullptr;
  if (n && !dev_words) return fail(DIC_EINVAL, "dev_words is NULL");
  dic_db *db = nullptr;
  TRY(new_db(n, m, &db));
  if (n == 0) { *out = db; return DIC_OK; }
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t *d_bad = nullptr, bad = 0;
  cudaError_t e = cudaMemcpyAsync(db->words, dev_words, (size_t)n * db->W * 8,
                                  cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_bad, 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, 4, s);
  if (e == cudaSuccess) e = launch_check_padding(db->words, n, m, db->W, d_bad, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (d_bad) cudaFreeAsync(d_bad, s);
  if (e != cudaSuccess || bad) {
    cudaStreamSynchronize(s);
    cudaFree(db->words);
    delete db;
    if (e != cudaSuccess) return fail(DIC_ECUDA, "device load: %s", cudaGetErrorString(e));
    return fail(DIC_EINVAL, "a row has a bit set at an item >= m");
  }
  *out = db;
  return DIC_OK;
}

extern "C" dic_status dic_db_free(dic_db *db) {
  if (!db) return DIC_OK;
  if (db->busy.load()) return fail(DIC_EBUSY, "database has queries in flight");
  if (db->words) cudaFree(db->words);
  delete db;
  return DIC_OK;
}

extern "C" uint64_t dic_db_rows(const dic_db *db) { return db ? db->n : 0; }
extern "C" uint32_t dic_db_items(const dic_db *db) { return db ? db->m : 0; }
extern "C" const uint64_t *dic_db_device_words(const dic_db *db) { return db ? db->words : nullptr; }

// ------------------------------------------------------------------ mining
extern "C" void dic_options_init(dic_options *o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->struct_size = sizeof *o;
  o->count_path = DIC_COUNT_AUTO;
  o->steps_per_sync = 0;
  o->use_graph = 1;
  o->profile = 0;
  o->max_candidates = 0;
}

namespace {

// A device allocation released on the mining stream.
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
};

class Miner {
 public:
  Miner(const dic_db *db, uint32_t minsup, uint64_t M, const dic_options &opt, cudaStream_t s)
      : db_(db), minsup_(minsup), M_(M), opt_(opt), s_(s), forced_tw_((int)opt.tile_words) {}
  ~Miner() { release(); }

  dic_status run(dic_result **out);
  // run() in phases, for the batched driver: begin() enqueues the first pass;
  // after a stream synchronisation prepare() builds the lattice; loop() runs
  // the remaining stops alone; collect() returns the result.
  dic_status begin();
  dic_status prepare();
  dic_status loop();
  dic_status collect(dic_result **out);
  // Use a loop-state record owned by the caller (device and pinned host
  // copies); call before begin().
  void use_external_ctrl(Ctrl *dev, Ctrl *host) { ext_ctrl_ = dev; h_ctrl_ = host; }
  bool has_loop() const { return has_loop_; }
  Lattice &lattice() { return L_; }
  Ctrl *host_ctrl() { return h_ctrl_; }
  bool bitslice_ready() const { return bs_ok_; }
  uint32_t l1p() const { return bs_l1p_; }
  int tile_words_per_rank() const { return bs_tw_; }
  uint64_t stop_max() const { return stop_max64_; }
  // Recover a stop that stalled (grow what it needs, re-run it from the
  // stalled phase with this query's own kernels); no-op without a stall.
  dic_status recover();
  // Grow what the next `stops` stops may need before they are enqueued.
  dic_status reserve(uint32_t stops);
  void set_forced_tw(int tw) { forced_tw_ = tw; }
  // Rebuild the BITSLICE column buffer for another tile width (the batched
  // count uses one width for all queries). False if it does not fit.
  dic_status set_tile_width(int tw, bool *ok);
  uint32_t launches() const { return launches_; }
  void add_launches(uint32_t k) { launches_ += k; }

 private:
  template <class T>
  dic_status alloc(T **p, size_t count, bool zero = false) {
    size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    if (injected_alloc_failure())
      return fail(DIC_ENOMEM, "device allocation of %zu bytes: injected failure", bytes);
    cudaError_t e = cudaMallocAsync((void **)p, bytes, s_);
    if (e != cudaSuccess) return fail(DIC_ENOMEM, "device allocation of %zu bytes: %s", bytes,
                                      cudaGetErrorString(e));
    bufs_.push_back(*p);
    if (zero) CU(cudaMemsetAsync(*p, 0, bytes, s_));
    return DIC_OK;
  }
  template <class T>
  void drop(T *p) {
    if (!p) return;
    auto it = std::find(bufs_.begin(), bufs_.end(), (void *)p);
    if (it != bufs_.end()) bufs_.erase(it);
    cudaFreeAsync(p, s_);
  }
  void release() {
    for (void *p : bufs_) cudaFreeAsync(p, s_);
    bufs_.clear();
    for (auto &sg : graphs_) retire_graph(sg.exec, sg.graph);
    graphs_.clear();
    for (cudaEvent_t ev : ev_pool_) retire_event(ev);
    ev_pool_.clear();
    ev_used_ = 0;
    if (h_ctrl_ && own_h_ctrl_) { pinned_free(h_ctrl_, sizeof(Ctrl)); h_ctrl_ = nullptr; }
    if (h_cnt1_) { pinned_free(h_cnt1_, (size_t)db_->m * 4); h_cnt1_ = nullptr; }
    if (fa_) { cudaEventDestroy(fa_); fa_ = nullptr; }
    if (fb_) { cudaEventDestroy(fb_); fb_ = nullptr; }
    if (ev_fork_) { cudaEventDestroy(ev_fork_); ev_fork_ = nullptr; }
    if (ev_join_) { cudaEventDestroy(ev_join_); ev_join_ = nullptr; }
    if (s2_) { cudaStreamDestroy(s2_); s2_ = nullptr; }
    if (ev_slice_) { cudaEventDestroy(ev_slice_); ev_slice_ = nullptr; }
    if (eg0_) { cudaEventDestroy(eg0_); eg0_ = nullptr; }
    if (eg1_) { cudaEventDestroy(eg1_); eg1_ = nullptr; }
    if (s3_) { cudaStreamDestroy(s3_); s3_ = nullptr; }
    if (evx_) { retire_graph(evx_, evg_); evx_ = nullptr; evg_ = nullptr; }
  }

  dic_status grow_candidates(uint32_t need);
  dic_status grow_hash(uint64_t entries);
  dic_status next_event(cudaEvent_t *ev);
  dic_status record(cudaEvent_t ev, cudaStream_t st);
  dic_status harvest_events();
  dic_status grow_trace(uint32_t need);
  dic_status launch_phase(int phase);
  dic_status launch_stop_from(int phase);
  dic_status sync_ctrl();
  int count_path_for_stop() const;
  uint32_t stop_profile_bits() const;

  const dic_db *db_;
  uint32_t minsup_;
  uint64_t M_;
  dic_options opt_;
  cudaStream_t s_;
  std::vector<void *> bufs_;
  std::vector<cudaEvent_t> ev_pool_;   // profiling events, reused every group
  size_t ev_used_ = 0;
  // profiled intervals: (start, end) pool indices and what they time
  enum IvKind { IV_COUNT = 0, IV_GRAM = 1, IV_SETTLE = 2, IV_GEN = 3 };
  struct Interval { size_t start, end; int kind; };
  std::vector<Interval> intervals_;
  size_t iv_start_ = 0;
  int iv_kind_ = 0;
  dic_status iv_open(int kind, cudaStream_t st);
  dic_status iv_close(cudaStream_t st);
  // profiling bits in force for the stop being enqueued (profile_every)
  uint32_t prof_now_ = 0;
  bool prof(uint32_t bit) const { return (prof_now_ & bit) != 0; }
  double settle_ms_ = 0, gen_ms_ = 0;
  uint64_t gen_timed_ = 0;
  double count_ms_ = 0;
  uint64_t count_timed_ = 0;
  Lattice L_{};
  Ctrl *h_ctrl_ = nullptr;
  uint32_t nw_ = 2;  // rows-kernel width bucket
  // BITSLICE path state
  bool bs_ok_ = false;     // the block's columns fit in shared memory
  int bs_tw_ = 16;         // 32-row words per tile
  uint32_t bs_l1p_ = 0;    // l1 rounded up to a multiple of 4
  uint32_t *bs_V_ = nullptr;
  uint64_t bs_V_words_ = 0;
  int bs_grid_ = 0;
  size_t smem_optin_ = 0;
  int cur_path_ = DIC_COUNT_ROWS;
  bool next_v_ready_ = false;  // the enqueued work builds V for the next count
  // TENSOR path (pair cohort on tcgen05)
  bool tc_ok_ = false;
  uint32_t tc_nkc_max_ = 0, tc_nsplit_ = 1;
  cudaStream_t s2_ = nullptr;  // side stream of the pair-cohort kernels
  cudaStream_t s3_ = nullptr;  // side stream of the next block's transposition
  cudaEvent_t ev_slice_ = nullptr;
  bool vdouble_ = false;       // double-buffered columns (single-query loop)
  bool direct_ = false;        // the counted window was small at the last sync
  cudaEvent_t ev_fork_ = nullptr, ev_join_ = nullptr;
  uint32_t pred_step_ = 1;     // stop number the next enqueued count runs at
  double gram_ms_ = 0;
  uint64_t gram_timed_ = 0;
  // CUDA graphs: one captured stop per variant, replayed stop after stop
  struct StopGraph {
    int path = 0, kre = 0;
    uint32_t nstops = 1;  // stops captured back to back in this graph
    bool gram = false, slice = false, direct = false;
    uint32_t profile = 0;  // DIC_PROFILE_* bits captured as event nodes
    uint32_t nw = 0;
    uint64_t version = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaGraphNode_t> ev_nodes;  // event records in recording order
    std::vector<Interval> ivs;              // intervals, relative to the first event
    uint32_t kernels = 0;
    uint32_t path_counts[4] = {0, 0, 0, 0};
  };
  std::vector<StopGraph> graphs_;
  uint64_t lat_version_ = 1;  // bumped whenever a buffer of the lattice changes
  // `nstops` stops: one graph replay (captured once per shape) or direct
  // launches
  dic_status launch_stop(uint32_t nstops = 1);
  int grid_ = 0;
  int gen_grid_ = 0;  // MAKECANDIDATES CTAs when no transposition rides along
  uint32_t launches_ = 0;
  uint32_t path_launches_[4] = {0, 0, 0, 0};
  uint64_t candidates_cap_limit_ = 0xFFFFFFF0ull;
  // phase state
  std::chrono::steady_clock::time_point t0_;
  std::unique_ptr<dic_result> res_;
  uint64_t n_ = 0, stop_max64_ = 0, tests_ = 0;
  uint32_t *h_cnt1_ = nullptr;
  cudaEvent_t fa_ = nullptr, fb_ = nullptr;
  std::vector<uint32_t> l1items_;
  // result itemsets, flat: items of itemset q at set_items_[set_off_[q] ..
  // set_off_[q + 1]) in ascending order, its support supps_[q]
  std::vector<uint32_t> set_items_, set_off_;
  std::vector<uint32_t> supps_;
  size_t n_first_ = 0;  // leading itemsets from the first pass (item order)
  size_t n_ordered_ = 0;  // leading itemsets already in canonical order
  bool has_loop_ = false;
  Ctrl *ext_ctrl_ = nullptr;
  bool own_h_ctrl_ = false;
  int forced_tw_ = 0;
  // every block's columns staged before the loop (L_.vall), the pair cohort
  // counted over the whole pass with precomputed events (L_.pair_events),
  // and the stop kernels chained by programmatic dependent launch
  bool vall_ = false, events_ = false, pc_wide_ = false, pdl_ = false;
  int32_t *d_rank_ = nullptr;  // rank of each item (-1: not frequent), chunk
                               // starts, then the item of each rank
  size_t item_of_off_ = 0;     // where the item of each rank starts in d_rank_
  bool rows_ready_ = false;    // L_.rows (compacted rows) built
  cudaEvent_t eg0_ = nullptr, eg1_ = nullptr;  // the all-blocks GEMM, profiled
  double setup_ms_ = 0, graph_ms_ = 0;         // host timings (dic_stats)
  dic_status ensure_rows();
  // event-driven loop (L_.events): the cohort pass and the generate kernel
  // replayed in a device-side WHILE loop of one graph (rebuilt when a buffer
  // of the lattice changes), or launched directly when they are profiled
  bool evmode_ = false;
  bool ev_ok_ = false;       // the event-driven form can take the loop
  bool ev_switched_ = false; // it took over from the per-stop form
  uint64_t switch_step_ = 0;  // first stop it closed
  dic_status switch_to_events();
  dic_status alloc_event_buffers();
  cudaGraph_t evg_ = nullptr;
  cudaGraphExec_t evx_ = nullptr;
  uint64_t evg_version_ = 0;
  cudaGraphConditionalHandle evh_ = 0;
  int cp_grid_ = 0;
  std::vector<uint32_t> prof_iters_;  // iterations launched with profiling
  dic_status alloc_event_tallies(uint32_t ehcap);
  dic_status launch_event_body(bool in_graph);
  dic_status ensure_event_graph();
  dic_status loop_events();
  dic_status recover_events();
};

// Compacted rows (only the frequent items, by rank) for the kernels that
// read rows: the ROWS count and the per-stop transposition.
dic_status Miner::ensure_rows() {
  if (rows_ready_) return DIC_OK;
  const uint32_t wc = std::max<uint32_t>(1, ((uint32_t)l1items_.size() + 63) / 64);
  uint64_t *d_rows = nullptr;
  TRY(alloc(&d_rows, (size_t)n_ * wc));
  CU(launch_compact_rows(db_->words, n_, db_->W, d_rank_, d_rows, wc, s_));
  ++launches_;
  L_.rows = d_rows;
  rows_ready_ = true;
  ++lat_version_;
  return DIC_OK;
}

// Count path for the next stops: BITSLICE whenever the block's columns fit in
// shared memory and every dashed itemset has at most KRMAX items, else ROWS.
int Miner::count_path_for_stop() const {
  if (opt_.count_path == DIC_COUNT_ROWS) return DIC_COUNT_ROWS;
  if (!bs_ok_ || h_ctrl_->max_k > (uint32_t)KRMAX) return DIC_COUNT_ROWS;
  return tc_ok_ ? DIC_COUNT_TENSOR : DIC_COUNT_BITSLICE;
}

static int kr_bucket(uint32_t max_k) {
  if (max_k <= 2) return 2;
  if (max_k <= 4) return 4;
  if (max_k <= 8) return 8;
  return 16;
}

// Record a profiling event; inside a stream capture it must become an event
// record node of the graph (a plain record would only add a dependency).
dic_status Miner::record(cudaEvent_t ev, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CU(cudaStreamIsCapturing(st, &cs));
  if (cs == cudaStreamCaptureStatusActive)
    CU(cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal));
  else
    CU(cudaEventRecord(ev, st));
  return DIC_OK;
}

dic_status Miner::next_event(cudaEvent_t *ev) {
  if (ev_used_ == ev_pool_.size()) {
    cudaEvent_t e;
    CU(cudaEventCreate(&e));
    ev_pool_.push_back(e);
  }
  *ev = ev_pool_[ev_used_++];
  return DIC_OK;
}

// Sum the count-kernel event pairs recorded since the last group (the
// stream has been synchronised).
dic_status Miner::iv_open(int kind, cudaStream_t st) {
  cudaEvent_t e;
  TRY(next_event(&e));
  TRY(record(e, st));
  iv_start_ = ev_used_ - 1;
  iv_kind_ = kind;
  return DIC_OK;
}

dic_status Miner::iv_close(cudaStream_t st) {
  cudaEvent_t e;
  TRY(next_event(&e));
  TRY(record(e, st));
  intervals_.push_back({iv_start_, ev_used_ - 1, iv_kind_});
  return DIC_OK;
}

dic_status Miner::harvest_events() {
  for (const Interval &iv : intervals_) {
    float ms = 0;
    CU(cudaEventElapsedTime(&ms, ev_pool_[iv.start], ev_pool_[iv.end]));
    if (iv.kind == IV_COUNT) { count_ms_ += ms; ++count_timed_; }
    else if (iv.kind == IV_GRAM) { gram_ms_ += ms; ++gram_timed_; }
    else if (iv.kind == IV_GEN) { gen_ms_ += ms; ++gen_timed_; }
    else settle_ms_ += ms;
  }
  intervals_.clear();
  ev_used_ = 0;
  return DIC_OK;
}

dic_status Miner::sync_ctrl() {
  CU(cudaMemcpyAsync(h_ctrl_, L_.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s_));
  CU(cudaStreamSynchronize(s_));
  if (opt_.profile) TRY(harvest_events());
  return DIC_OK;
}

dic_status Miner::launch_phase(int phase) {
  cudaError_t e = cudaSuccess;
  switch (phase) {
    case PH_COUNT: {
      if (cur_path_ == DIC_COUNT_BITSLICE || cur_path_ == DIC_COUNT_TENSOR) {
        // shared memory for the largest chunk that fits; the kernel sizes its
        // chunk from the live window
        const int kre = kr_bucket(std::max<uint32_t>(h_ctrl_->max_k, 4));
        const uint32_t chunk = std::min<uint32_t>(
            bitslice_max_chunk(bs_tw_, kre, bs_l1p_, smem_optin_), 1u << 20);
        if (!next_v_ready_ && !L_.vall) {
          e = launch_slice_block(L_, 0, s_);
          ++launches_;
        }
        next_v_ready_ = false;
        const bool gram =
            cur_path_ == DIC_COUNT_TENSOR && !L_.pair_events && pred_step_ <= L_.stop_max;
        if (e == cudaSuccess && (gram || L_.vdouble)) CU(cudaEventRecord(ev_fork_, s_));
        if (e == cudaSuccess && L_.vdouble) {
          // fork: the next stop's block is transposed into the other column
          // buffer on its own stream while this one is counted (the stop
          // number it reads changes only at the end of generation, which
          // waits for it)
          CU(cudaStreamWaitEvent(s3_, ev_fork_, 0));
          e = launch_slice_block(L_, 1, s3_);
          CU(cudaEventRecord(ev_slice_, s3_));
          ++launches_;
        }
        if (e == cudaSuccess && gram) {
          // fork: the pair cohort (in DASHED up to stop_max) is counted on the
          // tensor cores and pruned on the side stream while the rest of the
          // window is counted here; generation waits for both
          CU(cudaStreamWaitEvent(s2_, ev_fork_, 0));
          if (prof(DIC_PROFILE_GRAM)) TRY(iv_open(IV_GRAM, s2_));
          e = launch_gram_pairs(L_, tc_nsplit_, (uint32_t)kre, s2_);
          if (prof(DIC_PROFILE_GRAM)) TRY(iv_close(s2_));
          if (e == cudaSuccess) {
            if (prof(DIC_PROFILE_SETTLE)) TRY(iv_open(IV_SETTLE, s2_));
            e = launch_settle_pairs(L_, grid_, (uint32_t)kre, s2_);
            if (prof(DIC_PROFILE_SETTLE)) TRY(iv_close(s2_));
          }
          CU(cudaEventRecord(ev_join_, s2_));
          launches_ += 2;
          path_launches_[DIC_COUNT_TENSOR]++;
        }
        if (e == cudaSuccess) {
          if (prof(DIC_PROFILE_COUNT)) TRY(iv_open(IV_COUNT, s_));
          // (the direct form: one resident wave of CTAs at its register
          // use; warps stride over the records)
          e = launch_count_bitslice(L_, bs_V_, bs_tw_, kre, bs_l1p_, chunk, bs_V_words_,
                                    direct_ ? sm_count() * count_direct_ctas_per_sm(kre)
                                            : bs_grid_,
                                    direct_, s_);
          if (prof(DIC_PROFILE_COUNT)) TRY(iv_close(s_));
        }
        if (gram) CU(cudaStreamWaitEvent(s_, ev_join_, 0));  // join
        if (L_.vdouble) CU(cudaStreamWaitEvent(s_, ev_slice_, 0));
        path_launches_[DIC_COUNT_BITSLICE]++;
      } else {
        if (prof(DIC_PROFILE_COUNT)) TRY(iv_open(IV_COUNT, s_));
        e = launch_count_rows(L_, (int)nw_, grid_, s_);
        if (prof(DIC_PROFILE_COUNT)) TRY(iv_close(s_));
        path_launches_[DIC_COUNT_ROWS]++;
      }
      break;
    }
    case PH_PROMOTE: e = launch_promote(L_, grid_, s_); break;
    case PH_HASH: e = launch_hash_insert(L_, grid_, s_); break;
    case PH_GEN: {
      const bool fast = cur_path_ == DIC_COUNT_BITSLICE || cur_path_ == DIC_COUNT_TENSOR;
      if (prof(DIC_PROFILE_GEN)) TRY(iv_open(IV_GEN, s_));
      // (with double-buffered or staged columns the next block is ready)
      e = launch_generate_finish(L_, L_.vall ? gen_grid_ : grid_, fast && !L_.vdouble && !L_.vall,
                                 s_);
      if (prof(DIC_PROFILE_GEN)) TRY(iv_close(s_));
      next_v_ready_ = fast;
      ++pred_step_;
      break;
    }
  }
  ++launches_;
  if (e != cudaSuccess) return fail(DIC_ECUDA, "kernel launch (phase %d): %s", phase,
                                    cudaGetErrorString(e));
  return DIC_OK;
}

// The kernels of one stop from `phase` on. The ROWS path runs PRUNE and the
// box-set insert as kernels of their own; the BITSLICE count kernel applies
// both in its epilogue.
dic_status Miner::launch_stop_from(int phase) {
  struct PdlScope {  // the stop's kernels chained by programmatic launch
    bool prev;
    explicit PdlScope(bool on) : prev(pdl_enabled()) { pdl_enabled() = on; }
    ~PdlScope() { pdl_enabled() = prev; }
  } scope(pdl_);
  for (int p = phase; p <= PH_GEN; ++p) {
    if (cur_path_ != DIC_COUNT_ROWS && (p == PH_PROMOTE || p == PH_HASH)) continue;
    TRY(launch_phase(p));
  }
  return DIC_OK;
}

dic_status Miner::grow_candidates(uint32_t need) {
  uint64_t ncap = std::max<uint64_t>((uint64_t)L_.cap * 2, (uint64_t)need + need / 4 + 1024);
  if (opt_.max_candidates && ncap > opt_.max_candidates) ncap = opt_.max_candidates;
  if (ncap > candidates_cap_limit_) ncap = candidates_cap_limit_;
  if (ncap < need)
    return fail(DIC_ECAPACITY, "candidate store needs %u records, limit is %llu", need,
                (unsigned long long)ncap);
  const uint32_t keep = h_ctrl_->tail;
  const uint32_t nb = h_ctrl_->n_newbox;
  Lattice N = L_;
  N.cap = (uint32_t)ncap;
  TRY(alloc(&N.cmask, (size_t)ncap * L_.wc));
  TRY(alloc(&N.csupp, ncap));
  TRY(alloc(&N.cbirth, ncap));
  TRY(alloc(&N.cshape, ncap));
  TRY(alloc(&N.ck, ncap));
  TRY(alloc(&N.cranks, (size_t)ncap * KRMAX));
  TRY(alloc(&N.cpromo, ncap));
  TRY(alloc(&N.newbox, ncap));
  TRY(alloc(&N.newinfo, ncap));
  TRY(alloc(&N.newhash, ncap));
  CU(cudaMemcpyAsync(N.cpromo, L_.cpromo, (size_t)keep * 4, cudaMemcpyDeviceToDevice, s_));
  CU(cudaMemcpyAsync(N.ck, L_.ck, (size_t)keep, cudaMemcpyDeviceToDevice, s_));
  CU(cudaMemcpyAsync(N.cranks, L_.cranks, (size_t)keep * KRMAX * 2, cudaMemcpyDeviceToDevice, s_));
  CU(cudaMemcpyAsync(N.cmask, L_.cmask, (size_t)keep * L_.wc * 8, cudaMemcpyDeviceToDevice, s_));
  CU(cudaMemcpyAsync(N.csupp, L_.csupp, (size_t)keep * 4, cudaMemcpyDeviceToDevice, s_));
  CU(cudaMemcpyAsync(N.cbirth, L_.cbirth, (size_t)keep * 4, cudaMemcpyDeviceToDevice, s_));
  CU(cudaMemcpyAsync(N.cshape, L_.cshape, (size_t)keep, cudaMemcpyDeviceToDevice, s_));
  CU(cudaMemcpyAsync(N.newbox, L_.newbox, (size_t)nb * 4, cudaMemcpyDeviceToDevice, s_));
  CU(cudaMemcpyAsync(N.newinfo, L_.newinfo, (size_t)nb * 8, cudaMemcpyDeviceToDevice, s_));
  CU(cudaMemcpyAsync(N.newhash, L_.newhash, (size_t)nb * 8, cudaMemcpyDeviceToDevice, s_));
  drop(L_.cmask); drop(L_.csupp); drop(L_.cbirth); drop(L_.cshape); drop(L_.newbox);
  drop(L_.newinfo);
  drop(L_.newhash); drop(L_.ck); drop(L_.cranks); drop(L_.cpromo);
  L_ = N;
  ++lat_version_;
  return DIC_OK;
}

// Rebuild the box set with room for `entries` boxes at load factor 1/4.
dic_status Miner::grow_hash(uint64_t entries) {
  uint64_t ncap = std::max<uint64_t>((uint64_t)L_.hcap * 2, 4096);
  while (ncap < entries * 4) ncap *= 2;
  if (ncap > (1ull << 31)) return fail(DIC_ECAPACITY, "box set would exceed 2^31 slots");
  Lattice N = L_;
  N.hcap = (uint32_t)ncap;
  TRY(alloc(&N.hslot, ncap, true));
  CU(launch_rehash(N, L_.hslot, L_.hcap, s_));
  ++launches_;
  drop(L_.hslot);
  L_ = N;
  ++lat_version_;
  return DIC_OK;
}

dic_status Miner::grow_trace(uint32_t need) {
  if (need <= L_.tcap) return DIC_OK;
  uint32_t ncap = std::max<uint32_t>(need, L_.tcap * 2);
  Lattice N = L_;
  N.tcap = ncap;
  TRY(alloc(&N.trace, (size_t)ncap * TRACE_COLS));
  TRY(alloc(&N.trace_work, (size_t)ncap));
  CU(cudaMemcpyAsync(N.trace_work, L_.trace_work, (size_t)L_.tcap * 8, cudaMemcpyDeviceToDevice,
                     s_));
  TRY(alloc(&N.cohort_start, (size_t)ncap + 2));
  TRY(alloc(&N.cohort_birth, (size_t)ncap + 2));
  CU(cudaMemcpyAsync(N.trace, L_.trace, (size_t)L_.tcap * TRACE_COLS * 8,
                     cudaMemcpyDeviceToDevice, s_));
  CU(cudaMemcpyAsync(N.cohort_start, L_.cohort_start, ((size_t)L_.tcap + 2) * 4,
                     cudaMemcpyDeviceToDevice, s_));
  CU(cudaMemcpyAsync(N.cohort_birth, L_.cohort_birth, ((size_t)L_.tcap + 2) * 4,
                     cudaMemcpyDeviceToDevice, s_));
  drop(L_.trace); drop(L_.trace_work); drop(L_.cohort_start); drop(L_.cohort_birth);
  L_ = N;
  if (L_.events) TRY(alloc_event_tallies(ncap + L_.stop_max + 2));
  ++lat_version_;
  return DIC_OK;
}

// Per-stop tallies of the event-driven loop for stops < ehcap (the old
// entries copied, the rest zero).
dic_status Miner::alloc_event_tallies(uint32_t ehcap) {
  Lattice N = L_;
  N.ehcap = ehcap;
  TRY(alloc(&N.eh_box, ehcap, true));
  TRY(alloc(&N.eh_pruned, ehcap, true));
  TRY(alloc(&N.eh_solid, ehcap, true));
  TRY(alloc(&N.eb_list, (size_t)ehcap * EV_LIST));
  TRY(alloc(&N.ev_work, ehcap, true));
  if (L_.ehcap) {
    const size_t old = L_.ehcap;
    CU(cudaMemcpyAsync(N.eh_box, L_.eh_box, old * 4, cudaMemcpyDeviceToDevice, s_));
    CU(cudaMemcpyAsync(N.eh_pruned, L_.eh_pruned, old * 4, cudaMemcpyDeviceToDevice, s_));
    CU(cudaMemcpyAsync(N.eh_solid, L_.eh_solid, old * 4, cudaMemcpyDeviceToDevice, s_));
    CU(cudaMemcpyAsync(N.eb_list, L_.eb_list, old * EV_LIST * 4, cudaMemcpyDeviceToDevice, s_));
    CU(cudaMemcpyAsync(N.ev_work, L_.ev_work, old * 8, cudaMemcpyDeviceToDevice, s_));
    drop(L_.eh_box); drop(L_.eh_pruned); drop(L_.eh_solid); drop(L_.eb_list); drop(L_.ev_work);
  }
  L_ = N;
  ++lat_version_;
  return DIC_OK;
}

static dic_status device_error(uint32_t code) {
  if (code == DIC_INTERNAL_BOUNDS)
    return fail(DIC_ECUDA, "internal error: a kernel's bounds check caught an index outside its buffer");
  if (code == DIC_ECAPACITY) return fail(DIC_ECAPACITY, "trace capacity exceeded");
  return fail((dic_status)code, "device reported status %u", code);
}

// ---- phase 1: first pass launched, its counts copied to pinned memory
dic_status Miner::begin() {
  t0_ = std::chrono::steady_clock::now();
  n_ = db_->n;
  res_.reset(new dic_result());
  res_->W = db_->W;
  res_->stats.words = db_->W;
  grid_ = sm_count() * 4;
  gen_grid_ = sm_count() * 2;
  if (n_ == 0) return DIC_OK;
  if (M_ > n_) M_ = n_;
  stop_max64_ = (n_ + M_ - 1) / M_;
  if (!h_ctrl_) {
    CU(pinned_alloc((void **)&h_ctrl_, sizeof(Ctrl)));
    own_h_ctrl_ = true;
  }
  if (opt_.algorithm == 1) return DIC_OK;  // classic DIC: no first pass
  CU(pinned_alloc((void **)&h_cnt1_, (size_t)db_->m * 4));
  uint32_t *d_cnt1 = nullptr;
  TRY(alloc(&d_cnt1, db_->m));
  if (opt_.profile) {
    CU(cudaEventCreate(&fa_));
    CU(cudaEventCreate(&fb_));
    CU(cudaEventRecord(fa_, s_));
  }
  CU(launch_item_count(db_->words, n_, db_->W, db_->m, d_cnt1, s_));
  ++launches_;
  drain_retired();  // earlier mines' graphs, while the first pass runs
  if (opt_.profile) CU(cudaEventRecord(fb_, s_));
  CU(cudaMemcpyAsync(h_cnt1_, d_cnt1, (size_t)db_->m * 4, cudaMemcpyDeviceToHost, s_));
  return DIC_OK;
}

// ---- phase 2 (stream synchronised since begin): L1, compaction, lattice,
// pair join. Sets has_loop_ when there are candidate pairs.
dic_status Miner::prepare() {
  has_loop_ = false;
  if (n_ == 0) return DIC_OK;
  const uint64_t n = n_;
  const uint32_t m = db_->m, W = db_->W;
  const uint64_t stop_max64 = stop_max64_;
  const bool classic = opt_.algorithm == 1;
  if (opt_.profile && !classic) {
    float ms = 0;
    cudaEventElapsedTime(&ms, fa_, fb_);
    res_->stats.firstpass_ms = ms;
  }
  if (classic) {
    // Algorithm 1: no first pass; every item is a rank and a 1-itemset circle
    for (uint32_t i = 0; i < m; ++i) l1items_.push_back(i);
  } else {
    const uint32_t *cnt1 = h_cnt1_;
    for (uint32_t i = 0; i < m; ++i)
      if (cnt1[i] >= minsup_) l1items_.push_back(i);
  }
  const std::vector<uint32_t> &l1items = l1items_;
  const uint32_t l1 = (uint32_t)l1items.size();
  res_->stats.l1 = l1;
  const uint32_t wc = std::max<uint32_t>(1, (l1 + 63) / 64);
  res_->stats.words_compact = wc;
  tests_ = classic ? 0 : (uint64_t)m * n;
  if (!classic)
    for (uint32_t i : l1items) {
      set_off_.push_back((uint32_t)set_items_.size());
      set_items_.push_back(i);
      supps_.push_back(h_cnt1_[i]);
    }
  n_first_ = set_off_.size();
  // the first cohort: all pairs of frequent ranks, or (classic) all 1-itemsets
  const uint64_t npairs = classic ? (uint64_t)l1 : (uint64_t)l1 * (l1 - (l1 ? 1 : 0)) / 2;
  if (npairs > 0) {
    if (npairs > candidates_cap_limit_ ||
        (opt_.max_candidates && npairs > opt_.max_candidates))
      return fail(DIC_ECAPACITY, "%llu candidate pairs exceed the candidate limit",
                  (unsigned long long)npairs);
    if (stop_max64 > 0x7FFFFFFFull) return fail(DIC_EINVAL, "too many blocks");
    // ---- ranks of the frequent items
    // (followed by the first rank of every chunk of 512 items, for the
    // all-blocks transposition)
    const uint32_t nchunk = (W + 7) / 8;
    std::vector<int32_t> rank_of((size_t)W * 64 + nchunk + 1, -1);
    for (uint32_t r = 0; r < l1; ++r) rank_of[l1items[r]] = (int32_t)r;
    {
      uint32_t r = 0;
      for (uint32_t c = 0; c <= nchunk; ++c) {
        while (r < l1 && l1items[r] < c * 512u) ++r;
        rank_of[(size_t)W * 64 + c] = (int32_t)r;
      }
    }
    // (then the item of every rank, for the result's item ids)
    item_of_off_ = rank_of.size();
    for (uint32_t r = 0; r < l1; ++r) rank_of.push_back((int32_t)l1items[r]);
    TRY(alloc(&d_rank_, rank_of.size()));
    CU(cudaMemcpyAsync(d_rank_, rank_of.data(), rank_of.size() * 4, cudaMemcpyHostToDevice, s_));

    // ---- BITSLICE tiles: widest tile whose double buffer leaves room for
    // a useful candidate chunk in shared memory
    {
      int dev = 0, optin = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      smem_optin_ = (size_t)optin;
      bs_l1p_ = (l1 + 3) & ~3u;
      bs_ok_ = false;
      if (l1 <= 65535 && opt_.count_path != DIC_COUNT_ROWS) {
        for (int tw : {16, 8, 4}) {
          if (forced_tw_ && tw != forced_tw_) continue;
          if (bitslice_max_chunk(tw, 16, bs_l1p_, smem_optin_) >= 1024) {
            bs_tw_ = tw;
            bs_ok_ = true;
            break;
          }
        }
      }
    }
    const uint64_t blockmax = std::min<uint64_t>(M_, n);
    if (bs_ok_) {
      const uint64_t ntiles = ((blockmax + 31) / 32 + bs_tw_ - 1) / bs_tw_;
      bs_V_words_ = (uint64_t)ntiles * bitslice_tile_words(bs_tw_, bs_l1p_);
    }
    // Every block's columns are transposed once, before the loop, when this
    // query runs its own loop and they fit the memory rule (a quarter of the
    // free device memory, at most 16 GiB); otherwise the loop transposes
    // each stop's block (double-buffered, one stop ahead).
    const size_t free_b = free_device_memory();
    const uint64_t stage_cap = std::min<uint64_t>(free_b / 4, 16ull << 30);
    vall_ = false;
    if (bs_ok_ && vdouble_ && opt_.prestage == 0 &&
        stop_max64 * bs_V_words_ * 4 <= stage_cap)
      vall_ = true;

    // ---- compacted rows: the ROWS path and the per-stop transposition
    // read them; with every block staged they are built only if the loop
    // falls back to ROWS (itemsets beyond KRMAX items)
    rows_ready_ = false;
    if (!vall_) TRY(ensure_rows());

    // ---- lattice buffers
    L_.n = n;
    L_.M = M_;
    L_.stop_max = (uint32_t)stop_max64;
    L_.minsup = minsup_;
    L_.wc = wc;
    L_.l1 = l1;
    uint64_t cap = npairs + npairs / 8 + 4096;
    L_.pairs_lex = classic ? 0u : 1u;
    if (opt_.max_candidates && cap > opt_.max_candidates) cap = opt_.max_candidates;
    if (cap > candidates_cap_limit_) cap = candidates_cap_limit_;
    L_.cap = (uint32_t)cap;
    TRY(alloc(&L_.cmask, (size_t)cap * wc));
    TRY(alloc(&L_.csupp, cap));
    TRY(alloc(&L_.cbirth, cap));
    TRY(alloc(&L_.cshape, cap));
    TRY(alloc(&L_.ck, cap));
    TRY(alloc(&L_.cranks, (size_t)cap * KRMAX));
    TRY(alloc(&L_.cpromo, cap));
    TRY(alloc(&L_.newbox, cap));
    TRY(alloc(&L_.newinfo, cap));
    TRY(alloc(&L_.newhash, cap));
    L_.hcap = 1u << 12;
    while ((uint64_t)L_.hcap < npairs * 4 && L_.hcap < (1u << 31)) L_.hcap <<= 1;
    TRY(alloc(&L_.hslot, L_.hcap, true));
    L_.tcap = std::max<uint32_t>(64, (uint32_t)std::min<uint64_t>(stop_max64 * 3 + 16, 1u << 20));
    TRY(alloc(&L_.trace, (size_t)L_.tcap * TRACE_COLS));
    TRY(alloc(&L_.trace_work, (size_t)L_.tcap));
    TRY(alloc(&L_.cohort_start, (size_t)L_.tcap + 2));
    TRY(alloc(&L_.cohort_birth, (size_t)L_.tcap + 2, true));
    CU(cudaMemsetAsync(L_.cohort_start, 0, ((size_t)L_.tcap + 2) * 4, s_));
    if (!ext_ctrl_) TRY(alloc(&L_.ctrl, 1)); else L_.ctrl = ext_ctrl_;
    Ctrl c{};
    c.step = 1;
    c.head = 0;
    c.tail = (uint32_t)npairs;
    c.n_live = (uint32_t)npairs;
    c.n_cohorts = 1;
    c.max_k = classic ? 1 : 2;
    c.tests = tests_;
    c.ev_limit = ~0u;
    // ---- TENSOR path for the pair cohort: needs the BITSLICE path for the
    // rest, a block below 2^24 rows (exact fp32 sums), and enough pairs to
    // fill a tile (AUTO) or an explicit request. With every block staged and
    // room for the per-block counts, the pairs are counted over the whole
    // pass by one GEMM before the loop and their promotions and prunes are
    // precomputed per stop (pair events); otherwise a GEMM per stop runs
    // beside the BITSLICE count.
    const bool want_tc = !classic && (opt_.count_path == DIC_COUNT_TENSOR ||
                                      (opt_.count_path == DIC_COUNT_AUTO && l1 >= 256 &&
                                       blockmax >= 2048));
    tc_ok_ = false;
    events_ = false;
    if (want_tc && bs_ok_ && blockmax < (1ull << 24) && npairs <= 0xFFFFFFF0ull) {
      tc_ok_ = true;
      L_.pair_end = (uint32_t)npairs;
      pc_wide_ = blockmax > 65535;
      const uint64_t pc_bytes = stop_max64 * npairs * (pc_wide_ ? 4 : 2);
      if (vall_ && pc_bytes <= stage_cap && stop_max64 * gram_tile_pairs(l1) <= 0x7FFFFFFFull) {
        events_ = true;
        c.gram_rows = n;  // every row of the pass, counted once for the pairs
      } else {
        tc_nkc_max_ = gram_chunks(blockmax);
        const uint32_t ntp = gram_tile_pairs(l1);
        const uint32_t sms = (uint32_t)sm_count();
        // one CTA per SM (the rings take 192 KiB): a single wave of splits
        tc_nsplit_ = std::max<uint32_t>(1, std::min<uint32_t>(tc_nkc_max_, sms / ntp));
        if (!s2_) CU(cudaStreamCreateWithFlags(&s2_, cudaStreamNonBlocking));
        if (!ev_fork_) CU(cudaEventCreateWithFlags(&ev_fork_, cudaEventDisableTiming));
        if (!ev_join_) CU(cudaEventCreateWithFlags(&ev_join_, cudaEventDisableTiming));
      }
    }
    *h_ctrl_ = c;
    CU(cudaMemcpyAsync(L_.ctrl, h_ctrl_, sizeof(Ctrl), cudaMemcpyHostToDevice, s_));
    if (classic)
      CU(launch_singleton_join(L_, s_));
    else
      CU(launch_pair_join(L_, npairs, s_));
    ++launches_;
    nw_ = (uint32_t)rows_width_bucket(c.max_k, wc);

    // ---- BITSLICE column buffers: every block of the pass (staged), or two
    // blocks (this stop's and the next) / one block (batched forms)
    if (bs_ok_) {
      const uint64_t nbuf = vall_ ? stop_max64 : (vdouble_ ? 2 : 1);
      TRY(alloc(&bs_V_, bs_V_words_ * nbuf));
      L_.V = bs_V_;
      L_.vwords = bs_V_words_;
      L_.vall = vall_ ? 1u : 0u;
      L_.vdouble = (vdouble_ && !vall_) ? 1u : 0u;
      if (L_.vdouble) {
        if (!s3_) CU(cudaStreamCreateWithFlags(&s3_, cudaStreamNonBlocking));
        if (!ev_slice_) CU(cudaEventCreateWithFlags(&ev_slice_, cudaEventDisableTiming));
        if (!ev_fork_) CU(cudaEventCreateWithFlags(&ev_fork_, cudaEventDisableTiming));
      }
      L_.tw = (uint32_t)bs_tw_;
      L_.l1p = bs_l1p_;
      bs_grid_ = sm_count();
      if (vall_) {
        CU(launch_slice_all(L_, db_->words, W, d_rank_,
                            reinterpret_cast<const uint32_t *>(d_rank_) + (size_t)W * 64, s_));
        ++launches_;
      }
    }
    // ---- the pair cohort over every block at once, and its events
    if (events_) {
      void *pc = nullptr;
      uint32_t *ev = nullptr, *hist = nullptr, *cursor = nullptr;
      uint32_t *ev_off = nullptr, *ev_list = nullptr, *ev_pruned = nullptr;
      const uint64_t S = stop_max64;
      TRY(alloc((uint8_t **)&pc, (size_t)S * npairs * (pc_wide_ ? 4 : 2)));
      TRY(alloc(&ev, npairs));
      TRY(alloc(&hist, 2 * (S + 2)));
      TRY(alloc(&cursor, S + 2));
      TRY(alloc(&ev_off, S + 2));
      TRY(alloc(&ev_list, npairs));
      TRY(alloc(&ev_pruned, S + 1));
      if (opt_.profile & DIC_PROFILE_GRAM) {
        if (!eg0_) CU(cudaEventCreate(&eg0_));
        if (!eg1_) CU(cudaEventCreate(&eg1_));
        CU(cudaEventRecord(eg0_, s_));
      }
      CU(launch_gram_all_blocks(L_, pc, pc_wide_, s_));
      if (opt_.profile & DIC_PROFILE_GRAM) CU(cudaEventRecord(eg1_, s_));
      CU(launch_pair_events(L_, pc, pc_wide_, ev, hist, ev_off, cursor, ev_list, ev_pruned, s_));
      launches_ += 4;
      path_launches_[DIC_COUNT_TENSOR]++;
      drop((uint8_t *)pc); drop(ev); drop(hist); drop(cursor);
      L_.pair_events = 1;
      L_.ev_off = ev_off;
      L_.ev_list = ev_list;
      L_.ev_pruned = ev_pruned;
    }
    pdl_ = vall_;  // one stream per stop: kernels chained by programmatic launch
    // ---- event-driven loop: every block staged, the pairs' events
    // precomputed, a per-block counter array that fits shared memory
    evmode_ = false;
    ev_switched_ = false;
    L_.events = 0;
    ev_ok_ = events_ && opt_.stop_loop != 2 && stop_max64 <= EV_STOPMAX &&
             (L_.tw == 4 || L_.tw == 8 || L_.tw == 16) &&
             cohort_pass_smem((uint32_t)stop_max64, l1) + 1024 <= smem_optin_;
    cp_grid_ = sm_count() * 2;
    if (ev_ok_ && opt_.stop_loop == 1) {
      evmode_ = true;
      L_.events = 1;
      TRY(alloc_event_buffers());
    }

    has_loop_ = true;
  }
  return DIC_OK;
}

// ---- phase 3: the stop loop of Algorithm 2 for this query alone
// Stops the newest cohort still needs (more may follow if cohorts appear).
// Stops captured into one graph where the loop allows it.
constexpr uint32_t kStopsPerGraph = 8;
// Stops without promotions after which the per-stop loop hands over to the
// event-driven form (stop_loop 0), and the group size it checks at once the
// pair cohort has passed.
constexpr uint32_t kStopsQuiet = 10;
constexpr uint32_t kGroupAfterPairs = 16;

static uint32_t stops_needed(const Ctrl &c, uint32_t stop_max, uint32_t cap) {
  const uint64_t end = (uint64_t)c.last_birth + stop_max + 1;
  const uint64_t need = end > c.step ? end - c.step : 1;
  return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(need, cap));
}

dic_status Miner::reserve(uint32_t stops) {
  TRY(grow_trace(h_ctrl_->n_trace + stops + 2));
  if ((uint64_t)(h_ctrl_->hash_used + h_ctrl_->n_live) * 2 > L_.hcap)
    TRY(grow_hash((uint64_t)h_ctrl_->hash_used + h_ctrl_->n_live));
  return DIC_OK;
}

dic_status Miner::set_tile_width(int tw, bool *ok) {
  *ok = false;
  // the batched kernels count every record themselves
  tc_ok_ = false;
  L_.pair_end = 0;
  if (!bs_ok_) return DIC_OK;
  if (tw == bs_tw_) { *ok = true; return DIC_OK; }
  if (bitslice_max_chunk(tw, 16, bs_l1p_, smem_optin_) < 1024) return DIC_OK;
  const uint64_t blockmax = std::min<uint64_t>(M_, n_);
  const uint64_t ntiles = ((blockmax + 31) / 32 + tw - 1) / tw;
  drop(bs_V_);
  bs_tw_ = tw;
  bs_V_words_ = (uint64_t)ntiles * bitslice_tile_words(bs_tw_, bs_l1p_);
  TRY(alloc(&bs_V_, bs_V_words_ * (L_.vdouble ? 2 : 1)));
  L_.V = bs_V_;
  L_.vwords = bs_V_words_;
  L_.tw = (uint32_t)bs_tw_;
  next_v_ready_ = false;
  ++lat_version_;
  *ok = true;
  return DIC_OK;
}

dic_status Miner::recover() {
  const uint32_t wc = L_.wc;
  if (h_ctrl_->error) return device_error(h_ctrl_->error);
  if (h_ctrl_->stall) {
    int b = rows_width_bucket(h_ctrl_->max_k, wc);
    nw_ = b ? (uint32_t)b : 0;
    cur_path_ = count_path_for_stop();
    if (cur_path_ == DIC_COUNT_ROWS) TRY(ensure_rows());
  }
  while (h_ctrl_->stall) {
    const uint32_t st = h_ctrl_->stall;
    int phase = PH_COUNT;
    if (st == ST_WIDTH) {
      int b = rows_width_bucket(h_ctrl_->max_k, wc);
      nw_ = b ? (uint32_t)b : 0;
      cur_path_ = count_path_for_stop();
      if (cur_path_ == DIC_COUNT_ROWS) TRY(ensure_rows());
      phase = PH_COUNT;
    } else if (st == ST_HASH || st == ST_HASH_COUNT) {
      TRY(grow_hash((uint64_t)h_ctrl_->hash_used + h_ctrl_->n_live + h_ctrl_->n_newbox));
      phase = st == ST_HASH ? PH_HASH : PH_COUNT;
    } else if (st == ST_CAND) {
      TRY(grow_candidates(h_ctrl_->tail + n_gen_of(*h_ctrl_)));
      phase = PH_GEN;
    } else {
      return fail(DIC_ECUDA, "unknown stall code %u", st);
    }
    if (phase == PH_COUNT) next_v_ready_ = false;
    pred_step_ = h_ctrl_->step;
    h_ctrl_->stall = ST_NONE;
    h_ctrl_->gen_ticket = 0;  // no candidate drawn, no generate CTA done
    CU(cudaMemcpyAsync(L_.ctrl, h_ctrl_, sizeof(Ctrl), cudaMemcpyHostToDevice, s_));
    TRY(launch_stop_from(phase));
    TRY(sync_ctrl());
    if (h_ctrl_->error) return device_error(h_ctrl_->error);
  }
  return DIC_OK;
}

// Profiling bits that put CUDA events into a stop (the pair GEMM runs once
// before the loop when the pair events are precomputed).
uint32_t Miner::stop_profile_bits() const {
  uint32_t b = DIC_PROFILE_COUNT | DIC_PROFILE_GEN | DIC_PROFILE_SETTLE;
  if (!L_.pair_events) b |= DIC_PROFILE_GRAM;
  return opt_.profile & b;
}

dic_status Miner::launch_stop(uint32_t nstops) {
  prof_now_ = (opt_.profile_every <= 1 || pred_step_ % opt_.profile_every == 0)
                  ? stop_profile_bits()
                  : 0u;
  if (!opt_.use_graph) {
    for (uint32_t i = 0; i < nstops; ++i) TRY(launch_stop_from(PH_COUNT));
    return DIC_OK;
  }
  const bool fast = cur_path_ == DIC_COUNT_BITSLICE || cur_path_ == DIC_COUNT_TENSOR;
  StopGraph key;
  key.path = cur_path_;
  key.gram = cur_path_ == DIC_COUNT_TENSOR && !L_.pair_events && pred_step_ <= L_.stop_max;
  key.slice = fast && !next_v_ready_ && !L_.vall;
  key.kre = fast ? kr_bucket(std::max<uint32_t>(h_ctrl_->max_k, 4)) : 0;
  key.direct = fast && direct_;
  key.nw = cur_path_ == DIC_COUNT_ROWS ? nw_ : 0;
  key.profile = prof_now_;
  key.version = lat_version_;
  key.nstops = nstops;
  StopGraph *sg = nullptr;
  for (auto &g : graphs_)
    if (g.path == key.path && g.gram == key.gram && g.slice == key.slice && g.kre == key.kre &&
        g.direct == key.direct && g.nstops == key.nstops &&
        g.nw == key.nw && g.profile == key.profile && g.version == key.version)
      sg = &g;
  const uint32_t pred0 = pred_step_;
  if (!sg) {
    const auto tg0 = std::chrono::steady_clock::now();
    struct GraphTimer {  // host time of the capture and instantiation
      std::chrono::steady_clock::time_point t;
      double *acc;
      ~GraphTimer() {
        *acc += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t)
                    .count();
      }
    } gtimer{tg0, &graph_ms_};
    // capture this stop's launches once (the host-side bookkeeping of the
    // capture is undone; every replay applies it)
    for (size_t i = 0; i < 8; ++i) {  // pool events used by the capture
      cudaEvent_t e;
      TRY(next_event(&e));
    }
    ev_used_ -= 8;
    const size_t e0 = ev_used_, ni0 = intervals_.size();
    const uint32_t l0 = launches_;
    uint32_t p0[4];
    std::memcpy(p0, path_launches_, sizeof p0);
    const bool v0 = next_v_ready_;
    CU(cudaStreamBeginCapture(s_, cudaStreamCaptureModeThreadLocal));
    dic_status st = DIC_OK;
    for (uint32_t i = 0; i < nstops && st == DIC_OK; ++i) st = launch_stop_from(PH_COUNT);
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(s_, &graph);
    cudaError_t ie = cudaErrorUnknown;
    if (st == DIC_OK && ce == cudaSuccess) ie = cudaGraphInstantiate(&key.exec, graph, 0);
    if (st != DIC_OK || ce != cudaSuccess || ie != cudaSuccess) {
      // capture not possible here: undo its bookkeeping, launch directly from now on
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      launches_ = l0;
      std::memcpy(path_launches_, p0, sizeof p0);
      ev_used_ = e0;
      intervals_.resize(ni0);
      next_v_ready_ = v0;
      pred_step_ = pred0;
      opt_.use_graph = 0;
      for (uint32_t i = 0; i < nstops; ++i) TRY(launch_stop_from(PH_COUNT));
      return DIC_OK;
    }
    key.graph = graph;
    key.kernels = launches_ - l0;
    for (int i = 0; i < 4; ++i) key.path_counts[i] = path_launches_[i] - p0[i];
    if (key.profile) {
      size_t nn = 0;
      CU(cudaGraphGetNodes(graph, nullptr, &nn));
      std::vector<cudaGraphNode_t> nodes(nn);
      CU(cudaGraphGetNodes(graph, nodes.data(), &nn));
      std::vector<std::pair<size_t, cudaGraphNode_t>> evn;
      for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        CU(cudaGraphNodeGetType(nd, &t));
        if (t != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev;
        CU(cudaGraphEventRecordNodeGetEvent(nd, &ev));
        for (size_t i = e0; i < ev_used_; ++i)
          if (ev_pool_[i] == ev) evn.push_back({i, nd});
      }
      std::sort(evn.begin(), evn.end(),
                [](const std::pair<size_t, cudaGraphNode_t> &a,
                   const std::pair<size_t, cudaGraphNode_t> &b) { return a.first < b.first; });
      for (auto &p : evn) key.ev_nodes.push_back(p.second);
      for (size_t i = ni0; i < intervals_.size(); ++i)
        key.ivs.push_back({intervals_[i].start - e0, intervals_[i].end - e0, intervals_[i].kind});
    }
    launches_ = l0;
    std::memcpy(path_launches_, p0, sizeof p0);
    ev_used_ = e0;
    intervals_.resize(ni0);
    next_v_ready_ = v0;
    pred_step_ = pred0;
    graphs_.push_back(key);
    sg = &graphs_.back();
  }
  if (sg->profile) {
    // fresh events for this replay, in recording order: (gram start, gram
    // end,) count start, count end
    const size_t base = ev_used_;
    for (cudaGraphNode_t nd : sg->ev_nodes) {
      cudaEvent_t e;
      TRY(next_event(&e));
      CU(cudaGraphExecEventRecordNodeSetEvent(sg->exec, nd, e));
    }
    for (const Interval &iv : sg->ivs) intervals_.push_back({base + iv.start, base + iv.end, iv.kind});
  }
  CU(cudaGraphLaunch(sg->exec, s_));
  launches_ += sg->kernels;
  for (int i = 0; i < 4; ++i) path_launches_[i] += sg->path_counts[i];
  next_v_ready_ = fast;
  pred_step_ = pred0 + nstops;
  return DIC_OK;
}

// ---- phase 3, event-driven form (Lattice.events)
// Inactive stops closed per cohort pass at most (each advances the loop by
// one trace row).
constexpr uint32_t kEventBudget = 4096;

// One iteration: count the cohort of the stop generated last over its pass,
// close that stop and advance to the next stop with promotions, then
// MAKECANDIDATES at it.
dic_status Miner::launch_event_body(bool in_graph) {
  struct PdlScope {
    bool prev;
    explicit PdlScope(bool on) : prev(pdl_enabled()) { pdl_enabled() = on; }
    ~PdlScope() { pdl_enabled() = prev; }
  } scope(true);
  if (prof(DIC_PROFILE_COUNT)) TRY(iv_open(IV_COUNT, s_));
  cudaError_t e = launch_cohort_pass(L_, cp_grid_, kEventBudget, in_graph ? 1u : 0u, evh_, s_);
  if (e != cudaSuccess) return fail(DIC_ECUDA, "cohort pass launch: %s", cudaGetErrorString(e));
  if (prof(DIC_PROFILE_COUNT)) TRY(iv_close(s_));
  if (prof(DIC_PROFILE_GEN)) TRY(iv_open(IV_GEN, s_));
  e = launch_generate_finish(L_, gen_grid_, false, s_);
  if (e != cudaSuccess) return fail(DIC_ECUDA, "generate launch: %s", cudaGetErrorString(e));
  if (prof(DIC_PROFILE_GEN)) TRY(iv_close(s_));
  if (!in_graph) {
    launches_ += 2;
    path_launches_[DIC_COUNT_BITSLICE]++;
  }
  return DIC_OK;
}

// The loop graph: one WHILE node whose body is launch_event_body; the
// cohort pass ends it when DASHED is empty, a stop stalls or the iteration
// limit is reached.
dic_status Miner::ensure_event_graph() {
  if (evx_ && evg_version_ == lat_version_) return DIC_OK;
  if (evx_) {
    retire_graph(evx_, evg_);
    evx_ = nullptr;
    evg_ = nullptr;
  }
  const auto tg0 = std::chrono::steady_clock::now();
  CU(cudaGraphCreate(&evg_, 0));
  CU(cudaGraphConditionalHandleCreate(&evh_, evg_, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = evh_;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  CU(cudaGraphAddNode(&node, evg_, nullptr, nullptr, 0, &p));
  cudaGraph_t body = p.conditional.phGraph_out[0];
  CU(cudaStreamBeginCaptureToGraph(s_, body, nullptr, nullptr, 0,
                                   cudaStreamCaptureModeThreadLocal));
  const uint32_t pn = prof_now_;
  prof_now_ = 0;
  dic_status st = launch_event_body(true);
  prof_now_ = pn;
  cudaGraph_t outg = nullptr;
  cudaError_t ce = cudaStreamEndCapture(s_, &outg);
  if (st != DIC_OK) return st;
  if (ce != cudaSuccess) return fail(DIC_ECUDA, "loop graph capture: %s", cudaGetErrorString(ce));
  CU(cudaGraphInstantiate(&evx_, evg_, 0));
  evg_version_ = lat_version_;
  graph_ms_ += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tg0)
                   .count();
  return DIC_OK;
}

dic_status Miner::recover_events() {
  if (h_ctrl_->error) return device_error(h_ctrl_->error);
  while (h_ctrl_->stall) {
    const uint32_t st = h_ctrl_->stall;
    bool regen = false;
    if (st == ST_HASH_EV) {
      TRY(grow_hash((uint64_t)h_ctrl_->hash_used + h_ctrl_->n_live));
    } else if (st == ST_TRACE) {
      TRY(grow_trace(h_ctrl_->n_trace + 2 * L_.stop_max + 64));
    } else if (st == ST_CAND) {
      TRY(grow_candidates(h_ctrl_->tail + n_gen_of(*h_ctrl_)));
      regen = true;
    } else {
      return fail(DIC_ECUDA, "unexpected stall code %u in the event-driven loop", st);
    }
    h_ctrl_->stall = ST_NONE;
    if (regen) h_ctrl_->gen_ticket = 0;  // no candidate drawn, no generate CTA done
    CU(cudaMemcpyAsync(L_.ctrl, h_ctrl_, sizeof(Ctrl), cudaMemcpyHostToDevice, s_));
    if (regen) {
      // re-run the stop's generation into the grown store; the loop then
      // resumes with the cohort pass, which closes the stop
      cudaError_t e = launch_generate_finish(L_, gen_grid_, false, s_);
      if (e != cudaSuccess) return fail(DIC_ECUDA, "generate launch: %s", cudaGetErrorString(e));
      ++launches_;
      TRY(sync_ctrl());
      if (h_ctrl_->error) return device_error(h_ctrl_->error);
    }
  }
  return DIC_OK;
}

// The event-driven form's per-stop tallies and the split-count scratch of
// its cohort passes (cohorts of up to one record per CTA).
dic_status Miner::alloc_event_buffers() {
  TRY(alloc_event_tallies(L_.tcap + L_.stop_max + 2));
  L_.cp_records = (uint32_t)cp_grid_;
  TRY(alloc(&L_.cp_cnt, (size_t)L_.cp_records * L_.stop_max));
  TRY(alloc(&L_.cp_tick, L_.cp_records, true));
  return DIC_OK;
}

// Hand the rest of the loop to the event-driven form at the current stop
// boundary: the live records of three or more items are counted over the
// blocks left of their passes and their events tallied (the pair cohort has
// left the window: the hand-over waits for stop_max to pass).
dic_status Miner::switch_to_events() {
  if ((uint64_t)(h_ctrl_->hash_used + h_ctrl_->n_live) * 2 > L_.hcap)
    TRY(grow_hash((uint64_t)h_ctrl_->hash_used + h_ctrl_->n_live));
  TRY(alloc_event_buffers());
  L_.events = 1;
  evmode_ = true;
  ev_switched_ = true;
  switch_step_ = h_ctrl_->step;
  ++lat_version_;
  h_ctrl_->ev_pending = 0;
  h_ctrl_->ev_iter = 0;
  h_ctrl_->ev_limit = ~0u;
  h_ctrl_->ev_ticket = 0;
  CU(cudaMemcpyAsync(L_.ctrl, h_ctrl_, sizeof(Ctrl), cudaMemcpyHostToDevice, s_));
  const uint32_t lo = std::max(h_ctrl_->head, L_.pair_end), tail = h_ctrl_->tail;
  if (lo >= tail) return DIC_OK;
  const uint32_t batch = window_pass_batch(L_.stop_max, tail - lo);
  uint32_t *rows = nullptr, *tick = nullptr;
  TRY(alloc(&rows, (size_t)batch * L_.stop_max));
  TRY(alloc(&tick, batch, true));
  for (uint32_t b = lo; b < tail; b += batch) {
    const uint32_t hi = tail - b > batch ? b + batch : tail;
    cudaError_t e = launch_window_pass(L_, b, hi, h_ctrl_->step, rows, tick, cp_grid_, s_);
    if (e != cudaSuccess) return fail(DIC_ECUDA, "window pass launch: %s", cudaGetErrorString(e));
    ++launches_;
  }
  drop(rows);
  drop(tick);
  return DIC_OK;
}

dic_status Miner::loop_events() {
  if (!ev_switched_)
    setup_ms_ = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0_)
                    .count();
  // Profiling the count or generate kernels times whole iterations one
  // launch at a time: the graph runs up to the next profiled iteration (its
  // limit), that iteration is launched directly between CUDA events, and the
  // graph resumes. Without it one graph launch runs the whole loop.
  // (after a hand-over the per-stop stops alone are timed)
  const bool prof_iters =
      !ev_switched_ && (opt_.profile & (DIC_PROFILE_COUNT | DIC_PROFILE_GEN)) != 0;
  const uint32_t every = opt_.profile_every > 1 ? opt_.profile_every : 1u;
  const bool graph = opt_.use_graph && !(prof_iters && every == 1);
  while (!h_ctrl_->done) {
    const uint32_t it0 = h_ctrl_->ev_iter;
    uint32_t graph_runs = 0, direct_runs = 0;
    if (!prof_iters && graph) {
      TRY(ensure_event_graph());
      CU(cudaGraphLaunch(evx_, s_));
      graph_runs = 1;
    } else {
      // segments up to the next iteration that is a multiple of `every`
      // (iterations launched after the loop has ended do nothing; without
      // the graph fewer are enqueued between checks)
      const uint32_t group = opt_.steps_per_sync ? opt_.steps_per_sync : graph ? 64u : 8u;
      uint32_t it = it0;
      for (uint32_t seg = 0; seg < group;) {
        const uint32_t p = prof_iters ? (it + every - 1) / every * every : it + group;
        if (graph && p > it) {
          TRY(ensure_event_graph());
          cudaError_t e = launch_set_ev_limit(L_.ctrl, p, s_);
          if (e != cudaSuccess) return fail(DIC_ECUDA, "launch: %s", cudaGetErrorString(e));
          ++launches_;
          CU(cudaGraphLaunch(evx_, s_));
          ++graph_runs;
          seg += p - it;
          it = p;
        } else if (p > it) {  // graphs off: plain launches up to p
          prof_now_ = 0;
          TRY(launch_event_body(false));
          ++direct_runs;
          ++seg;
          ++it;
          continue;
        }
        prof_now_ = prof_iters ? opt_.profile : 0u;
        prof_iters_.push_back(it);
        TRY(launch_event_body(false));
        prof_now_ = 0;
        ++direct_runs;
        ++seg;
        ++it;
      }
      if (graph) {
        cudaError_t e = launch_set_ev_limit(L_.ctrl, ~0u, s_);
        if (e != cudaSuccess) return fail(DIC_ECUDA, "launch: %s", cudaGetErrorString(e));
        ++launches_;
      }
    }
    TRY(sync_ctrl());
    if (graph_runs) {
      // two kernels per graph iteration (a launch ending early runs one more)
      const uint32_t done_it = h_ctrl_->ev_iter - it0;
      const uint32_t n = (done_it > direct_runs ? done_it - direct_runs : 0u) +
                         (h_ctrl_->done ? 0u : 1u);
      launches_ += 2 * n;
      path_launches_[DIC_COUNT_BITSLICE] += n;
    }
    TRY(recover_events());
  }
  return DIC_OK;
}

dic_status Miner::loop() {
  if (!has_loop_) return DIC_OK;
  if (evmode_) return loop_events();
  setup_ms_ = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0_)
                  .count();
  const uint32_t wc = L_.wc;
  // stops enqueued per group: those the newest cohort still needs, at most
  // 64 between host checks
  const uint32_t group_max = opt_.steps_per_sync ? opt_.steps_per_sync : 64;
  while (!h_ctrl_->done) {
    uint32_t group = stops_needed(*h_ctrl_, L_.stop_max, group_max);
    // after the pair cohort, shorter groups let the hand-over to the
    // event-driven form come soon after promotions stop
    if (ev_ok_ && opt_.stop_loop == 0 && !opt_.steps_per_sync && h_ctrl_->step > L_.stop_max)
      group = std::min(group, kGroupAfterPairs);
    TRY(reserve(group));
    int bucket = rows_width_bucket(h_ctrl_->max_k, wc);
    nw_ = bucket ? (uint32_t)bucket : 0;
    cur_path_ = count_path_for_stop();
    if (cur_path_ == DIC_COUNT_ROWS) TRY(ensure_rows());
    pred_step_ = h_ctrl_->step;
    {
      // the window the BITSLICE kernel counts (the pair cohort aside while
      // the tensor path has it); small ones take the direct form
      const Ctrl &c = *h_ctrl_;
      const uint32_t skip = (L_.pair_end && c.step <= L_.stop_max) ? L_.pair_end : 0u;
      // (pair_end is set whenever the tensor path has the pair cohort)
      const uint32_t lo = skip > c.head ? std::min(skip, c.tail) : c.head;
      direct_ = opt_.count_form == 2 ||
                (opt_.count_form == 0 && c.tail - lo <= BS_DIRECT_HOST_MAX);
    }
    // with staged columns and no per-stop host state, runs of stops are
    // captured together (stops without profiling events only)
    const bool multi = L_.vall && opt_.use_graph && (cur_path_ != DIC_COUNT_TENSOR ||
                                                     L_.pair_events);
    for (uint32_t i = 0; i < group;) {
      // the run ends before the next stop that carries profiling events
      uint32_t u = 1;
      if (multi) {
        const uint32_t cap = std::min<uint32_t>(kStopsPerGraph, group - i);
        u = 0;
        const bool prof_stops = stop_profile_bits() != 0;
        while (u < cap && !(prof_stops && (opt_.profile_every <= 1 ||
                                           (pred_step_ + u) % opt_.profile_every == 0)))
          ++u;
        if (u == 0) u = 1;  // the profiled stop itself, alone
      }
      TRY(launch_stop(u));
      i += u;
    }
    TRY(sync_ctrl());
    TRY(recover());
    // once the pair cohort has passed and the last kStopsQuiet stops promoted
    // nothing, the stops left are mostly ones without promotions: the
    // event-driven form closes those from tallies (stop_loop 0)
    if (ev_ok_ && !h_ctrl_->done && h_ctrl_->step > L_.stop_max &&
        h_ctrl_->step > h_ctrl_->last_promo + kStopsQuiet) {
      TRY(switch_to_events());
      return loop_events();
    }
  }
  return DIC_OK;
}

// ---- phase 4: SOLID boxes to the host, canonical order
dic_status Miner::collect(dic_result **out) {
  const auto tc0 = std::chrono::steady_clock::now();
  const uint32_t W = db_->W;
  std::unique_ptr<dic_result> res(std::move(res_));
  std::vector<uint32_t> &supps = supps_;
  const std::vector<uint32_t> &l1items = l1items_;
  uint64_t tests = tests_;
  if (has_loop_) {
    const uint32_t wc = L_.wc;
    tests = h_ctrl_->tests;
    res->stats.count_ops = h_ctrl_->work;
    res->stats.gram_flops = 2ull * ((uint64_t)L_.l1 * (L_.l1 - 1) / 2) * h_ctrl_->gram_rows;
    const uint32_t tail = h_ctrl_->tail;
    res->stats.candidates = tail;

    // ---- SOLID boxes (k >= 2) to the host, in record order, as item ids
    const uint32_t nch = collect_chunks(tail);
    uint32_t *d_idx = nullptr, *d_cnt = nullptr;
    TRY(alloc(&d_idx, std::max<uint32_t>(tail, 1)));
    TRY(alloc(&d_cnt, (size_t)nch + 1));
    CU(launch_collect_boxes(L_, tail, d_cnt, d_idx, s_));
    launches_ += 3;
    PinnedBuf<uint32_t> h_nbox;
    CU(h_nbox.get(1));
    CU(cudaMemcpyAsync(h_nbox.p, d_cnt + nch, 4, cudaMemcpyDeviceToHost, s_));
    CU(cudaStreamSynchronize(s_));
    const uint32_t nbox = tail ? *h_nbox.p : 0u;
    // masks only when some itemset has more items than a record's ranks
    const bool long_sets = h_ctrl_->max_k > (uint32_t)KRMAX;
    uint32_t *d_k = nullptr, *d_s = nullptr, *d_it = nullptr;
    uint64_t *d_om = nullptr;
    TRY(alloc(&d_k, nbox));
    TRY(alloc(&d_s, nbox));
    TRY(alloc(&d_it, (size_t)nbox * KRMAX));
    if (long_sets) TRY(alloc(&d_om, (size_t)nbox * wc));
    CU(launch_gather_boxes(L_, d_idx, nbox,
                           reinterpret_cast<const uint32_t *>(d_rank_) + item_of_off_, d_k, d_s,
                           d_it, d_om, s_));
    ++launches_;
    // staged in reused page-locked host blocks
    PinnedBuf<uint32_t> hk_b, hs_b, hi_b, hx_b;
    PinnedBuf<uint64_t> hm_b;
    PinnedBuf<unsigned long long> tr_b;
    const uint32_t ntr = h_ctrl_->n_trace;
    CU(hk_b.get(nbox));
    CU(hs_b.get(nbox));
    CU(hi_b.get((size_t)nbox * KRMAX));
    CU(hx_b.get(nbox));
    if (long_sets) CU(hm_b.get((size_t)nbox * wc));
    CU(tr_b.get((size_t)ntr * TRACE_COLS));
    if (nbox) {
      CU(cudaMemcpyAsync(hk_b.p, d_k, (size_t)nbox * 4, cudaMemcpyDeviceToHost, s_));
      CU(cudaMemcpyAsync(hs_b.p, d_s, (size_t)nbox * 4, cudaMemcpyDeviceToHost, s_));
      CU(cudaMemcpyAsync(hi_b.p, d_it, (size_t)nbox * KRMAX * 4, cudaMemcpyDeviceToHost, s_));
      CU(cudaMemcpyAsync(hx_b.p, d_idx, (size_t)nbox * 4, cudaMemcpyDeviceToHost, s_));
      if (long_sets)
        CU(cudaMemcpyAsync(hm_b.p, d_om, (size_t)nbox * wc * 8, cudaMemcpyDeviceToHost, s_));
    }
    if (ntr)
      CU(cudaMemcpyAsync(tr_b.p, L_.trace, (size_t)ntr * TRACE_COLS * 8, cudaMemcpyDeviceToHost,
                         s_));
    CU(cudaStreamSynchronize(s_));
    const unsigned long long *tr = tr_b.p;
    res->trace.assign(tr, tr + (size_t)ntr * TRACE_COLS);
    res->stats.stops = ntr;
    if (evmode_ && !ev_switched_ && (opt_.profile & DIC_PROFILE_COUNT)) {
      // count work of the profiled iterations' cohort passes
      const uint32_t ni = std::min<uint32_t>(h_ctrl_->ev_iter, L_.ehcap);
      std::vector<unsigned long long> ew(ni);
      if (ni) CU(cudaMemcpy(ew.data(), L_.ev_work, (size_t)ni * 8, cudaMemcpyDeviceToHost));
      uint64_t timed = 0;
      for (uint32_t i : prof_iters_)
        if (i < ni) timed += ew[i] - (i ? ew[i - 1] : 0ull);
      res->stats.count_ops_timed = timed;
    } else if (ntr && (opt_.profile & DIC_PROFILE_COUNT)) {
      // count work of the stops whose count kernel was bracketed by events
      std::vector<unsigned long long> tw(ntr);
      CU(cudaMemcpy(tw.data(), L_.trace_work, (size_t)ntr * 8, cudaMemcpyDeviceToHost));
      uint64_t timed = 0;
      for (uint32_t i = 0; i < ntr; ++i) {
        const uint64_t step = tr[(size_t)i * TRACE_COLS];
        const bool profiled = (opt_.profile_every <= 1 || step % opt_.profile_every == 0) &&
                              (!ev_switched_ || step < switch_step_);
        if (profiled) timed += tw[i] - (i ? tw[i - 1] : 0ull);
      }
      res->stats.count_ops_timed = timed;
    }
    // item lists (items come out ascending: rank order is item order)
    const uint32_t *hk = hk_b.p, *hsup = hs_b.p, *hit = hi_b.p;
    set_items_.reserve(set_items_.size() + (size_t)nbox * 3);
    for (uint32_t q = 0; q < nbox; ++q) {
      set_off_.push_back((uint32_t)set_items_.size());
      const uint32_t k = hk[q];
      if (k <= (uint32_t)KRMAX) {
        set_items_.insert(set_items_.end(), hit + (size_t)q * KRMAX, hit + (size_t)q * KRMAX + k);
      } else {
        for (uint32_t w = 0; w < wc; ++w)
          for (uint64_t x = hm_b.p[(size_t)q * wc + w]; x; x &= x - 1)
            set_items_.push_back(l1items[w * 64 + (uint32_t)__builtin_ctzll(x)]);
      }
      supps.push_back(hsup[q]);
    }
    // boxes of the first pass's pair cohort (records below pair_lex_end)
    // are already in canonical order and precede all longer itemsets
    n_ordered_ = n_first_;
    if (L_.pairs_lex) {
      const uint32_t pend = (uint32_t)((uint64_t)L_.l1 * (L_.l1 - (L_.l1 ? 1 : 0)) / 2);
      const uint32_t *hx = hx_b.p;
      uint32_t q = 0;
      while (q < nbox && hx[q] < pend) ++q;
      n_ordered_ += q;
    }
  } else {
    res->stats.candidates = 0;
    n_ordered_ = n_first_;
  }
  // ---- canonical order (size, then lexicographic), original item space.
  // The 1-itemsets and the pair cohort's boxes come first and already in
  // order; the rest are sorted by size and a key holding their first eight
  // item ids (16 bits each, first item most significant), comparing whole
  // item lists only on equal keys.
  const size_t nset = set_off_.size();
  set_off_.push_back((uint32_t)set_items_.size());
  const uint32_t *items = set_items_.data();
  const uint32_t *off = set_off_.data();
  std::vector<uint32_t> order(nset);
  for (uint32_t i = 0; i < nset; ++i) order[i] = i;
  {
    const size_t n1 = std::min(nset, n_ordered_);
    struct Key { uint64_t hi, lo; uint32_t k, idx; };
    std::vector<Key> keys(nset - n1);
    const bool narrow = db_->m <= 65536u;
    for (size_t q = n1; q < nset; ++q) {
      Key &kq = keys[q - n1];
      kq.k = off[q + 1] - off[q];
      kq.idx = (uint32_t)q;
      kq.hi = kq.lo = 0;
      if (narrow)
        for (uint32_t j = 0; j < 8 && j < kq.k; ++j) {
          const uint64_t v = items[off[q] + j];
          if (j < 4) kq.hi |= v << (48 - 16 * j);
          else kq.lo |= v << (48 - 16 * (j - 4));
        }
    }
    std::sort(keys.begin(), keys.end(), [&](const Key &a, const Key &b) {
      if (a.k != b.k) return a.k < b.k;
      if (a.hi != b.hi) return a.hi < b.hi;
      if (a.lo != b.lo) return a.lo < b.lo;
      return std::lexicographical_compare(items + off[a.idx], items + off[a.idx + 1],
                                          items + off[b.idx], items + off[b.idx + 1]);
    });
    for (size_t q = n1; q < nset; ++q) order[q] = keys[q - n1].idx;
  }
  res->masks = take_mask_array(nset * W);
  res->k.resize(nset);
  res->supp.resize(nset);
  for (size_t q = 0; q < nset; ++q) {
    const uint32_t o = order[q];
    for (uint32_t j = off[o]; j < off[o + 1]; ++j)
      res->masks[q * W + (items[j] >> 6)] |= 1ull << (items[j] & 63);
    res->k[q] = off[o + 1] - off[o];
    res->supp[q] = supps[o];
  }
  res->stats.tests = tests;
  res->stats.event_loop = ev_switched_ ? 2u : evmode_ ? 1u : 0u;
  res->stats.event_iters = evmode_ && has_loop_ ? h_ctrl_->ev_iter : 0u;
  res->stats.frequent = order.size();
  res->stats.kernel_launches = launches_;
  for (int i = 0; i < 4; ++i) res->stats.path_launches[i] = path_launches_[i];
  if (eg0_ && eg1_) {  // the all-blocks pair GEMM (once per mine)
    float ms = 0;
    if (cudaEventElapsedTime(&ms, eg0_, eg1_) == cudaSuccess) {
      gram_ms_ += ms;
      ++gram_timed_;
    }
  }
  if (opt_.profile) {
    res->stats.count_ms = count_ms_;
    res->stats.count_launches = count_timed_;
    res->stats.gram_ms = gram_ms_;
    res->stats.gram_launches = gram_timed_;
    res->stats.settle_ms = settle_ms_;
    res->stats.gen_ms = gen_ms_;
    res->stats.gen_launches = gen_timed_;
  }
  release();
  cudaError_t e = cudaStreamSynchronize(s_);
  if (e != cudaSuccess) return fail(DIC_ECUDA, "finalise: %s", cudaGetErrorString(e));
  const auto tend = std::chrono::steady_clock::now();
  res->stats.mine_ms = std::chrono::duration<double, std::milli>(tend - t0_).count();
  res->stats.setup_ms = setup_ms_;
  res->stats.graph_ms = graph_ms_;
  res->stats.collect_ms = std::chrono::duration<double, std::milli>(tend - tc0).count();
  *out = res.release();
  return DIC_OK;
}


dic_status Miner::run(dic_result **out) {
  vdouble_ = true;  // this query's own stop loop: transpose the next block beside the count
  TRY(begin());
  CU(cudaStreamSynchronize(s_));
  TRY(prepare());
  TRY(loop());
  return collect(out);
}

}  // namespace

// Checks of the option fields with a closed set of values.
static dic_status check_options(const dic_options &o) {
  if (o.tile_words != 0 && o.tile_words != 4 && o.tile_words != 8 && o.tile_words != 16)
    return fail(DIC_EINVAL, "tile_words must be 0, 4, 8 or 16 (got %u)", o.tile_words);
  if (o.count_form > 2) return fail(DIC_EINVAL, "count_form must be 0, 1 or 2 (got %u)", o.count_form);
  if (o.count_path > DIC_COUNT_TENSOR)
    return fail(DIC_EINVAL, "unknown count_path %u", o.count_path);
  if (o.algorithm > 1) return fail(DIC_EINVAL, "algorithm must be 0 or 1 (got %u)", o.algorithm);
  if (o.prestage > 1) return fail(DIC_EINVAL, "prestage must be 0 or 1 (got %u)", o.prestage);
  if (o.stop_loop > 2) return fail(DIC_EINVAL, "stop_loop must be 0, 1 or 2 (got %u)", o.stop_loop);
  return DIC_OK;
}

extern "C" dic_status dic_mine_ex(const dic_db *db, uint32_t minsup_count, uint64_t M,
                                  const dic_options *opt, void *stream, dic_result **out) {
  if (!out) return fail(DIC_EINVAL, "out is NULL");
  *out = nullptr;
  if (!db) return fail(DIC_EINVAL, "db is NULL");
  if (minsup_count == 0) return fail(DIC_EINVAL, "minsup_count must be >= 1");
  if (M == 0) return fail(DIC_EINVAL, "M must be >= 1");
  dic_options o;
  dic_options_init(&o);
  if (opt) std::memcpy(&o, opt, std::min<size_t>(sizeof o, opt->struct_size ? opt->struct_size : sizeof o));
  TRY(check_options(o));
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != db->device) cudaSetDevice(db->device);
  // The mine runs on a stream of its own (it captures graphs there, which a
  // stream shared with other host threads would not allow), ordered after
  // the caller's stream by an event and rejoining it at the end.
  cudaStream_t s = nullptr, user = (cudaStream_t)stream;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaError_t e = take_stream(db->device, &s);
  if (e == cudaSuccess && user) {
    e = cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev_in, user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_in, 0);
  }
  if (e != cudaSuccess) {
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (s) give_stream(db->device, s);
    if (prev != db->device) cudaSetDevice(prev);
    return fail(DIC_ECUDA, "stream setup: %s", cudaGetErrorString(e));
  }
  const_cast<dic_db *>(db)->busy.fetch_add(1);
  dic_status st;
  {
    Miner mn(db, minsup_count, M, o, s);
    st = mn.run(out);
  }
  if (st != DIC_OK) cudaStreamSynchronize(s);
  if (user) {  // the caller's later work waits for the mine
    cudaEventRecord(ev_out, s);
    cudaStreamWaitEvent(user, ev_out, 0);
    retire_event(ev_in);
    retire_event(ev_out);
  }
  const_cast<dic_db *>(db)->busy.fetch_sub(1);
  cudaStreamSynchronize(s);
  give_stream(db->device, s);
  if (prev != db->device) cudaSetDevice(prev);
  return st;
}

extern "C" dic_status dic_mine(const dic_db *db, uint32_t minsup_count, uint64_t M,
                               dic_result **out) {
  return dic_mine_ex(db, minsup_count, M, nullptr, nullptr, out);
}

// ------------------------------------------------------------ async mining
// A mine whose host side (the group loop of Algorithm 2: enqueue stops, read
// the loop state back, grow buffers) runs on a worker thread of its own, so
// the caller gets control back at once and several mines can be in flight on
// different streams.
struct dic_mine_job {
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv;
  bool finished = false;
  dic_status status = DIC_OK;
  std::string error;
  dic_result *result = nullptr;
};

extern "C" dic_status dic_mine_async(const dic_db *db, uint32_t minsup_count, uint64_t M,
                                     const dic_options *opt, void *stream, dic_mine_job **out) {
  if (!out) return fail(DIC_EINVAL, "out is NULL");
  *out = nullptr;
  if (!db) return fail(DIC_EINVAL, "db is NULL");
  if (minsup_count == 0) return fail(DIC_EINVAL, "minsup_count must be >= 1");
  if (M == 0) return fail(DIC_EINVAL, "M must be >= 1");
  dic_options o;
  dic_options_init(&o);
  if (opt) std::memcpy(&o, opt, std::min<size_t>(sizeof o, opt->struct_size ? opt->struct_size : sizeof o));
  TRY(check_options(o));
  std::unique_ptr<dic_mine_job> job(new (std::nothrow) dic_mine_job());
  if (!job) return fail(DIC_ENOMEM, "host allocation");
  dic_mine_job *j = job.get();
  const_cast<dic_db *>(db)->busy.fetch_add(1);  // held until the worker ends
  try {
    j->worker = std::thread([j, db, minsup_count, M, o, stream]() {
      cudaSetDevice(db->device);
      dic_result *res = nullptr;
      const dic_status st = dic_mine_ex(db, minsup_count, M, &o, stream, &res);
      const std::string err = st == DIC_OK ? std::string() : std::string(dic_last_error());
      const_cast<dic_db *>(db)->busy.fetch_sub(1);
      std::lock_guard<std::mutex> lk(j->mu);
      j->status = st;
      j->error = err;
      j->result = res;
      j->finished = true;
      j->cv.notify_all();
    });
  } catch (...) {
    const_cast<dic_db *>(db)->busy.fetch_sub(1);
    return fail(DIC_ENOMEM, "could not start the mining thread");
  }
  *out = job.release();
  return DIC_OK;
}

extern "C" dic_status dic_mine_wait(dic_mine_job *job, int64_t timeout_ms, dic_result **out) {
  if (!job || !out) return fail(DIC_EINVAL, "NULL argument");
  *out = nullptr;
  {
    std::unique_lock<std::mutex> lk(job->mu);
    auto ready = [&] { return job->finished; };
    if (timeout_ms < 0) job->cv.wait(lk, ready);
    else if (!job->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
      return fail(DIC_ETIMEOUT, "mining job not finished after %lld ms", (long long)timeout_ms);
  }
  job->worker.join();
  const dic_status st = job->status;
  dic_result *res = job->result;
  const std::string err = job->error;
  delete job;
  if (st != DIC_OK) return fail(st, "%s", err.c_str());
  *out = res;
  return DIC_OK;
}


// --------------------------------------------------- batched round graphs
// The four launches of a batched round (count, generation plan, generation,
// plan) read every argument from device arrays, so a run of rounds is
// captured once per shape (tile width, rank width, chunk size, shared memory,
// rounds) and replayed.
namespace {

struct RoundArgs {
  const Lattice *Ls;
  uint32_t Q;
  int tw, kre;
  uint32_t *items, *chunk;
  uint64_t *gen, *slice;
  uint32_t smem, chunk_cap;
  int grid, gen_grid;
};

cudaError_t enqueue_round(const RoundArgs &a, cudaStream_t s) {
  cudaError_t e = launch_batch_count(a.Ls, a.Q, a.tw, a.kre, a.items, a.chunk, a.smem, a.grid, s);
  if (e == cudaSuccess) e = launch_batch_plan_gen(a.Ls, a.Q, 1, a.gen, a.slice, s);
  if (e == cudaSuccess) e = launch_batch_gen(a.Ls, a.Q, 1, a.gen, a.slice, a.gen_grid, s);
  if (e == cudaSuccess)
    e = launch_batch_plan(a.Ls, a.Q, true, a.grid, a.chunk_cap, a.items, a.chunk, s);
  return e;
}

class RoundGraphs {
 public:
  ~RoundGraphs() {
    for (auto &g : cache_) retire_graph(g.exec, g.graph);
  }
  // `rounds` rounds on stream s: replays of captured runs of up to kRun
  // rounds (direct launches if capture is not possible).
  cudaError_t run(const RoundArgs &a, uint32_t rounds, cudaStream_t s) {
    while (rounds > 0) {
      const uint32_t u = rounds < kRun ? rounds : kRun;
      cudaGraphExec_t ex = get(a, u, s);
      cudaError_t e = cudaSuccess;
      if (ex) {
        e = cudaGraphLaunch(ex, s);
      } else {
        for (uint32_t i = 0; i < u && e == cudaSuccess; ++i) e = enqueue_round(a, s);
      }
      if (e != cudaSuccess) return e;
      rounds -= u;
    }
    return cudaSuccess;
  }

 private:
  static constexpr uint32_t kRun = 8;
  struct Entry {
    RoundArgs a;
    uint32_t rounds;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
  };
  std::vector<Entry> cache_;
  bool broken_ = false;
  static bool same(const RoundArgs &x, const RoundArgs &y) {
    return x.Ls == y.Ls && x.Q == y.Q && x.tw == y.tw && x.kre == y.kre && x.items == y.items &&
           x.chunk == y.chunk && x.gen == y.gen && x.slice == y.slice && x.smem == y.smem &&
           x.chunk_cap == y.chunk_cap && x.grid == y.grid && x.gen_grid == y.gen_grid;
  }
  cudaGraphExec_t get(const RoundArgs &a, uint32_t u, cudaStream_t s) {
    if (broken_) return nullptr;
    for (auto &g : cache_)
      if (g.rounds == u && same(g.a, a)) return g.exec;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    cudaError_t le = cudaSuccess;
    for (uint32_t i = 0; i < u && e == cudaSuccess && le == cudaSuccess; ++i)
      le = enqueue_round(a, s);
    if (e == cudaSuccess) e = cudaStreamEndCapture(s, &graph);
    if (e == cudaSuccess && le == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess || le != cudaSuccess || !exec) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      broken_ = true;  // launch directly from now on
      return nullptr;
    }
    cache_.push_back({a, u, graph, exec});
    return exec;
  }
};

}  // namespace

// ------------------------------------------------------------ batch driver
// Mines many queries together: every query keeps its own lattice; a round
// advances every active query by one stop and each phase of a round is one
// launch for all of them (kernels_batch.cu). Queries whose BITSLICE columns
// do not fit the common tile width, or whose itemsets outgrow the ranks the
// batched count handles, finish alone afterwards ("solo").
namespace {

class BatchMiner {
 public:
  BatchMiner(const dic_db *const *dbs, const uint32_t *minsup, const uint64_t *M, uint32_t Q,
             const dic_options &opt, cudaStream_t s)
      : dbs_(dbs), minsup_(minsup), M_(M), Q_(Q), opt_(opt), s_(s) {}
  ~BatchMiner() {
    ms_.clear();
    for (void *p : bufs_) cudaFreeAsync(p, s_);
    cudaStreamSynchronize(s_);
    if (h_ctrls_) pinned_free(h_ctrls_, (size_t)Q_ * sizeof(Ctrl));
    if (h_Ls_) pinned_free(h_Ls_, (size_t)Q_ * sizeof(Lattice));
  }
  dic_status run(dic_result **out);
  uint32_t batch_launches() const { return launches_; }

 private:
  template <class T>
  dic_status alloc(T **p, size_t count) {
    if (injected_alloc_failure()) return fail(DIC_ENOMEM, "batch allocation: injected failure");
    cudaError_t e = cudaMallocAsync((void **)p, std::max<size_t>(count * sizeof(T), 16), s_);
    if (e != cudaSuccess) return fail(DIC_ENOMEM, "batch allocation: %s", cudaGetErrorString(e));
    bufs_.push_back(*p);
    return DIC_OK;
  }
  dic_status upload_lattices();
  dic_status sync_ctrls();

  const dic_db *const *dbs_;
  const uint32_t *minsup_;
  const uint64_t *M_;
  uint32_t Q_;
  dic_options opt_;
  cudaStream_t s_;
  std::vector<void *> bufs_;
  std::vector<std::unique_ptr<Miner>> ms_;
  Ctrl *d_ctrls_ = nullptr, *h_ctrls_ = nullptr;
  Lattice *d_Ls_ = nullptr, *h_Ls_ = nullptr;
  uint32_t launches_ = 0;
  RoundGraphs rounds_;
};

dic_status BatchMiner::upload_lattices() {
  for (uint32_t q = 0; q < Q_; ++q) {
    h_Ls_[q] = ms_[q]->has_loop() ? ms_[q]->lattice() : Lattice{};
    h_Ls_[q].ctrl = d_ctrls_ + q;
  }
  CU(cudaMemcpyAsync(d_Ls_, h_Ls_, (size_t)Q_ * sizeof(Lattice), cudaMemcpyHostToDevice, s_));
  return DIC_OK;
}

dic_status BatchMiner::sync_ctrls() {
  CU(cudaMemcpyAsync(h_ctrls_, d_ctrls_, (size_t)Q_ * sizeof(Ctrl), cudaMemcpyDeviceToHost, s_));
  CU(cudaStreamSynchronize(s_));
  return DIC_OK;
}

dic_status BatchMiner::run(dic_result **out) {
  const uint32_t Q = Q_;
  CU(pinned_alloc((void **)&h_ctrls_, (size_t)Q * sizeof(Ctrl)));
  CU(pinned_alloc((void **)&h_Ls_, (size_t)Q * sizeof(Lattice)));
  TRY(alloc(&d_ctrls_, Q));
  TRY(alloc(&d_Ls_, Q));
  uint32_t *d_items = nullptr, *d_chunk = nullptr;
  uint64_t *d_gen = nullptr, *d_slice = nullptr;
  TRY(alloc(&d_items, (size_t)Q + 1));
  TRY(alloc(&d_chunk, 1));
  TRY(alloc(&d_gen, (size_t)Q + 1));
  TRY(alloc(&d_slice, (size_t)Q + 1));
  // every loop-state record starts as "done" (queries without candidate
  // pairs keep it); prepare() initialises the others
  for (uint32_t q = 0; q < Q; ++q) {
    h_ctrls_[q] = Ctrl{};
    h_ctrls_[q].done = 1;
  }
  CU(cudaMemcpyAsync(d_ctrls_, h_ctrls_, (size_t)Q * sizeof(Ctrl), cudaMemcpyHostToDevice, s_));
  for (uint32_t q = 0; q < Q; ++q) {
    ms_.emplace_back(new Miner(dbs_[q], minsup_[q], M_[q], opt_, s_));
    ms_[q]->use_external_ctrl(d_ctrls_ + q, h_ctrls_ + q);
    TRY(ms_[q]->begin());
  }
  CU(cudaStreamSynchronize(s_));
  int tw = 16;
  for (uint32_t q = 0; q < Q; ++q) {
    TRY(ms_[q]->prepare());
    if (ms_[q]->has_loop() && ms_[q]->bitslice_ready())
      tw = std::min(tw, ms_[q]->tile_words_per_rank());
  }
  // one tile width for the batch; queries that cannot use it go solo
  std::vector<bool> solo(Q, false);
  uint32_t max_l1p = 4;
  for (uint32_t q = 0; q < Q; ++q) {
    if (!ms_[q]->has_loop()) continue;
    bool ok = false;
    TRY(ms_[q]->set_tile_width(tw, &ok));
    solo[q] = !ok;
    if (ok) max_l1p = std::max(max_l1p, ms_[q]->l1p());
    h_ctrls_[q].solo = solo[q] ? 1 : 0;
  }
  int dev = 0, optin = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  CU(cudaMemcpyAsync(d_ctrls_, h_ctrls_, (size_t)Q * sizeof(Ctrl), cudaMemcpyHostToDevice, s_));
  TRY(upload_lattices());
  const int grid = sms, gen_grid = sms * 4;
  // bit columns of every query's first stop, then the first plan
  CU(launch_batch_plan_gen(d_Ls_, Q, 0, d_gen, d_slice, s_));
  CU(launch_batch_gen(d_Ls_, Q, 0, d_gen, d_slice, gen_grid, s_));
  launches_ += 2;
  const uint32_t group_max = opt_.steps_per_sync ? opt_.steps_per_sync : 64;
  for (;;) {
    uint32_t max_k = 2, group = 0;
    for (uint32_t q = 0; q < Q; ++q) {
      const Ctrl &c = h_ctrls_[q];
      if (c.done || solo[q]) continue;
      max_k = std::max(max_k, c.max_k);
      group = std::max(group, stops_needed(c, ms_[q]->lattice().stop_max, group_max));
    }
    if (group == 0) break;
    if (max_k > (uint32_t)KRMAX) {  // these queries continue alone
      for (uint32_t q = 0; q < Q; ++q)
        if (!h_ctrls_[q].done && !solo[q] && h_ctrls_[q].max_k > (uint32_t)KRMAX) {
          solo[q] = true;
          h_ctrls_[q].solo = 1;
          CU(cudaMemcpyAsync(d_ctrls_ + q, h_ctrls_ + q, sizeof(Ctrl), cudaMemcpyHostToDevice,
                             s_));
        }
      continue;
    }
    const int kre = kr_bucket(std::max<uint32_t>(max_k, 4));
    for (uint32_t q = 0; q < Q; ++q)
      if (!h_ctrls_[q].done && !solo[q]) TRY(ms_[q]->reserve(group));
    TRY(upload_lattices());
    const uint32_t chunk_cap = bitslice_max_chunk(tw, kre, max_l1p, (size_t)optin);
    const uint32_t smem = (uint32_t)bitslice_smem(tw, kre, max_l1p, chunk_cap);
    CU(launch_batch_plan(d_Ls_, Q, false, grid, chunk_cap, d_items, d_chunk, s_));
    ++launches_;
    const RoundArgs ra{d_Ls_, Q, tw, kre, d_items, d_chunk, d_gen, d_slice, smem, chunk_cap, grid,
                       gen_grid};
    CU(rounds_.run(ra, group, s_));
    launches_ += 4 * group;
    TRY(sync_ctrls());
    bool changed = false;
    for (uint32_t q = 0; q < Q; ++q) {
      if (solo[q] || !ms_[q]->has_loop()) continue;
      if (h_ctrls_[q].error) return device_error(h_ctrls_[q].error);
      if (h_ctrls_[q].stall) {
        TRY(ms_[q]->recover());
        changed = true;
      }
    }
    (void)changed;
  }
  // queries that left the batch finish alone
  for (uint32_t q = 0; q < Q; ++q)
    if (solo[q] && ms_[q]->has_loop()) {
      h_ctrls_[q].solo = 0;
      TRY(ms_[q]->loop());
    }
  for (uint32_t q = 0; q < Q; ++q) {
    if (q == 0) ms_[q]->add_launches(launches_);
    TRY(ms_[q]->collect(&out[q]));
  }
  return DIC_OK;
}

}  // namespace

extern "C" dic_status dic_mine_batch(const dic_db *const *dbs, const uint32_t *minsup,
                                     const uint64_t *M, uint32_t count, const dic_options *opt,
                                     dic_result **out) {
  if (!out || (count && (!dbs || !minsup || !M))) return fail(DIC_EINVAL, "NULL argument");
  for (uint32_t i = 0; i < count; ++i) out[i] = nullptr;
  if (count == 0) return DIC_OK;
  for (uint32_t i = 0; i < count; ++i) {
    if (!dbs[i]) return fail(DIC_EINVAL, "dbs[%u] is NULL", i);
    if (minsup[i] == 0) return fail(DIC_EINVAL, "minsup[%u] must be >= 1", i);
    if (M[i] == 0) return fail(DIC_EINVAL, "M[%u] must be >= 1", i);
    if (dbs[i]->device != dbs[0]->device) return fail(DIC_EINVAL, "databases on different devices");
  }
  dic_options o;
  dic_options_init(&o);
  if (opt) std::memcpy(&o, opt, std::min<size_t>(sizeof o, opt->struct_size ? opt->struct_size : sizeof o));
  TRY(check_options(o));
  if (o.algorithm != 0) return fail(DIC_EINVAL, "classic DIC runs single queries only");
  if (o.count_path == DIC_COUNT_ROWS) {  // plain per-query GPU DIC, one after another
    for (uint32_t i = 0; i < count; ++i) {
      dic_status st = dic_mine_ex(dbs[i], minsup[i], M[i], &o, nullptr, &out[i]);
      if (st != DIC_OK) {
        for (uint32_t j = 0; j <= i; ++j) { dic_result_free(out[j]); out[j] = nullptr; }
        return st;
      }
    }
    return DIC_OK;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != dbs[0]->device) cudaSetDevice(dbs[0]->device);
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
    return fail(DIC_ECUDA, "stream creation failed");
  for (uint32_t i = 0; i < count; ++i) const_cast<dic_db *>(dbs[i])->busy.fetch_add(1);
  dic_status st;
  {
    BatchMiner bm(dbs, minsup, M, count, o, s);
    st = bm.run(out);
    if (st != DIC_OK)
      for (uint32_t j = 0; j < count; ++j) { dic_result_free(out[j]); out[j] = nullptr; }
  }
  cudaStreamSynchronize(s);
  for (uint32_t i = 0; i < count; ++i) const_cast<dic_db *>(dbs[i])->busy.fetch_sub(1);
  cudaStreamDestroy(s);
  if (prev != dbs[0]->device) cudaSetDevice(prev);
  return st;
}


// ------------------------------------------------------------- request server
// Continuous batching of mining queries. A worker thread owns a stream and a
// table of slots; requests wait in arrival order and are admitted at every
// group boundary while a slot is free and their estimated device footprint
// fits the HBM budget. Admitted queries run their first pass and setup, then
// join the active slots, which all advance one stop per round through the
// batched kernels (one launch per phase for every slot); a query that
// finishes completes its ticket and frees its slot and memory at once.
namespace {

struct ServerRequest {
  uint64_t ticket = 0;
  const dic_db *db = nullptr;
  uint32_t minsup = 0;
  uint64_t M = 0;
  uint64_t est_bytes = 0;
  std::chrono::steady_clock::time_point t_submit, t_done;
  dic_result *result = nullptr;
  dic_status status = DIC_OK;
  std::string error;
  bool done = false;
};

// Upper bound of a query's device footprint before its first pass (all m
// items taken as frequent).
uint64_t estimate_bytes(const dic_db *db, uint64_t M) {
  const uint64_t m = db->m, W = db->W, n = db->n;
  const uint64_t pairs = m * (m - 1) / 2;
  const uint64_t cap = pairs + pairs / 8 + 4096;
  const uint64_t record = W * 8 + 4 + 4 + 1 + 1 + 2 * KRMAX + 4 + 4 + 8;
  uint64_t hcap = 4096;
  while (hcap < pairs * 4) hcap *= 2;
  const uint64_t block = std::min<uint64_t>(M, n ? n : 1);
  const uint64_t vbytes = ((block + 31) / 32 / 16 + 1) * 16 * ((m + 3) & ~3ull) * 20 * 4;
  return n * W * 8 + cap * record + hcap * 4 + vbytes + (1u << 20);
}

}  // namespace

struct dic_server {
  uint64_t budget = 0;
  uint32_t max_slots = 0;
  dic_options opt{};
  int device = 0;
  int tw = 16;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<ServerRequest>> pending;
  std::unordered_map<uint64_t, std::shared_ptr<ServerRequest>> tickets;
  uint64_t next_ticket = 1;
  bool stopping = false;
  std::thread worker;
  // statistics (under mu)
  std::vector<double> lat_ms;
  uint64_t submitted = 0, completed = 0, rejected = 0, rounds = 0;
  uint32_t peak_slots = 0;
  uint64_t used_bytes = 0, peak_bytes = 0;
  bool have_first = false;
  std::chrono::steady_clock::time_point t_first, t_last;
  std::string fatal;
  // worker-owned device state
  cudaStream_t s = nullptr;
  Ctrl *d_ctrls = nullptr, *h_ctrls = nullptr;
  Lattice *d_Ls = nullptr, *h_Ls = nullptr;
  uint32_t *d_items = nullptr, *d_chunk = nullptr;
  uint64_t *d_gen = nullptr, *d_slice = nullptr;
  std::vector<std::unique_ptr<Miner>> miner;
  std::vector<std::shared_ptr<ServerRequest>> req;
  // queries on databases of at least solo_rows rows, each mined alone by the
  // single-query path on a thread of its own (under mu: solo_running)
  uint64_t solo_rows = 0;
  uint32_t solo_running = 0;
  uint64_t solo_served = 0;
  struct Solo {
    std::thread th;
    std::shared_ptr<std::atomic<bool>> done;
  };
  std::vector<Solo> solos;  // worker-owned
  std::unique_ptr<RoundGraphs> round_graphs;  // worker-owned
};

namespace {

void server_complete(dic_server *sv, uint32_t slot, dic_status st) {
  std::shared_ptr<ServerRequest> r = sv->req[slot];
  dic_result *res = nullptr;
  if (st == DIC_OK) st = sv->miner[slot]->collect(&res);
  std::string err = st == DIC_OK ? std::string() : std::string(dic_last_error());
  sv->miner[slot].reset();  // buffers released on the stream
  sv->req[slot].reset();
  sv->h_ctrls[slot] = Ctrl{};
  sv->h_ctrls[slot].done = 1;
  cudaMemcpyAsync(sv->d_ctrls + slot, sv->h_ctrls + slot, sizeof(Ctrl), cudaMemcpyHostToDevice,
                  sv->s);
  const_cast<dic_db *>(r->db)->busy.fetch_sub(1);
  std::lock_guard<std::mutex> lk(sv->mu);
  r->done = true;
  r->status = st;
  r->error = err;
  r->result = res;
  r->t_done = std::chrono::steady_clock::now();
  sv->used_bytes -= r->est_bytes;
  sv->lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
  ++sv->completed;
  sv->t_last = r->t_done;
  sv->cv_done.notify_all();
}

dic_status server_upload(dic_server *sv) {
  for (uint32_t q = 0; q < sv->max_slots; ++q) {
    sv->h_Ls[q] = sv->miner[q] && sv->miner[q]->has_loop() ? sv->miner[q]->lattice() : Lattice{};
    sv->h_Ls[q].ctrl = sv->d_ctrls + q;
  }
  CU(cudaMemcpyAsync(sv->d_Ls, sv->h_Ls, (size_t)sv->max_slots * sizeof(Lattice),
                     cudaMemcpyHostToDevice, sv->s));
  return DIC_OK;
}

// One pass of the worker: admit, set up, run a group of rounds, retire.
dic_status server_step(dic_server *sv, const std::vector<std::shared_ptr<ServerRequest>> &adm,
                       const std::vector<uint32_t> &slots) {
  const uint32_t Q = sv->max_slots;
  // setup of newly admitted queries: first passes together, one sync
  for (size_t i = 0; i < adm.size(); ++i) {
    const uint32_t q = slots[i];
    sv->req[q] = adm[i];
    sv->miner[q].reset(new Miner(adm[i]->db, adm[i]->minsup, adm[i]->M, sv->opt, sv->s));
    sv->miner[q]->use_external_ctrl(sv->d_ctrls + q, sv->h_ctrls + q);
    dic_status st = sv->miner[q]->begin();
    if (st != DIC_OK) { server_complete(sv, q, st); continue; }
  }
  if (!adm.empty()) CU(cudaStreamSynchronize(sv->s));
  for (size_t i = 0; i < adm.size(); ++i) {
    const uint32_t q = slots[i];
    if (!sv->miner[q]) continue;
    dic_status st = sv->miner[q]->prepare();
    if (st != DIC_OK || !sv->miner[q]->has_loop()) { server_complete(sv, q, st); continue; }
    bool ok = false;
    st = sv->miner[q]->set_tile_width(sv->tw, &ok);
    if (st == DIC_OK && !ok) st = sv->miner[q]->loop();  // cannot join the batch
    if (st != DIC_OK || !ok) { server_complete(sv, q, st); continue; }
  }
  uint32_t max_k = 2, group = 0, max_l1p = 4, active = 0;
  const uint32_t group_cap = sv->opt.steps_per_sync ? sv->opt.steps_per_sync : 8;
  for (uint32_t q = 0; q < Q; ++q) {
    if (!sv->miner[q]) continue;
    const Ctrl &c = sv->h_ctrls[q];
    if (c.done) { server_complete(sv, q, DIC_OK); continue; }
    if (c.max_k > (uint32_t)KRMAX) {  // outgrew the batched count: finish alone
      server_complete(sv, q, sv->miner[q]->loop());
      continue;
    }
    ++active;
    max_k = std::max(max_k, c.max_k);
    max_l1p = std::max(max_l1p, sv->miner[q]->l1p());
    group = std::max(group, stops_needed(c, sv->miner[q]->lattice().stop_max, group_cap));
  }
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->peak_slots = std::max(sv->peak_slots, active);
  }
  if (active == 0) return DIC_OK;
  for (uint32_t q = 0; q < Q; ++q)
    if (sv->miner[q]) TRY(sv->miner[q]->reserve(group));
  TRY(server_upload(sv));
  int dev = 0, optin = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int kre = kr_bucket(std::max<uint32_t>(max_k, 4));
  const uint32_t chunk_cap = bitslice_max_chunk(sv->tw, kre, max_l1p, (size_t)optin);
  const uint32_t smem = (uint32_t)bitslice_smem(sv->tw, kre, max_l1p, chunk_cap);
  // bit columns of every active query's current stop (cheap; covers the
  // newly admitted and any recovered query), then the plan
  CU(launch_batch_plan_gen(sv->d_Ls, Q, 0, sv->d_gen, sv->d_slice, sv->s));
  CU(launch_batch_gen(sv->d_Ls, Q, 0, sv->d_gen, sv->d_slice, sms * 4, sv->s));
  CU(launch_batch_plan(sv->d_Ls, Q, false, sms, chunk_cap, sv->d_items, sv->d_chunk, sv->s));
  {
    const RoundArgs ra{sv->d_Ls, Q, sv->tw, kre, sv->d_items, sv->d_chunk, sv->d_gen, sv->d_slice,
                       smem, chunk_cap, sms, sms * 4};
    CU(sv->round_graphs->run(ra, group, sv->s));
  }
  CU(cudaMemcpyAsync(sv->h_ctrls, sv->d_ctrls, (size_t)Q * sizeof(Ctrl), cudaMemcpyDeviceToHost,
                     sv->s));
  CU(cudaStreamSynchronize(sv->s));
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->rounds += group;
  }
  for (uint32_t q = 0; q < Q; ++q) {
    if (!sv->miner[q]) continue;
    const Ctrl &c = sv->h_ctrls[q];
    if (c.error || c.stall) {
      dic_status st = sv->miner[q]->recover();
      if (st != DIC_OK) { server_complete(sv, q, st); continue; }
    }
    if (sv->h_ctrls[q].done) server_complete(sv, q, DIC_OK);
  }
  return DIC_OK;
}

// A query mined alone by the single-query path (every block staged, the pair
// cohort counted over the whole pass on the tensor cores) on a thread of its
// own, beside the batched rounds; it completes its own ticket.
void server_solo(dic_server *sv, std::shared_ptr<ServerRequest> r,
                 std::shared_ptr<std::atomic<bool>> done) {
  cudaSetDevice(sv->device);
  dic_result *res = nullptr;
  const dic_status st = dic_mine_ex(r->db, r->minsup, r->M, &sv->opt, nullptr, &res);
  const std::string err = st == DIC_OK ? std::string() : std::string(dic_last_error());
  const_cast<dic_db *>(r->db)->busy.fetch_sub(1);
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    r->done = true;
    r->status = st;
    r->error = err;
    r->result = res;
    r->t_done = std::chrono::steady_clock::now();
    sv->used_bytes -= r->est_bytes;
    sv->lat_ms.push_back(
        std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
    ++sv->completed;
    ++sv->solo_served;
    sv->t_last = r->t_done;
    --sv->solo_running;
    done->store(true);
  }
  sv->cv_done.notify_all();
  sv->cv_work.notify_all();
}

void server_main(dic_server *sv) {
  cudaSetDevice(sv->device);
  const uint32_t Q = sv->max_slots;
  for (;;) {
    std::vector<std::shared_ptr<ServerRequest>> adm;
    std::vector<uint32_t> slots;
    {
      // join the threads of solo queries that have finished
      for (size_t i = 0; i < sv->solos.size();) {
        if (sv->solos[i].done->load()) {
          sv->solos[i].th.join();
          sv->solos[i] = std::move(sv->solos.back());
          sv->solos.pop_back();
        } else {
          ++i;
        }
      }
      std::unique_lock<std::mutex> lk(sv->mu);
      bool any_active = false;
      for (uint32_t q = 0; q < Q; ++q) any_active |= (bool)sv->miner[q];
      // the head request can start now: nothing at all is running, or its
      // footprint fits the budget (all slots are free when none is active)
      auto admissible = [&] {
        if (sv->pending.empty()) return false;
        if (!any_active && sv->solo_running == 0) return true;
        return sv->used_bytes + sv->pending.front()->est_bytes <= sv->budget;
      };
      if (!any_active) {
        while (!admissible()) {
          if (sv->stopping && sv->pending.empty() && sv->solo_running == 0) {
            lk.unlock();
            for (auto &so : sv->solos) so.th.join();
            sv->solos.clear();
            return;
          }
          sv->cv_work.wait(lk);  // a submission, a solo query ending, or shutdown
        }
      }
      std::vector<uint32_t> free_slots;
      for (uint32_t q = 0; q < Q; ++q)
        if (!sv->miner[q]) free_slots.push_back(q);
      size_t f = 0;
      while (!sv->pending.empty()) {
        std::shared_ptr<ServerRequest> r = sv->pending.front();
        const bool alone = !any_active && adm.empty() && sv->solo_running == 0;
        if (sv->used_bytes + r->est_bytes > sv->budget && !alone) break;  // wait for memory
        const bool solo = r->db->n >= sv->solo_rows;
        if (!solo && f >= free_slots.size()) break;  // wait for a slot
        sv->pending.pop_front();
        sv->used_bytes += r->est_bytes;
        sv->peak_bytes = std::max(sv->peak_bytes, sv->used_bytes);
        if (solo) {
          ++sv->solo_running;
          auto done = std::make_shared<std::atomic<bool>>(false);
          sv->solos.push_back({std::thread(server_solo, sv, r, done), done});
          continue;
        }
        adm.push_back(r);
        slots.push_back(free_slots[f++]);
      }
    }
    dic_status st = server_step(sv, adm, slots);
    if (st != DIC_OK) {  // device failure: fail every query in flight
      std::string err = dic_last_error();
      for (uint32_t q = 0; q < Q; ++q)
        if (sv->miner[q]) server_complete(sv, q, st);
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->fatal = err;
    }
  }
}

}  // namespace

extern "C" dic_status dic_server_create(uint64_t hbm_budget_bytes, uint32_t max_slots,
                                        const dic_options *opt, dic_server **out) {
  if (!out) return fail(DIC_EINVAL, "out is NULL");
  *out = nullptr;
  if (max_slots == 0 || max_slots > 65536) return fail(DIC_EINVAL, "max_slots must be 1..65536");
  if (hbm_budget_bytes == 0) return fail(DIC_EINVAL, "hbm budget must be > 0");
  std::unique_ptr<dic_server> sv(new (std::nothrow) dic_server());
  if (!sv) return fail(DIC_ENOMEM, "host allocation");
  sv->budget = hbm_budget_bytes;
  sv->max_slots = max_slots;
  sv->solo_rows = opt && opt->struct_size >= offsetof(dic_options, solo_rows) + 4 &&
                          opt->solo_rows
                      ? opt->solo_rows
                      : (1ull << 19);
  dic_options_init(&sv->opt);
  if (opt) std::memcpy(&sv->opt, opt, std::min<size_t>(sizeof sv->opt, opt->struct_size ? opt->struct_size : sizeof sv->opt));
  TRY(check_options(sv->opt));
  if (sv->opt.algorithm != 0) return fail(DIC_EINVAL, "classic DIC runs single queries only");
  cudaGetDevice(&sv->device);
  init_pool(sv->device);
  CU(cudaStreamCreateWithFlags(&sv->s, cudaStreamNonBlocking));
  CU(cudaMallocHost((void **)&sv->h_ctrls, (size_t)max_slots * sizeof(Ctrl)));
  CU(cudaMallocHost((void **)&sv->h_Ls, (size_t)max_slots * sizeof(Lattice)));
  CU(cudaMalloc(&sv->d_ctrls, (size_t)max_slots * sizeof(Ctrl)));
  CU(cudaMalloc(&sv->d_Ls, (size_t)max_slots * sizeof(Lattice)));
  CU(cudaMalloc(&sv->d_items, ((size_t)max_slots + 1) * 4));
  CU(cudaMalloc(&sv->d_chunk, 16));
  CU(cudaMalloc(&sv->d_gen, ((size_t)max_slots + 1) * 8));
  CU(cudaMalloc(&sv->d_slice, ((size_t)max_slots + 1) * 8));
  for (uint32_t q = 0; q < max_slots; ++q) {
    sv->h_ctrls[q] = Ctrl{};
    sv->h_ctrls[q].done = 1;
  }
  CU(cudaMemcpy(sv->d_ctrls, sv->h_ctrls, (size_t)max_slots * sizeof(Ctrl),
                cudaMemcpyHostToDevice));
  sv->miner.resize(max_slots);
  sv->req.resize(max_slots);
  sv->round_graphs.reset(new RoundGraphs());
  dic_server *p = sv.release();
  p->worker = std::thread(server_main, p);
  *out = p;
  return DIC_OK;
}

extern "C" dic_status dic_server_submit(dic_server *sv, const dic_db *db, uint32_t minsup_count,
                                        uint64_t M, uint64_t *ticket) {
  if (!sv || !db || !ticket) return fail(DIC_EINVAL, "NULL argument");
  if (minsup_count == 0 || M == 0) return fail(DIC_EINVAL, "minsup_count and M must be >= 1");
  if (db->device != sv->device) return fail(DIC_EINVAL, "database on another device");
  std::shared_ptr<ServerRequest> r(new ServerRequest());
  r->db = db;
  r->minsup = minsup_count;
  r->M = M;
  r->est_bytes = estimate_bytes(db, M);
  r->t_submit = std::chrono::steady_clock::now();
  const_cast<dic_db *>(db)->busy.fetch_add(1);
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stopping) {
      const_cast<dic_db *>(db)->busy.fetch_sub(1);
      return fail(DIC_EBUSY, "server is shutting down");
    }
    r->ticket = sv->next_ticket++;
    sv->tickets[r->ticket] = r;
    sv->pending.push_back(r);
    ++sv->submitted;
    if (!sv->have_first) { sv->have_first = true; sv->t_first = r->t_submit; }
  }
  sv->cv_work.notify_one();
  *ticket = r->ticket;
  return DIC_OK;
}

extern "C" dic_status dic_server_wait(dic_server *sv, uint64_t ticket, int64_t timeout_ms,
                                      dic_result **out) {
  if (!sv || !out) return fail(DIC_EINVAL, "NULL argument");
  *out = nullptr;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->tickets.find(ticket);
  if (it == sv->tickets.end()) return fail(DIC_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
  std::shared_ptr<ServerRequest> r = it->second;
  auto ready = [&] { return r->done; };
  if (timeout_ms < 0) sv->cv_done.wait(lk, ready);
  else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
    return fail(DIC_ETIMEOUT, "ticket %llu not finished", (unsigned long long)ticket);
  sv->tickets.erase(ticket);
  if (r->status != DIC_OK) return fail(r->status, "%s", r->error.c_str());
  *out = r->result;
  r->result = nullptr;
  return DIC_OK;
}

extern "C" dic_status dic_server_stats(dic_server *sv, dic_server_metrics *out) {
  if (!sv || !out) return fail(DIC_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  std::memset(out, 0, sizeof *out);
  out->submitted = sv->submitted;
  out->completed = sv->completed;
  out->rounds = sv->rounds;
  out->peak_slots = sv->peak_slots;
  out->peak_bytes = sv->peak_bytes;
  out->solo = sv->solo_served;
  std::vector<double> v = sv->lat_ms;
  if (!v.empty()) {
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) { return v[std::min<size_t>(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    double sum = 0;
    for (double x : v) sum += x;
    out->mean_ms = sum / v.size();
  }
  if (sv->completed && sv->have_first) {
    const double secs = std::chrono::duration<double>(sv->t_last - sv->t_first).count();
    out->qps = secs > 0 ? sv->completed / secs : 0;
  }
  return DIC_OK;
}

extern "C" dic_status dic_server_destroy(dic_server *sv) {
  if (!sv) return DIC_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stopping = true;
  }
  sv->cv_work.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  for (auto &kv : sv->tickets) dic_result_free(kv.second->result);
  cudaStreamSynchronize(sv->s);
  cudaFree(sv->d_ctrls); cudaFree(sv->d_Ls); cudaFree(sv->d_items); cudaFree(sv->d_chunk);
  cudaFree(sv->d_gen); cudaFree(sv->d_slice);
  cudaFreeHost(sv->h_ctrls); cudaFreeHost(sv->h_Ls);
  cudaStreamDestroy(sv->s);
  delete sv;
  return DIC_OK;
}

// ----------------------------------------------------------------- results
extern "C" uint64_t dic_result_count(const dic_result *r) { return r ? r->k.size() : 0; }
extern "C" uint32_t dic_result_words(const dic_result *r) { return r ? r->W : 0; }
extern "C" dic_status dic_result_copy(const dic_result *r, uint64_t *masks, uint32_t *k,
                                      uint32_t *support) {
  if (!r) return fail(DIC_EINVAL, "result is NULL");
  if (masks && !r->masks.empty()) std::memcpy(masks, r->masks.data(), r->masks.size() * 8);
  if (k && !r->k.empty()) std::memcpy(k, r->k.data(), r->k.size() * 4);
  if (support && !r->supp.empty()) std::memcpy(support, r->supp.data(), r->supp.size() * 4);
  return DIC_OK;
}
extern "C" uint64_t dic_result_trace_len(const dic_result *r) {
  return r ? r->trace.size() / TRACE_COLS : 0;
}
extern "C" dic_status dic_result_trace(const dic_result *r, uint64_t *rows) {
  if (!r || !rows) return fail(DIC_EINVAL, "NULL argument");
  if (!r->trace.empty()) std::memcpy(rows, r->trace.data(), r->trace.size() * 8);
  return DIC_OK;
}
extern "C" dic_status dic_result_stats(const dic_result *r, dic_stats *out) {
  if (!r || !out) return fail(DIC_EINVAL, "NULL argument");
  *out = r->stats;
  return DIC_OK;
}
extern "C" void dic_result_free(dic_result *r) {
  if (!r) return;
  give_mask_array(std::move(r->masks));
  delete r;
}

// ------------------------------------------------------ association rules
namespace {
// A device buffer of the rules call, allocated and freed on its stream.
struct RuleBuf {
  void *p = nullptr;
  cudaStream_t s;
  explicit RuleBuf(cudaStream_t st) : s(st) {}
  dic_status alloc(size_t bytes) {
    cudaError_t e = cudaMallocAsync(&p, bytes < 16 ? 16 : bytes, s);
    if (e != cudaSuccess) {
      p = nullptr;
      return fail(DIC_ENOMEM, "device allocation of %zu bytes: %s", bytes, cudaGetErrorString(e));
    }
    return DIC_OK;
  }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
  }
  ~RuleBuf() { release(); }
};
}  // namespace

struct dic_rules {
  uint32_t W = 1;
  std::vector<uint64_t> ante, cons;  // [count][W]
  std::vector<uint32_t> supp, supp_ante;
};

extern "C" dic_status dic_rules_from_itemsets(const uint64_t *masks, const uint32_t *k,
                                              const uint32_t *support, uint64_t count,
                                              uint32_t m, uint32_t conf_num, uint32_t conf_den,
                                              dic_rules **out) {
  if (!out) return fail(DIC_EINVAL, "out is NULL");
  *out = nullptr;
  if (m == 0) return fail(DIC_EINVAL, "m must be >= 1");
  if (conf_den == 0) return fail(DIC_EINVAL, "conf_den must be >= 1");
  if (count && (!masks || !k || !support)) return fail(DIC_EINVAL, "NULL argument");
  if (count >= 0xFFFFFFFFull) return fail(DIC_ECAPACITY, "too many itemsets");
  const uint32_t W = (m + 63) / 64;
  // host checks: sizes are the popcounts, no item >= m, the work fits
  std::vector<uint64_t> prefix((size_t)count + 1, 0);
  for (uint64_t i = 0; i < count; ++i) {
    uint32_t pc = 0;
    for (uint32_t w = 0; w < W; ++w) pc += (uint32_t)__builtin_popcountll(masks[i * W + w]);
    if (pc != k[i]) return fail(DIC_EINVAL, "k[%llu] is not the popcount of its mask",
                                (unsigned long long)i);
    if (m % 64 && (masks[i * W + W - 1] >> (m % 64)))
      return fail(DIC_EINVAL, "itemset %llu holds an item >= m", (unsigned long long)i);
    if (pc > 31) return fail(DIC_ECAPACITY, "itemset %llu has more than 31 items",
                             (unsigned long long)i);
    prefix[i + 1] = prefix[i] + (pc >= 2 ? (1ull << pc) - 2 : 0);
  }
  const uint64_t total = prefix[count];
  if (total > 0xFFFFFFFFull) return fail(DIC_ECAPACITY, "more than 2^32 splits");
  std::unique_ptr<dic_rules> r(new (std::nothrow) dic_rules());
  if (!r) return fail(DIC_ENOMEM, "host allocation");
  r->W = W;
  if (total == 0) { *out = r.release(); return DIC_OK; }
  uint32_t hcap = 1024;
  while ((uint64_t)hcap < 2 * count) hcap <<= 1;
  cudaStream_t s;
  CU(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  RuleBuf d_masks(s), d_k(s), d_supp(s), d_prefix(s), d_hslot(s), d_cursor(s), d_z(s),
      d_code(s), d_sx(s), d_err(s);
  dic_status st = DIC_OK;
  uint32_t herr = 0;
  unsigned long long nrules = 0;
  do {
    if ((st = d_masks.alloc(count * W * 8)) != DIC_OK) break;
    if ((st = d_k.alloc(count * 4)) != DIC_OK) break;
    if ((st = d_supp.alloc(count * 4)) != DIC_OK) break;
    if ((st = d_prefix.alloc((count + 1) * 8)) != DIC_OK) break;
    if ((st = d_hslot.alloc((uint64_t)hcap * 4)) != DIC_OK) break;
    if ((st = d_cursor.alloc(8)) != DIC_OK) break;
    if ((st = d_z.alloc(total * 4)) != DIC_OK) break;
    if ((st = d_code.alloc(total * 4)) != DIC_OK) break;
    if ((st = d_sx.alloc(total * 4)) != DIC_OK) break;
    if ((st = d_err.alloc(4)) != DIC_OK) break;
    cudaError_t e = cudaMemcpyAsync(d_masks.p, masks, count * W * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_k.p, k, count * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_supp.p, support, count * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_prefix.p, prefix.data(), (count + 1) * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_hslot.p, 0, (size_t)hcap * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cursor.p, 0, 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err.p, 0, 4, s);
    if (e == cudaSuccess)
      e = launch_rules((const uint64_t *)d_masks.p, (const uint32_t *)d_k.p,
                       (const uint32_t *)d_supp.p, (const uint64_t *)d_prefix.p,
                       (uint32_t *)d_hslot.p, count, W, hcap, conf_num, conf_den, total,
                       (unsigned long long *)d_cursor.p, (uint32_t *)d_z.p,
                       (uint32_t *)d_code.p, (uint32_t *)d_sx.p, (uint32_t *)d_err.p, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nrules, d_cursor.p, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, d_err.p, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { st = fail(DIC_ECUDA, "rules: %s", cudaGetErrorString(e)); break; }
    if (herr & 1u) { st = fail(DIC_EINVAL, "the itemsets are not downward closed"); break; }
    if (herr & 2u) { st = fail(DIC_ECUDA, "rules: internal table sizing error"); break; }
    if (nrules > total) nrules = total;
    std::vector<uint32_t> hz(nrules), hc(nrules), hs(nrules);
    if (nrules) {
      e = cudaMemcpyAsync(hz.data(), d_z.p, nrules * 4, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(hc.data(), d_code.p, nrules * 4, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), d_sx.p, nrules * 4, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) { st = fail(DIC_ECUDA, "rules: %s", cudaGetErrorString(e)); break; }
    }
    // expand (itemset, split code) into item lists and sort canonically
    struct Rule { std::vector<uint32_t> x, y; uint32_t sz, sx; };
    std::vector<Rule> rules(nrules);
    for (uint64_t q = 0; q < nrules; ++q) {
      const uint64_t *Z = masks + (uint64_t)hz[q] * W;
      uint32_t t = 0;
      for (uint32_t w = 0; w < W; ++w)
        for (uint64_t y = Z[w]; y; y &= y - 1, ++t) {
          const uint32_t item = w * 64 + (uint32_t)__builtin_ctzll(y);
          ((hc[q] >> t) & 1u ? rules[q].x : rules[q].y).push_back(item);
        }
      rules[q].sz = support[hz[q]];
      rules[q].sx = hs[q];
    }
    std::sort(rules.begin(), rules.end(), [](const Rule &a, const Rule &b) {
      if (a.x.size() != b.x.size()) return a.x.size() < b.x.size();
      if (a.x != b.x) return a.x < b.x;
      if (a.y.size() != b.y.size()) return a.y.size() < b.y.size();
      return a.y < b.y;
    });
    r->ante.assign(nrules * W, 0);
    r->cons.assign(nrules * W, 0);
    r->supp.resize(nrules);
    r->supp_ante.resize(nrules);
    for (uint64_t q = 0; q < nrules; ++q) {
      for (uint32_t it : rules[q].x) r->ante[q * W + it / 64] |= 1ull << (it % 64);
      for (uint32_t it : rules[q].y) r->cons[q * W + it / 64] |= 1ull << (it % 64);
      r->supp[q] = rules[q].sz;
      r->supp_ante[q] = rules[q].sx;
    }
  } while (false);
  d_masks.release(); d_k.release(); d_supp.release(); d_prefix.release(); d_hslot.release();
  d_cursor.release(); d_z.release(); d_code.release(); d_sx.release(); d_err.release();
  cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  if (st != DIC_OK) return st;
  *out = r.release();
  return DIC_OK;
}

extern "C" uint64_t dic_rules_count(const dic_rules *r) { return r ? r->supp.size() : 0; }

extern "C" dic_status dic_rules_copy(const dic_rules *r, uint64_t *antecedent,
                                     uint64_t *consequent, uint32_t *support,
                                     uint32_t *antecedent_support) {
  if (!r) return fail(DIC_EINVAL, "rules is NULL");
  if (antecedent) std::memcpy(antecedent, r->ante.data(), r->ante.size() * 8);
  if (consequent) std::memcpy(consequent, r->cons.data(), r->cons.size() * 8);
  if (support) std::memcpy(support, r->supp.data(), r->supp.size() * 4);
  if (antecedent_support)
    std::memcpy(antecedent_support, r->supp_ante.data(), r->supp_ante.size() * 4);
  return DIC_OK;
}

extern "C" void dic_rules_free(dic_rules *r) { delete r; }

// -------------------------------------------------------------------- misc
namespace dic {
cudaError_t measure_alu_peak(double *tops);
}

extern "C" dic_status dic_debug_fail_device_alloc(int64_t after) {
  g_fail_alloc_after = after < 0 ? -1 : after;
  return DIC_OK;
}

extern "C" dic_status dic_debug_pool_used(uint64_t *bytes) {
  if (!bytes) return fail(DIC_EINVAL, "out is NULL");
  *bytes = 0;
  int dev = 0;
  cudaMemPool_t pool;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetDefaultMemPool(&pool, dev));
  uint64_t used = 0;
  CU(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
  *bytes = used;
  return DIC_OK;
}

extern "C" dic_status dic_measure_alu_peak(double *tera_ops_per_s) {
  if (!tera_ops_per_s) return fail(DIC_EINVAL, "out is NULL");
  *tera_ops_per_s = 0;
  cudaError_t e = dic::measure_alu_peak(tera_ops_per_s);
  if (e != cudaSuccess) return fail(DIC_ECUDA, "ALU peak: %s", cudaGetErrorString(e));
  return DIC_OK;
}

extern "C" uint32_t dic_minsup_count(uint64_t n, double frac) {
  if (!(frac > 0)) return 1;
  double v = std::ceil(frac * (double)n - 1e-9);
  if (v < 1) v = 1;
  if (v > 4294967295.0) v = 4294967295.0;
  return (uint32_t)v;
}

extern "C" const char *dic_status_str(dic_status s) {
  switch (s) {
    case DIC_OK: return "ok";
    case DIC_EINVAL: return "invalid argument";
    case DIC_ENOMEM: return "out of memory";
    case DIC_ECUDA: return "CUDA error";
    case DIC_ECAPACITY: return "capacity exceeded";
    case DIC_ETIMEOUT: return "device wait timed out";
    case DIC_EBUSY: return "busy";
  }
  return "unknown status";
}

extern "C" const char *dic_last_error(void) { return g_last_error.c_str(); }
extern "C" uint32_t dic_abi_version(void) { return DIC_ABI_VERSION; }
