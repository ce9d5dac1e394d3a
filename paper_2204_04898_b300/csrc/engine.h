// Host-side engine internals: context, device buffers, kernel timing, status
// handling and the declarations shared by the .cu files.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/pm4g.h"

namespace pm4g {

// Activity alphabets: codes fit 16 bits of a bucketed record; the global edge
// table is dense over the A * A pairs up to kDenseMaxActivities.
constexpr int32_t kMaxActivities = 65536;
constexpr int32_t kDenseMaxActivities = 4096;

void set_error(const char *fmt, ...);

#define PM4G_CK(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      ::pm4g::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                     \
      return PM4G_ECUDA;                                                               \
    }                                                                                  \
  } while (0)

#define PM4G_TRY(expr)           \
  do {                           \
    int st_ = (expr);            \
    if (st_ != PM4G_OK) return st_; \
  } while (0)

// Records a CUDA event pair around every launch when timing is on.
struct TimingRec {
  std::string name;
  cudaEvent_t a, b;
};

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool has_alloc = false;
  pm4g_allocator alloc{};
  int num_sms = 148;
  int smem_optin = 227 * 1024;
  // options
  int timing = 0;  // PM4G_OPT_TIMING: 0 off, 1 every launch, 2 the dominant kernels
  int test_hash_bits = 0;
  int test_bucket_cap = 0;
  // launch choices of the single-log pass (PM4G_OPT_EDGE_TABLE, _LOAD_CLB,
  // _LOAD_SPLITS, _STREAM_WARPS, _STREAM_OFF, _PART1_ITEMS, _PART2_ITEMS;
  // 0 = default)
  int edge_table = 0;
  int load_clb = 0;
  int load_splits = 0;
  int stream_warps = 0;
  int stream_off = 0;
  int part1_items = 0;
  int part2_items = 0;
  int part_fbits = 0;
  // launch choices of the batched drill-down (PM4G_OPT_BATCH_*; 0 = default)
  int batch_chunk = 0;
  int batch_stages = 0;
  int batch_items_per_sm = 0;
  // timing
  std::vector<TimingRec> pending;
  std::vector<cudaEvent_t> free_events;
  std::map<std::string, std::pair<int64_t, double>> totals;
  int64_t live_logs = 0;
  int64_t launches = 0;  // kernels launched by this context
  // pinned host staging for device-to-host results
  void *pin = nullptr;
  size_t pin_bytes = 0;
  // second stream for result copies that overlap later kernels, and the
  // event that orders it after the context stream (created when first used)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t copy_ready = nullptr;
  // page-locked, device-mapped bytes for small results (counts, totals): a
  // kernel writes them over the bus, so reading one does not queue behind
  // bulk result copies on the copy engines (allocated when first used)
  void *small = nullptr;
  void *small_dev = nullptr;
  // page-locked, device-mapped result staging: kernels write a query's
  // results straight to host memory, so the query needs one wait in all
  // (grown when first needed; at most kMappedMax bytes)
  void *mapped = nullptr;
  void *mapped_dev = nullptr;
  size_t mapped_bytes = 0;
  // device blocks freed by this context, kept for reuse in stream order
  // (rounded size -> blocks); every kernel of the context runs on its stream
  std::multimap<size_t, void *> cache;
  size_t cached_bytes = 0;
  size_t cache_limit = 0;
};

// Device memory through the context's allocator (stream ordered).
void *dalloc(Ctx *c, size_t bytes);
void dfree(Ctx *c, void *p, size_t bytes);

// A device array owned by a log or a scope.
template <class T>
struct DBuf {
  T *p = nullptr;
  size_t n = 0;
};

// Scope holding temporary device buffers, released in stream order.
struct Scratch {
  Ctx *c;
  std::vector<std::pair<void *, size_t>> bufs;
  explicit Scratch(Ctx *ctx) : c(ctx) {}
  ~Scratch() {
    for (auto &b : bufs) dfree(c, b.first, b.second);
  }
  template <class T>
  T *get(size_t n) {
    size_t bytes = (n ? n : 1) * sizeof(T);
    void *p = dalloc(c, bytes);
    if (p) bufs.push_back({p, bytes});
    return (T *)p;
  }
};

// Kernel timing scope: begin/end events on the context stream.
struct KTime {
  Ctx *c;
  const char *name;
  cudaEvent_t a = nullptr, b = nullptr;
  KTime(Ctx *ctx, const char *nm);
  ~KTime();
};

int check_launch(Ctx *c, const char *what);

// NVTX range over an ABI call (visible to profilers; no cost without one).
struct ApiRange {
  explicit ApiRange(const char *name) { nvtxRangePushA(name); }
  ~ApiRange() { nvtxRangePop(); }
  ApiRange(const ApiRange &) = delete;
  ApiRange &operator=(const ApiRange &) = delete;
};

// A kernel's dynamic shared-memory limit is one setting per function, shared by
// every thread and context of the process, so it is always set to the
// device's opt-in maximum (a launch still uses only what it asks for):
// concurrent calls with different needs cannot undo each other's setting.
inline int smem_optin_max() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

// Device arrays of a log or context, through the context's allocator.
template <class T>
inline void free_buf(Ctx *c, DBuf<T> &b) {
  if (b.p) dfree(c, b.p, (b.n ? b.n : 1) * sizeof(T));
  b.p = nullptr;
  b.n = 0;
}

// A buffer that already holds an array gives it back first (in stream order):
// a call retried after failing part way through its allocations, such as a
// variant request that ran out of memory, leaves nothing behind.
template <class T>
inline int alloc_buf(Ctx *c, DBuf<T> &b, size_t n) {
  free_buf(c, b);
  b.n = n;
  b.p = (T *)dalloc(c, (n ? n : 1) * sizeof(T));
  if (!b.p) {
    b.n = 0;
    set_error("device allocation of %zu bytes failed", (n ? n : 1) * sizeof(T));
    return PM4G_ENOMEM;
  }
  return PM4G_OK;
}

// Pinned host staging owned by the context (grown on demand): device-to-host
// copies land there asynchronously, so a batch of them costs one
// synchronisation; the bytes then move to their destinations on the host.
char *pinned(Ctx *c, size_t bytes);

// A batch of device-to-host copies through the staging area. The caller
// states an upper bound of the batch's bytes (each copy adds up to 15 bytes of
// alignment) before the first add; nothing else may use the staging area
// until finish().
struct D2HBatch {
  Ctx *c;
  char *base = nullptr;
  size_t cap = 0, used = 0;
  int st = PM4G_OK;
  std::vector<std::tuple<void *, size_t, size_t>> items;
  D2HBatch(Ctx *ctx, size_t bound) : c(ctx), cap(bound) {
    base = pinned(c, bound < 16 ? 16 : bound);
    if (!base) {
      set_error("out of pinned host memory for results");
      st = PM4G_ENOMEM;
    }
  }
  void add(void *dst, const void *src, size_t bytes) {
    if (st != PM4G_OK || bytes == 0) return;
    used = (used + 15) & ~(size_t)15;
    if (used + bytes > cap) {
      set_error("internal: result staging bound exceeded");
      st = PM4G_ECUDA;
      return;
    }
    const cudaError_t e = cudaMemcpyAsync(base + used, src, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) {
      set_error("device-to-host copy failed: %s", cudaGetErrorString(e));
      st = PM4G_ECUDA;
      return;
    }
    items.emplace_back(dst, used, bytes);
    used += bytes;
  }
  int finish() {
    if (st != PM4G_OK) return st;
    PM4G_CK(cudaStreamSynchronize(c->stream));
    for (auto &it : items) memcpy(std::get<0>(it), base + std::get<1>(it), std::get<2>(it));
    return PM4G_OK;
  }
};

// One device-to-host copy, synchronised (up to 256 bytes through the mapped
// bytes of the context).
int d2h(Ctx *c, void *dst, const void *src, size_t bytes);
// Reads n (1..8) 32-bit device words with one wait on the context stream.
int d2h_words(Ctx *c, uint32_t *const *dst, const uint32_t *const *src, int n);
// Device-mapped staging of at least `bytes` (host pointer; *dev the device
// view), or NULL if bytes > kMappedMax or the allocation fails. Growing it
// waits for the context stream.
constexpr size_t kMappedMax = (size_t)64 << 20;
char *mapped_buf(Ctx *c, size_t bytes, char **dev);
bool small_buffer(Ctx *c);

}  // namespace pm4g
struct pm4g_log;
namespace pm4g {
// Log helpers (capi.cu): the formatted log in export order into device arrays
// (any may be NULL), and the per-slot case offsets L->off.
int run_export(pm4g_log *L, int32_t *ec, int32_t *ea, int64_t *et, int64_t *er);
int ensure_offsets(pm4g_log *L);
// The edges of a hashed global table: their keys (src * A + dst), ascending,
// and slot indices, in arrays of the scope S.
int hashed_edges(pm4g_log *L, Scratch &S, uint32_t *&keys, uint32_t *&slots, uint32_t &E);


// ---- primitives (prims.cu) ----
// Exclusive scan of n uint32 values; out must hold n + 1 entries, out[n] = total.
int scan_u32(Ctx *c, const uint32_t *in, uint32_t *out, int64_t n);
// Stable LSD radix sort of (key, value) pairs by key bits [begin_bit, end_bit).
// Sorts in place using the given temporaries of the same length.
int radix_sort_u32(Ctx *c, uint32_t *keys, uint32_t *vals, uint32_t *keys_tmp, uint32_t *vals_tmp,
                   int64_t n, int begin_bit, int end_bit);
int radix_sort_u64(Ctx *c, uint64_t *keys, uint32_t *vals, uint64_t *keys_tmp, uint32_t *vals_tmp,
                   int64_t n, int begin_bit, int end_bit);
// Stream compaction helpers
int iota_u32(Ctx *c, uint32_t *out, int64_t n);

inline int bits_for(uint64_t maxval) {  // bits to represent values in [0, maxval]
  int b = 0;
  while (b < 64 && (maxval >> b)) ++b;
  return b;
}

inline unsigned grid_for(int64_t n, int per_block, unsigned cap = 1u << 20) {
  int64_t g = (n + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > (int64_t)cap) g = cap;
  return (unsigned)g;
}

}  // namespace pm4g

// Handles of the C ABI.
struct pm4g_ctx : public pm4g::Ctx {};

struct pm4g_log {
  pm4g::Ctx *ctx = nullptr;
  int64_t n = 0;
  int32_t A = 1;
  int64_t C = 0;
  int32_t min_case = 0;
  uint64_t R = 0;  // case slots
  int clb = 0;
  int act_bits = 0;
  uint32_t nb = 0;
  bool has_attr = false;
  pm4g::DBuf<uint4> rec;
  pm4g::DBuf<uint32_t> bucket_off;
  pm4g::DBuf<uint16_t> act_s;  // activities in formatted order (16 bits: at most 65,536 activities)
  pm4g::DBuf<uint32_t> len;
  pm4g::DBuf<int32_t> cattr;
  pm4g::DBuf<int32_t> uniq;  // sorted distinct case ids when renumbered
  // global edge table: 5 arrays of gcells cells (cnt, lo, hi, min, max),
  // dense over the A * A pairs, or (ghash) open addressing whose keys
  // (key + 1, 0 = empty) are in gkey
  pm4g::DBuf<unsigned long long> dfg;
  uint64_t gcells = 0;
  bool ghash = false;
  pm4g::DBuf<unsigned long long> gkey;
  pm4g::DBuf<unsigned long long> ends; // 2 * A: start, end
  // every bucket's records are in row order (the stable partition bucketed
  // them, or a filter of such a log): only then may the streaming pass run
  bool row_ordered = false;
  // one device word: bit 0 an activity outside [0, A) was seen
  pm4g::DBuf<uint32_t> status;
  // caches
  bool edges_ready = false;
  std::vector<int32_t> e_src, e_dst;
  std::vector<uint64_t> e_cnt, e_lo, e_hi, e_min, e_max, h_start, h_end, h_freq;
  std::vector<double> e_mean;
  bool span_ready = false;
  pm4g::DBuf<int64_t> span;  // first_ts[R], last_ts[R]
  bool var_ready = false;
  uint32_t V = 0;
  pm4g::DBuf<uint32_t> off, rep_slots, order, vcount, rep_of;
  bool off_ready = false;  // off holds the case offsets (else ensure_offsets forms them)
  pm4g::DBuf<uint32_t> rep_pos;  // exclusive prefix of the representative flags (the case variants' input)
  pm4g::DBuf<int32_t> cvar;      // variant rank of every case slot, formed when first asked for
  // drill-down index (batched drill-down; built on first use)
  bool dd_ready = false;
  pm4g::DBuf<int64_t> ts_s;       // timestamps in (case, timestamp, row) order
  pm4g::DBuf<int64_t> row_s;      // original rows in that order (paths filter; built on first use)
  pm4g::DBuf<uint32_t> aslots;    // present case slots ordered by (attribute, slot)
  pm4g::DBuf<uint32_t> apre;      // events before each entry of aslots (C + 1)
  pm4g::DBuf<uint32_t> aoff, alen; // first formatted position and length of each entry of aslots
  pm4g::DBuf<uint32_t> eidx_s;     // edge index of the pair (event, next event of its case), ~0 at case ends
  std::vector<int32_t> attr_vals; // distinct attribute values, ascending
  std::vector<uint32_t> attr_lo;  // their first entry in aslots (one more at the end)
  std::vector<uint32_t> attr_ev;  // events before that entry
  pm4g::DBuf<uint32_t> emap;      // A * A: edge index of a directly-follows pair, or ~0
  pm4g::DBuf<int32_t> e_pair;     // 2 * E: src and dst of every edge, (src, dst) order
  pm4g::DBuf<uint32_t> ekey;      // E: src * A + dst of every edge, ascending (hashed table only)
  uint32_t n_edges = 0;
};

