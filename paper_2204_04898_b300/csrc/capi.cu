// C ABI of the engine (include/pm4g.h): contexts, log handles, the formatting
// and segment passes, and the queries of Section 3 (DFG, performance DFG,
// start/end activities, variants, drill-down filters, formatted-log export).
#include <algorithm>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "device_common.cuh"
#include "engine.h"
#include "kernels.h"
#include "variants.h"

using namespace pm4g;

// ---------------------------------------------------------------------------
// errors, memory, timing
// ---------------------------------------------------------------------------
namespace pm4g {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int check_launch(Ctx *c, const char *what) {
  c->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("launch of %s failed: %s", what, cudaGetErrorString(e));
    return PM4G_ECUDA;
  }
  return PM4G_OK;
}

// Without a caller-supplied allocator, device memory comes from the stream-
// ordered pool, and blocks the context frees are kept in its cache: a later
// request of the same rounded size reuses one at once. Reuse is safe because
// every kernel and copy of the context runs on its one stream, in order. The
// cache is emptied when the pool cannot satisfy a request, and when it would
// exceed its limit the freed block goes back to the pool.
static size_t cache_round(size_t bytes) {
  if (bytes <= 4096) return (bytes + 255) & ~(size_t)255;
  size_t p2 = 4096;
  while (p2 < bytes) p2 <<= 1;
  const size_t g = p2 >> 4;  // sizes round up by at most 1/16
  return (bytes + g - 1) / g * g;
}

static void cache_flush(Ctx *c) {
  for (auto &kv : c->cache) cudaFreeAsync(kv.second, c->stream);
  c->cache.clear();
  c->cached_bytes = 0;
}

void *dalloc(Ctx *c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (c->has_alloc) {
    void *p = c->alloc.alloc(bytes, (void *)c->stream, c->alloc.user);
    if (p && ((uintptr_t)p & 15u)) {  // bulk copies and vector loads need 16-byte alignment
      c->alloc.free(p, bytes, (void *)c->stream, c->alloc.user);
      set_error("the context's allocator returned memory not aligned to 16 bytes");
      return nullptr;
    }
    return p;
  }
  const size_t key = cache_round(bytes);
  auto it = c->cache.find(key);
  if (it != c->cache.end()) {
    void *p = it->second;
    c->cache.erase(it);
    c->cached_bytes -= key;
    return p;
  }
  void *p = nullptr;
  if (cudaMallocAsync(&p, key, c->stream) != cudaSuccess) {
    cudaGetLastError();
    if (c->cache.empty()) return nullptr;
    cache_flush(c);
    if (cudaMallocAsync(&p, key, c->stream) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
  }
  return p;
}

void dfree(Ctx *c, void *p, size_t bytes) {
  if (!p) return;
  if (bytes == 0) bytes = 16;
  if (c->has_alloc) {
    c->alloc.free(p, bytes, (void *)c->stream, c->alloc.user);
    return;
  }
  const size_t key = cache_round(bytes);
  if (c->cached_bytes + key <= c->cache_limit) {
    c->cache.emplace(key, p);
    c->cached_bytes += key;
  } else {
    cudaFreeAsync(p, c->stream);
  }
}

// Adds the durations of the finished timing pairs at the front of the pending
// list to the totals and returns their events to the pool (no wait).
static void settle_finished(Ctx *c) {
  size_t k = 0;
  for (; k < c->pending.size(); ++k) {
    const TimingRec &p = c->pending[k];
    if (cudaEventQuery(p.b) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    auto &t = c->totals[p.name];
    t.first += 1;
    t.second += ms;
    c->free_events.push_back(p.a);
    c->free_events.push_back(p.b);
  }
  cudaGetLastError();  // a query of an unfinished event is not an error
  c->pending.erase(c->pending.begin(), c->pending.begin() + k);
}

static cudaEvent_t get_event(Ctx *c) {
  if (c->free_events.empty()) settle_finished(c);
  if (!c->free_events.empty()) {
    cudaEvent_t e = c->free_events.back();
    c->free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// The kernels PM4G_OPT_TIMING = 2 times: each is one launch carrying most of
// its call's device time.
static bool dominant_kernel(const char *nm) {
  static const char *const names[] = {"segment", "segment_sort", "partition", "batch_dfg", "efg", "filter"};
  for (const char *x : names)
    if (strcmp(nm, x) == 0) return true;
  return false;
}

KTime::KTime(Ctx *ctx, const char *nm) : c(ctx), name(nm) {
  if (c->timing == 1 || (c->timing == 2 && dominant_kernel(nm))) {
    a = get_event(c);
    cudaEventRecord(a, c->stream);
  }
}

KTime::~KTime() {
  if (c->timing && a) {
    b = get_event(c);
    cudaEventRecord(b, c->stream);
    c->pending.push_back({name, a, b});
  }
}

char *pinned(Ctx *c, size_t bytes) {
  if (bytes <= c->pin_bytes) return (char *)c->pin;
  if (c->pin) {
    cudaStreamSynchronize(c->stream);
    cudaFreeHost(c->pin);
    c->pin = nullptr;
    c->pin_bytes = 0;
  }
  size_t want = (size_t)1 << 20;
  while (want < bytes) want <<= 1;
  if (cudaHostAlloc(&c->pin, want, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    c->pin = nullptr;
    return nullptr;
  }
  c->pin_bytes = want;
  return (char *)c->pin;
}

namespace {
constexpr size_t kSmallBytes = 256;
__global__ void k_small_copy(const unsigned char *__restrict__ src, unsigned char *dst, uint32_t n) {
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}
struct WordSrcs {
  const uint32_t *p[8];
};
__global__ void k_words_copy(WordSrcs w, int n, uint32_t *dst) {
  if ((int)threadIdx.x < n) dst[threadIdx.x] = *w.p[threadIdx.x];
}
}  // namespace

bool small_buffer(Ctx *c) {
  if (!c->small) {
    if (cudaHostAlloc(&c->small, kSmallBytes, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(&c->small_dev, c->small, 0) != cudaSuccess) {
      cudaGetLastError();
      if (c->small) cudaFreeHost(c->small);
      c->small = nullptr;
      c->small_dev = nullptr;
    }
  }
  return c->small != nullptr;
}

char *mapped_buf(Ctx *c, size_t bytes, char **dev) {
  if (bytes > kMappedMax) return nullptr;
  if (bytes > c->mapped_bytes) {
    if (c->mapped) {
      cudaStreamSynchronize(c->stream);  // kernels in flight may still write the old buffer
      cudaFreeHost(c->mapped);
      c->mapped = c->mapped_dev = nullptr;
      c->mapped_bytes = 0;
    }
    size_t want = (size_t)1 << 20;
    while (want < bytes) want <<= 1;
    if (cudaHostAlloc(&c->mapped, want, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(&c->mapped_dev, c->mapped, 0) != cudaSuccess) {
      cudaGetLastError();
      if (c->mapped) cudaFreeHost(c->mapped);
      c->mapped = c->mapped_dev = nullptr;
      return nullptr;
    }
    c->mapped_bytes = want;
  }
  *dev = (char *)c->mapped_dev;
  return (char *)c->mapped;
}

int d2h_words(Ctx *c, uint32_t *const *dst, const uint32_t *const *src, int n) {
  if (n < 1 || n > 8) return PM4G_EINVAL;
  if (!small_buffer(c)) {
    for (int i = 0; i < n; ++i) PM4G_TRY(d2h(c, dst[i], src[i], 4));
    return PM4G_OK;
  }
  WordSrcs w{};
  for (int i = 0; i < n; ++i) w.p[i] = src[i];
  k_words_copy<<<1, 32, 0, c->stream>>>(w, n, (uint32_t *)c->small_dev);
  PM4G_TRY(check_launch(c, "k_words_copy"));
  PM4G_CK(cudaStreamSynchronize(c->stream));
  for (int i = 0; i < n; ++i) *dst[i] = ((const uint32_t *)c->small)[i];
  return PM4G_OK;
}

int d2h(Ctx *c, void *dst, const void *src, size_t bytes) {
  if (!bytes) return PM4G_OK;
  if (bytes <= kSmallBytes) {
    if (small_buffer(c)) {
      k_small_copy<<<1, 64, 0, c->stream>>>((const unsigned char *)src, (unsigned char *)c->small_dev,
                                            (uint32_t)bytes);
      PM4G_TRY(check_launch(c, "k_small_copy"));
      PM4G_CK(cudaStreamSynchronize(c->stream));
      memcpy(dst, c->small, bytes);
      return PM4G_OK;
    }
  }
  D2HBatch b(c, bytes);
  b.add(dst, src, bytes);
  return b.finish();
}

}  // namespace pm4g

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------
static void release_log(pm4g_log *L) {
  if (!L) return;
  Ctx *c = L->ctx;
  free_buf(c, L->rec);
  free_buf(c, L->bucket_off);
  free_buf(c, L->act_s);
  free_buf(c, L->len);
  free_buf(c, L->cattr);
  free_buf(c, L->uniq);
  free_buf(c, L->dfg);
  free_buf(c, L->gkey);
  free_buf(c, L->ekey);
  free_buf(c, L->ends);
  free_buf(c, L->span);
  free_buf(c, L->off);
  free_buf(c, L->rep_slots);
  free_buf(c, L->order);
  free_buf(c, L->vcount);
  free_buf(c, L->rep_of);
  free_buf(c, L->cvar);
  free_buf(c, L->rep_pos);
  free_buf(c, L->status);
  free_buf(c, L->ts_s);
  free_buf(c, L->row_s);
  free_buf(c, L->aslots);
  free_buf(c, L->apre);
  free_buf(c, L->aoff);
  free_buf(c, L->alen);
  free_buf(c, L->eidx_s);
  free_buf(c, L->emap);
  free_buf(c, L->e_pair);
  c->live_logs--;
  delete L;
}



// ---------------------------------------------------------------------------
// segment pass configuration
// ---------------------------------------------------------------------------
struct SegConfig {
  int cap, a_s, tbl_mode, tbl_slots;
  size_t smem;
};

static SegConfig seg_config(Ctx *c, int clb, int32_t A) {
  SegConfig s;
  const int ncl = 1 << clb;
  s.a_s = A <= 2048 ? A : 0;
  const int64_t cells = (int64_t)A * A;
  if (cells <= 4096) {
    s.tbl_mode = 0;
    s.tbl_slots = (int)cells;
  } else {
    s.tbl_mode = 1;
    s.tbl_slots = 4096;
  }
  // the largest multiple of 32 records whose layout fits the opt-in shared memory
  int64_t lo = 0, hi = std::min(65535, kSegThreads * kSegChunks) / 32;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if (seg_smem_layout((int)(mid * 32), ncl, s.a_s, s.tbl_slots, s.tbl_mode).total + 64 <= (size_t)c->smem_optin)
      lo = mid;
    else
      hi = mid - 1;
  }
  int64_t cap = lo * 32;
  if (c->test_bucket_cap > 0) cap = std::min<int64_t>(cap, c->test_bucket_cap);
  s.cap = (int)std::max<int64_t>(cap, 0);
  s.smem = seg_smem_layout(s.cap, ncl, s.a_s, s.tbl_slots, s.tbl_mode).total;
  return s;
}

static SegArgs seg_args(pm4g_log *L, const SegConfig &sc, uint32_t *work, uint32_t *ovf, uint32_t *n_ovf,
                        unsigned long long *n_cases) {
  SegArgs a{};
  a.rec = L->rec.p;
  a.bucket_off = L->bucket_off.p;
  a.nb = L->nb;
  a.clb = L->clb;
  a.act_bits = L->act_bits;
  a.n_act = (uint32_t)L->A;
  a.n_slots = L->R;
  a.cap = sc.cap;
  a.ep_smem = sc.a_s > 0;
  a.tbl_mode = sc.tbl_mode;
  a.tbl_slots = sc.tbl_slots;
  a.work = work;
  a.act_s = L->act_s.p;
  a.len = L->len.p;
  const size_t cells = L->gcells;
  a.g.cnt = L->dfg.p;
  a.g.lo = L->dfg.p + cells;
  a.g.hi = L->dfg.p + 2 * cells;
  a.g.mn = L->dfg.p + 3 * cells;
  a.g.mx = L->dfg.p + 4 * cells;
  a.g.key = L->ghash ? L->gkey.p : nullptr;
  a.g.mask = L->ghash ? cells - 1 : 0;
  a.g_start = L->ends.p;
  a.g_end = L->ends.p + L->A;
  a.ovf = ovf;
  a.n_ovf = n_ovf;
  a.n_cases = n_cases;
  a.min_case = L->min_case;
  a.uniq = L->uniq.p;
  return a;
}

// Global-memory path for one bucket (too many events, or a case too long to
// sort on chip): radix sort by (case slot, timestamp, row), then the same
// per-position computation with global atomics.
static int fallback_bucket(pm4g_log *L, const SegArgs &a, uint32_t b, bool exp) {
  Ctx *c = L->ctx;
  uint32_t lohi[2];
  PM4G_TRY(d2h(c, lohi, L->bucket_off.p + b, sizeof(lohi)));
  const uint32_t lo = lohi[0], n = lohi[1] - lohi[0];
  const int ncl = 1 << L->clb;
  Scratch S(c);
  uint32_t *keys = S.get<uint32_t>(n), *vals = S.get<uint32_t>(n);
  uint32_t *keys2 = S.get<uint32_t>(n), *vals2 = S.get<uint32_t>(n);
  uint64_t *k64 = S.get<uint64_t>(n), *k64b = S.get<uint64_t>(n);
  uint4 *srec = S.get<uint4>(n);
  uint32_t *ccnt = S.get<uint32_t>(ncl), *cstart = S.get<uint32_t>(ncl + 1);
  if (!keys || !vals || !keys2 || !vals2 || !k64 || !k64b || !srec || !ccnt || !cstart) {
    set_error("bucket fallback: out of device memory");
    return PM4G_ENOMEM;
  }
  const uint4 *rec = L->rec.p + lo;
  const unsigned g = grid_for(n, 256, 8192);
  {
    KTime t(c, "fallback");
    k_fb_keys_row<<<g, 256, 0, c->stream>>>(rec, n, keys, vals);
    PM4G_TRY(check_launch(c, "k_fb_keys_row"));
  }
  PM4G_TRY(radix_sort_u32(c, keys, vals, keys2, vals2, n, 0, 32));
  {
    KTime t(c, "fallback");
    k_fb_keys_ts<<<g, 256, 0, c->stream>>>(rec, vals, n, k64);
    PM4G_TRY(check_launch(c, "k_fb_keys_ts"));
  }
  PM4G_TRY(radix_sort_u64(c, k64, vals, k64b, vals2, n, 0, 64));
  if (L->clb > 0) {
    {
      KTime t(c, "fallback");
      k_fb_keys_case<<<g, 256, 0, c->stream>>>(rec, vals, n, L->act_bits, (uint32_t)ncl - 1, keys);
      PM4G_TRY(check_launch(c, "k_fb_keys_case"));
    }
    PM4G_TRY(radix_sort_u32(c, keys, vals, keys2, vals2, n, 0, L->clb));
  }
  PM4G_CK(cudaMemsetAsync(ccnt, 0, ncl * sizeof(uint32_t), c->stream));
  {
    KTime t(c, "fallback");
    k_fb_gather<<<g, 256, 0, c->stream>>>(rec, vals, n, srec);
    PM4G_TRY(check_launch(c, "k_fb_gather"));
    k_fb_hist<<<g, 256, 0, c->stream>>>(srec, n, L->act_bits, (uint32_t)ncl - 1, ccnt);
    PM4G_TRY(check_launch(c, "k_fb_hist"));
  }
  PM4G_TRY(scan_u32(c, ccnt, cstart, ncl));
  KTime t(c, "fallback");
  c->launches++;
  PM4G_CK(launch_fb_compute(exp, a, srec, n, b, cstart, g, c->stream));
  k_fb_cases<<<(ncl + 255) / 256, 256, 0, c->stream>>>(a, srec, b, ccnt, cstart, ncl, exp ? 0 : 1);
  return check_launch(c, "k_fb_cases");
}

// Runs the segment pass over a bucketed log: fills act_s, len, the DFG table,
// the endpoint counts and (at load) the per-case attribute, and the case
// offsets when the streaming pass formats the log; sets C.
// err_in (optional): a device word to read back with the pass's own counters
// (one synchronisation for both); its value goes to *err_out.
// keys (optional): the first word of every bucketed record, in bucket order,
// written by the partition; with it, the streaming pass takes the log first
// (it gives up on a log with a case out of timestamp order, which the sorting
// pass then formats).
static int run_segment(pm4g_log *L, const int32_t *attr_in, bool write_cattr, const uint32_t *err_in = nullptr,
                       uint32_t *err_out = nullptr, const uint32_t *keys = nullptr) {
  Ctx *c = L->ctx;
  // The global edge table: dense over the A * A pairs up to A = 4096 (at most
  // 670 MB); beyond that, or when a test asks for it, open addressing with
  // twice as many slots as the log can have distinct pairs (a power of two).
  L->ghash = L->A > kDenseMaxActivities || c->edge_table == 1;
  size_t cells = (size_t)L->A * L->A;
  if (L->ghash) {
    const uint64_t pairs = std::min<uint64_t>((uint64_t)L->A * (uint64_t)L->A, (uint64_t)std::max<int64_t>(L->n, 1));
    uint64_t T = 4096;
    while (T < 2 * pairs) T <<= 1;
    cells = T;
    PM4G_TRY(alloc_buf(c, L->gkey, cells));
    PM4G_CK(cudaMemsetAsync(L->gkey.p, 0, cells * sizeof(unsigned long long), c->stream));
  }
  L->gcells = cells;
  PM4G_TRY(alloc_buf(c, L->act_s, L->n));
  if (!L->len.p) PM4G_TRY(alloc_buf(c, L->len, L->R));
  PM4G_TRY(alloc_buf(c, L->dfg, 5 * cells));
  PM4G_TRY(alloc_buf(c, L->ends, 2 * (size_t)L->A));
  PM4G_CK(cudaMemsetAsync(L->dfg.p, 0, 3 * cells * sizeof(unsigned long long), c->stream));
  PM4G_CK(cudaMemsetAsync(L->dfg.p + 3 * cells, 0xFF, cells * sizeof(unsigned long long), c->stream));
  PM4G_CK(cudaMemsetAsync(L->dfg.p + 4 * cells, 0, cells * sizeof(unsigned long long), c->stream));
  PM4G_CK(cudaMemsetAsync(L->ends.p, 0, 2 * L->A * sizeof(unsigned long long), c->stream));
  if (write_cattr) {
    PM4G_TRY(alloc_buf(c, L->cattr, L->R));
    PM4G_CK(cudaMemsetAsync(L->cattr.p, 0, L->R * sizeof(int32_t), c->stream));
  }
  PM4G_CK(cudaMemsetAsync(L->len.p, 0, L->R * sizeof(uint32_t), c->stream));
  if (L->n == 0 || L->nb == 0) {
    L->C = 0;
    return PM4G_OK;
  }
  Scratch S(c);
  // status block: counters {work, n_ovf, -, -}, {cases, sorted windows}, caller's word
  struct Status {
    uint32_t ctr[4];
    unsigned long long nc[2];
    uint32_t err[4];
  };
  Status *blk = S.get<Status>(1);
  uint32_t *ovf = S.get<uint32_t>(L->nb);
  if (!blk || !ovf) {
    set_error("segment pass: out of device memory");
    return PM4G_ENOMEM;
  }
  uint32_t *ctr = blk->ctr;
  unsigned long long *n_cases = blk->nc;
  PM4G_CK(cudaMemsetAsync(blk, 0, sizeof(Status), c->stream));
  const SegConfig sc = seg_config(c, L->clb, L->A);
  SegArgs a = seg_args(L, sc, ctr, ovf, ctr + 1, n_cases);
  a.n_sorted = n_cases + 1;
  a.attr_in = attr_in;
  a.cattr = write_cattr ? L->cattr.p : nullptr;
  a.err = ctr + 2;
  a.g.err = ctr + 2;
  if (keys && L->row_ordered && c->test_bucket_cap == 0 && sc.cap >= 32 && !L->ghash && L->A <= 2048 &&
      !c->stream_off) {
    // the streaming pass, for logs whose cases' events come in timestamp
    // order (it checks this itself; a log where it finds a case out of order
    // is cleared of its partial sums and redone by the sorting pass below)
    int w = stream_segment_warps(L->clb, sc.a_s, (size_t)c->smem_optin);
    if (c->stream_warps > 0) w = std::min(w, c->stream_warps);
    const size_t cells = (size_t)L->A * L->A;
    uint32_t *emap = w > 0 ? S.get<uint32_t>(cells) : nullptr;
    uint32_t *key_of = w > 0 ? S.get<uint32_t>(kStSlots) : nullptr;
    if (w > 0 && (!emap || !key_of)) {
      set_error("segment pass: out of device memory for the edge ids");
      return PM4G_ENOMEM;
    }
    if (w > 0 && !L->off.p) PM4G_TRY(alloc_buf(c, L->off, L->R + 1));
    if (w > 0) {
      PM4G_CK(cudaMemsetAsync(emap, 0xFF, cells * sizeof(uint32_t), c->stream));
      a.off_out = L->off.p;
      a.ran = blk->err + 1;
      a.keys = keys;
      a.emap = emap;
      a.key_of = key_of;
      a.n_ids = ctr + 3;
      const size_t smem = st_smem_layout(1 << L->clb, sc.a_s, w).total;
      const unsigned grid = std::min<unsigned>((L->nb + w - 1) / w, (unsigned)c->num_sms);
      {
        KTime t(c, "segment");
        c->launches++;
        PM4G_CK(launch_stream_segment(a, w, grid, smem, c->stream));
      }
      c->launches++;
      PM4G_CK(launch_stream_undo(a, (uint32_t)L->A, (unsigned)c->num_sms, c->stream));
      a.skip_ordered = 1;
    }
  }
  if (sc.cap >= 32) {
    const unsigned grid = std::min<unsigned>(L->nb, (unsigned)c->num_sms);
    KTime t(c, "segment_sort");
    c->launches++;
    PM4G_CK(launch_segment(false, a, grid, sc.smem, c->stream));
  } else {
    // nothing fits on chip: every bucket takes the global-memory path
    std::vector<uint32_t> all(L->nb);
    for (uint32_t b = 0; b < L->nb; ++b) all[b] = b;
    PM4G_CK(cudaMemcpyAsync(ovf, all.data(), L->nb * sizeof(uint32_t), cudaMemcpyHostToDevice, c->stream));
    const uint32_t nbv = L->nb;
    PM4G_CK(cudaMemcpyAsync(ctr + 1, &nbv, sizeof(uint32_t), cudaMemcpyHostToDevice, c->stream));
  }
  if (err_in) PM4G_CK(cudaMemcpyAsync(blk->err, err_in, 4, cudaMemcpyDeviceToDevice, c->stream));
  Status h{};
  PM4G_TRY(d2h(c, &h, blk, sizeof(Status)));
  if (err_out) *err_out = h.err[0];
  if (h.ctr[2] & 1u) {
    set_error("internal: case lengths counted by the partition disagree with the bucketed records");
    return PM4G_ECUDA;
  }
  if (h.ctr[2] & 2u) {
    set_error("internal: the hashed edge table is full");
    return PM4G_ECUDA;
  }
  const uint32_t n_ovf = h.ctr[1];
  if (n_ovf) {
    std::vector<uint32_t> list(n_ovf);
    PM4G_TRY(d2h(c, list.data(), ovf, n_ovf * sizeof(uint32_t)));
    std::sort(list.begin(), list.end());
    for (uint32_t b : list) PM4G_TRY(fallback_bucket(L, a, b, false));
    PM4G_TRY(d2h(c, h.nc, n_cases, sizeof(h.nc)));  // the global path adds its cases
  }
  L->C = (int64_t)h.nc[0];
  L->off_ready = h.err[1] != 0 && !(h.ctr[2] & kStDisorder);  // the streaming pass wrote the case offsets
  auto &sw = c->totals["sorted_windows"];
  sw.first += (int64_t)h.nc[1];
  return PM4G_OK;
}

// Chooses the bucket width (2^clb case slots) so that a bucket's expected
// events stay well inside the on-chip capacity.
static int choose_clb(Ctx *c, int64_t n, uint64_t R, int32_t A, int act_bits) {
  if (c->load_clb > 0) return std::min(c->load_clb, 32 - act_bits);  // a launch choice (autotuner)
  const double avg = (double)n / (double)std::max<uint64_t>(R, 1);
  int best = 0;
  for (int clb = 8; clb >= 0; --clb) {  // per-warp case counts hold at most 256 slots
    if (clb + act_bits > 32) continue;
    const SegConfig sc = seg_config(c, clb, A);
    if (avg * (double)(1 << clb) <= 0.8 * (double)sc.cap) {
      best = clb;
      break;
    }
  }
  // keep at least two buckets per SM when the log allows it
  while (best > 3 && ((R + (1ull << best) - 1) >> best) < 2ull * (uint64_t)c->num_sms) --best;
  return best;
}

// The API functions below take C linkage from their declarations in pm4g.h.

const char *pm4g_last_error(void) { return pm4g::g_err; }

const char *pm4g_kernel_names(void) {
  return "stats,bucket_hist,bucket_scatter,partition,segment,segment_sort,fallback,scan,radix_sort,filter,variants,dfg,"
         "export,batch,batch_dfg,efg";
}

int pm4g_ctx_create(pm4g_ctx **out, int device, void *cuda_stream, const pm4g_allocator *alloc) {
  if (!out) {
    set_error("pm4g_ctx_create: out is NULL");
    return PM4G_EINVAL;
  }
  *out = nullptr;
  int ndev = 0;
  PM4G_CK(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) {
    set_error("pm4g_ctx_create: device %d out of range (%d devices)", device, ndev);
    return PM4G_EINVAL;
  }
  if (alloc && (!alloc->alloc || !alloc->free)) {
    set_error("pm4g_ctx_create: allocator needs both alloc and free");
    return PM4G_EINVAL;
  }
  PM4G_CK(cudaSetDevice(device));
  pm4g_ctx *c = new (std::nothrow) pm4g_ctx();
  if (!c) return PM4G_ENOMEM;
  c->device = device;
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      set_error("pm4g_ctx_create: stream creation failed");
      return PM4G_ECUDA;
    }
    c->own_stream = true;
  }
  if (alloc) {
    c->alloc = *alloc;
    c->has_alloc = true;
  } else {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;  // keep freed blocks cached in this process
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  }
  {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) c->cache_limit = tot / 2;
    cudaGetLastError();
  }
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  *out = c;
  return PM4G_OK;
}

int pm4g_ctx_destroy(pm4g_ctx *c) {
  if (!c) return PM4G_OK;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  for (auto &p : c->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : c->free_events) cudaEventDestroy(e);
  cache_flush(c);
  cudaStreamSynchronize(c->stream);
  if (c->pin) cudaFreeHost(c->pin);
  if (c->small) cudaFreeHost(c->small);
  if (c->mapped) cudaFreeHost(c->mapped);
  if (c->copy_stream) {
    cudaStreamSynchronize(c->copy_stream);
    cudaStreamDestroy(c->copy_stream);
  }
  if (c->copy_ready) cudaEventDestroy(c->copy_ready);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return PM4G_OK;
}

int pm4g_ctx_set_option(pm4g_ctx *c, int option, int64_t value) {
  if (!c) {
    set_error("pm4g_ctx_set_option: ctx is NULL");
    return PM4G_EINVAL;
  }
  switch (option) {
    case PM4G_OPT_TIMING:
      if (value < 0 || value > 2) break;
      c->timing = (int)value;
      return PM4G_OK;
    case PM4G_OPT_TEST_HASH_BITS:
      if (value < 0 || value > 63) break;
      c->test_hash_bits = (int)value;
      return PM4G_OK;
    case PM4G_OPT_BATCH_CHUNK:
      if (value != 0 && value != 8 && value != 16 && value != 32) break;
      c->batch_chunk = (int)value;
      return PM4G_OK;
    case PM4G_OPT_BATCH_STAGES:
      if (value < 0 || value > 16) break;
      c->batch_stages = (int)value;
      return PM4G_OK;
    case PM4G_OPT_BATCH_ITEMS_PER_SM:
      if (value < 0 || value > 32) break;
      c->batch_items_per_sm = (int)value;
      return PM4G_OK;
    case PM4G_OPT_TEST_BUCKET_CAP:
      if (value != 0 && (value < 32 || value > 65535)) break;
      c->test_bucket_cap = (int)value;
      return PM4G_OK;
    case PM4G_OPT_EDGE_TABLE:
      if (value < 0 || value > 1) break;
      c->edge_table = (int)value;
      return PM4G_OK;
    case PM4G_OPT_LOAD_CLB:
      if (value < 0 || value > 8) break;
      c->load_clb = (int)value;
      return PM4G_OK;
    case PM4G_OPT_LOAD_SPLITS:
      if (value < 0 || value > 64) break;
      c->load_splits = (int)value;
      return PM4G_OK;
    case PM4G_OPT_STREAM_WARPS:
      if (value < 0 || value > kStMaxThreads / 32) break;
      c->stream_warps = (int)value;
      return PM4G_OK;
    case PM4G_OPT_STREAM_OFF:
      if (value < 0 || value > 1) break;
      c->stream_off = (int)value;
      return PM4G_OK;
    case PM4G_OPT_PART_FBITS:
      if (value < 0 || value > 9) break;
      c->part_fbits = (int)value;
      return PM4G_OK;
    case PM4G_OPT_PART1_ITEMS:
    case PM4G_OPT_PART2_ITEMS:
      if (value != 0 && value != 4 && value != 8) break;
      (option == PM4G_OPT_PART1_ITEMS ? c->part1_items : c->part2_items) = (int)value;
      return PM4G_OK;
    default:
      break;
  }
  set_error("pm4g_ctx_set_option: bad option %d or value %lld", option, (long long)value);
  return PM4G_EINVAL;
}

int pm4g_ctx_timing(pm4g_ctx *c, const char *name, int64_t *launches, double *total_ms) {
  if (!c || !name || !launches || !total_ms) {
    set_error("pm4g_ctx_timing: NULL argument");
    return PM4G_EINVAL;
  }
  cudaSetDevice(c->device);
  PM4G_CK(cudaStreamSynchronize(c->stream));
  for (auto &p : c->pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    auto &t = c->totals[p.name];
    t.first += 1;
    t.second += ms;
    c->free_events.push_back(p.a);
    c->free_events.push_back(p.b);
  }
  c->pending.clear();
  if (strcmp(name, "launches") == 0) {
    *launches = c->launches;
    *total_ms = 0.0;
    return PM4G_OK;
  }
  auto it = c->totals.find(name);
  *launches = it == c->totals.end() ? 0 : it->second.first;
  *total_ms = it == c->totals.end() ? 0.0 : it->second.second;
  return PM4G_OK;
}

int pm4g_ctx_timing_reset(pm4g_ctx *c) {
  if (!c) return PM4G_EINVAL;
  int64_t l;
  double ms;
  pm4g_ctx_timing(c, "", &l, &ms);
  c->totals.clear();
  c->launches = 0;
  return PM4G_OK;
}

int pm4g_load_log(pm4g_ctx *c, const int32_t *case_id, const int32_t *activity, const int64_t *ts_ns,
                  const int32_t *case_attr, int64_t n, int32_t A, uint32_t flags, pm4g_log **out) {
  pm4g::ApiRange nvtx_range("pm4g_load_log");
  if (!c || !out) {
    set_error("pm4g_load_log: ctx or out is NULL");
    return PM4G_EINVAL;
  }
  *out = nullptr;
  if (n < 0 || n > INT32_MAX) {
    set_error("pm4g_load_log: n_events %lld outside [0, 2^31-1]", (long long)n);
    return PM4G_EINVAL;
  }
  if (A < 1 || A > kMaxActivities) {
    set_error("pm4g_load_log: n_activities %d outside [1, %d]", A, kMaxActivities);
    return PM4G_EINVAL;
  }
  if (flags != PM4G_HOST_PTRS && flags != PM4G_DEVICE_PTRS) {
    set_error("pm4g_load_log: flags must be PM4G_HOST_PTRS or PM4G_DEVICE_PTRS");
    return PM4G_EINVAL;
  }
  if (n > 0 && (!case_id || !activity || !ts_ns)) {
    set_error("pm4g_load_log: NULL column");
    return PM4G_EINVAL;
  }
  PM4G_CK(cudaSetDevice(c->device));
  pm4g_log *L = new (std::nothrow) pm4g_log();
  if (!L) return PM4G_ENOMEM;
  L->ctx = c;
  c->live_logs++;
  L->n = n;
  L->A = A;
  L->has_attr = case_attr != nullptr;
  L->act_bits = bits_for((uint64_t)(A - 1));
  int st = PM4G_OK;
  {
    Scratch S(c);
    const int32_t *dcase = case_id, *dact = activity, *dattr = case_attr;
    const int64_t *dts = ts_ns;
    auto fail = [&](int s) {
      st = s;
      return s;
    };
    do {
      if (flags == PM4G_HOST_PTRS && n > 0) {
        int32_t *hc = S.get<int32_t>(n), *ha = S.get<int32_t>(n);
        int64_t *ht = S.get<int64_t>(n);
        int32_t *hat = case_attr ? S.get<int32_t>(n) : nullptr;
        if (!hc || !ha || !ht || (case_attr && !hat)) {
          set_error("pm4g_load_log: out of device memory for input columns");
          fail(PM4G_ENOMEM);
          break;
        }
        KTime t(c, "h2d");
        if (cudaMemcpyAsync(hc, case_id, n * 4, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
            cudaMemcpyAsync(ha, activity, n * 4, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
            cudaMemcpyAsync(ht, ts_ns, n * 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
            (hat && cudaMemcpyAsync(hat, case_attr, n * 4, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)) {
          set_error("pm4g_load_log: host-to-device copy failed: %s", cudaGetErrorString(cudaGetLastError()));
          fail(PM4G_ECUDA);
          break;
        }
        dcase = hc;
        dact = ha;
        dts = ht;
        dattr = hat;
      }
      if (n == 0) {
        L->R = 0;
        L->nb = 0;
        if (fail(alloc_buf(c, L->bucket_off, 1))) break;
        if (cudaMemsetAsync(L->bucket_off.p, 0, 4, c->stream) != cudaSuccess) {
          fail(PM4G_ECUDA);
          break;
        }
        if (fail(run_segment(L, nullptr, L->has_attr))) break;
        break;
      }
      // Case id range (the column reduction of Section 2.1). The buckets are
      // laid out for a guess that should enclose every id: the smallest and
      // largest of kRangeSamples evenly spaced rows, widened by 1/256 of
      // their span on each side (slots outside the ids only stay empty). The
      // bucket histogram checks every id against it on its own read of the
      // column; only when an id falls outside, or when the guess would take
      // the ids for sparse, does the reduction run (and the histogram again).
      int mn = 0, mx = 0;
      {
        int2 smp = make_int2(INT32_MAX, INT32_MIN);
        if (flags == PM4G_HOST_PTRS) {
          for (int k = 0; k < kRangeSamples; ++k) {
            const int32_t v = case_id[(n - 1) * k / (kRangeSamples - 1)];
            smp.x = std::min(smp.x, v);
            smp.y = std::max(smp.y, v);
          }
        } else {
          int2 *d = S.get<int2>(1);
          if (!d) {
            fail(PM4G_ENOMEM);
            break;
          }
          k_sample_range<<<1, 1024, 0, c->stream>>>(dcase, n, d);
          if (fail(check_launch(c, "k_sample_range"))) break;
          if (fail(d2h(c, &smp, d, sizeof(int2)))) break;
        }
        const int64_t pad = ((int64_t)smp.y - (int64_t)smp.x) / 256 + 1;
        mn = (int)std::max<int64_t>(INT32_MIN, (int64_t)smp.x - pad);
        mx = (int)std::min<int64_t>(INT32_MAX, (int64_t)smp.y + pad);
      }
      bool range_exact = false;
      uint32_t *range_err = S.get<uint32_t>(1);
      if (!range_err) {
        fail(PM4G_ENOMEM);
        break;
      }
    case_range:
      if (range_exact) {
        const unsigned gs = (unsigned)c->num_sms * 4;
        int2 *part = S.get<int2>(gs);
        if (!part) {
          fail(PM4G_ENOMEM);
          break;
        }
        {
          KTime t(c, "stats");
          k_stats<<<gs, 256, 0, c->stream>>>(dcase, n, part);
          if (fail(check_launch(c, "k_stats"))) break;
        }
        std::vector<int2> hp(gs);
        if (fail(d2h(c, hp.data(), part, gs * sizeof(int2)))) break;
        mn = INT32_MAX;
        mx = INT32_MIN;
        for (auto &p : hp) {
          mn = std::min(mn, p.x);
          mx = std::max(mx, p.y);
        }
      }
      uint64_t R = (uint64_t)((int64_t)mx - (int64_t)mn + 1);
      const int32_t *keycol = dcase;
      L->min_case = mn;
      const bool sparse = R > std::max<uint64_t>(2 * (uint64_t)n, 1u << 20);
      if (sparse && !range_exact) {  // decided on the exact range only
        range_exact = true;
        goto case_range;
      }
      if (sparse) {
        // sparse case ids: dense renumbering by rank of the distinct ids
        uint32_t *keys = S.get<uint32_t>(n), *vals = S.get<uint32_t>(n);
        uint32_t *k2 = S.get<uint32_t>(n), *v2 = S.get<uint32_t>(n);
        uint32_t *head = S.get<uint32_t>(n), *hpos = S.get<uint32_t>(n + 1);
        int32_t *dense = S.get<int32_t>(n);
        if (!keys || !vals || !k2 || !v2 || !head || !hpos || !dense) {
          set_error("pm4g_load_log: out of device memory for case renumbering");
          fail(PM4G_ENOMEM);
          break;
        }
        const unsigned g = grid_for(n, 256, 8192);
        k_case_keys<<<g, 256, 0, c->stream>>>(dcase, n, keys, vals);
        if (fail(check_launch(c, "k_case_keys"))) break;
        if (fail(radix_sort_u32(c, keys, vals, k2, v2, n, 0, 32))) break;
        k_case_heads<<<g, 256, 0, c->stream>>>(keys, n, head);
        if (fail(check_launch(c, "k_case_heads"))) break;
        if (fail(scan_u32(c, head, hpos, n))) break;
        uint32_t Cu = 0;
        if (fail(d2h(c, &Cu, hpos + n, 4))) break;
        if (fail(alloc_buf(c, L->uniq, Cu))) break;
        k_case_dense<<<g, 256, 0, c->stream>>>(keys, vals, head, hpos, n, dense, L->uniq.p);
        if (fail(check_launch(c, "k_case_dense"))) break;
        keycol = dense;
        L->min_case = 0;
        R = Cu;
      }
      L->R = R;
      L->clb = choose_clb(c, n, R, A, L->act_bits);
      const int ncl = 1 << L->clb;
      const uint64_t nb64 = (R + ncl - 1) >> L->clb;
      if (nb64 > 0xFFFFFFF0ull) {
        set_error("pm4g_load_log: too many buckets");
        fail(PM4G_EINVAL);
        break;
      }
      L->nb = (uint32_t)nb64;
      // bucket histogram, offsets and partition. Row chunks: one per
      // resident first-level partition block (two per SM at 4,096-record
      // tiles, three at 2,048-record ones).
      const int64_t n_chunks = (c->part1_items == 4 ? 3 : 2) * (int64_t)c->num_sms;
      int64_t chunk = (n + n_chunks - 1) / n_chunks;
      chunk = (chunk + 3) / 4 * 4;
      const int p_ctas = (int)((n + chunk - 1) / chunk);
      uint32_t *mat = S.get<uint32_t>((size_t)p_ctas * L->nb);
      uint32_t *total = S.get<uint32_t>(L->nb);
      if (!mat || !total) {
        set_error("pm4g_load_log: out of device memory for the bucket matrix");
        fail(PM4G_ENOMEM);
        break;
      }
      FormatArgs fa{};
      fa.case_id = keycol;
      fa.activity = dact;
      fa.ts = dts;
      fa.n = n;
      fa.chunk = chunk;
      fa.min_case = L->min_case;
      fa.clb = L->clb;
      fa.act_bits = L->act_bits;
      fa.n_act = A;
      fa.nb = L->nb;
      fa.mat = mat;
      fa.slot_hi = range_exact ? 0xFFFFFFFFu : (uint32_t)(R - 1);
      fa.range_err = range_exact ? nullptr : range_err;
      if (!range_exact && cudaMemsetAsync(range_err, 0, 4, c->stream) != cudaSuccess) {
        fail(PM4G_ECUDA);
        break;
      }
      const uint32_t nbs_max = (uint32_t)std::min<int64_t>(((int64_t)c->smem_optin - 1024) / 4, 1 << 20);
      cudaFuncSetAttribute(k_bucket_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin_max());
      cudaFuncSetAttribute(k_bucket_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin_max());
      if (L->nb > nbs_max && L->nb <= 2 * nbs_max - 2) {
        // one pass with 16-bit counters instead of two with 32-bit ones
        cudaFuncSetAttribute(k_bucket_hist16, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin_max());
        KTime t(c, "bucket_hist");
        k_bucket_hist16<<<p_ctas, 1024, ((size_t)(L->nb + 1) / 2 + 1) * 4, c->stream>>>(fa);
        fail(check_launch(c, "k_bucket_hist16"));
      } else {
        for (uint32_t b0 = 0; b0 < L->nb && st == PM4G_OK; b0 += nbs_max) {
          const uint32_t nbs = std::min(nbs_max, L->nb - b0);
          KTime t(c, "bucket_hist");
          k_bucket_hist<<<p_ctas, 1024, nbs * 4, c->stream>>>(fa, b0, nbs);
          fail(check_launch(c, "k_bucket_hist"));
        }
      }
      if (st) break;
      if (!range_exact) {
        uint32_t outside = 0;
        if (fail(d2h(c, &outside, range_err, 4))) break;
        if (outside) {
          range_exact = true;
          goto case_range;
        }
      }
      if (fail(alloc_buf(c, L->bucket_off, (size_t)L->nb + 1))) break;
      if (fail(alloc_buf(c, L->rec, n))) break;
      if (fail(alloc_buf(c, L->status, 1))) break;
      uint32_t *err = L->status.p;
      if (cudaMemsetAsync(err, 0, 4, c->stream) != cudaSuccess) {
        fail(PM4G_ECUDA);
        break;
      }
      fa.bucket_off = L->bucket_off.p;
      fa.rec = L->rec.p;
      fa.err_flags = err;
      // the first word of every record in bucket order, written by the
      // partition's final level (the streaming pass counts cases from it)
      uint32_t *keys = nullptr;
      // Partition levels: one level when the buckets fit the bins of a pass,
      // two when coarse buckets of 2^fbits final buckets do; the record-by-
      // record scatter otherwise.
      int fbits = 0;
      while (fbits < 8 && ((L->nb + (1u << fbits) - 1) >> fbits) > kPartMaxBins) ++fbits;
      // a launch choice may ask for fewer, larger coarse buckets (more final
      // buckets in each), as long as the second level's digits fit a pass
      if (c->part_fbits > fbits && (1u << c->part_fbits) <= kPartMaxBins && L->clb + c->part_fbits <= 16)
        fbits = c->part_fbits;
      const uint32_t nc = (L->nb + (1u << fbits) - 1) >> fbits;
      const bool two_level = fbits > 0 && nc <= kPartMaxBins && L->clb + fbits <= 16;
      uint32_t *mat1 = mat;
      if (two_level) {
        mat1 = S.get<uint32_t>((size_t)p_ctas * nc);
        if (!mat1) {
          fail(PM4G_ENOMEM);
          break;
        }
        KTime t(c, "scan");
        const int64_t k = (int64_t)p_ctas * nc;
        k_coarse_counts<<<(unsigned)((k * 32 + 255) / 256), 256, 0, c->stream>>>(mat, L->nb, p_ctas, fbits, nc, mat1);
        if (fail(check_launch(c, "k_coarse_counts"))) break;
      }
      {
        KTime t(c, "scan");
        k_bucket_colprefix<<<(L->nb + 31) / 32, 256, 0, c->stream>>>(mat, L->nb, p_ctas, total);
        if (fail(check_launch(c, "k_bucket_colprefix"))) break;
      }
      if (fail(scan_u32(c, total, L->bucket_off.p, L->nb))) break;
      L->row_ordered = fbits == 0 || two_level;
      if (fbits == 0 || two_level) {
        PartArgs pa{};
        pa.case_id = keycol;
        pa.activity = dact;
        pa.ts = dts;
        pa.n = n;
        pa.chunk = chunk;
        pa.min_case = L->min_case;
        pa.n_act = A;
        pa.act_bits = L->act_bits;
        pa.clb = L->clb;
        pa.fbits = fbits;
        pa.bucket_off = L->bucket_off.p;
        pa.nb = L->nb;
        pa.err_flags = err;
        keys = S.get<uint32_t>(n);
        pa.keys_out = keys;
        uint4 *tmp = nullptr;
        if (two_level) {
          {
            KTime t(c, "scan");
            const int64_t k = (int64_t)p_ctas * nc;
            k_bucket_colprefix<<<(nc + 31) / 32, 256, 0, c->stream>>>(mat1, nc, p_ctas, total);
            if (fail(check_launch(c, "k_bucket_colprefix"))) break;
            k_add_base<<<(unsigned)((k + 255) / 256), 256, 0, c->stream>>>(mat1, p_ctas, nc, L->bucket_off.p, fbits);
            if (fail(check_launch(c, "k_add_base"))) break;
          }
          tmp = S.get<uint4>(n);
          if (!tmp) {
            set_error("pm4g_load_log: out of device memory for the partition buffer");
            fail(PM4G_ENOMEM);
            break;
          }
          pa.nbins = nc;
          pa.cur1 = mat1;
          pa.rec_out = tmp;
          {
            KTime t(c, "partition");
            c->launches++;
            if (const cudaError_t le = launch_partition(1, pa, (unsigned)p_ctas, c->stream, c->part1_items == 4 ? 4 : 8)) {
              set_error("launch of k_partition<1> failed: %s", cudaGetErrorString(le));
              fail(PM4G_ECUDA);
              break;
            }
          }
          pa.nbins = 1u << fbits;
          pa.rec_in = tmp;
          pa.rec_out = L->rec.p;
          pa.mat = mat;
          pa.p_ctas = p_ctas;
          // split coarse buckets at row-chunk boundaries into about four
          // waves of units, so that no short last wave idles most SMs
          pa.splits = (int)std::max<int64_t>(
              1, std::min<int64_t>(p_ctas, c->load_splits > 0 ? (int64_t)c->load_splits
                                                              : (8 * (int64_t)c->num_sms + nc - 1) / (int64_t)nc));
          {
            KTime t(c, "partition");
            c->launches++;
            if (const cudaError_t le = launch_partition(2, pa, nc * (unsigned)pa.splits, c->stream, c->part2_items == 8 ? 8 : 4)) {
              set_error("launch of k_partition<2> failed: %s", cudaGetErrorString(le));
              fail(PM4G_ECUDA);
              break;
            }
          }
        } else {
          {
            KTime t(c, "scan");
            const int64_t k = (int64_t)p_ctas * L->nb;
            k_add_base<<<(unsigned)((k + 255) / 256), 256, 0, c->stream>>>(mat, p_ctas, L->nb, L->bucket_off.p, 0);
            if (fail(check_launch(c, "k_add_base"))) break;
          }
          pa.nbins = L->nb;
          pa.cur1 = mat;
          pa.rec_out = L->rec.p;
          KTime t(c, "partition");
          c->launches++;
          if (const cudaError_t le = launch_partition(1, pa, (unsigned)p_ctas, c->stream, c->part1_items == 4 ? 4 : 8)) {
            set_error("launch of k_partition<1> failed: %s", cudaGetErrorString(le));
            fail(PM4G_ECUDA);
            break;
          }
        }
      } else {
        // the record scatter may reorder a case's events: no key words are
        // written, so the sorting pass (which checks every case's order)
        // takes the log
        for (uint32_t b0 = 0; b0 < L->nb && st == PM4G_OK; b0 += nbs_max) {
          const uint32_t nbs = std::min(nbs_max, L->nb - b0);
          KTime t(c, "bucket_scatter");
          k_bucket_scatter<<<p_ctas, 1024, nbs * 4, c->stream>>>(fa, b0, nbs);
          fail(check_launch(c, "k_bucket_scatter"));
        }
      }
      if (st) break;
      uint32_t errv = 0;
      if (fail(run_segment(L, dattr, L->has_attr, err, &errv, keys))) break;
      if (errv & 1u) {
        set_error("pm4g_load_log: activity code outside [0, %d)", A);
        fail(PM4G_ERANGE);
        break;
      }
    } while (0);
  }
  if (st != PM4G_OK) {
    release_log(L);
    return st;
  }
  *out = L;
  return PM4G_OK;
}

int pm4g_log_activities(const pm4g_log *L, int32_t *n_activities) {
  if (!L || !n_activities) {
    set_error("pm4g_log_activities: NULL argument");
    return PM4G_EINVAL;
  }
  *n_activities = L->A;
  return PM4G_OK;
}

int pm4g_log_info(const pm4g_log *L, int64_t *n_events, int64_t *n_cases) {
  if (!L) {
    set_error("pm4g_log_info: log is NULL");
    return PM4G_EINVAL;
  }
  if (n_events) *n_events = L->n;
  if (n_cases) *n_cases = L->C;
  return PM4G_OK;
}

int pm4g_log_free(pm4g_log *L) {
  pm4g::ApiRange nvtx_range("pm4g_log_free");
  if (!L) return PM4G_OK;
  cudaSetDevice(L->ctx->device);
  release_log(L);
  return PM4G_OK;
}

// Runs the segment pass in export mode: the formatted log in (case,
// timestamp, row) order into the given device arrays (any may be NULL).
namespace pm4g {
// The formatted activities widened to the export's 32-bit codes (act_s is
// already in formatted order).
__global__ void k_widen_acts(const uint16_t *__restrict__ src, int64_t n, int32_t *__restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}
}  // namespace pm4g

int pm4g::run_export(pm4g_log *L, int32_t *ec, int32_t *ea, int64_t *et, int64_t *er) {
  Ctx *c = L->ctx;
  if (L->n == 0) return PM4G_OK;
  if (ea) {
    k_widen_acts<<<grid_for(L->n, 256, 65535), 256, 0, c->stream>>>(L->act_s.p, L->n, ea);
    PM4G_TRY(check_launch(c, "k_widen_acts"));
  }
  if (!ec && !et && !er) return PM4G_OK;
  Scratch S(c);
  uint32_t *ctr = S.get<uint32_t>(4);
  uint32_t *ovf = S.get<uint32_t>(L->nb);
  unsigned long long *dummy = S.get<unsigned long long>(1);
  if (!ctr || !ovf || !dummy) {
    set_error("export: out of device memory");
    return PM4G_ENOMEM;
  }
  PM4G_CK(cudaMemsetAsync(ctr, 0, 16, c->stream));
  const SegConfig sc = seg_config(c, L->clb, L->A);
  SegArgs a = seg_args(L, sc, ctr, ovf, ctr + 1, dummy);
  a.act_s = nullptr;  // widened from act_s above
  a.ex_case = ec;
  a.ex_ts = et;
  a.ex_row = er;
  uint32_t n_ovf = 0;
  if (sc.cap >= 32) {
    KTime t(c, "export");
    c->launches++;
    PM4G_CK(launch_segment(true, a, std::min<unsigned>(L->nb, (unsigned)c->num_sms), sc.smem, c->stream));
    PM4G_TRY(d2h(c, &n_ovf, ctr + 1, 4));
  } else {
    n_ovf = L->nb;
  }
  std::vector<uint32_t> list(n_ovf);
  if (sc.cap >= 32) {
    PM4G_TRY(d2h(c, list.data(), ovf, n_ovf * 4));
  } else {
    for (uint32_t b = 0; b < n_ovf; ++b) list[b] = b;
  }
  for (uint32_t b : list) PM4G_TRY(fallback_bucket(L, a, b, true));
  return PM4G_OK;
}

int pm4g_log_export(pm4g_log *L, int32_t *case_out, int32_t *act_out, int64_t *ts_out, int64_t *row_out) {
  pm4g::ApiRange nvtx_range("pm4g_log_export");
  if (!L) {
    set_error("pm4g_log_export: log is NULL");
    return PM4G_EINVAL;
  }
  Ctx *c = L->ctx;
  PM4G_CK(cudaSetDevice(c->device));
  if (L->n == 0) return PM4G_OK;
  Scratch S(c);
  int32_t *ec = S.get<int32_t>(L->n), *ea = S.get<int32_t>(L->n);
  int64_t *et = S.get<int64_t>(L->n), *er = S.get<int64_t>(L->n);
  if (!ec || !ea || !et || !er) {
    set_error("pm4g_log_export: out of device memory");
    return PM4G_ENOMEM;
  }
  PM4G_TRY(run_export(L, ec, ea, et, er));
  if (case_out) PM4G_CK(cudaMemcpyAsync(case_out, ec, L->n * 4, cudaMemcpyDeviceToHost, c->stream));
  if (act_out) PM4G_CK(cudaMemcpyAsync(act_out, ea, L->n * 4, cudaMemcpyDeviceToHost, c->stream));
  if (ts_out) PM4G_CK(cudaMemcpyAsync(ts_out, et, L->n * 8, cudaMemcpyDeviceToHost, c->stream));
  if (row_out) PM4G_CK(cudaMemcpyAsync(row_out, er, L->n * 8, cudaMemcpyDeviceToHost, c->stream));
  PM4G_CK(cudaStreamSynchronize(c->stream));
  return PM4G_OK;
}

// Case offsets: exclusive prefix of the per-slot lengths (R + 1 entries).
int pm4g::ensure_offsets(pm4g_log *L) {
  if (L->off_ready) return PM4G_OK;
  if (!L->off.p) PM4G_TRY(alloc_buf(L->ctx, L->off, L->R + 1));
  PM4G_TRY(scan_u32(L->ctx, L->len.p, L->off.p, (int64_t)L->R));
  L->off_ready = true;
  return PM4G_OK;
}

// ---------------------------------------------------------------------------
// DFG / endpoints
// ---------------------------------------------------------------------------
int pm4g::hashed_edges(pm4g_log *L, Scratch &S, uint32_t *&keys, uint32_t *&slots, uint32_t &E) {
  Ctx *c = L->ctx;
  const uint64_t T = L->gcells;
  uint32_t *flags = S.get<uint32_t>(T), *pos = S.get<uint32_t>(T + 1);
  if (!flags || !pos) {
    set_error("dfg: out of device memory");
    return PM4G_ENOMEM;
  }
  const unsigned gT = grid_for((int64_t)T, 256, 65535);
  {
    KTime t(c, "dfg");
    k_gkey_flags<<<gT, 256, 0, c->stream>>>(L->gkey.p, T, flags);
    PM4G_TRY(check_launch(c, "k_gkey_flags"));
  }
  PM4G_TRY(scan_u32(c, flags, pos, (int64_t)T));
  E = 0;
  PM4G_TRY(d2h(c, &E, pos + T, 4));
  keys = S.get<uint32_t>(E);
  slots = S.get<uint32_t>(E);
  uint32_t *k2 = S.get<uint32_t>(E), *v2 = S.get<uint32_t>(E);
  if (!keys || !slots || !k2 || !v2) {
    set_error("dfg: out of device memory");
    return PM4G_ENOMEM;
  }
  {
    KTime t(c, "dfg");
    k_gkey_compact<<<gT, 256, 0, c->stream>>>(L->gkey.p, T, flags, pos, keys, slots);
    PM4G_TRY(check_launch(c, "k_gkey_compact"));
  }
  const int kb = std::max(1, bits_for((uint64_t)L->A * (uint64_t)L->A - 1));
  if (E > 1) PM4G_TRY(radix_sort_u32(c, keys, slots, k2, v2, E, 0, kb));
  return PM4G_OK;
}

static int ensure_edges(pm4g_log *L) {
  if (L->edges_ready) return PM4G_OK;
  Ctx *c = L->ctx;
  const int64_t cells = (int64_t)L->gcells;
  const uint32_t A = (uint32_t)L->A;
  Scratch S(c);
  unsigned long long *freq = S.get<unsigned long long>(A);
  if (!freq) {
    set_error("dfg: out of device memory");
    return PM4G_ENOMEM;
  }
  DfgTable t{L->dfg.p, L->dfg.p + cells, L->dfg.p + 2 * cells, L->dfg.p + 3 * cells, L->dfg.p + 4 * cells};
  uint32_t E = 0;
  int32_t *src = nullptr, *dst = nullptr;
  unsigned long long *o[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  double *mean = nullptr;
  auto alloc_out = [&]() {
    src = S.get<int32_t>(E);
    dst = S.get<int32_t>(E);
    for (auto &p : o) p = S.get<unsigned long long>(E);
    mean = S.get<double>(E);
    return src && dst && o[0] && o[1] && o[2] && o[3] && o[4] && mean;
  };
  if (L->ghash) {
    // the occupied slots in (src, dst) order; frequencies from the edges
    uint32_t *keys = nullptr, *slots = nullptr;
    PM4G_TRY(hashed_edges(L, S, keys, slots, E));
    if (!alloc_out()) return PM4G_ENOMEM;
    KTime tk(c, "dfg");
    PM4G_CK(cudaMemsetAsync(freq, 0, (size_t)A * sizeof(unsigned long long), c->stream));
    if (E) {
      k_dfg_gather<<<grid_for(E, 256, 4096), 256, 0, c->stream>>>(t, keys, slots, E, A, src, dst, o[0], o[1], o[2],
                                                                   o[3], o[4], mean);
      PM4G_TRY(check_launch(c, "k_dfg_gather"));
      k_freq_edges<<<grid_for(E, 256, 4096), 256, 0, c->stream>>>(src, o[0], E, freq);
      PM4G_TRY(check_launch(c, "k_freq_edges"));
    }
    k_freq_end<<<grid_for(A, 256, 4096), 256, 0, c->stream>>>(L->ends.p + A, A, freq);
    PM4G_TRY(check_launch(c, "k_freq_end"));
  } else {
    uint32_t *flags = S.get<uint32_t>(cells), *pos = S.get<uint32_t>(cells + 1);
    if (!flags || !pos) {
      set_error("dfg: out of device memory");
      return PM4G_ENOMEM;
    }
    {
      KTime tk(c, "dfg");
      k_dfg_flags<<<grid_for(cells, 256, 4096), 256, 0, c->stream>>>(L->dfg.p, cells, flags);
      PM4G_TRY(check_launch(c, "k_dfg_flags"));
    }
    PM4G_TRY(scan_u32(c, flags, pos, cells));
    // the compacted edges, frequencies and endpoint counts written straight
    // to mapped host memory (room for every cell): one wait for the query
    const size_t need = (size_t)cells * 56 + (size_t)A * 24 + 16;
    char *md = nullptr;
    char *mh = mapped_buf(c, need, &md);
    if (mh) {
      int32_t *msrc = (int32_t *)md, *mdst = msrc + cells;
      unsigned long long *mo = (unsigned long long *)(mdst + cells);
      double *mmean = (double *)(mo + 5 * cells);
      unsigned long long *mfreq = (unsigned long long *)(mmean + cells), *mends = mfreq + A;
      {
        KTime tk(c, "dfg");
        k_dfg_compact<<<grid_for(cells, 256, 4096), 256, 0, c->stream>>>(t, cells, A, flags, pos, msrc, mdst, mo,
                                                                         mo + cells, mo + 2 * cells, mo + 3 * cells,
                                                                         mo + 4 * cells, mmean);
        PM4G_TRY(check_launch(c, "k_dfg_compact"));
        k_freq<<<A, 256, 0, c->stream>>>(t.cnt, L->ends.p + A, A, mfreq);
        PM4G_TRY(check_launch(c, "k_freq"));
      }
      char *hends = mh + ((char *)mends - md);
      uint32_t *hE = (uint32_t *)(hends + (size_t)A * 16);
      PM4G_CK(cudaMemcpyAsync(hends, L->ends.p, (size_t)A * 16, cudaMemcpyDeviceToHost, c->stream));
      PM4G_CK(cudaMemcpyAsync(hE, pos + cells, 4, cudaMemcpyDeviceToHost, c->stream));
      PM4G_CK(cudaStreamSynchronize(c->stream));
      E = *hE;
      const int32_t *hsrc = (const int32_t *)mh, *hdst = hsrc + cells;
      const unsigned long long *ho = (const unsigned long long *)(hdst + cells);
      const double *hmean = (const double *)(ho + 5 * cells);
      const unsigned long long *hfreq = (const unsigned long long *)(hmean + cells), *he = hfreq + A;
      L->e_src.assign(hsrc, hsrc + E);
      L->e_dst.assign(hdst, hdst + E);
      L->e_cnt.assign(ho, ho + E);
      L->e_lo.assign(ho + cells, ho + cells + E);
      L->e_hi.assign(ho + 2 * cells, ho + 2 * cells + E);
      L->e_min.assign(ho + 3 * cells, ho + 3 * cells + E);
      L->e_max.assign(ho + 4 * cells, ho + 4 * cells + E);
      L->e_mean.assign(hmean, hmean + E);
      L->h_start.assign(he, he + A);
      L->h_end.assign(he + A, he + 2 * A);
      L->h_freq.assign(hfreq, hfreq + A);
      L->edges_ready = true;
      return PM4G_OK;
    }
    PM4G_TRY(d2h(c, &E, pos + cells, 4));
    if (!alloc_out()) return PM4G_ENOMEM;
    KTime tk(c, "dfg");
    k_dfg_compact<<<grid_for(cells, 256, 4096), 256, 0, c->stream>>>(t, cells, A, flags, pos, src, dst, o[0], o[1],
                                                                     o[2], o[3], o[4], mean);
    PM4G_TRY(check_launch(c, "k_dfg_compact"));
    k_freq<<<A, 256, 0, c->stream>>>(t.cnt, L->ends.p + A, A, freq);
    PM4G_TRY(check_launch(c, "k_freq"));
  }
  L->e_src.resize(E);
  L->e_dst.resize(E);
  L->e_cnt.resize(E);
  L->e_lo.resize(E);
  L->e_hi.resize(E);
  L->e_min.resize(E);
  L->e_max.resize(E);
  L->e_mean.resize(E);
  L->h_start.resize(A);
  L->h_end.resize(A);
  L->h_freq.resize(A);
  D2HBatch hb(c, (size_t)E * 56 + (size_t)A * 24 + 11 * 16);
  hb.add(L->e_src.data(), src, E * 4);
  hb.add(L->e_dst.data(), dst, E * 4);
  hb.add(L->e_cnt.data(), o[0], E * 8);
  hb.add(L->e_lo.data(), o[1], E * 8);
  hb.add(L->e_hi.data(), o[2], E * 8);
  hb.add(L->e_min.data(), o[3], E * 8);
  hb.add(L->e_max.data(), o[4], E * 8);
  hb.add(L->e_mean.data(), mean, E * 8);
  hb.add(L->h_start.data(), L->ends.p, A * 8);
  hb.add(L->h_end.data(), L->ends.p + A, A * 8);
  hb.add(L->h_freq.data(), freq, A * 8);
  PM4G_TRY(hb.finish());
  L->edges_ready = true;
  return PM4G_OK;
}

template <class T>
static T *host_copy(const std::vector<T> &v) {
  T *p = (T *)malloc(std::max<size_t>(v.size(), 1) * sizeof(T));
  if (p && !v.empty()) memcpy(p, v.data(), v.size() * sizeof(T));
  return p;
}

int pm4g_dfg(pm4g_log *L, pm4g_dfg_t *out) {
  pm4g::ApiRange nvtx_range("pm4g_dfg");
  if (!L || !out) {
    set_error("pm4g_dfg: NULL argument");
    return PM4G_EINVAL;
  }
  memset(out, 0, sizeof(*out));
  PM4G_CK(cudaSetDevice(L->ctx->device));
  PM4G_TRY(ensure_edges(L));
  out->n_edges = (int64_t)L->e_src.size();
  out->src = host_copy(L->e_src);
  out->dst = host_copy(L->e_dst);
  out->count = host_copy(L->e_cnt);
  if (!out->src || !out->dst || !out->count) {
    pm4g_dfg_free(out);
    return PM4G_ENOMEM;
  }
  return PM4G_OK;
}

int pm4g_dfg_free(pm4g_dfg_t *r) {
  if (!r) return PM4G_OK;
  free(r->src);
  free(r->dst);
  free(r->count);
  memset(r, 0, sizeof(*r));
  return PM4G_OK;
}

int pm4g_perf_dfg(pm4g_log *L, pm4g_perf_dfg_t *out) {
  pm4g::ApiRange nvtx_range("pm4g_perf_dfg");
  if (!L || !out) {
    set_error("pm4g_perf_dfg: NULL argument");
    return PM4G_EINVAL;
  }
  memset(out, 0, sizeof(*out));
  PM4G_CK(cudaSetDevice(L->ctx->device));
  PM4G_TRY(ensure_edges(L));
  const size_t E = L->e_src.size();
  out->n_edges = (int64_t)E;
  out->src = host_copy(L->e_src);
  out->dst = host_copy(L->e_dst);
  out->count = host_copy(L->e_cnt);
  out->sum_lo = host_copy(L->e_lo);
  out->sum_hi = host_copy(L->e_hi);
  out->min = host_copy(L->e_min);
  out->max = host_copy(L->e_max);
  out->mean = host_copy(L->e_mean);  // formed on the device from the exact sums
  if (!out->src || !out->dst || !out->count || !out->sum_lo || !out->sum_hi || !out->min || !out->max || !out->mean) {
    pm4g_perf_dfg_free(out);
    return PM4G_ENOMEM;
  }
  return PM4G_OK;
}

int pm4g_perf_dfg_free(pm4g_perf_dfg_t *r) {
  if (!r) return PM4G_OK;
  free(r->src);
  free(r->dst);
  free(r->count);
  free(r->sum_lo);
  free(r->sum_hi);
  free(r->min);
  free(r->max);
  free(r->mean);
  memset(r, 0, sizeof(*r));
  return PM4G_OK;
}

int pm4g_start_end(pm4g_log *L, uint64_t *start, uint64_t *end, uint64_t *freq) {
  pm4g::ApiRange nvtx_range("pm4g_start_end");
  if (!L || !start || !end) {
    set_error("pm4g_start_end: NULL argument");
    return PM4G_EINVAL;
  }
  PM4G_CK(cudaSetDevice(L->ctx->device));
  PM4G_TRY(ensure_edges(L));
  memcpy(start, L->h_start.data(), L->A * 8);
  memcpy(end, L->h_end.data(), L->A * 8);
  if (freq) memcpy(freq, L->h_freq.data(), L->A * 8);
  return PM4G_OK;
}

// ---------------------------------------------------------------------------
// variants
// ---------------------------------------------------------------------------
static uint64_t next_pow2(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

int pm4g::group_variants(Ctx *c, VarArgs a, uint64_t n_items, uint32_t *rep_pos, uint32_t *n_reps) {
  const uint64_t R = a.n_slots;
  Scratch S(c);
  // table of about 1.5 slots per item (load at most 2/3), a power of two
  const uint64_t T = next_pow2(std::max<uint64_t>(n_items + n_items / 2, 1024));
  VarSlot *tab = S.get<VarSlot>(T);
  uint32_t *grp = S.get<uint32_t>(R);
  uint8_t *isbad = S.get<uint8_t>(R);
  uint32_t *listA = S.get<uint32_t>(n_items), *listB = S.get<uint32_t>(n_items);
  uint32_t *n_bad = S.get<uint32_t>(1);
  if (!tab || !grp || !isbad || !listA || !listB || !n_bad) {
    set_error("variants: out of device memory");
    return PM4G_ENOMEM;
  }
  a.tab = tab;
  a.grp = grp;
  a.isbad = isbad;
  const uint32_t *list = nullptr;
  uint32_t n_list = 0;
  uint32_t *out_list = listA;
  for (uint32_t round = 0;; ++round) {
    const uint64_t items = list ? n_list : R;
    const uint64_t ni = list ? n_list : n_items;
    const uint64_t Tr = next_pow2(std::max<uint64_t>(ni + ni / 2, 1024));
    a.tmask = (uint32_t)(Tr - 1);
    PM4G_CK(cudaMemsetAsync(tab, 0, Tr * sizeof(VarSlot), c->stream));
    PM4G_CK(cudaMemsetAsync(n_bad, 0, 4, c->stream));
    const unsigned g = grid_for((int64_t)items, 256, 65535);
    {
      KTime t(c, "variants");
      if (round == 0 && !a.hash && !list) {
        k_var_hash_insert<<<grid_for((int64_t)((R + 31) / 32) * 32, kHiThreads, 16 * (unsigned)c->num_sms),
                            kHiThreads, 0, c->stream>>>(a);
        PM4G_TRY(check_launch(c, "k_var_hash_insert"));
      } else {
        k_var_insert<<<g, 256, 0, c->stream>>>(a, list, n_list, round);
        PM4G_TRY(check_launch(c, "k_var_insert"));
      }
      k_var_verify<<<g, 256, 0, c->stream>>>(a, list, n_list, out_list, n_bad);
      PM4G_TRY(check_launch(c, "k_var_verify"));
      k_var_final<<<g, 256, 0, c->stream>>>(a, list, n_list);
      PM4G_TRY(check_launch(c, "k_var_final"));
    }
    uint32_t nb = 0;
    if (rep_pos) {
      // the representatives' positions, read back with the round's count of
      // differing cases (one wait; the scan is repeated if a round follows)
      PM4G_TRY(scan_u32(c, a.rep_flag, rep_pos, (int64_t)R));
      uint32_t *dst[2] = {&nb, n_reps};
      const uint32_t *src[2] = {n_bad, rep_pos + R};
      PM4G_TRY(d2h_words(c, dst, src, 2));
    } else {
      PM4G_TRY(d2h(c, &nb, n_bad, 4));
    }
    c->totals["variant_regrouped"].first += nb;  // cases whose sequence differed from their group's
    if (nb == 0) break;
    if (round > 1000000) {
      set_error("variants: collision rounds did not converge");
      return PM4G_ETIMEOUT;
    }
    list = out_list;
    n_list = nb;
    out_list = (out_list == listA) ? listB : listA;
  }
  return PM4G_OK;
}

static int ensure_variants(pm4g_log *L) {
  if (L->var_ready) return PM4G_OK;
  Ctx *c = L->ctx;
  const uint64_t R = L->R;
  PM4G_TRY(ensure_offsets(L));
  PM4G_TRY(alloc_buf(c, L->vcount, R));
  PM4G_TRY(alloc_buf(c, L->rep_of, R));
  if (L->C == 0) {
    L->V = 0;
    PM4G_TRY(alloc_buf(c, L->rep_slots, 0));
    PM4G_TRY(alloc_buf(c, L->order, 0));
    L->var_ready = true;
    return PM4G_OK;
  }
  Scratch S(c);
  VarArgs a{};
  a.n_slots = R;
  a.len = L->len.p;
  a.hash = nullptr;  // formed from the formatted activities in the first round
  {
    unsigned long long *gtab = S.get<unsigned long long>((size_t)std::max<int64_t>(L->A, 1));
    if (!gtab) return PM4G_ENOMEM;
    KTime t(c, "variants");
    k_var_gtab<<<grid_for(L->A, 256, 256), 256, 0, c->stream>>>(gtab, (uint32_t)L->A);
    PM4G_TRY(check_launch(c, "k_var_gtab"));
    a.gtab = gtab;
  }
  a.off = L->off.p;
  a.act_s = L->act_s.p;
  a.n_events = L->n;
  a.bits = c->test_hash_bits;
  a.rep_of = L->rep_of.p;
  a.vcount = L->vcount.p;
  uint32_t *flags = S.get<uint32_t>(R);  // representative flags, set by the grouping rounds
  if (!flags) return PM4G_ENOMEM;
  a.rep_flag = flags;
  // representatives in slot order (their positions and count come with the
  // grouping's last round), then ranked by (count desc, smallest case asc)
  PM4G_TRY(alloc_buf(c, L->rep_pos, R + 1));
  uint32_t *pos = L->rep_pos.p;
  uint32_t V = 0;
  PM4G_TRY(group_variants(c, a, (uint64_t)L->C, pos, &V));
  const unsigned gR = grid_for((int64_t)R, 256, 65535);
  L->V = V;
  PM4G_TRY(alloc_buf(c, L->rep_slots, V));
  PM4G_TRY(alloc_buf(c, L->order, V));
  uint32_t *keys = S.get<uint32_t>(V), *k2 = S.get<uint32_t>(V), *v2 = S.get<uint32_t>(V);
  if (!keys || !k2 || !v2) return PM4G_ENOMEM;
  const int cbits = bits_for((uint64_t)L->C);
  const uint32_t cmask = cbits >= 32 ? 0xFFFFFFFFu : ((1u << cbits) - 1);
  {
    KTime t(c, "variants");
    k_rep_compact<<<gR, 256, 0, c->stream>>>(a, flags, pos, cmask, L->rep_slots.p, keys, L->order.p);
    PM4G_TRY(check_launch(c, "k_rep_compact"));
  }
  PM4G_TRY(radix_sort_u32(c, keys, L->order.p, k2, v2, V, 0, cbits));
  // (no synchronisation: the callers' work follows on the same stream, and
  // their own result copies report any failure)
  L->var_ready = true;
  return PM4G_OK;
}

// The variant rank of every case slot (for PM4G_VARIANTS_CASES), from the
// ranking and the representatives' positions.
static int ensure_case_variants(pm4g_log *L) {
  if (L->cvar.p || L->R == 0) return PM4G_OK;
  Ctx *c = L->ctx;
  const uint64_t R = L->R;
  const uint32_t V = L->V;
  // the scratch first: cvar, once allocated, marks the ranks as formed
  Scratch S(c);
  uint32_t *rank_of = L->C ? S.get<uint32_t>(V) : nullptr;
  if (L->C && !rank_of) return PM4G_ENOMEM;
  PM4G_TRY(alloc_buf(c, L->cvar, R));
  if (L->C == 0) return PM4G_OK;  // no case reads it
  VarArgs a{};
  a.n_slots = R;
  a.len = L->len.p;
  a.rep_of = L->rep_of.p;
  KTime t(c, "variants");
  k_rank_scatter<<<grid_for(V, 256, 65535), 256, 0, c->stream>>>(L->order.p, V, rank_of);
  int st = check_launch(c, "k_rank_scatter");
  if (st == PM4G_OK) {
    k_case_variant<<<grid_for((int64_t)R, 256, 65535), 256, 0, c->stream>>>(a, L->rep_pos.p, rank_of, L->cvar.p);
    st = check_launch(c, "k_case_variant");
  }
  if (st != PM4G_OK) free_buf(c, L->cvar);  // unfilled: the next request forms it again
  return st;
}

int pm4g_variants(pm4g_log *L, int64_t top_k, uint32_t flags, pm4g_variants_t *out) {
  pm4g::ApiRange nvtx_range("pm4g_variants");
  if (!L || !out) {
    set_error("pm4g_variants: NULL argument");
    return PM4G_EINVAL;
  }
  memset(out, 0, sizeof(*out));
  if (flags & ~PM4G_VARIANTS_CASES) {
    set_error("pm4g_variants: unknown flags");
    return PM4G_EINVAL;
  }
  Ctx *c = L->ctx;
  PM4G_CK(cudaSetDevice(c->device));
  PM4G_TRY(ensure_variants(L));
  const uint32_t V = L->V;
  const uint32_t k = top_k < 0 ? V : (uint32_t)std::min<int64_t>(top_k, V);
  out->n_variants = V;
  out->n_out = k;
  Scratch S(c);
  unsigned long long *oc = S.get<unsigned long long>(k);
  int32_t *om = S.get<int32_t>(k);
  uint32_t *ol = S.get<uint32_t>(k), *oo = S.get<uint32_t>(k + 1);
  if (!oc || !om || !ol || !oo) return PM4G_ENOMEM;
  VarArgs a{};
  a.n_slots = L->R;
  a.len = L->len.p;
  a.off = L->off.p;
  a.act_s = L->act_s.p;
  a.vcount = L->vcount.p;
  a.rep_of = L->rep_of.p;
  uint32_t total = 0;
  if (k > 0) {
    KTime t(c, "variants");
    k_var_out_head<<<grid_for(k, 256, 65535), 256, 0, c->stream>>>(a, L->order.p, L->rep_slots.p, k, L->min_case,
                                                                    L->uniq.p, oc, om, ol);
    PM4G_TRY(check_launch(c, "k_var_out_head"));
  }
  PM4G_TRY(scan_u32(c, ol, oo, k));
  // the sequences go straight to mapped host memory, with room for 64
  // activities a variant (at least 64k in all); longer top lists take a
  // second pass sized from the offsets
  const uint64_t cap = std::max<uint64_t>(65536, (uint64_t)k * 64);
  char *md = nullptr;
  char *mh = mapped_buf(c, (size_t)cap * 4, &md);
  if (mh && k > 0) {
    KTime t(c, "variants");
    k_var_out_acts<<<grid_for((int64_t)k * 32, 256, 65535), 256, 0, c->stream>>>(a, L->order.p, L->rep_slots.p, k, oo,
                                                                    (int32_t *)md, cap);
    PM4G_TRY(check_launch(c, "k_var_out_acts"));
  }
  out->count = (uint64_t *)malloc(std::max<size_t>(k, 1) * 8);
  out->min_case = (int32_t *)malloc(std::max<size_t>(k, 1) * 4);
  out->off = (int64_t *)malloc(((size_t)k + 1) * 8);
  std::vector<uint32_t> hoff((size_t)k + 1);
  if (!out->count || !out->min_case || !out->off) {
    pm4g_variants_free(out);
    return PM4G_ENOMEM;
  }
  cudaStream_t s = c->stream;
  const bool want_cases = (flags & PM4G_VARIANTS_CASES) != 0;
  {
    D2HBatch hb(c, (size_t)k * 16 + 4 + (want_cases ? (size_t)L->C * 8 : 0) + 6 * 16);
    hb.add(out->count, oc, (size_t)k * 8);
    hb.add(out->min_case, om, (size_t)k * 4);
    hb.add(hoff.data(), oo, ((size_t)k + 1) * 4);
    if (want_cases) {
      if (const int st = ensure_case_variants(L)) {
        pm4g_variants_free(out);
        return st;
      }
      const uint64_t R = L->R;
      uint32_t *pf = S.get<uint32_t>(R), *pp = S.get<uint32_t>(R + 1);
      int32_t *cid = S.get<int32_t>(L->C), *cv = S.get<int32_t>(L->C);
      if (!pf || !pp || !cid || !cv) {
        pm4g_variants_free(out);
        return PM4G_ENOMEM;
      }
      const unsigned gR = grid_for((int64_t)R, 256, 65535);
      k_present_flags<<<gR, 256, 0, s>>>(L->len.p, R, pf);
      int st = check_launch(c, "k_present_flags");
      if (!st) st = scan_u32(c, pf, pp, (int64_t)R);
      if (!st) {
        k_cases_out<<<gR, 256, 0, s>>>(L->len.p, R, pp, L->cvar.p, L->min_case, L->uniq.p, cid, cv);
        st = check_launch(c, "k_cases_out");
      }
      if (st) {
        pm4g_variants_free(out);
        return st;
      }
      out->n_cases = L->C;
      out->case_ids = (int32_t *)malloc(std::max<size_t>(L->C, 1) * 4);
      out->case_variant = (int32_t *)malloc(std::max<size_t>(L->C, 1) * 4);
      if (!out->case_ids || !out->case_variant) {
        pm4g_variants_free(out);
        return PM4G_ENOMEM;
      }
      hb.add(out->case_ids, cid, L->C * 4);
      hb.add(out->case_variant, cv, L->C * 4);
    }
    const int st = hb.finish();  // waits for the mapped sequences too
    if (st != PM4G_OK) {
      pm4g_variants_free(out);
      return st;
    }
  }
  total = hoff[k];
  out->acts = (int32_t *)malloc(std::max<size_t>(total, 1) * 4);
  if (!out->acts) {
    pm4g_variants_free(out);
    return PM4G_ENOMEM;
  }
  if (mh && total <= cap) {
    if (total) memcpy(out->acts, mh, (size_t)total * 4);
  } else if (total > 0) {
    int32_t *oa = S.get<int32_t>(total);
    if (!oa) {
      pm4g_variants_free(out);
      return PM4G_ENOMEM;
    }
    {
      KTime t(c, "variants");
      k_var_out_acts<<<grid_for((int64_t)k * 32, 256, 65535), 256, 0, c->stream>>>(a, L->order.p, L->rep_slots.p, k, oo, oa,
                                                                      ~0ull);
    }
    if (const int st = check_launch(c, "k_var_out_acts")) {
      pm4g_variants_free(out);
      return st;
    }
    D2HBatch hb(c, (size_t)total * 4 + 16);
    hb.add(out->acts, oa, (size_t)total * 4);
    const int st = hb.finish();
    if (st != PM4G_OK) {
      pm4g_variants_free(out);
      return st;
    }
  }
  for (size_t i = 0; i <= k; ++i) out->off[i] = hoff[i];
  return PM4G_OK;
}

int pm4g_variants_free(pm4g_variants_t *r) {
  if (!r) return PM4G_OK;
  free(r->count);
  free(r->min_case);
  free(r->off);
  free(r->acts);
  free(r->case_ids);
  free(r->case_variant);
  memset(r, 0, sizeof(*r));
  return PM4G_OK;
}

// ---------------------------------------------------------------------------
// filter
// ---------------------------------------------------------------------------
// First and last timestamp of every case slot (cached on the log).
static int ensure_span(pm4g_log *L) {
  if (L->span_ready) return PM4G_OK;
  Ctx *c = L->ctx;
  const uint64_t R = L->R;
  PM4G_TRY(alloc_buf(c, L->span, 2 * R));
  FilterArgs fa{};
  fa.rec = L->rec.p;
  fa.bucket_off = L->bucket_off.p;
  fa.nb = L->nb;
  fa.clb = L->clb;
  fa.act_bits = L->act_bits;
  fa.n_slots = R;
  fa.first_ts = L->span.p;
  fa.last_ts = L->span.p + R;
  KTime t(c, "filter");
  const int ncl = 1 << L->clb;
  k_case_span<<<std::min<unsigned>(L->nb, 4u * c->num_sms), 256, (size_t)ncl * 16, c->stream>>>(fa);
  PM4G_TRY(check_launch(c, "k_case_span"));
  L->span_ready = true;
  return PM4G_OK;
}

// A new log holding the records of L that the predicate of `fa` keeps (case_ok
// per slot with the window, or row_keep per original row), formatted by the
// segment pass. `fa`'s device arrays must stay valid until this returns.
static int extract_sublog(pm4g_log *L, FilterArgs fa, pm4g_log **out) {
  Ctx *c = L->ctx;
  pm4g_log *F = new (std::nothrow) pm4g_log();
  if (!F) return PM4G_ENOMEM;
  F->ctx = c;
  c->live_logs++;
  F->A = L->A;
  F->min_case = L->min_case;
  F->R = L->R;
  F->clb = L->clb;
  F->act_bits = L->act_bits;
  F->nb = L->nb;
  F->has_attr = L->has_attr;
  int st = PM4G_OK;
  do {
    const uint64_t R = L->R;
    if ((st = alloc_buf(c, F->bucket_off, (size_t)L->nb + 1))) break;
    if (L->has_attr) {
      if ((st = alloc_buf(c, F->cattr, R))) break;
      if (R && cudaMemcpyAsync(F->cattr.p, L->cattr.p, R * 4, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess) {
        st = PM4G_ECUDA;
        break;
      }
    }
    if (L->uniq.p) {
      if ((st = alloc_buf(c, F->uniq, L->uniq.n))) break;
      if (cudaMemcpyAsync(F->uniq.p, L->uniq.p, L->uniq.n * 4, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess) {
        st = PM4G_ECUDA;
        break;
      }
    }
    if (L->n == 0 || L->nb == 0) {
      F->n = 0;
      if (cudaMemsetAsync(F->bucket_off.p, 0, 4 * ((size_t)L->nb + 1), c->stream) != cudaSuccess) {
        st = PM4G_ECUDA;
        break;
      }
      st = run_segment(F, nullptr, false);
      break;
    }
    Scratch S(c);
    uint32_t *kept = S.get<uint32_t>(L->nb);
    if (!kept) {
      st = PM4G_ENOMEM;
      break;
    }
    fa.rec = L->rec.p;
    fa.bucket_off = L->bucket_off.p;
    fa.nb = L->nb;
    fa.clb = L->clb;
    fa.act_bits = L->act_bits;
    fa.n_slots = R;
    fa.kept = kept;
    fa.new_off = F->bucket_off.p;
    const unsigned gb = std::min<unsigned>(L->nb, 8u * c->num_sms);
    {
      KTime t(c, "filter");
      k_filter_count<<<gb, 256, 0, c->stream>>>(fa);
      if ((st = check_launch(c, "k_filter_count"))) break;
    }
    if ((st = scan_u32(c, kept, F->bucket_off.p, L->nb))) break;
    uint32_t nsub = 0;
    if ((st = d2h(c, &nsub, F->bucket_off.p + L->nb, 4))) break;
    F->n = nsub;
    if ((st = alloc_buf(c, F->rec, nsub))) break;
    fa.out = F->rec.p;
    // A sub-log keeps each bucket's records in the order of the log it comes
    // from, so its cases are in timestamp order when that log's are: it then
    // takes the streaming segment pass, which counts cases from the key words.
    uint32_t *keys = nullptr;
    F->row_ordered = L->row_ordered;
    if (L->status.p) {
      if ((st = alloc_buf(c, F->status, 1))) break;
      if (cudaMemcpyAsync(F->status.p, L->status.p, 4, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess) {
        st = PM4G_ECUDA;
        break;
      }
      if (F->row_ordered) keys = S.get<uint32_t>(nsub);  // NULL (no streaming pass) if memory is short
    }
    fa.keys_out = keys;
    {
      KTime t(c, "filter");
      k_filter_write<<<gb, 256, 0, c->stream>>>(fa);
      if ((st = check_launch(c, "k_filter_write"))) break;
    }
    st = run_segment(F, nullptr, false, nullptr, nullptr, keys);
  } while (0);
  if (st != PM4G_OK) {
    if (st == PM4G_ENOMEM) set_error("filter: out of device memory");
    release_log(F);
    return st;
  }
  *out = F;
  return PM4G_OK;
}

int pm4g_filter(pm4g_log *L, const pm4g_filter_spec *spec, pm4g_log **out) {
  pm4g::ApiRange nvtx_range("pm4g_filter");
  if (!L || !spec || !out) {
    set_error("pm4g_filter: NULL argument");
    return PM4G_EINVAL;
  }
  *out = nullptr;
  if (spec->mode < PM4G_TW_NONE || spec->mode > PM4G_TW_CASES_INTERSECTING || spec->n_attr < 0 ||
      (spec->n_attr > 0 && !spec->attr_set)) {
    set_error("pm4g_filter: bad mode or attribute set");
    return PM4G_EINVAL;
  }
  if (spec->n_attr > 0 && !L->has_attr) {
    set_error("pm4g_filter: the log was loaded without a case attribute");
    return PM4G_EINVAL;
  }
  Ctx *c = L->ctx;
  PM4G_CK(cudaSetDevice(c->device));
  if (L->n == 0 || L->nb == 0) return extract_sublog(L, FilterArgs{}, out);
  PM4G_TRY(ensure_span(L));
  const uint64_t R = L->R;
  Scratch S(c);
  std::vector<int32_t> aset(spec->attr_set, spec->attr_set + spec->n_attr);
  std::sort(aset.begin(), aset.end());
  aset.erase(std::unique(aset.begin(), aset.end()), aset.end());
  int32_t *dset = S.get<int32_t>(aset.size());
  uint8_t *ok = S.get<uint8_t>(R);
  if (!ok || (!aset.empty() && !dset)) {
    set_error("pm4g_filter: out of device memory");
    return PM4G_ENOMEM;
  }
  if (!aset.empty())
    PM4G_CK(cudaMemcpyAsync(dset, aset.data(), aset.size() * 4, cudaMemcpyHostToDevice, c->stream));
  FilterArgs fa{};
  fa.n_slots = R;
  fa.first_ts = L->span.p;
  fa.last_ts = L->span.p + R;
  fa.cattr = L->cattr.p;
  fa.attr_set = dset;
  fa.n_attr = (int32_t)aset.size();
  fa.t_lo = spec->t_lo;
  fa.t_hi = spec->t_hi;
  fa.mode = spec->mode;
  fa.case_ok = ok;
  fa.len = L->len.p;
  {
    KTime t(c, "filter");
    k_case_ok<<<grid_for((int64_t)R, 256, 65535), 256, 0, c->stream>>>(fa);
    PM4G_TRY(check_launch(c, "k_case_ok"));
  }
  return extract_sublog(L, fa, out);
}

// Bitmap of the activity codes of a host set (NULL when the set is empty);
// PM4G_EINVAL for a code outside [0, A).
static int activity_bits(Ctx *c, Scratch &S, const int32_t *set, int32_t n, int32_t A, const char *what,
                         uint32_t **out) {
  *out = nullptr;
  if (n == 0) return PM4G_OK;
  std::vector<uint32_t> bits(((size_t)A + 31) / 32, 0u);
  for (int32_t k = 0; k < n; ++k) {
    if (set[k] < 0 || set[k] >= A) {
      set_error("pm4g_filter_cases: %s holds activity %d outside [0, %d)", what, set[k], A);
      return PM4G_EINVAL;
    }
    bits[(uint32_t)set[k] >> 5] |= 1u << (set[k] & 31);
  }
  uint32_t *d = S.get<uint32_t>(bits.size());
  if (!d) return PM4G_ENOMEM;
  PM4G_CK(cudaMemcpyAsync(d, bits.data(), bits.size() * 4, cudaMemcpyHostToDevice, c->stream));
  *out = d;
  return PM4G_OK;
}

int pm4g_filter_cases(pm4g_log *L, const pm4g_case_filter *spec, pm4g_log **out) {
  pm4g::ApiRange nvtx_range("pm4g_filter_cases");
  if (!L || !spec || !out) {
    set_error("pm4g_filter_cases: NULL argument");
    return PM4G_EINVAL;
  }
  *out = nullptr;
  if (spec->n_start < 0 || spec->n_end < 0 || spec->n_act < 0 || spec->n_variant < 0 ||
      (spec->n_start > 0 && !spec->start_set) || (spec->n_end > 0 && !spec->end_set) ||
      (spec->n_act > 0 && !spec->act_set) || (spec->n_variant > 0 && !spec->variant_set)) {
    set_error("pm4g_filter_cases: negative set size or NULL set");
    return PM4G_EINVAL;
  }
  Ctx *c = L->ctx;
  PM4G_CK(cudaSetDevice(c->device));
  Scratch S(c);
  CaseFilterArgs ca{};
  PM4G_TRY(activity_bits(c, S, spec->start_set, spec->n_start, L->A, "start_set", (uint32_t **)&ca.start_bits));
  PM4G_TRY(activity_bits(c, S, spec->end_set, spec->n_end, L->A, "end_set", (uint32_t **)&ca.end_bits));
  PM4G_TRY(activity_bits(c, S, spec->act_set, spec->n_act, L->A, "act_set", (uint32_t **)&ca.act_bits));
  if (L->n == 0 || L->nb == 0) return extract_sublog(L, FilterArgs{}, out);
  PM4G_TRY(ensure_span(L));
  PM4G_TRY(ensure_offsets(L));
  std::vector<int32_t> vset(spec->variant_set, spec->variant_set + spec->n_variant);
  std::sort(vset.begin(), vset.end());
  vset.erase(std::unique(vset.begin(), vset.end()), vset.end());
  if (!vset.empty()) {
    PM4G_TRY(ensure_variants(L));
    PM4G_TRY(ensure_case_variants(L));
    int32_t *dv = S.get<int32_t>(vset.size());
    if (!dv) return PM4G_ENOMEM;
    PM4G_CK(cudaMemcpyAsync(dv, vset.data(), vset.size() * 4, cudaMemcpyHostToDevice, c->stream));
    ca.variants = dv;
    ca.n_variants = (int32_t)vset.size();
    ca.cvar = L->cvar.p;
  }
  const uint64_t R = L->R;
  uint8_t *ok = S.get<uint8_t>(R);
  if (!ok) return PM4G_ENOMEM;
  ca.n_slots = R;
  ca.len = L->len.p;
  ca.off = L->off.p;
  ca.act_s = L->act_s.p;
  ca.first_ts = L->span.p;
  ca.last_ts = L->span.p + R;
  ca.min_events = spec->min_events;
  ca.max_events = spec->max_events;
  ca.min_duration = spec->min_duration;
  ca.max_duration = spec->max_duration;
  ca.exclude = spec->exclude;
  ca.case_ok = ok;
  {
    KTime t(c, "filter");
    k_case_filter<<<grid_for((int64_t)R, 256, 65535), 256, 0, c->stream>>>(ca);
    PM4G_TRY(check_launch(c, "k_case_filter"));
  }
  FilterArgs fa{};
  fa.case_ok = ok;
  fa.mode = PM4G_TW_NONE;
  fa.len = L->len.p;
  return extract_sublog(L, fa, out);
}

int pm4g_filter_paths(pm4g_log *L, const int32_t *src, const int32_t *dst, int32_t n_pairs, int32_t exclude,
                      pm4g_log **out) {
  pm4g::ApiRange nvtx_range("pm4g_filter_paths");
  if (!L || !out || n_pairs < 0 || (n_pairs > 0 && (!src || !dst))) {
    set_error("pm4g_filter_paths: NULL argument or negative pair count");
    return PM4G_EINVAL;
  }
  *out = nullptr;
  const uint32_t A = (uint32_t)L->A;
  std::vector<uint64_t> keys((size_t)n_pairs);
  for (int32_t k = 0; k < n_pairs; ++k) {
    if (src[k] < 0 || (uint32_t)src[k] >= A || dst[k] < 0 || (uint32_t)dst[k] >= A) {
      set_error("pm4g_filter_paths: pair %d holds an activity outside [0, %u)", k, A);
      return PM4G_EINVAL;
    }
    keys[k] = (uint64_t)src[k] * A + (uint32_t)dst[k];
  }
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  Ctx *c = L->ctx;
  PM4G_CK(cudaSetDevice(c->device));
  if (L->n == 0 || L->nb == 0) return extract_sublog(L, FilterArgs{}, out);
  PM4G_TRY(ensure_offsets(L));
  const uint64_t n = L->n, R = L->R;
  // the original row of every formatted position, kept on the log for later
  // path filters (the export pass that forms it costs about as much as a
  // filter's other kernels)
  if (!L->row_s.p) {
    PM4G_TRY(alloc_buf(c, L->row_s, (size_t)n));
    const int st = run_export(L, nullptr, nullptr, nullptr, L->row_s.p);
    if (st != PM4G_OK) {
      free_buf(c, L->row_s);
      return st;
    }
  }
  const int64_t *row_s = L->row_s.p;
  Scratch S(c);
  uint8_t *start = S.get<uint8_t>(n);
  uint32_t *keep = S.get<uint32_t>((n + 31) / 32);
  uint64_t *dkeys = S.get<uint64_t>(keys.size());
  if (!start || !keep || (!keys.empty() && !dkeys)) {
    set_error("pm4g_filter_paths: out of device memory");
    return PM4G_ENOMEM;
  }
  if (!keys.empty())
    PM4G_CK(cudaMemcpyAsync(dkeys, keys.data(), keys.size() * 8, cudaMemcpyHostToDevice, c->stream));
  // where cases start
  PM4G_CK(cudaMemsetAsync(start, 0, n, c->stream));
  PM4G_CK(cudaMemsetAsync(keep, 0, (n + 31) / 32 * 4, c->stream));
  {
    KTime t(c, "filter");
    k_mark_case_starts<<<grid_for((int64_t)R, 256, 65535), 256, 0, c->stream>>>(L->len.p, L->off.p, R, start);
    PM4G_TRY(check_launch(c, "k_mark_case_starts"));
    k_path_keep<<<grid_for((int64_t)n, 256, 65535), 256, 0, c->stream>>>(n, L->act_s.p, start, row_s, dkeys,
                                                                         (int32_t)keys.size(), A, exclude, keep);
    PM4G_TRY(check_launch(c, "k_path_keep"));
  }
  FilterArgs fa{};
  fa.row_keep = keep;
  return extract_sublog(L, fa, out);
}


