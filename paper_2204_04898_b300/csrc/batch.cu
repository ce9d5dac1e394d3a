// Batched drill-down (Section 1: drill-down into sub-logs; Section 3: the
// attribute and timestamp filters followed by the frequency and performance
// DFG and the start/end activities).
//
// A sub-log keeps the cases whose attribute is in its set and, by its window
// mode, the events (EVENTS) or whole cases (CONTAINED, INTERSECTING) that meet
// its window. A case's kept events are a contiguous run of its events in
// (timestamp, row) order, because the window is a closed timestamp interval.
// So the sub-log's directly-follows pairs are exactly the resident log's pairs
// whose two events are both kept, and every sub-log result can be computed
// from the resident formatted log without forming the sub-log.
//
// The resident log gets a drill-down index once: timestamps in formatted
// order (ts_s; activities are act_s), case offsets, the present cases ordered
// by (attribute, slot) with event prefixes, the distinct attribute values with
// their case ranges (host copy), and the map from a pair (a, b) to the index
// of edge (a, b) among the resident log's edges (any sub-log edge is one).
//
// A call plans work items on the host: each sub-log becomes one or more items,
// an item being a list of case ranges of the attribute order with at most
// about W events; items run largest first. One persistent CTA per SM takes
// items from a counter. For an item it aggregates the pairs of its cases in a
// shared-memory table keyed by edge index (the segment pass's table, hashed),
// counts start/end activities in shared memory, and at the end of the item
// adds its table and counts to the sub-log's dense accumulators (one row of
// E entries per sub-log, E = the resident log's edge count). A compaction
// then lists each sub-log's edges with a non-zero count in edge order, which
// is (src, dst) order.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <type_traits>
#include <vector>

#include "device_common.cuh"
#include "engine.h"
#include "kernels.h"
#include "sink.cuh"
#include "variants.h"

using namespace pm4g;

namespace pm4g {
namespace {

constexpr int kBtThreads = 1024;
constexpr int kBtWarps = kBtThreads / 32;
constexpr int kBtSlots = 8192;  // shared edge table (hashed)
// Defaults of the tunable launch choices (PM4G_OPT_BATCH_*): groups a
// pipelined batch is cut into, cases a warp takes at once, work items per SM.
constexpr int kBtStages = 4;
constexpr int kBtChunk = 16;
constexpr int kBtItemsPerSm = 4;
static_assert(kBtChunk == 8 || kBtChunk == 16 || kBtChunk == 32, "the launch switch covers 8, 16 and 32");

struct BatchArgs {
  const uint32_t *aslots;  // present slots in (attribute, slot) order
  const uint32_t *aoff;    // first formatted position of each entry of aslots
  const uint32_t *alen;    // events of each entry of aslots
  const uint16_t *act_s;
  const int64_t *ts_s;
  const uint32_t *eidx_s;  // edge index of each event's pair with the next event of its case
  uint32_t n_act;
  uint32_t a_s;  // endpoint counters kept in shared memory (n_act, or 0 for large alphabets: global adds)
  uint32_t n_edges;
  const uint4 *items;   // {sub, first range, end range, 0}
  uint32_t n_items;
  const uint2 *ranges;  // [k0, k1) of aslots
  uint32_t *work;
  const int64_t *t_lo, *t_hi;
  const int32_t *mode;
  DfgTable acc;                   // each array: n_sub rows of n_edges
  unsigned long long *start, *end;  // n_sub rows of n_act
  unsigned long long *n_ev, *n_cs;  // n_sub
  // variant records (NULL rlen: no variants): one per (sub-log, case of its
  // ranges) at rbase[range] + position in the range; rlen 0 = nothing kept
  const uint32_t *rbase;
  uint32_t *rq, *rslot, *rpos, *rlen;
  uint64_t *rhash;
};

__host__ __device__ inline size_t bt_smem_bytes(uint32_t n_act) {
  return (size_t)kBtSlots * 24 + (size_t)n_act * 8 + 64 + (size_t)kBtWarps * 64 * 4;
}

// First index of the non-decreasing t[0, L) whose value is >= v (strict: > v).
template <bool kStrict>
__device__ __forceinline__ uint32_t ts_bound(const int64_t *__restrict__ t, uint32_t L, int64_t v) {
  uint32_t lo = 0, n = L;
  while (n > 0) {
    const uint32_t h = n >> 1;
    const int64_t x = t[lo + h];
    if (kStrict ? x <= v : x < v) {
      lo += h + 1;
      n -= h + 1;
    } else {
      n = h;
    }
  }
  return lo;
}

// Kept run [j0, j1) of one case of L events at formatted position o, found by
// one lane. Timestamps are non-decreasing along a case, so EVENTS keeps the
// events from the first at or after t_lo up to the last at or before t_hi;
// cases wholly inside or outside the window (most of them) take two loads.
__device__ __forceinline__ void kept_run(const BatchArgs &a, uint32_t o, uint32_t L, int mode, int64_t t_lo,
                                         int64_t t_hi, uint32_t &j0, uint32_t &j1) {
  j0 = 0;
  j1 = L;
  if (mode == PM4G_TW_NONE || L == 0) return;
  const int64_t first = a.ts_s[o], last = a.ts_s[o + L - 1];
  if (mode == PM4G_TW_EVENTS) {
    if (first >= t_lo && last <= t_hi) return;
    if (last < t_lo || first > t_hi) {
      j1 = 0;
      return;
    }
    j0 = first >= t_lo ? 0u : ts_bound<false>(a.ts_s + o, L, t_lo);
    j1 = last <= t_hi ? L : ts_bound<true>(a.ts_s + o, L, t_hi);
    j1 = max(j1, j0);
    return;
  }
  const bool keep = mode == PM4G_TW_CASES_CONTAINED ? (first >= t_lo && last <= t_hi)
                                                    : (first <= t_hi && last >= t_lo);
  if (!keep) j1 = 0;
}

template <int kChunk>  // cases a warp takes at once: a power of two, at most 32
__global__ void __launch_bounds__(kBtThreads, 1) k_batch_dfg(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t *tl = reinterpret_cast<uint32_t *>(smem);
  uint32_t *tm = tl + kBtSlots;
  uint32_t *tkey = tm + kBtSlots;
  uint32_t *tcnt = tkey + kBtSlots;
  uint32_t *tminh = tcnt + kBtSlots;
  uint32_t *tmaxh = tminh + kBtSlots;
  uint32_t *st = tmaxh + kBtSlots;
  uint32_t *en = st + a.a_s;
  uint32_t *misc = en + a.a_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // per warp: sequence hash words (low, high) of its chunk's cases
  uint32_t *wl = misc + 16 + warp * 64, *wh = wl + 32;
  const uint32_t A = a.n_act;
  for (;;) {
    if (tid == 0) {
      misc[0] = atomicAdd(a.work, 1u);
      misc[1] = 0;  // next chunk of the item
    }
    for (int i = tid; i < kBtSlots; i += kBtThreads) {
      tkey[i] = kEmptyKey;
      tcnt[i] = 0;
      tl[i] = 0;
      tm[i] = 0;
      tminh[i] = kGuardMinInit;
      tmaxh[i] = kGuardMaxInit;
    }
    for (uint32_t i = tid; i < a.a_s; i += kBtThreads) {
      st[i] = 0;
      en[i] = 0;
    }
    __syncthreads();
    const uint32_t it = misc[0];
    if (it >= a.n_items) break;
    const uint4 item = a.items[it];
    const uint32_t sub = item.x;
    const int mode = a.mode[sub];
    const int64_t t_lo = a.t_lo[sub], t_hi = a.t_hi[sub];
    const uint64_t row = (uint64_t)sub * a.n_edges;
    const DfgTable g{a.acc.cnt + row, a.acc.lo + row, a.acc.hi + row, a.acc.mn + row, a.acc.mx + row};
    SmemSink sink{tkey, tcnt, tminh, tmaxh, tl, tm, (uint32_t)(kBtSlots - 1),
                  (uint32_t)__clz((uint32_t)kBtSlots) + 1u, 1, a.a_s ? st : nullptr,
                  a.a_s ? en : nullptr, g,
                  a.start + (uint64_t)sub * A, a.end + (uint64_t)sub * A};
    sink.probes = 16;
    uint64_t ev = 0, cs = 0;  // this lane's kept events and cases
    // The item's ranges are cut into chunks of kChunk consecutive cases,
    // numbered across the ranges; warps take chunks from a shared counter.
    // A warp takes a chunk one case per lane: each lane finds its case's kept
    // run, then the warp walks the runs' events 32 at a time across case
    // boundaries (lane-dense), each lane locating its event's case by a
    // binary search over the runs' prefix.
    uint32_t r = item.y, qb = 0, nch = 0;  // the warp's range; it holds chunks [qb, qb + nch)
    uint2 rg = make_uint2(0, 0);
    if (r < item.z) {
      rg = a.ranges[r];
      nch = (rg.y - rg.x + kChunk - 1) / kChunk;
    }
    for (;;) {
      uint32_t q = 0;
      if (lane == 0) q = atomicAdd(&misc[1], 1u);
      q = __shfl_sync(kFull, q, 0);
      while (r < item.z && q >= qb + nch) {
        qb += nch;
        if (++r < item.z) {
          rg = a.ranges[r];
          nch = (rg.y - rg.x + kChunk - 1) / kChunk;
        }
      }
      if (r >= item.z) break;
      {
        const uint32_t jc = q - qb;
        const uint32_t k = rg.x + jc * kChunk + (uint32_t)lane;
        const bool have = lane < kChunk && k < rg.y;
        uint32_t o = 0, L = 0, j0 = 0, j1 = 0;
        if (have) {
          o = a.aoff[k];
          L = a.alen[k];
          kept_run(a, o, L, mode, t_lo, t_hi, j0, j1);
        }
        const uint32_t n = j1 - j0, pos0 = o + j0;
        uint32_t incl = n;  // inclusive prefix over lanes [0, kChunk)
#pragma unroll
        for (int d = 1; d < kChunk; d <<= 1) {
          const uint32_t v = __shfl_up_sync(kFull, incl, d);
          if (lane >= d) incl += v;
        }
        const uint32_t excl = incl - n, T = __shfl_sync(kFull, incl, kChunk - 1);
        if (a.rlen) {
          wl[lane] = 0;
          wh[lane] = 0;
          __syncwarp();
        }
        for (uint32_t b = 0; b < T; b += 32) {
          const uint32_t x = b + (uint32_t)lane;
          const bool valid = x < T;
          // the case of x: the last lane whose prefix is at most x (it has a
          // non-empty run containing x)
          uint32_t c = 0;
#pragma unroll
          for (uint32_t d = kChunk / 2; d >= 1; d >>= 1) {
            const uint32_t e = __shfl_sync(kFull, excl, (int)(c + d));
            if (e <= x) c += d;
          }
          const uint32_t ce = __shfl_sync(kFull, excl, (int)c);
          const uint32_t cn = __shfl_sync(kFull, n, (int)c);
          const uint32_t cp = __shfl_sync(kFull, pos0, (int)c);
          const uint32_t i = x - ce, p = cp + i;
          const bool first = valid && i == 0, last = valid && i + 1 == cn;
          const bool has_edge = valid && !last;
          uint32_t act = 0, e = 0;
          int64_t ts = 0;
          if (valid) {
            ts = a.ts_s[p];
            if (a.rlen || first || last) act = (uint32_t)a.act_s[p];
            if (has_edge) e = a.eidx_s[p];
          }
          if (first) sink.start(act);
          if (last) sink.end(act);
          int64_t nts = __shfl_down_sync(kFull, ts, 1);
          if (lane == 31 && has_edge) nts = a.ts_s[p + 1];
          aggregate_edges(sink, has_edge, e, (uint64_t)nts - (uint64_t)ts);
          if (a.rlen && valid) {
            // the sequence hash of the kept run, as the segment pass forms it
            const uint64_t t = event_hash(act, i, 0);
            atomicAdd(&wl[c], (uint32_t)t);
            atomicAdd(&wh[c], (uint32_t)(t >> 32));
          }
        }
        ev += n;
        cs += n ? 1u : 0u;
        if (a.rlen) {
          __syncwarp();
          if (have) {
            const uint32_t rec = a.rbase[r] + (k - rg.x);
            if (n == 0) {
              a.rlen[rec] = 0;
            } else {
              a.rq[rec] = sub;
              a.rslot[rec] = a.aslots[k];
              a.rpos[rec] = pos0;
              a.rlen[rec] = n;
              a.rhash[rec] = ((uint64_t)wh[lane] << 32) | wl[lane];
            }
          }
          __syncwarp();
        }
      }
    }
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
      ev += __shfl_down_sync(kFull, ev, d);
      cs += __shfl_down_sync(kFull, cs, d);
    }
    if (lane == 0 && cs) {
      atomicAdd(&a.n_ev[sub], (unsigned long long)ev);
      atomicAdd(&a.n_cs[sub], (unsigned long long)cs);
    }
    __syncthreads();
    for (int s = tid; s < kBtSlots; s += kBtThreads) {
      const uint32_t c = tcnt[s];
      if (c) global_edge_group(g, tkey[s], c, tl[s] | ((uint64_t)tm[s] << 32), 0);
    }
    for (uint32_t i = tid; i < a.a_s; i += kBtThreads) {
      if (st[i]) atomicAdd(&sink.g_start[i], (unsigned long long)st[i]);
      if (en[i]) atomicAdd(&sink.g_end[i], (unsigned long long)en[i]);
    }
    __syncthreads();
  }
}

// ---- drill-down index ----
__global__ void k_dd_present_keys(const uint32_t *__restrict__ len, uint64_t R, const uint32_t *__restrict__ pos,
                                  const int32_t *__restrict__ cattr, uint32_t *keys, uint32_t *vals) {
  for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < R; s += (uint64_t)gridDim.x * blockDim.x) {
    if (!len[s]) continue;
    const uint32_t p = pos[s];
    keys[p] = cattr ? ((uint32_t)cattr[s] ^ 0x80000000u) : 0x80000000u;  // signed order
    vals[p] = (uint32_t)s;
  }
}
__global__ void k_dd_lens(const uint32_t *__restrict__ aslots, const uint32_t *__restrict__ len, uint32_t C,
                          uint32_t *out) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < C; k += gridDim.x * blockDim.x) out[k] = len[aslots[k]];
}
__global__ void k_dd_heads(const uint32_t *__restrict__ keys, uint32_t C, uint32_t *flags) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < C; k += gridDim.x * blockDim.x)
    flags[k] = (k == 0 || keys[k] != keys[k - 1]) ? 1u : 0u;
}
__global__ void k_dd_groups(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ flags,
                            const uint32_t *__restrict__ pos, const uint32_t *__restrict__ apre, uint32_t C,
                            int32_t *vals, uint32_t *lo, uint32_t *ev) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < C; k += gridDim.x * blockDim.x) {
    if (!flags[k]) continue;
    const uint32_t u = pos[k];
    vals[u] = (int32_t)(keys[k] ^ 0x80000000u);
    lo[u] = k;
    ev[u] = apre[k];
  }
}
__global__ void k_dd_emap(const uint32_t *__restrict__ flags, const uint32_t *__restrict__ pos, int64_t cells,
                          uint32_t n_act, uint32_t *emap, int32_t *pair, uint32_t E) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cells; i += (int64_t)gridDim.x * blockDim.x) {
    if (flags[i]) {
      const uint32_t e = pos[i];
      emap[i] = e;
      pair[e] = (int32_t)(i / n_act);
      pair[E + e] = (int32_t)(i % n_act);
    } else {
      emap[i] = 0xFFFFFFFFu;
    }
  }
}

__global__ void k_dd_case_cols(const uint32_t *__restrict__ aslots, const uint32_t *__restrict__ off,
                               const uint32_t *__restrict__ len, uint32_t C, uint32_t *aoff, uint32_t *alen) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < C; k += gridDim.x * blockDim.x) {
    const uint32_t s = aslots[k];
    aoff[k] = off[s];
    alen[k] = len[s];
  }
}
// One warp per case: the edge index of every event's pair with the next
// event of its case (~0 for the case's last event).
// Edge e of a hashed table's ascending keys: its key and its (src, dst).
__global__ void k_dd_pairs_of_keys(const uint32_t *__restrict__ keys, uint32_t E, uint32_t A, uint32_t *ekey,
                                   int32_t *pair) {
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
    const uint32_t k = keys[e];
    ekey[e] = k;
    pair[e] = (int32_t)(k / A);
    pair[E + e] = (int32_t)(k % A);
  }
}
// With no dense map (large alphabets), the edge index is found by binary
// search over the log's edge keys (src * A + dst), ascending.
__device__ __forceinline__ uint32_t edge_of(const uint32_t *__restrict__ emap, const uint32_t *__restrict__ ekey,
                                            uint32_t E, uint32_t key) {
  if (emap) return emap[key];
  uint32_t lo = 0, n = E;
  while (n > 0) {
    const uint32_t h = n >> 1;
    if (ekey[lo + h] < key) {
      lo += h + 1;
      n -= h + 1;
    } else {
      n = h;
    }
  }
  return lo < E && ekey[lo] == key ? lo : 0xFFFFFFFFu;
}
__global__ void k_dd_eidx(const uint32_t *__restrict__ aoff, const uint32_t *__restrict__ alen, uint32_t C,
                          const uint16_t *__restrict__ act_s, const uint32_t *__restrict__ emap,
                          const uint32_t *__restrict__ ekey, uint32_t E, uint32_t A, uint32_t *eidx) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t k = w0; k < C; k += nw) {
    const uint32_t o = aoff[k], L = alen[k];
    for (uint32_t base = 0; base < L; base += 32) {
      const uint32_t j = base + lane;
      const uint32_t act = j < L ? (uint32_t)act_s[o + j] : 0u;
      uint32_t nact = __shfl_down_sync(kFull, act, 1);
      if (lane == 31 && j + 1 < L) nact = (uint32_t)act_s[o + j + 1];
      if (j + 1 < L) eidx[o + j] = edge_of(emap, ekey, E, act * A + nact);
      else if (j + 1 == L) eidx[o + j] = 0xFFFFFFFFu;
    }
  }
}

// ---- outputs ----
__global__ void k_bt_flags(const unsigned long long *__restrict__ cnt, uint64_t n, uint32_t *flags) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    flags[i] = cnt[i] ? 1u : 0u;
}
__global__ void k_bt_compact(DfgTable acc, const uint32_t *__restrict__ flags, const uint32_t *__restrict__ pos,
                             uint64_t n, uint32_t E, uint32_t A, const int32_t *__restrict__ pair, int32_t *src,
                             int32_t *dst, unsigned long long *cnt, unsigned long long *lo, unsigned long long *hi,
                             unsigned long long *mn, unsigned long long *mx, double *mean,
                             unsigned long long *freq) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    if (!flags[i]) continue;
    const uint32_t p = pos[i];
    const uint32_t e = (uint32_t)(i % E);
    const uint64_t q = i / E;
    const unsigned long long c = acc.cnt[i], l = acc.lo[i], h = acc.hi[i];
    src[p] = pair[e];
    dst[p] = pair[E + e];
    cnt[p] = c;
    lo[p] = l;
    hi[p] = h;
    mn[p] = acc.mn[i];
    mx[p] = acc.mx[i];
    mean[p] = edge_mean(h, l, c);
    atomicAdd(&freq[q * A + (uint32_t)pair[e]], c);  // out-edges of src
  }
}
__global__ void k_bt_offsets(const uint32_t *__restrict__ pos, uint32_t Qg, uint32_t E, int64_t *off) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q <= Qg; q += gridDim.x * blockDim.x)
    off[q] = pos[(uint64_t)q * E];
}
__global__ void k_bt_add(unsigned long long *freq, const unsigned long long *__restrict__ end, uint64_t n) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    freq[i] += end[i];
}

// ---- variants of the sub-logs ----
__global__ void k_bv_flags(const uint32_t *__restrict__ rlen, uint32_t n, uint32_t *flags) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    flags[i] = rlen[i] ? 1u : 0u;
}
// kept records keyed by (sub-log, case slot), so that sorting puts each
// sub-log's cases in ascending case order
__global__ void k_bv_keys(const uint32_t *__restrict__ rlen, const uint32_t *__restrict__ rq,
                          const uint32_t *__restrict__ rslot, const uint32_t *__restrict__ pos, uint32_t n,
                          int sbits, uint64_t *keys, uint32_t *idx) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (!rlen[i]) continue;
    const uint32_t p = pos[i];
    keys[p] = ((uint64_t)rq[i] << sbits) | rslot[i];  // (view, slot), slot < 2^sbits
    idx[p] = i;
  }
}
__global__ void k_bv_gather(const uint32_t *__restrict__ idx, uint32_t n, const uint32_t *__restrict__ rq,
                            const uint32_t *__restrict__ rslot, const uint32_t *__restrict__ rpos,
                            const uint32_t *__restrict__ rlen, const uint64_t *__restrict__ rhash, uint32_t *sq,
                            uint32_t *sslot, uint32_t *spos, uint32_t *slen, uint64_t *shash) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const uint32_t i = idx[p];
    sq[p] = rq[i];
    sslot[p] = rslot[i];
    spos[p] = rpos[i];
    slen[p] = rlen[i];
    shash[p] = rhash[i];
  }
}
// after the sort by count: the sub-log of each representative, for the
// stable second sort
__global__ void k_bv_qkeys(const uint32_t *__restrict__ order, const uint32_t *__restrict__ rep_idx,
                           const uint32_t *__restrict__ sq, uint32_t V, uint32_t *qk) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < V; t += gridDim.x * blockDim.x)
    qk[t] = sq[rep_idx[order[t]]];
}
// after the sort by sub-log: each sub-log's first representative and count
// (absent sub-logs keep 0 from the memset)
__global__ void k_bv_bounds(const uint32_t *__restrict__ qk, uint32_t V, uint32_t *vbeg, uint32_t *vq) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < V; t += gridDim.x * blockDim.x) {
    const uint32_t q = qk[t];
    if (t == 0 || qk[t - 1] != q) vbeg[q] = t;
    if (t + 1 == V || qk[t + 1] != q) vq[q] = t + 1;  // end, made a count below
  }
}
__global__ void k_bv_counts(const uint32_t *__restrict__ vbeg, uint32_t Qg, uint32_t *vq) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < Qg; q += gridDim.x * blockDim.x)
    if (vq[q]) vq[q] -= vbeg[q];
}
// sequence offsets of the output rows as 64-bit positions in the call's result
__global__ void k_bv_seq64(const uint32_t *__restrict__ seq, uint32_t n, int64_t base, int64_t *out) {
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
    out[r] = base + (int64_t)seq[r];
}
__global__ void k_bv_take(const uint32_t *__restrict__ vq, uint32_t Qg, int64_t top_k, uint32_t *take) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < Qg; q += gridDim.x * blockDim.x)
    take[q] = (top_k < 0 || (uint64_t)vq[q] <= (uint64_t)top_k) ? vq[q] : (uint32_t)top_k;
}
// output rows: the first take[q] representatives of every sub-log, in
// (count desc, smallest case asc) order
__global__ void k_bv_head(const uint32_t *__restrict__ order, const uint32_t *__restrict__ qk,
                          const uint32_t *__restrict__ vstart, const uint32_t *__restrict__ take,
                          const uint32_t *__restrict__ row0, const uint32_t *__restrict__ rep_idx,
                          const uint32_t *__restrict__ vcount, const uint32_t *__restrict__ sslot,
                          const uint32_t *__restrict__ slen, uint32_t V, int32_t min_case,
                          const int32_t *__restrict__ uniq, unsigned long long *o_count, int32_t *o_min,
                          uint32_t *o_len, uint32_t *o_rep) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < V; t += gridDim.x * blockDim.x) {
    const uint32_t q = qk[t], i = t - vstart[q];
    if (i >= take[q]) continue;
    const uint32_t row = row0[q] + i, r = rep_idx[order[t]];
    const uint32_t slot = sslot[r];
    o_count[row] = vcount[r];
    o_min[row] = uniq ? uniq[slot] : (int32_t)((uint32_t)min_case + slot);
    o_len[row] = slen[r];
    o_rep[row] = r;
  }
}
__global__ void k_bv_acts(const uint32_t *__restrict__ o_rep, const uint32_t *__restrict__ seq,
                          const uint32_t *__restrict__ spos, const uint32_t *__restrict__ slen,
                          const uint16_t *__restrict__ act_s, uint32_t rows, int32_t *o_acts) {
  for (uint32_t row = blockIdx.x * blockDim.x + threadIdx.x; row < rows; row += gridDim.x * blockDim.x) {
    const uint32_t r = o_rep[row], L = slen[r];
    const uint16_t *src = act_s + spos[r];
    int32_t *dst = o_acts + seq[row];
    for (uint32_t k = 0; k < L; ++k) dst[k] = src[k];
  }
}

// Builds the drill-down index of L (once).
int ensure_drilldown(pm4g_log *L) {
  if (L->dd_ready) return PM4G_OK;
  Ctx *c = L->ctx;
  const uint32_t C = (uint32_t)L->C;
  PM4G_TRY(ensure_offsets(L));
  // timestamps in formatted order: shared with the eventually-follows graph,
  // which may have formed them already; dropped again if forming them fails
  if (!L->ts_s.p) {
    PM4G_TRY(alloc_buf(c, L->ts_s, (size_t)L->n));
    const int st = run_export(L, nullptr, nullptr, L->ts_s.p, nullptr);
    if (st != PM4G_OK) {
      free_buf(c, L->ts_s);
      return st;
    }
  }
  // what an earlier attempt that failed part way left behind
  free_buf(c, L->aslots);
  free_buf(c, L->apre);
  free_buf(c, L->emap);
  free_buf(c, L->ekey);
  free_buf(c, L->e_pair);
  free_buf(c, L->aoff);
  free_buf(c, L->alen);
  free_buf(c, L->eidx_s);
  // present cases in (attribute, slot) order
  PM4G_TRY(alloc_buf(c, L->aslots, C));
  PM4G_TRY(alloc_buf(c, L->apre, (size_t)C + 1));
  {
    Scratch S(c);
    const uint64_t R = L->R;
    uint32_t *pf = S.get<uint32_t>(R), *pp = S.get<uint32_t>(R + 1);
    uint32_t *keys = S.get<uint32_t>(C), *k2 = S.get<uint32_t>(C), *v2 = S.get<uint32_t>(C);
    uint32_t *lens = S.get<uint32_t>(C), *hf = S.get<uint32_t>(C), *hp = S.get<uint32_t>((size_t)C + 1);
    if (!pf || !pp || !keys || !k2 || !v2 || !lens || !hf || !hp) {
      set_error("drill-down index: out of device memory");
      return PM4G_ENOMEM;
    }
    const unsigned gR = grid_for((int64_t)R, 256, 65535), gC = grid_for((int64_t)C, 256, 65535);
    k_present_flags<<<gR, 256, 0, c->stream>>>(L->len.p, R, pf);
    PM4G_TRY(check_launch(c, "k_present_flags"));
    PM4G_TRY(scan_u32(c, pf, pp, (int64_t)R));
    k_dd_present_keys<<<gR, 256, 0, c->stream>>>(L->len.p, R, pp, L->has_attr ? L->cattr.p : nullptr, keys,
                                                  L->aslots.p);
    PM4G_TRY(check_launch(c, "k_dd_present_keys"));
    if (L->has_attr && C > 1) PM4G_TRY(radix_sort_u32(c, keys, L->aslots.p, k2, v2, C, 0, 32));
    k_dd_lens<<<gC, 256, 0, c->stream>>>(L->aslots.p, L->len.p, C, lens);
    PM4G_TRY(check_launch(c, "k_dd_lens"));
    PM4G_TRY(scan_u32(c, lens, L->apre.p, C));
    k_dd_heads<<<gC, 256, 0, c->stream>>>(keys, C, hf);
    PM4G_TRY(check_launch(c, "k_dd_heads"));
    PM4G_TRY(scan_u32(c, hf, hp, C));
    uint32_t U = 0;
    PM4G_TRY(d2h(c, &U, hp + C, 4));
    int32_t *gv = S.get<int32_t>(U);
    uint32_t *glo = S.get<uint32_t>(U), *gev = S.get<uint32_t>(U);
    if (!gv || !glo || !gev) return PM4G_ENOMEM;
    if (C) {
      k_dd_groups<<<gC, 256, 0, c->stream>>>(keys, hf, hp, L->apre.p, C, gv, glo, gev);
      PM4G_TRY(check_launch(c, "k_dd_groups"));
    }
    L->attr_vals.assign(U, 0);
    L->attr_lo.assign((size_t)U + 1, C);
    L->attr_ev.assign((size_t)U + 1, (uint32_t)L->n);
    D2HBatch hb(c, (size_t)U * 12 + 64);
    hb.add(L->attr_vals.data(), gv, (size_t)U * 4);
    hb.add(L->attr_lo.data(), glo, (size_t)U * 4);
    hb.add(L->attr_ev.data(), gev, (size_t)U * 4);
    PM4G_TRY(hb.finish());
  }
  // edge index of every directly-follows pair of the resident log
  if (!L->ghash) {
    Scratch S(c);
    const int64_t cells = (int64_t)L->gcells;
    uint32_t *flags = S.get<uint32_t>(cells), *pos = S.get<uint32_t>(cells + 1);
    if (!flags || !pos) return PM4G_ENOMEM;
    k_dfg_flags<<<grid_for(cells, 256, 4096), 256, 0, c->stream>>>(L->dfg.p, cells, flags);
    PM4G_TRY(check_launch(c, "k_dfg_flags"));
    PM4G_TRY(scan_u32(c, flags, pos, cells));
    uint32_t E = 0;
    PM4G_TRY(d2h(c, &E, pos + cells, 4));
    L->n_edges = E;
    PM4G_TRY(alloc_buf(c, L->emap, (size_t)cells));
    PM4G_TRY(alloc_buf(c, L->e_pair, 2 * (size_t)E));
    k_dd_emap<<<grid_for(cells, 256, 4096), 256, 0, c->stream>>>(flags, pos, cells, (uint32_t)L->A, L->emap.p,
                                                                 L->e_pair.p, E);
    PM4G_TRY(check_launch(c, "k_dd_emap"));
  } else {
    // large alphabets: the edges' keys, ascending, searched per pair
    Scratch S(c);
    uint32_t *keys = nullptr, *slots = nullptr, E = 0;
    PM4G_TRY(hashed_edges(L, S, keys, slots, E));
    L->n_edges = E;
    PM4G_TRY(alloc_buf(c, L->ekey, (size_t)E));
    PM4G_TRY(alloc_buf(c, L->e_pair, 2 * (size_t)E));
    if (E) {
      k_dd_pairs_of_keys<<<grid_for(E, 256, 4096), 256, 0, c->stream>>>(keys, E, (uint32_t)L->A, L->ekey.p,
                                                                         L->e_pair.p);
      PM4G_TRY(check_launch(c, "k_dd_pairs_of_keys"));
    }
  }
  // per-entry case columns in attribute order, and the edge index of every pair
  PM4G_TRY(alloc_buf(c, L->aoff, C));
  PM4G_TRY(alloc_buf(c, L->alen, C));
  PM4G_TRY(alloc_buf(c, L->eidx_s, (size_t)L->n));
  if (C) {
    k_dd_case_cols<<<grid_for((int64_t)C, 256, 65535), 256, 0, c->stream>>>(L->aslots.p, L->off.p, L->len.p, C,
                                                                            L->aoff.p, L->alen.p);
    PM4G_TRY(check_launch(c, "k_dd_case_cols"));
    k_dd_eidx<<<grid_for((int64_t)C * 32, 256, 65535), 256, 0, c->stream>>>(
        L->aoff.p, L->alen.p, C, L->act_s.p, L->emap.p, L->ekey.p, L->n_edges, (uint32_t)L->A, L->eidx_s.p);
    PM4G_TRY(check_launch(c, "k_dd_eidx"));
  }
  L->dd_ready = true;
  return PM4G_OK;
}

struct Plan {
  std::vector<uint4> items;   // {sub (group-local), r0, r1, events}
  std::vector<uint2> ranges;
  std::vector<uint32_t> rbase;  // first variant record of each range
  uint32_t n_rec = 0;
};

}  // namespace
}  // namespace pm4g

int pm4g_batch_dfg_free(pm4g_batch_dfg_t *r) {
  if (!r) return PM4G_OK;
  free(r->n_events);
  free(r->n_cases);
  free(r->edge_off);
  free(r->src);
  free(r->dst);
  free(r->count);
  free(r->sum_lo);
  free(r->sum_hi);
  free(r->min);
  free(r->max);
  free(r->mean);
  free(r->start);
  free(r->end);
  free(r->freq);
  free(r->n_variants);
  free(r->var_off);
  free(r->var_count);
  free(r->var_min_case);
  free(r->var_seq_off);
  free(r->var_acts);
  memset(r, 0, sizeof(*r));
  return PM4G_OK;
}

// The batched drill-down. With caller buffers (cap >= 0) the results go
// straight into out's arrays, edges only while they fit cap (the required
// count is reported through edge_off either way); otherwise the library
// allocates every array.
static int batch_dfg(pm4g_log *L, const pm4g_batch_spec *spec, pm4g_batch_dfg_t *out, int64_t cap) {
  if (!L || !spec || !out) {
    set_error("pm4g_batch_dfg: NULL argument");
    return PM4G_EINVAL;
  }
  const bool caller = cap >= 0;
  if (!caller) memset(out, 0, sizeof(*out));
  const int32_t Q = spec->n_sub;
  if (Q < 0 || (Q > 0 && (!spec->attr_off || !spec->t_lo || !spec->t_hi || !spec->mode))) {
    set_error("pm4g_batch_dfg: bad spec (n_sub < 0 or NULL arrays)");
    return PM4G_EINVAL;
  }
  if (Q > 0 && spec->attr_off[0] != 0) {
    set_error("pm4g_batch_dfg: attr_off[0] must be 0");
    return PM4G_EINVAL;
  }
  for (int32_t i = 0; i < Q; ++i) {
    if (spec->attr_off[i + 1] < spec->attr_off[i]) {
      set_error("pm4g_batch_dfg: attr_off decreases at sub-log %d", i);
      return PM4G_EINVAL;
    }
    if (spec->mode[i] < PM4G_TW_NONE || spec->mode[i] > PM4G_TW_CASES_INTERSECTING) {
      set_error("pm4g_batch_dfg: bad window mode %d at sub-log %d", spec->mode[i], i);
      return PM4G_EINVAL;
    }
    if (spec->attr_off[i + 1] > spec->attr_off[i] && !L->has_attr) {
      set_error("pm4g_batch_dfg: attribute filter on a log loaded without case_attr");
      return PM4G_EINVAL;
    }
  }
  if (Q > 0 && spec->attr_off[Q] > 0 && !spec->attr_vals) {
    set_error("pm4g_batch_dfg: attr_vals is NULL");
    return PM4G_EINVAL;
  }
  Ctx *c = L->ctx;
  PM4G_CK(cudaSetDevice(c->device));
  const uint32_t A = (uint32_t)L->A;
  out->n_sub = Q;
  out->n_activities = (int32_t)A;
  const bool want_var = spec->var_top_k != 0;
  if (caller) {
    if (!out->n_events || !out->n_cases || !out->edge_off || (Q > 0 && (!out->start || !out->end || !out->freq)) ||
        (cap > 0 && (!out->src || !out->dst || !out->count || !out->sum_lo || !out->sum_hi || !out->min ||
                     !out->max || !out->mean)) ||
        (want_var && (!out->n_variants || !out->var_off || !out->var_seq_off || out->var_capacity < 0 ||
                      out->acts_capacity < 0 ||
                      (out->var_capacity > 0 && (!out->var_count || !out->var_min_case)) ||
                      (out->acts_capacity > 0 && !out->var_acts)))) {
      set_error("pm4g_batch_dfg_into: NULL result array or negative capacity");
      return PM4G_EINVAL;
    }
    if (want_var) {
      memset(out->var_off, 0, ((size_t)Q + 1) * 8);
      out->var_seq_off[0] = 0;
      if (Q > 0) memset(out->n_variants, 0, (size_t)Q * 8);
    }
    memset(out->edge_off, 0, ((size_t)Q + 1) * 8);
    if (Q > 0) {
      memset(out->n_events, 0, (size_t)Q * 8);
      memset(out->n_cases, 0, (size_t)Q * 8);
      // the endpoint rows are zeroed only where no group copies them (a log
      // without cases); otherwise every row is written by its group's copy
      if (L->C == 0) {
        memset(out->start, 0, (size_t)Q * A * 8);
        memset(out->end, 0, (size_t)Q * A * 8);
        memset(out->freq, 0, (size_t)Q * A * 8);
      }
    }
  } else {
    out->n_events = (int64_t *)calloc(std::max(Q, 1), 8);
    out->n_cases = (int64_t *)calloc(std::max(Q, 1), 8);
    out->edge_off = (int64_t *)calloc((size_t)Q + 1, 8);
    out->start = (uint64_t *)calloc(std::max<size_t>((size_t)Q * A, 1), 8);
    out->end = (uint64_t *)calloc(std::max<size_t>((size_t)Q * A, 1), 8);
    out->freq = (uint64_t *)calloc(std::max<size_t>((size_t)Q * A, 1), 8);
    out->n_variants = (int64_t *)calloc(std::max(Q, 1), 8);
    out->var_off = (int64_t *)calloc((size_t)Q + 1, 8);
    out->var_seq_off = (int64_t *)calloc(1, 8);
    if (!out->n_events || !out->n_cases || !out->edge_off || !out->start || !out->end || !out->freq ||
        !out->n_variants || !out->var_off || !out->var_seq_off) {
      pm4g_batch_dfg_free(out);
      return PM4G_ENOMEM;
    }
  }
  const int64_t var_cap = caller ? out->var_capacity : -1, acts_cap = caller ? out->acts_capacity : -1;
  auto fail_out = [&](int code) {
    if (!caller) pm4g_batch_dfg_free(out);
    return code;
  };
  size_t Et = 0;  // edges so far
  // room for n edges in the result arrays
  auto room = [&](size_t n) {
    if (caller) return n <= (size_t)cap;
    const size_t m = std::max<size_t>(n, 1);
    bool ok = true;
    auto re = [&](auto *&p, size_t el) {
      void *q = realloc(p, m * el);
      if (!q) ok = false;
      else p = (std::remove_reference_t<decltype(p)>)q;
    };
    re(out->src, 4);
    re(out->dst, 4);
    re(out->count, 8);
    re(out->sum_lo, 8);
    re(out->sum_hi, 8);
    re(out->min, 8);
    re(out->max, 8);
    re(out->mean, 8);
    return ok;
  };
  size_t Vt = 0, At = 0;  // variant rows and their activities so far
  // room for n variant rows with m activities
  auto room_var = [&](size_t n, size_t m) {
    if (caller) return (int64_t)n <= var_cap && (int64_t)m <= acts_cap;
    bool ok = true;
    auto re = [&](auto *&p, size_t cnt, size_t el) {
      void *q = realloc(p, std::max<size_t>(cnt, 1) * el);
      if (!q) ok = false;
      else p = (std::remove_reference_t<decltype(p)>)q;
    };
    re(out->var_count, n, 8);
    re(out->var_min_case, n, 4);
    re(out->var_seq_off, n + 1, 8);
    re(out->var_acts, m, 4);
    return ok;
  };
  if (Q == 0 || L->C == 0) {
    if (!room(0) || (!caller && !room_var(0, 0))) return fail_out(PM4G_ENOMEM);
    return PM4G_OK;
  }
  int st = ensure_drilldown(L);
  if (st != PM4G_OK) return fail_out(st);
  const uint32_t E = L->n_edges;
  const uint32_t C = (uint32_t)L->C;
  // per sub-log: its case ranges and their events
  std::vector<std::vector<uint2>> sub_ranges(Q);
  std::vector<std::vector<uint32_t>> sub_ev(Q);
  uint64_t total_ev = 0;
  for (int32_t i = 0; i < Q; ++i) {
    const int64_t a0 = spec->attr_off[i], a1 = spec->attr_off[i + 1];
    if (a1 == a0) {
      sub_ranges[i].push_back(make_uint2(0, C));
      sub_ev[i].push_back((uint32_t)L->n);
      total_ev += (uint64_t)L->n;
      continue;
    }
    std::vector<int32_t> v(spec->attr_vals + a0, spec->attr_vals + a1);
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    for (int32_t x : v) {
      const auto it = std::lower_bound(L->attr_vals.begin(), L->attr_vals.end(), x);
      if (it == L->attr_vals.end() || *it != x) continue;
      const size_t u = (size_t)(it - L->attr_vals.begin());
      sub_ranges[i].push_back(make_uint2(L->attr_lo[u], L->attr_lo[u + 1]));
      sub_ev[i].push_back(L->attr_ev[u + 1] - L->attr_ev[u]);
      total_ev += L->attr_ev[u + 1] - L->attr_ev[u];
    }
  }
  // groups of consecutive sub-logs whose accumulators (and variant records)
  // fit the memory budget
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  const size_t per_sub = (size_t)E * 40 + (size_t)A * 24 + 64 + (size_t)E * 8;
  const size_t rec_bytes = want_var ? 128 : 0;  // records, their sort and the variant table, per case
  // Into caller-owned arrays (which never move), a batch of many sub-logs
  // runs as a pipeline of about kBtStages groups: a group's result copies
  // (copy stream) overlap the next group's kernels (context stream). Two
  // groups' scratch is then alive at once, so each gets half the budget.
  const int stages = c->batch_stages ? c->batch_stages : kBtStages;
  const bool pipelined = caller && Q >= 64 && stages > 1;
  const size_t budget =
      std::max<size_t>(std::min<size_t>(fr / (pipelined ? 6 : 3), (size_t)(pipelined ? 16 : 32) << 30), per_sub);
  const int32_t group_cap = pipelined ? (Q + stages - 1) / stages : Q;
  std::vector<std::pair<int32_t, int32_t>> groups;
  {
    int32_t g0 = 0;
    size_t mem = 0;
    uint64_t recs = 0;
    for (int32_t i = 0; i < Q; ++i) {
      uint64_t ci = 0;
      for (const uint2 &rg : sub_ranges[i]) ci += rg.y - rg.x;
      const size_t m = per_sub + (size_t)ci * rec_bytes;
      if (i > g0 && (mem + m > budget || (want_var && recs + ci > (1ull << 31)) || i - g0 >= group_cap)) {
        groups.emplace_back(g0, i - g0);
        g0 = i;
        mem = 0;
        recs = 0;
      }
      mem += m;
      recs += ci;
    }
    groups.emplace_back(g0, Q - g0);
  }
  const uint64_t per_sm = (uint64_t)(c->batch_items_per_sm ? c->batch_items_per_sm : kBtItemsPerSm);
  const uint64_t W = std::max<uint64_t>(1 << 15, total_ev / ((uint64_t)c->num_sms * per_sm) + 1);
  bool overflow = false;
  // A group whose results are still being copied out: its scratch (the
  // copies' sources), the host vectors the copies land in, and the events
  // after its last work on each stream. Destroying it waits for both.
  struct Pending {
    std::unique_ptr<Scratch> S;
    std::vector<int64_t> goff;
    std::vector<unsigned long long> gcnt;
    std::vector<uint32_t> gvq, grow0;
    int32_t q0 = 0, Qg = 0;
    size_t base = 0, vbase = 0;
    cudaEvent_t ev_s = nullptr, ev_cs = nullptr;
    ~Pending() {
      if (ev_s) cudaEventSynchronize(ev_s);
      if (ev_cs) cudaEventSynchronize(ev_cs);
      if (ev_s) cudaEventDestroy(ev_s);
      if (ev_cs) cudaEventDestroy(ev_cs);
    }
  };
  // Waits for a group's copies and fills the per-sub-log host results.
  auto finish = [&](Pending &p) -> int {
    cudaError_t ce = cudaEventSynchronize(p.ev_s);
    const cudaError_t ce2 = cudaEventSynchronize(p.ev_cs);
    if (ce == cudaSuccess) ce = ce2;
    if (ce != cudaSuccess) {
      set_error("pm4g_batch_dfg: result copy failed: %s", cudaGetErrorString(ce));
      return PM4G_ECUDA;
    }
    for (int32_t q = 0; q < p.Qg; ++q) {
      out->n_events[p.q0 + q] = (int64_t)p.gcnt[q];
      out->n_cases[p.q0 + q] = (int64_t)p.gcnt[p.Qg + q];
      out->edge_off[p.q0 + q] = (int64_t)p.base + p.goff[q];
    }
    out->edge_off[p.q0 + p.Qg] = (int64_t)p.base + p.goff[p.Qg];
    if (want_var) {
      for (int32_t q = 0; q < p.Qg; ++q) {
        out->n_variants[p.q0 + q] = p.gvq[q];
        out->var_off[p.q0 + q] = (int64_t)p.vbase + p.grow0[q];
      }
      out->var_off[p.q0 + p.Qg] = (int64_t)p.vbase + p.grow0[p.Qg];
    }
    return PM4G_OK;
  };
  std::unique_ptr<Pending> prev;
  for (const auto &grp : groups) {
    if (st != PM4G_OK) break;
    const int32_t q0 = grp.first, Qg = grp.second;
    Plan P;
    for (int32_t q = 0; q < Qg; ++q) {
      const int32_t i = q0 + q;
      uint32_t r_first = (uint32_t)P.ranges.size();
      uint64_t ev = 0;
      auto close = [&]() {
        if ((uint32_t)P.ranges.size() > r_first)
          P.items.push_back(make_uint4((uint32_t)q, r_first, (uint32_t)P.ranges.size(), (uint32_t)std::min<uint64_t>(ev, 0xFFFFFFFFu)));
        r_first = (uint32_t)P.ranges.size();
        ev = 0;
      };
      for (size_t r = 0; r < sub_ranges[i].size(); ++r) {
        const uint2 rg = sub_ranges[i][r];
        const uint64_t rev = sub_ev[i][r];
        const uint32_t ncase = rg.y - rg.x;
        if (ncase == 0) continue;
        // split a large range into pieces of about W events
        const uint64_t pieces = std::max<uint64_t>(1, (rev + W - 1) / W);
        const uint32_t step = (uint32_t)((ncase + pieces - 1) / pieces);
        for (uint32_t k = rg.x; k < rg.y; k += step) {
          const uint32_t k1 = std::min(rg.y, k + step);
          const uint64_t pev = rev * (k1 - k) / ncase;
          if (ev > 0 && ev + pev > W) close();
          P.ranges.push_back(make_uint2(k, k1));
          P.rbase.push_back(P.n_rec);
          P.n_rec += k1 - k;
          ev += pev;
        }
      }
      close();
    }
    std::stable_sort(P.items.begin(), P.items.end(), [](const uint4 &x, const uint4 &y) { return x.w > y.w; });
    const uint64_t cellsg = (uint64_t)Qg * E;
    auto Sp = std::make_unique<Scratch>(c);
    Scratch &S = *Sp;
    unsigned long long *acc = S.get<unsigned long long>(5 * cellsg);
    unsigned long long *se = S.get<unsigned long long>(3 * (size_t)Qg * A);  // start, end, freq
    unsigned long long *cnts = S.get<unsigned long long>(2 * (size_t)Qg);
    uint4 *ditems = S.get<uint4>(P.items.size());
    uint2 *dranges = S.get<uint2>(P.ranges.size());
    uint32_t *dwork = S.get<uint32_t>(1);
    int64_t *dtlo = S.get<int64_t>(Qg), *dthi = S.get<int64_t>(Qg);
    int32_t *dmode = S.get<int32_t>(Qg);
    uint32_t *drbase = nullptr, *rq = nullptr, *rslot = nullptr, *rpos = nullptr, *rlen = nullptr;
    uint64_t *rhash = nullptr;
    if (want_var) {
      drbase = S.get<uint32_t>(P.rbase.size());
      rq = S.get<uint32_t>(P.n_rec);
      rslot = S.get<uint32_t>(P.n_rec);
      rpos = S.get<uint32_t>(P.n_rec);
      rlen = S.get<uint32_t>(P.n_rec);
      rhash = S.get<uint64_t>(P.n_rec);
      if (!drbase || !rq || !rslot || !rpos || !rlen || !rhash) {
        set_error("pm4g_batch_dfg: out of device memory for variant records");
        st = PM4G_ENOMEM;
        break;
      }
      if (!P.rbase.empty() && cudaMemcpyAsync(drbase, P.rbase.data(), P.rbase.size() * 4, cudaMemcpyHostToDevice,
                                              c->stream) != cudaSuccess) {
        st = PM4G_ECUDA;
        break;
      }
    }
    if (!acc || !se || !cnts || !ditems || !dranges || !dwork || !dtlo || !dthi || !dmode) {
      set_error("pm4g_batch_dfg: out of device memory");
      st = PM4G_ENOMEM;
      break;
    }
    cudaStream_t s = c->stream;
    if (cudaMemsetAsync(acc, 0, 3 * cellsg * 8, s) != cudaSuccess ||
        cudaMemsetAsync(acc + 3 * cellsg, 0xFF, cellsg * 8, s) != cudaSuccess ||
        cudaMemsetAsync(acc + 4 * cellsg, 0, cellsg * 8, s) != cudaSuccess ||
        cudaMemsetAsync(se, 0, 3 * (size_t)Qg * A * 8, s) != cudaSuccess ||
        cudaMemsetAsync(cnts, 0, 2 * (size_t)Qg * 8, s) != cudaSuccess ||
        cudaMemsetAsync(dwork, 0, 4, s) != cudaSuccess ||
        (!P.items.empty() &&
         cudaMemcpyAsync(ditems, P.items.data(), P.items.size() * sizeof(uint4), cudaMemcpyHostToDevice, s) != cudaSuccess) ||
        (!P.ranges.empty() &&
         cudaMemcpyAsync(dranges, P.ranges.data(), P.ranges.size() * sizeof(uint2), cudaMemcpyHostToDevice, s) != cudaSuccess) ||
        cudaMemcpyAsync(dtlo, spec->t_lo + q0, (size_t)Qg * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(dthi, spec->t_hi + q0, (size_t)Qg * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(dmode, spec->mode + q0, (size_t)Qg * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      set_error("pm4g_batch_dfg: copy failed: %s", cudaGetErrorString(cudaGetLastError()));
      st = PM4G_ECUDA;
      break;
    }
    BatchArgs a{};
    a.aslots = L->aslots.p;
    a.aoff = L->aoff.p;
    a.alen = L->alen.p;
    a.act_s = L->act_s.p;
    a.ts_s = L->ts_s.p;
    a.eidx_s = L->eidx_s.p;
    a.n_act = A;
    a.a_s = A <= 2048 ? A : 0;
    a.n_edges = E;
    a.items = ditems;
    a.n_items = (uint32_t)P.items.size();
    a.ranges = dranges;
    a.work = dwork;
    a.t_lo = dtlo;
    a.t_hi = dthi;
    a.mode = dmode;
    a.acc = DfgTable{acc, acc + cellsg, acc + 2 * cellsg, acc + 3 * cellsg, acc + 4 * cellsg};
    a.start = se;
    a.end = se + (size_t)Qg * A;
    a.n_ev = cnts;
    a.n_cs = cnts + Qg;
    a.rbase = drbase;
    a.rq = rq;
    a.rslot = rslot;
    a.rpos = rpos;
    a.rlen = rlen;
    a.rhash = rhash;
    unsigned long long *freq = se + 2 * (size_t)Qg * A;
    if (!P.items.empty()) {
      const size_t smem = bt_smem_bytes(A <= 2048 ? A : 0);
      const int chunk = c->batch_chunk ? c->batch_chunk : kBtChunk;
      void (*kern)(BatchArgs) = chunk == 8 ? k_batch_dfg<8> : chunk == 32 ? k_batch_dfg<32> : k_batch_dfg<16>;
      if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin_max()) != cudaSuccess) {
        set_error("pm4g_batch_dfg: shared memory attribute: %s", cudaGetErrorString(cudaGetLastError()));
        st = PM4G_ECUDA;
        break;
      }
      KTime t(c, "batch_dfg");
      kern<<<std::min<unsigned>(a.n_items, (unsigned)c->num_sms), kBtThreads, smem, s>>>(a);
      if ((st = check_launch(c, "k_batch_dfg")) != PM4G_OK) break;
    }
    // compaction of the group's edges, sub-log by sub-log in edge order
    uint32_t *flags = S.get<uint32_t>(cellsg), *pos = S.get<uint32_t>(cellsg + 1);
    int64_t *doff = S.get<int64_t>((size_t)Qg + 1);
    if (!flags || !pos || !doff) {
      st = PM4G_ENOMEM;
      break;
    }
    const unsigned gN = grid_for((int64_t)cellsg, 256, 65535);
    {
      KTime t(c, "batch");
      k_bt_flags<<<gN, 256, 0, s>>>(acc, cellsg, flags);
      if ((st = check_launch(c, "k_bt_flags")) != PM4G_OK) break;
    }
    if ((st = scan_u32(c, flags, pos, (int64_t)cellsg)) != PM4G_OK) break;
    uint32_t Eg = 0;
    if ((st = d2h(c, &Eg, pos + cellsg, 4)) != PM4G_OK) break;
    int32_t *osrc = S.get<int32_t>(Eg), *odst = S.get<int32_t>(Eg);
    unsigned long long *o5 = S.get<unsigned long long>(5 * (size_t)Eg);
    double *omean = S.get<double>(Eg);
    if (!osrc || !odst || !o5 || !omean) {
      st = PM4G_ENOMEM;
      break;
    }
    {
      KTime t(c, "batch");
      k_bt_compact<<<gN, 256, 0, s>>>(a.acc, flags, pos, cellsg, E, A, L->e_pair.p, osrc, odst, o5, o5 + Eg,
                                      o5 + 2 * (size_t)Eg, o5 + 3 * (size_t)Eg, o5 + 4 * (size_t)Eg, omean, freq);
      if ((st = check_launch(c, "k_bt_compact")) != PM4G_OK) break;
      k_bt_add<<<grid_for((int64_t)Qg * A, 256, 65535), 256, 0, s>>>(freq, a.end, (uint64_t)Qg * A);
      if ((st = check_launch(c, "k_bt_add")) != PM4G_OK) break;
      k_bt_offsets<<<grid_for((int64_t)Qg + 1, 256, 65535), 256, 0, s>>>(pos, (uint32_t)Qg, E, doff);
      if ((st = check_launch(c, "k_bt_offsets")) != PM4G_OK) break;
    }
    // The group's edge and endpoint results are final: they are copied out on
    // the copy stream while the variant kernels run on the context stream.
    const size_t base = Et;
    const bool fits = !overflow && room(base + Eg);
    if (!fits) {
      if (!caller) {
        st = PM4G_ENOMEM;
        break;
      }
      overflow = true;  // keep counting to report the size needed
    }
    std::vector<int64_t> goff((size_t)Qg + 1);
    std::vector<unsigned long long> gcnt(2 * (size_t)Qg);
    cudaError_t ce = cudaSuccess;
    if (!c->copy_stream && cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
      c->copy_stream = nullptr;
      st = PM4G_ECUDA;
      break;
    }
    if (!c->copy_ready && cudaEventCreateWithFlags(&c->copy_ready, cudaEventDisableTiming) != cudaSuccess) {
      c->copy_ready = nullptr;
      st = PM4G_ECUDA;
      break;
    }
    cudaStream_t cs = c->copy_stream;
    ce = cudaEventRecord(c->copy_ready, s);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(cs, c->copy_ready, 0);
    auto cpc = [&](void *dst, const void *src, size_t bytes) {
      if (ce == cudaSuccess && bytes) ce = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, cs);
    };
    if (fits) {
      cpc(out->src + base, osrc, (size_t)Eg * 4);
      cpc(out->dst + base, odst, (size_t)Eg * 4);
      cpc(out->count + base, o5, (size_t)Eg * 8);
      cpc(out->sum_lo + base, o5 + Eg, (size_t)Eg * 8);
      cpc(out->sum_hi + base, o5 + 2 * (size_t)Eg, (size_t)Eg * 8);
      cpc(out->min + base, o5 + 3 * (size_t)Eg, (size_t)Eg * 8);
      cpc(out->max + base, o5 + 4 * (size_t)Eg, (size_t)Eg * 8);
      cpc(out->mean + base, omean, (size_t)Eg * 8);
    }
    cpc(out->start + (size_t)q0 * A, a.start, (size_t)Qg * A * 8);
    cpc(out->end + (size_t)q0 * A, a.end, (size_t)Qg * A * 8);
    cpc(out->freq + (size_t)q0 * A, freq, (size_t)Qg * A * 8);
    // leaving the group by any path waits for these copies before the
    // group's scratch (their sources) goes back to the block cache
    struct CopyWait {
      cudaStream_t cs;
      bool armed;
      ~CopyWait() {
        if (armed) cudaStreamSynchronize(cs);
      }
    } copy_wait{cs, true};
    // variants of the group's sub-logs
    uint32_t rows_g = 0, acts_g = 0;
    uint32_t *vq = nullptr, *row0 = nullptr, *o_seq = nullptr;
    int64_t *o_seq64 = nullptr;
    unsigned long long *o_count = nullptr;
    int32_t *o_min = nullptr, *o_acts = nullptr;
    if (want_var) {
      const uint32_t NR = P.n_rec;
      uint32_t *kf = S.get<uint32_t>(NR), *kp = S.get<uint32_t>((size_t)NR + 1);
      vq = S.get<uint32_t>(Qg);
      row0 = S.get<uint32_t>((size_t)Qg + 1);
      uint32_t *take = S.get<uint32_t>(Qg), *vstart = S.get<uint32_t>((size_t)Qg + 1);
      if (!kf || !kp || !vq || !row0 || !take || !vstart) {
        st = PM4G_ENOMEM;
        break;
      }
      const unsigned gR = grid_for((int64_t)NR, 256, 65535);
      if (NR) {
        KTime t(c, "variants");
        k_bv_flags<<<gR, 256, 0, s>>>(rlen, NR, kf);
        if ((st = check_launch(c, "k_bv_flags")) != PM4G_OK) break;
      }
      if ((st = scan_u32(c, kf, kp, (int64_t)NR)) != PM4G_OK) break;
      uint32_t NK = 0;
      if ((st = d2h(c, &NK, kp + NR, 4)) != PM4G_OK) break;
      uint64_t *k64 = S.get<uint64_t>(NK), *k64b = S.get<uint64_t>(NK);
      uint32_t *idx = S.get<uint32_t>(NK), *idxb = S.get<uint32_t>(NK);
      uint32_t *sq = S.get<uint32_t>(NK), *sslot = S.get<uint32_t>(NK), *spos = S.get<uint32_t>(NK);
      uint32_t *slen = S.get<uint32_t>(NK), *rep_of = S.get<uint32_t>(NK), *vcount = S.get<uint32_t>(NK);
      uint64_t *shash = S.get<uint64_t>(NK);
      uint32_t *rf = S.get<uint32_t>(NK), *rp = S.get<uint32_t>((size_t)NK + 1);
      if (!k64 || !k64b || !idx || !idxb || !sq || !sslot || !spos || !slen || !rep_of || !vcount || !shash || !rf ||
          !rp) {
        set_error("pm4g_batch_dfg: out of device memory for variants");
        st = PM4G_ENOMEM;
        break;
      }
      const unsigned gK = grid_for((int64_t)NK, 256, 65535);
      const int sbits = std::max(1, bits_for(L->R - 1));  // bits of a case slot
      if (NK) {
        {
          KTime t(c, "variants");
          k_bv_keys<<<gR, 256, 0, s>>>(rlen, rq, rslot, kp, NR, sbits, k64, idx);
          if ((st = check_launch(c, "k_bv_keys")) != PM4G_OK) break;
        }
        const int qb = bits_for((uint64_t)std::max(Qg - 1, 0));
        if ((st = radix_sort_u64(c, k64, idx, k64b, idxb, NK, 0, sbits + qb)) != PM4G_OK) break;
        KTime t(c, "variants");
        k_bv_gather<<<gK, 256, 0, s>>>(idx, NK, rq, rslot, rpos, rlen, rhash, sq, sslot, spos, slen, shash);
        if ((st = check_launch(c, "k_bv_gather")) != PM4G_OK) break;
      }
      VarArgs va{};
      va.n_slots = NK;
      va.len = slen;
      va.hash = shash;
      va.off = spos;
      va.act_s = L->act_s.p;
      va.bits = c->test_hash_bits;
      va.rep_of = rep_of;
      va.vcount = vcount;
      va.cls = sq;
      if (NK && (st = group_variants(c, va, NK)) != PM4G_OK) break;
      if (NK) {
        KTime t(c, "variants");
        k_rep_flags<<<gK, 256, 0, s>>>(va, rf);
        if ((st = check_launch(c, "k_rep_flags")) != PM4G_OK) break;
      }
      if ((st = scan_u32(c, rf, rp, (int64_t)NK)) != PM4G_OK) break;
      uint32_t V = 0;
      if ((st = d2h(c, &V, rp + NK, 4)) != PM4G_OK) break;
      uint32_t *rep_idx = S.get<uint32_t>(V), *ck = S.get<uint32_t>(V), *ckb = S.get<uint32_t>(V);
      uint32_t *order = S.get<uint32_t>(V), *orderb = S.get<uint32_t>(V), *qk = S.get<uint32_t>(V);
      if (!rep_idx || !ck || !ckb || !order || !orderb || !qk) {
        st = PM4G_ENOMEM;
        break;
      }
      if (cudaMemsetAsync(vq, 0, (size_t)Qg * 4, s) != cudaSuccess ||
          cudaMemsetAsync(vstart, 0, ((size_t)Qg + 1) * 4, s) != cudaSuccess) {
        st = PM4G_ECUDA;
        break;
      }
      if (V) {
        const int cbits = bits_for((uint64_t)NK);
        const uint32_t cmask = cbits >= 32 ? 0xFFFFFFFFu : ((1u << cbits) - 1);
        {
          KTime t(c, "variants");
          k_rep_compact<<<gK, 256, 0, s>>>(va, rf, rp, cmask, rep_idx, ck, order);
          if ((st = check_launch(c, "k_rep_compact")) != PM4G_OK) break;
        }
        // (sub-log asc, count desc, smallest case asc): stable sort by count,
        // then by sub-log; representatives start in (sub-log, case) order
        if ((st = radix_sort_u32(c, ck, order, ckb, orderb, V, 0, cbits)) != PM4G_OK) break;
        {
          KTime t(c, "variants");
          k_bv_qkeys<<<grid_for(V, 256, 65535), 256, 0, s>>>(order, rep_idx, sq, V, qk);
          if ((st = check_launch(c, "k_bv_qkeys")) != PM4G_OK) break;
        }
        const int qb = bits_for((uint64_t)std::max(Qg - 1, 0));
        if (qb > 0 && (st = radix_sort_u32(c, qk, order, ckb, orderb, V, 0, qb)) != PM4G_OK) break;
        KTime t(c, "variants");
        k_bv_bounds<<<grid_for(V, 256, 65535), 256, 0, s>>>(qk, V, vstart, vq);
        if ((st = check_launch(c, "k_bv_bounds")) != PM4G_OK) break;
        k_bv_counts<<<grid_for(Qg, 256, 65535), 256, 0, s>>>(vstart, (uint32_t)Qg, vq);
        if ((st = check_launch(c, "k_bv_counts")) != PM4G_OK) break;
      }
      {
        KTime t(c, "variants");
        k_bv_take<<<grid_for(Qg, 256, 65535), 256, 0, s>>>(vq, (uint32_t)Qg, spec->var_top_k, take);
        if ((st = check_launch(c, "k_bv_take")) != PM4G_OK) break;
      }
      if ((st = scan_u32(c, take, row0, Qg)) != PM4G_OK) break;
      if ((st = d2h(c, &rows_g, row0 + Qg, 4)) != PM4G_OK) break;
      o_count = S.get<unsigned long long>(rows_g);
      o_min = S.get<int32_t>(rows_g);
      uint32_t *o_len = S.get<uint32_t>(rows_g), *o_rep = S.get<uint32_t>(rows_g);
      o_seq = S.get<uint32_t>((size_t)rows_g + 1);
      o_seq64 = S.get<int64_t>((size_t)rows_g + 1);
      if (!o_count || !o_min || !o_len || !o_rep || !o_seq || !o_seq64) {
        st = PM4G_ENOMEM;
        break;
      }
      if (V) {
        KTime t(c, "variants");
        k_bv_head<<<grid_for(V, 256, 65535), 256, 0, s>>>(order, qk, vstart, take, row0, rep_idx, vcount, sslot, slen,
                                                          V, L->min_case, L->uniq.p, o_count, o_min, o_len, o_rep);
        if ((st = check_launch(c, "k_bv_head")) != PM4G_OK) break;
      }
      if ((st = scan_u32(c, o_len, o_seq, rows_g)) != PM4G_OK) break;
      if ((st = d2h(c, &acts_g, o_seq + rows_g, 4)) != PM4G_OK) break;
      o_acts = S.get<int32_t>(acts_g);
      if (!o_acts) {
        st = PM4G_ENOMEM;
        break;
      }
      if (rows_g) {
        KTime t(c, "variants");
        k_bv_acts<<<grid_for(rows_g, 256, 65535), 256, 0, s>>>(o_rep, o_seq, spos, slen, L->act_s.p, rows_g, o_acts);
        if ((st = check_launch(c, "k_bv_acts")) != PM4G_OK) break;
      }
    }
    // The group's remaining results go out on the copy stream too, after the
    // variant kernels: the context stream carries no copy that the next
    // group's kernels would queue behind.
    std::vector<uint32_t> gvq, grow0;
    bool vfits = false;
    const size_t vbase = Vt, abase = At;
    if (want_var) {
      vfits = !overflow && room_var(vbase + rows_g, abase + acts_g);
      if (!vfits && !caller) {
        st = PM4G_ENOMEM;
        break;
      }
      if (!vfits) overflow = true;
      gvq.resize(Qg);
      grow0.resize((size_t)Qg + 1);
      if (vfits && rows_g + 1 > 0) {
        k_bv_seq64<<<grid_for((int64_t)rows_g + 1, 256, 65535), 256, 0, s>>>(o_seq, rows_g + 1, (int64_t)abase,
                                                                            o_seq64);
        if (ce == cudaSuccess) ce = cudaGetLastError();
      }
    }
    if (ce == cudaSuccess) ce = cudaEventRecord(c->copy_ready, s);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(cs, c->copy_ready, 0);
    cpc(goff.data(), doff, ((size_t)Qg + 1) * 8);
    cpc(gcnt.data(), cnts, 2 * (size_t)Qg * 8);
    if (want_var) {
      cpc(gvq.data(), vq, (size_t)Qg * 4);
      cpc(grow0.data(), row0, ((size_t)Qg + 1) * 4);
      if (vfits) {
        cpc(out->var_seq_off + vbase, o_seq64, ((size_t)rows_g + 1) * 8);
        cpc(out->var_count + vbase, o_count, (size_t)rows_g * 8);
        cpc(out->var_min_case + vbase, o_min, (size_t)rows_g * 4);
        cpc(out->var_acts + abase, o_acts, (size_t)acts_g * 4);
      }
    }
    auto pend = std::make_unique<Pending>();
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&pend->ev_s, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&pend->ev_cs, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventRecord(pend->ev_s, s);
    if (ce == cudaSuccess) ce = cudaEventRecord(pend->ev_cs, cs);
    if (ce != cudaSuccess) {
      set_error("pm4g_batch_dfg: result copy failed: %s", cudaGetErrorString(ce));
      st = PM4G_ECUDA;
      break;
    }
    pend->S = std::move(Sp);
    pend->goff = std::move(goff);
    pend->gcnt = std::move(gcnt);
    pend->gvq = std::move(gvq);
    pend->grow0 = std::move(grow0);
    pend->q0 = q0;
    pend->Qg = Qg;
    pend->base = base;
    pend->vbase = vbase;
    copy_wait.armed = false;  // the pending group now waits for its copies
    Et = base + Eg;
    if (want_var) {
      Vt = vbase + rows_g;
      At = abase + acts_g;
    }
    if (prev) {
      st = finish(*prev);
      prev.reset();
      if (st != PM4G_OK) break;
    }
    prev = std::move(pend);
    if (!pipelined) {
      st = finish(*prev);
      prev.reset();
      if (st != PM4G_OK) break;
    }
  }
  if (prev) {
    if (st == PM4G_OK) st = finish(*prev);
    prev.reset();
  }
  if (st == PM4G_OK && !caller && (!room(Et) || !room_var(Vt, At))) st = PM4G_ENOMEM;  // arrays exist even when empty
  if (st != PM4G_OK) return fail_out(st);
  if (overflow) {
    if (want_var) out->acts_capacity = (int64_t)At;
    set_error("pm4g_batch_dfg_into: %zu edges, %zu variant rows, %zu activities do not fit the buffers", Et, Vt, At);
    return PM4G_ERANGE;
  }
  return PM4G_OK;
}

int pm4g_batch_dfg(pm4g_log *L, const pm4g_batch_spec *spec, pm4g_batch_dfg_t *out) {
  pm4g::ApiRange nvtx_range("pm4g_batch_dfg");
  return batch_dfg(L, spec, out, -1);
}

int pm4g_batch_dfg_into(pm4g_log *L, const pm4g_batch_spec *spec, pm4g_batch_dfg_t *out, int64_t edge_capacity) {
  pm4g::ApiRange nvtx_range("pm4g_batch_dfg_into");
  if (edge_capacity < 0) {
    set_error("pm4g_batch_dfg_into: negative edge capacity");
    return PM4G_EINVAL;
  }
  return batch_dfg(L, spec, out, edge_capacity);
}
