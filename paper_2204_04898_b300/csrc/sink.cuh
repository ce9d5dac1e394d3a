// Directly-follows pair aggregation shared by the segment pass and the
// batched drill-down: a shared-memory table of per-edge sums with exact
// 128-bit durations (see the segment pass for the layout), its global
// fallbacks, and the warp-level pre-aggregation of equal edges.
#pragma once

#include "device_common.cuh"
#include "kernels.h"

namespace pm4g {

constexpr uint32_t kEmptyKey = 0xFFFFFFFFu;

// Index of a pair's cell in the global table: the key itself when the table
// is dense; otherwise the slot holding key + 1, claimed by compare-and-swap
// when the pair is new (~0 if the table is full, which the host's sizing
// rules out and the error word reports).
__device__ __forceinline__ uint64_t g_index(const DfgTable &g, uint32_t key) {
  if (!g.key) return key;
  const unsigned long long k1 = (unsigned long long)key + 1ull;
  uint64_t h = fmix64(k1) & g.mask;
  for (uint64_t it = 0; it <= g.mask; ++it) {
    const unsigned long long k = *(volatile unsigned long long *)&g.key[h];
    if (k == k1) return h;
    if (k == 0) {
      const unsigned long long old = atomicCAS(&g.key[h], 0ull, k1);
      if (old == 0 || old == k1) return h;
    }
    h = (h + 1) & g.mask;
  }
  atomicOr(g.err, 1u);
  return ~0ull;
}

__device__ __forceinline__ void global_sum_at(const DfgTable &g, uint64_t i, uint64_t lo, uint64_t hi) {
  const unsigned long long old = atomicAdd(&g.lo[i], (unsigned long long)lo);
  const unsigned long long h2 = hi + (old + lo < old ? 1ull : 0ull);
  if (h2) red_add_u64(&g.hi[i], h2);
}

// Adds cnt pairs with exact sum (hi:lo) and extremes mn, mx to the pair's cell.
__device__ __forceinline__ void global_edge_add(const DfgTable &g, uint32_t key, uint32_t cnt, uint64_t lo,
                                                uint64_t hi, uint64_t mn, uint64_t mx) {
  const uint64_t i = g_index(g, key);
  if (i == ~0ull) return;
  red_add_u64(&g.cnt[i], cnt);
  global_sum_at(g, i, lo, hi);
  red_min_u64(&g.mn[i], mn);
  red_max_u64(&g.mx[i], mx);
}

// The same without extremes (a shared table's flush: its extremes were pushed
// as they came).
__device__ __forceinline__ void global_edge_group(const DfgTable &g, uint32_t key, uint32_t cnt, uint64_t lo,
                                                  uint64_t hi) {
  const uint64_t i = g_index(g, key);
  if (i == ~0ull) return;
  red_add_u64(&g.cnt[i], cnt);
  global_sum_at(g, i, lo, hi);
}

struct SmemSink {
  uint32_t *tkey, *tcnt, *tminh, *tmaxh;  // tminh/tmaxh: float guards (device_common.cuh)
  uint32_t *tl, *tm;  // low and middle 32-bit words of the slot's sum
  uint32_t mask;
  uint32_t shift;  // 32 - log2(slots), for the multiplicative slot hash
  int mode;
  uint32_t *st, *en;
  DfgTable g;         // global accumulators (misses and carries)
  unsigned long long *g_start, *g_end;
  int probes = 64;    // hashed mode: slots tried before a pair goes to g

  __device__ __forceinline__ int find(uint32_t key) {
    if (mode == 0) return (int)key;
    if (key == kEmptyKey) return -1;  // the pair (65535, 65535) of a 65,536-activity log: global table
    uint32_t h = (key * 0x9E3779B1u) >> shift;
    for (int it = 0; it < probes; ++it) {
      const uint32_t k = *(volatile uint32_t *)&tkey[h];
      if (k == key) return (int)h;
      if (k == kEmptyKey) {
        const uint32_t old = atomicCAS(&tkey[h], kEmptyKey, key);
        if (old == kEmptyKey || old == key) return (int)h;
      }
      h = (h + 1) & mask;
    }
    return -1;
  }
  // The shared sum of a slot is two 32-bit words (low, middle) updated with
  // native 32-bit atomics; every carry out of bit 63 goes to the global high
  // word at once.
  __device__ __forceinline__ void edge_group(uint32_t key, uint32_t cnt, u128 sum, uint64_t mn, uint64_t mx) {
    const uint64_t lo64 = (uint64_t)sum;
    uint64_t top = (uint64_t)(sum >> 64);
    const int s = find(key);
    if (s >= 0) {
      atomicAdd(&tcnt[s], cnt);
      const uint32_t l = (uint32_t)lo64;
      const uint32_t old_l = atomicAdd(&tl[s], l);
      const uint64_t madd = (lo64 >> 32) + (old_l + l < old_l ? 1u : 0u);
      if (madd >> 32) {
        top += 1;
      } else if (madd) {
        const uint32_t old_m = atomicAdd(&tm[s], (uint32_t)madd);
        if (old_m + (uint32_t)madd < old_m) top += 1;
      }
      // extremes pushed (fire-and-forget) only when the float guards of what
      // this block already pushed allow them to improve
      const bool pmn = __float_as_uint(__ull2float_rd(mn)) < *(volatile uint32_t *)&tminh[s];
      const bool pmx = __float_as_uint(__ull2float_ru(mx)) > *(volatile uint32_t *)&tmaxh[s];
      if (top || pmn || pmx) {
        const uint64_t i = g_index(g, key);
        if (i != ~0ull) {
          if (top) red_add_u64(&g.hi[i], top);
          if (pmn) red_min_u64(&g.mn[i], mn);
          if (pmx) red_max_u64(&g.mx[i], mx);
        }
        if (pmn) atomicMin(&tminh[s], guard_up(mn));
        if (pmx) atomicMax(&tmaxh[s], guard_down(mx));
      }
    } else {
      global_edge_add(g, key, cnt, lo64, top, mn, mx);
    }
  }
  __device__ __forceinline__ void start(uint32_t act) {
    if (st) atomicAdd(&st[act], 1u);
    else atomicAdd(&g_start[act], 1ull);
  }
  __device__ __forceinline__ void end(uint32_t act) {
    if (en) atomicAdd(&en[act], 1u);
    else atomicAdd(&g_end[act], 1ull);
  }
};

// Aggregates the warp's directly-follows pairs with full-warp operations.
// Up to twice, the pending lanes whose edge equals the first pending lane's
// edge are reduced together (count, exact 128-bit sum, min, max; non-members
// add neutral values) when there are at least two of them. Then a single pass
// updates the sink: each group through its first lane, every other pending
// lane on its own.
template <class Sink>
__device__ __forceinline__ void aggregate_edges(Sink &sink, bool has_edge, uint32_t key, uint64_t d) {
  const int lane = (int)lane_id();
  uint32_t rem = __ballot_sync(kFull, has_edge);
  if (rem == 0) return;
  const uint32_t hi = (uint32_t)(d >> 32), lo = (uint32_t)d;
  uint32_t u_cnt = 1;
  u128 u_sum = (u128)d;
  uint64_t u_mn = d, u_mx = d;
  bool leader = false;
#pragma unroll
  for (int round = 0; round < 2; ++round) {
    if (rem == 0) break;
    const int src = __ffs(rem) - 1;
    const uint32_t cand = __shfl_sync(kFull, key, src);
    const bool mem = ((rem >> lane) & 1u) && key == cand;
    const uint32_t grp = __ballot_sync(kFull, mem);
    if (__popc(grp) < 2) break;
    const uint32_t s0 = __reduce_add_sync(kFull, mem ? (uint32_t)(d & 0x3FFFFF) : 0u);
    const uint32_t s1 = __reduce_add_sync(kFull, mem ? (uint32_t)((d >> 22) & 0x3FFFFF) : 0u);
    const uint32_t s2 = __reduce_add_sync(kFull, mem ? (uint32_t)(d >> 44) : 0u);
    const uint32_t mnh = __reduce_min_sync(kFull, mem ? hi : 0xFFFFFFFFu);
    const uint32_t mnl = __reduce_min_sync(kFull, (mem && hi == mnh) ? lo : 0xFFFFFFFFu);
    const uint32_t mxh = __reduce_max_sync(kFull, mem ? hi : 0u);
    const uint32_t mxl = __reduce_max_sync(kFull, (mem && hi == mxh) ? lo : 0u);
    if (lane == src) {
      u_cnt = (uint32_t)__popc(grp);
      u_sum = (u128)s0 + ((u128)s1 << 22) + ((u128)s2 << 44);
      u_mn = ((uint64_t)mnh << 32) | mnl;
      u_mx = ((uint64_t)mxh << 32) | mxl;
      leader = true;
    }
    rem &= ~grp;
  }
  if (leader || ((rem >> lane) & 1u)) sink.edge_group(key, u_cnt, u_sum, u_mn, u_mx);
}

}  // namespace pm4g
