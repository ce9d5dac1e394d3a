// Filters that return a sub-log (a new bucketed log formatted by the segment
// pass): the drill-down filter (Section 3, timestamp.py and attributes.py) and
// the filters on derived results (Section 3, the directly-follows, case and
// variant levels).

#include <cstdint>

#include "device_common.cuh"
#include "kernels.h"
#include "../../include/pm4g.h"

namespace pm4g {

// ---------------------------------------------------------------------------
// Drill-down filter (Section 3, timestamp.py / attributes.py).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_case_span(FilterArgs a) {
  extern __shared__ unsigned long long s_span[];
  const int ncl = 1 << a.clb;
  unsigned long long *mn = s_span, *mx = s_span + ncl;
  for (uint32_t b = blockIdx.x; b < a.nb; b += gridDim.x) {
    for (int c = threadIdx.x; c < ncl; c += blockDim.x) {
      mn[c] = ~0ull;
      mx[c] = 0ull;
    }
    __syncthreads();
    const uint32_t lo = a.bucket_off[b], hi = a.bucket_off[b + 1];
    for (uint32_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      const uint4 r = a.rec[i];
      const uint32_t c = (r.x >> a.act_bits) & ((1u << a.clb) - 1);
      const unsigned long long k = ts_key(rec_ts(r));
      atomicMin(&mn[c], k);
      atomicMax(&mx[c], k);
    }
    __syncthreads();
    const uint64_t slot0 = (uint64_t)b << a.clb;
    for (int c = threadIdx.x; c < ncl; c += blockDim.x) {
      const uint64_t slot = slot0 + (uint64_t)c;
      if (slot < a.n_slots) {
        a.first_ts[slot] = (int64_t)(mn[c] ^ 0x8000000000000000ULL);
        a.last_ts[slot] = (int64_t)(mx[c] ^ 0x8000000000000000ULL);
      }
    }
    __syncthreads();
  }
}

__global__ void k_case_ok(FilterArgs a) {
  for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.n_slots;
       s += (uint64_t)gridDim.x * blockDim.x) {
    bool ok = true;
    if (a.n_attr > 0) {
      const int32_t v = a.cattr[s];
      int lo = 0, hi = a.n_attr;  // first index with attr_set[i] >= v
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a.attr_set[mid] < v) lo = mid + 1;
        else hi = mid;
      }
      ok = lo < a.n_attr && a.attr_set[lo] == v;
    }
    const int64_t f = a.first_ts[s], l = a.last_ts[s];
    if (ok && a.mode == PM4G_TW_CASES_CONTAINED) ok = f >= a.t_lo && l <= a.t_hi;
    if (ok && a.mode == PM4G_TW_CASES_INTERSECTING) ok = f <= a.t_hi && l >= a.t_lo;
    a.case_ok[s] = ok ? 1 : 0;
  }
}

__device__ __forceinline__ bool filter_keep(const FilterArgs &a, uint32_t b, uint4 r) {
  if (a.row_keep) return (a.row_keep[r.y >> 5] >> (r.y & 31)) & 1u;
  const uint64_t slot = ((uint64_t)b << a.clb) + ((r.x >> a.act_bits) & ((1u << a.clb) - 1));
  if (!a.case_ok[slot]) return false;
  if (a.mode == PM4G_TW_EVENTS) {
    const int64_t t = rec_ts(r);
    return t >= a.t_lo && t <= a.t_hi;
  }
  return true;
}

// Kept events per bucket: a predicate on whole cases (no row flags, no event
// window) sums the lengths of the bucket's kept case slots; otherwise every
// record is tested.
__global__ void __launch_bounds__(256) k_filter_count(FilterArgs a) {
  const bool by_case = a.len && !a.row_keep && a.mode != PM4G_TW_EVENTS;
  for (uint32_t b = blockIdx.x; b < a.nb; b += gridDim.x) {
    uint32_t k = 0;
    if (by_case) {
      const uint64_t s0 = (uint64_t)b << a.clb, s1 = min((uint64_t)a.n_slots, s0 + ((uint64_t)1 << a.clb));
      for (uint64_t s = s0 + threadIdx.x; s < s1; s += blockDim.x) k += a.case_ok[s] ? a.len[s] : 0u;
    } else {
      const uint32_t lo = a.bucket_off[b], hi = a.bucket_off[b + 1];
      uint32_t i = lo + threadIdx.x;
      for (; i + 3 * blockDim.x < hi; i += 4 * blockDim.x) {  // four loads in flight
        uint4 r[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) r[u] = a.rec[i + u * blockDim.x];
#pragma unroll
        for (int u = 0; u < 4; ++u) k += filter_keep(a, b, r[u]) ? 1u : 0u;
      }
      for (; i < hi; i += blockDim.x) k += filter_keep(a, b, a.rec[i]) ? 1u : 0u;
    }
    k = __reduce_add_sync(kFull, k);
    __shared__ uint32_t s_k;
    if (threadIdx.x == 0) s_k = 0;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) atomicAdd(&s_k, k);
    __syncthreads();
    if (threadIdx.x == 0) a.kept[b] = s_k;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_filter_write(FilterArgs a) {
  __shared__ uint32_t s_warp[32];
  for (uint32_t b = blockIdx.x; b < a.nb; b += gridDim.x) {
    const uint32_t lo = a.bucket_off[b], hi = a.bucket_off[b + 1];
    uint32_t out = a.new_off[b];
    const uint32_t kept = a.new_off[b + 1] - out;
    if (kept == 0) continue;  // nothing of this bucket is kept
    if (kept == hi - lo) {    // all of it: a straight copy
      for (uint32_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const uint4 r = a.rec[i];
        a.out[out + (i - lo)] = r;
        if (a.keys_out) a.keys_out[out + (i - lo)] = r.x;
      }
      continue;
    }
    // 2,048 records a step: each warp takes 256 consecutive records, eight
    // rounds of 32 (one load each, all in flight before the tests); a
    // record's rank among the warp's kept ones comes from one ballot a round,
    // and one block scan of the eight warps' totals places the warps
    constexpr int kR = 8;
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5, lt = (1u << lane) - 1u;
    for (uint32_t t0 = lo; t0 < hi; t0 += 256 * kR) {
      const uint32_t wb = t0 + w * 32 * kR + lane;
      uint4 r[kR];
#pragma unroll
      for (int j = 0; j < kR; ++j)
        if (wb + 32 * j < hi) r[j] = a.rec[wb + 32 * j];
      uint32_t m[kR], cnt = 0;
#pragma unroll
      for (int j = 0; j < kR; ++j) {
        m[j] = __ballot_sync(kFull, wb + 32 * j < hi && filter_keep(a, b, r[j]));
        cnt += __popc(m[j]);
      }
      if (lane == 0) s_warp[w] = cnt;
      __syncthreads();
      uint32_t base = out, tot = 0;
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        const uint32_t c = s_warp[v];
        base += v < (int)w ? c : 0u;
        tot += c;
      }
      __syncthreads();  // s_warp is read before the next step writes it
#pragma unroll
      for (int j = 0; j < kR; ++j) {
        if ((m[j] >> lane) & 1u) {
          const uint32_t dst = base + __popc(m[j] & lt);
          a.out[dst] = r[j];
          if (a.keys_out) a.keys_out[dst] = r[j].x;
        }
        base += __popc(m[j]);
      }
      out += tot;
    }
  }
}

// ---------------------------------------------------------------------------
// Filters on derived results (Section 3: the case and variant levels, the
// directly-follows level).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool bit_of(const uint32_t *bits, uint32_t v) { return (bits[v >> 5] >> (v & 31)) & 1u; }

__global__ void k_case_filter(CaseFilterArgs a) {
  for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.n_slots;
       s += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t L = a.len[s];
    if (L == 0) {
      a.case_ok[s] = 0;  // no case: nothing to keep
      continue;
    }
    bool ok = true;
    if (a.min_events >= 0 && (int64_t)L < a.min_events) ok = false;
    if (a.max_events >= 0 && (int64_t)L > a.max_events) ok = false;
    const uint64_t dur = (uint64_t)a.last_ts[s] - (uint64_t)a.first_ts[s];
    if (a.min_duration >= 0 && dur < (uint64_t)a.min_duration) ok = false;
    if (a.max_duration >= 0 && dur > (uint64_t)a.max_duration) ok = false;
    const uint32_t o = a.off[s];
    if (ok && a.start_bits && !bit_of(a.start_bits, (uint32_t)a.act_s[o])) ok = false;
    if (ok && a.end_bits && !bit_of(a.end_bits, (uint32_t)a.act_s[o + L - 1])) ok = false;
    if (ok && a.act_bits) {
      bool any = false;
      for (uint32_t j = 0; j < L && !any; ++j) any = bit_of(a.act_bits, (uint32_t)a.act_s[o + j]);
      ok = any;
    }
    if (ok && a.n_variants > 0) {
      const int32_t v = a.cvar[s];
      int lo = 0, hi = a.n_variants;  // first index with variants[i] >= v
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a.variants[mid] < v) lo = mid + 1;
        else hi = mid;
      }
      ok = lo < a.n_variants && a.variants[lo] == v;
    }
    a.case_ok[s] = ok != (a.exclude != 0) ? 1 : 0;
  }
}

__global__ void k_mark_case_starts(const uint32_t *len, const uint32_t *off, uint64_t n_slots, uint8_t *start) {
  for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_slots;
       s += (uint64_t)gridDim.x * blockDim.x)
    if (len[s]) start[off[s]] = 1;
}

// An event at formatted position p > 0 that does not start its case has the
// event at p - 1 as its previous one; its pair key is prev * A + act.
__global__ void k_path_keep(uint64_t n, const uint16_t *act_s, const uint8_t *start, const int64_t *row_s,
                            const uint64_t *keys, int32_t n_keys, uint32_t n_act, int32_t exclude,
                            uint32_t *row_keep) {
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (uint64_t)gridDim.x * blockDim.x) {
    bool m = false;
    if (!start[p]) {
      const uint64_t key = (uint64_t)(uint32_t)act_s[p - 1] * n_act + (uint32_t)act_s[p];
      int lo = 0, hi = n_keys;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (keys[mid] < key) lo = mid + 1;
        else hi = mid;
      }
      m = lo < n_keys && keys[lo] == key;
    }
    // one bit per original row (the array, 1/8 of a byte per row, stays in
    // L2 for the random accesses); bits start clear and kept rows set theirs
    if (m != (exclude != 0)) {
      const uint64_t row = (uint64_t)row_s[p];
      atomicOr(&row_keep[row >> 5], 1u << (row & 31));
    }
  }
}

}  // namespace pm4g
