// Segment pass: per bucket, order the events by (case, timestamp, row) on chip
// and derive every summary in the same pass (Section 3: the second formatting
// step adds each event's previous activity and timestamp; the DFG, performance
// DFG, start/end activities and the per-case variant features follow from
// consecutive events of a case).
//
// One persistent CTA per SM takes buckets from a work counter. For a bucket it
//  1. loads the bucket's 16-byte records into shared memory;
//  2. counting-sorts them by case slot into an index array;
//  3. orders each case by (timestamp, row) with a warp bitonic sort (skipped
//     when the case is already in order, e.g. for time-ordered input);
//  4. walks the ordered positions warp by warp: writes the activity sequence,
//     counts start/end activities, forms the directly-follows pair
//     (a_i, a_{i+1}) with duration ts_{i+1} - ts_i, aggregates pairs of a warp
//     with equal edges (match + redux) into a shared-memory edge table, and
//     adds each event's term of the case's sequence hash.
// The shared edge table is dense over A*A cells when that fits, otherwise an
// open-addressing table keyed by src*A+dst; misses fall back to global
// atomics. Duration sums are exact: a 64-bit add whose carry-out is added to a
// high word. Minimum and maximum go straight to global memory, guarded by a
// plain read (a stale value is never wrong for a monotone min/max, it only
// costs an extra atomic).
//
// Buckets that do not fit (too many events, or a case longer than
// kMaxCaseSmem) are listed and handled by the global-memory path below, which
// sorts the bucket with the device radix sort and runs the same per-position
// code on global memory.
#include "device_common.cuh"
#include "engine.h"
#include "kernels.h"

namespace pm4g {

namespace {

constexpr uint32_t kEmptyKey = 0xFFFFFFFFu;

__device__ __forceinline__ void global_edge_group(const DfgTable &g, uint32_t key, uint32_t cnt, uint64_t lo,
                                                  uint64_t hi) {
  atomicAdd(&g.cnt[key], (unsigned long long)cnt);
  const unsigned long long old = atomicAdd(&g.lo[key], (unsigned long long)lo);
  const unsigned long long h2 = hi + (old + lo < old ? 1ull : 0ull);
  if (h2) atomicAdd(&g.hi[key], h2);
}

__device__ __forceinline__ void global_minmax(const DfgTable &g, uint32_t key, uint64_t d) {
  unsigned long long *pm = g.mn + key;
  if (d < *(volatile unsigned long long *)pm) atomicMin(pm, (unsigned long long)d);
  unsigned long long *px = g.mx + key;
  if (d > *(volatile unsigned long long *)px) atomicMax(px, (unsigned long long)d);
}

struct SmemSink {
  uint32_t *tkey, *tcnt, *thi;
  unsigned long long *tlo;
  uint32_t mask;
  int mode;
  uint32_t *st, *en;
  unsigned long long *chash;
  const SegArgs *a;

  __device__ __forceinline__ int find(uint32_t key) {
    if (mode == 0) return (int)key;
    uint32_t h = fmix32(key) & mask;
    for (int it = 0; it < 64; ++it) {
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
  __device__ __forceinline__ void edge_group(uint32_t key, uint32_t cnt, u128 sum) {
    const unsigned long long lo = (unsigned long long)sum;
    const uint32_t hi = (uint32_t)(sum >> 64);
    const int s = find(key);
    if (s >= 0) {
      atomicAdd(&tcnt[s], cnt);
      const unsigned long long old = atomicAdd(&tlo[s], lo);
      const uint32_t h2 = hi + (old + lo < old ? 1u : 0u);
      if (h2) atomicAdd(&thi[s], h2);
    } else {
      global_edge_group(a->g, key, cnt, lo, hi);
    }
  }
  __device__ __forceinline__ void start(uint32_t act) {
    if (st) atomicAdd(&st[act], 1u);
    else atomicAdd(&a->g_start[act], 1ull);
  }
  __device__ __forceinline__ void end(uint32_t act) {
    if (en) atomicAdd(&en[act], 1u);
    else atomicAdd(&a->g_end[act], 1ull);
  }
  __device__ __forceinline__ void hash_add(uint32_t c, uint64_t v) { atomicAdd(&chash[c], (unsigned long long)v); }
};

struct GlobalSink {
  const SegArgs *a;
  uint64_t slot_base;
  __device__ __forceinline__ void edge_group(uint32_t key, uint32_t cnt, u128 sum) {
    global_edge_group(a->g, key, cnt, (uint64_t)sum, (uint64_t)(sum >> 64));
  }
  __device__ __forceinline__ void start(uint32_t act) { atomicAdd(&a->g_start[act], 1ull); }
  __device__ __forceinline__ void end(uint32_t act) { atomicAdd(&a->g_end[act], 1ull); }
  __device__ __forceinline__ void hash_add(uint32_t c, uint64_t v) {
    atomicAdd((unsigned long long *)&a->hash[slot_base + c], (unsigned long long)v);
  }
};

// One warp handles 32 consecutive ordered positions p = base + lane of a
// bucket. fetch(p) returns the record at ordered position p; cstart[c] is the
// first ordered position of case slot c (cstart[ncl] = n).
template <bool kExport, class Sink, class Fetch>
__device__ __forceinline__ void process_warp_tile(const SegArgs &a, Sink &sink, const Fetch &fetch,
                                                  const uint32_t *cstart, int p, int n, int64_t out_base,
                                                  uint64_t slot_base, uint32_t act_mask) {
  const int lane = (int)lane_id();
  const bool valid = p < n;
  uint32_t c = 0xFFFFFFFFu, act = 0, row = 0, cs = 0, ce = 0;
  int64_t ts = 0;
  if (valid) {
    const uint4 r = fetch(p);
    c = r.x >> a.act_bits;
    act = r.x & act_mask;
    ts = rec_ts(r);
    row = r.y;
    cs = cstart[c];
    ce = cstart[c + 1];
  }
  if (kExport) {
    if (valid) {
      const uint64_t slot = slot_base + c;
      a.act_s[out_base + p] = (int32_t)act;
      a.ex_case[out_base + p] = a.uniq ? a.uniq[slot] : (int32_t)((uint32_t)a.min_case + (uint32_t)slot);
      a.ex_ts[out_base + p] = ts;
      a.ex_row[out_base + p] = (int64_t)row;
    }
    return;
  }
  const bool first = valid && (uint32_t)p == cs;
  const bool last = valid && (uint32_t)p + 1 == ce;
  if (valid) a.act_s[out_base + p] = (int32_t)act;
  if (first) sink.start(act);
  if (last) sink.end(act);
  const bool has_edge = valid && !last;
  uint32_t key = 0;
  uint64_t delta = 0;
  if (has_edge) {
    const uint4 r2 = fetch(p + 1);
    key = act * a.n_act + (r2.x & act_mask);
    delta = (uint64_t)rec_ts(r2) - (uint64_t)ts;
  }
  const uint32_t emask = __ballot_sync(kFull, has_edge);
  if (has_edge) {
    const uint32_t peers = __match_any_sync(emask, key);
    const u128 sum = peer_sum_u64(peers, delta);
    if (lane == __ffs(peers) - 1) sink.edge_group(key, (uint32_t)__popc(peers), sum);
    global_minmax(a.g, key, delta);
  }
  // variant hash: segmented inclusive sum over lanes holding the same case
  uint64_t v = valid ? event_hash(act, (uint32_t)p - cs, a.seed) : 0ull;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(kFull, v, o);
    const uint32_t cy = __shfl_up_sync(kFull, c, o);
    if (lane >= o && cy == c) v += y;
  }
  const uint32_t cn = __shfl_down_sync(kFull, c, 1);
  if (valid && (lane == 31 || cn != c)) sink.hash_add(c, v);
}

template <int E>
__device__ __forceinline__ void sort_case(const uint4 *rec_s, uint16_t *idx_s, uint32_t s0, uint32_t L) {
  uint64_t key[E];
  uint32_t row[E], pay[E];
  const int lane = (int)lane_id();
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t i = (uint32_t)(lane * E + e);
    if (i < L) {
      const uint32_t ix = idx_s[s0 + i];
      const uint4 r = rec_s[ix];
      key[e] = ts_key(rec_ts(r));
      row[e] = r.y;
      pay[e] = ix;
    } else {
      key[e] = ~0ull;
      row[e] = ~0u;
      pay[e] = 0;
    }
  }
  __syncwarp();
  warp_bitonic_sort<E>(key, row, pay);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t i = (uint32_t)(lane * E + e);
    if (i < L) idx_s[s0 + i] = (uint16_t)pay[e];
  }
  __syncwarp();
}

}  // namespace

template <bool kExport>
__global__ void __launch_bounds__(kSegThreads, 1) k_segment(SegArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int ncl = 1 << a.clb;
  const int a_s = a.ep_smem ? (int)a.n_act : 0;
  const SegSmem L = seg_smem_layout(a.cap, ncl, a_s, a.tbl_slots, a.tbl_mode);
  uint4 *rec_s = reinterpret_cast<uint4 *>(smem + L.rec);
  unsigned long long *tlo = reinterpret_cast<unsigned long long *>(smem + L.tlo);
  unsigned long long *chash = reinterpret_cast<unsigned long long *>(smem + L.chash);
  uint16_t *idx_s = reinterpret_cast<uint16_t *>(smem + L.idx);
  uint32_t *ccnt = reinterpret_cast<uint32_t *>(smem + L.ccnt);
  uint32_t *cstart = reinterpret_cast<uint32_t *>(smem + L.cstart);
  uint32_t *ccur = reinterpret_cast<uint32_t *>(smem + L.ccur);
  uint32_t *st = reinterpret_cast<uint32_t *>(smem + L.st);
  uint32_t *en = reinterpret_cast<uint32_t *>(smem + L.en);
  uint32_t *tkey = reinterpret_cast<uint32_t *>(smem + L.tkey);
  uint32_t *tcnt = reinterpret_cast<uint32_t *>(smem + L.tcnt);
  uint32_t *thi = reinterpret_cast<uint32_t *>(smem + L.thi);
  uint32_t *misc = reinterpret_cast<uint32_t *>(smem + L.misc);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kWarps = kSegThreads / 32;
  const uint32_t act_mask = (1u << a.act_bits) - 1;

  if (!kExport) {
    for (int i = tid; i < a.tbl_slots; i += kSegThreads) {
      tcnt[i] = 0;
      thi[i] = 0;
      tlo[i] = 0;
      if (a.tbl_mode) tkey[i] = kEmptyKey;
    }
    for (int i = tid; i < a_s; i += kSegThreads) {
      st[i] = 0;
      en[i] = 0;
    }
  }
  SmemSink sink{tkey, tcnt, thi, tlo, (uint32_t)(a.tbl_slots - 1), a.tbl_mode, a_s ? st : nullptr,
                a_s ? en : nullptr, chash, &a};
  __syncthreads();

  for (;;) {
    if (tid == 0) misc[0] = atomicAdd(a.work, 1u);
    __syncthreads();
    const uint32_t b = misc[0];
    if (b >= a.nb) break;
    const uint32_t lo = a.bucket_off[b];
    const uint32_t n = a.bucket_off[b + 1] - lo;
    if (n > (uint32_t)a.cap) {
      if (tid == 0) a.ovf[atomicAdd(a.n_ovf, 1u)] = b;
      __syncthreads();
      continue;
    }
    const uint4 *src = a.rec + lo;
    for (uint32_t i = tid; i < n; i += kSegThreads) rec_s[i] = __ldcs(src + i);
    for (int c = tid; c < ncl; c += kSegThreads) {
      ccnt[c] = 0;
      chash[c] = 0;
    }
    __syncthreads();
    for (uint32_t i = tid; i < n; i += kSegThreads) atomicAdd(&ccnt[rec_s[i].x >> a.act_bits], 1u);
    __syncthreads();
    {
      const int c0 = 2 * tid;
      const uint32_t v0 = c0 < ncl ? ccnt[c0] : 0u, v1 = c0 + 1 < ncl ? ccnt[c0 + 1] : 0u;
      uint32_t tot;
      const uint32_t pre = block_exclusive_scan<kSegThreads>(v0 + v1, misc + 8, tot);
      if (c0 < ncl) cstart[c0] = ccur[c0] = pre;
      if (c0 + 1 < ncl) cstart[c0 + 1] = ccur[c0 + 1] = pre + v0;
      if (tid == 0) cstart[ncl] = n;
      const int too_long = __syncthreads_or(max(v0, v1) > (uint32_t)kMaxCaseSmem);
      if (too_long) {
        if (tid == 0) a.ovf[atomicAdd(a.n_ovf, 1u)] = b;
        __syncthreads();
        continue;
      }
    }
    for (uint32_t i = tid; i < n; i += kSegThreads) {
      const uint32_t p = atomicAdd(&ccur[rec_s[i].x >> a.act_bits], 1u);
      idx_s[p] = (uint16_t)i;
    }
    __syncthreads();
    // order each case by (timestamp, row)
    for (int c = warp; c < ncl; c += kWarps) {
      const uint32_t Lc = ccnt[c];
      if (Lc < 2) continue;
      const uint32_t s0 = cstart[c];
      bool ok = true;
      for (uint32_t j = lane; j + 1 < Lc; j += 32) {
        const uint4 x = rec_s[idx_s[s0 + j]], y = rec_s[idx_s[s0 + j + 1]];
        if (!kr_less(ts_key(rec_ts(x)), x.y, ts_key(rec_ts(y)), y.y)) ok = false;
      }
      if (__all_sync(kFull, ok)) continue;
      if (Lc <= 32) sort_case<1>(rec_s, idx_s, s0, Lc);
      else if (Lc <= 64) sort_case<2>(rec_s, idx_s, s0, Lc);
      else if (Lc <= 128) sort_case<4>(rec_s, idx_s, s0, Lc);
      else if (Lc <= 256) sort_case<8>(rec_s, idx_s, s0, Lc);
      else sort_case<16>(rec_s, idx_s, s0, Lc);
    }
    __syncthreads();
    {
      const uint64_t slot_base = (uint64_t)b << a.clb;
      auto fetch = [&](int p) { return rec_s[idx_s[p]]; };
      for (int base = warp * 32; base < (int)n; base += kSegThreads)
        process_warp_tile<kExport>(a, sink, fetch, cstart, base + lane, (int)n, (int64_t)lo, slot_base, act_mask);
    }
    __syncthreads();
    if (!kExport) {
      const uint64_t slot0 = (uint64_t)b << a.clb;
      uint32_t present = 0;
      for (int c = tid; c < ncl; c += kSegThreads) {
        const uint64_t slot = slot0 + (uint64_t)c;
        if (slot < a.n_slots) {
          const uint32_t Lc = ccnt[c];
          a.len[slot] = Lc;
          a.hash[slot] = chash[c];
          if (a.cattr) a.cattr[slot] = (Lc && a.attr_in) ? a.attr_in[rec_s[idx_s[cstart[c]]].y] : 0;
          present += Lc ? 1u : 0u;
        }
      }
      present = __reduce_add_sync(kFull, present);
      if (lane == 0 && present) atomicAdd(a.n_cases, (unsigned long long)present);
    }
    __syncthreads();
  }
  if (!kExport) {
    for (int s = tid; s < a.tbl_slots; s += kSegThreads) {
      const uint32_t cnt = tcnt[s];
      if (cnt) global_edge_group(a.g, a.tbl_mode ? tkey[s] : (uint32_t)s, cnt, tlo[s], thi[s]);
    }
    for (int i = tid; i < a_s; i += kSegThreads) {
      if (st[i]) atomicAdd(&a.g_start[i], (unsigned long long)st[i]);
      if (en[i]) atomicAdd(&a.g_end[i], (unsigned long long)en[i]);
    }
  }
}

cudaError_t launch_segment(bool exp, const SegArgs &a, unsigned grid, size_t smem, cudaStream_t s) {
  cudaError_t e;
  if (exp) {
    e = cudaFuncSetAttribute(k_segment<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_segment<true><<<grid, kSegThreads, smem, s>>>(a);
  } else {
    e = cudaFuncSetAttribute(k_segment<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_segment<false><<<grid, kSegThreads, smem, s>>>(a);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Global-memory path for buckets that do not fit on chip.
// ---------------------------------------------------------------------------
__global__ void k_fb_keys_row(const uint4 *__restrict__ rec, uint32_t n, uint32_t *keys, uint32_t *vals) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    keys[i] = rec[i].y;
    vals[i] = i;
  }
}
__global__ void k_fb_keys_ts(const uint4 *__restrict__ rec, const uint32_t *__restrict__ perm, uint32_t n,
                             uint64_t *keys) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    keys[i] = ts_key(rec_ts(rec[perm[i]]));
}
__global__ void k_fb_keys_case(const uint4 *__restrict__ rec, const uint32_t *__restrict__ perm, uint32_t n,
                               int act_bits, uint32_t *keys) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    keys[i] = rec[perm[i]].x >> act_bits;
}
__global__ void k_fb_gather(const uint4 *__restrict__ rec, const uint32_t *__restrict__ perm, uint32_t n,
                            uint4 *out) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = rec[perm[i]];
}
__global__ void k_fb_hist(const uint4 *__restrict__ srec, uint32_t n, int act_bits, uint32_t *ccnt) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    atomicAdd(&ccnt[srec[i].x >> act_bits], 1u);
}

template <bool kExport>
__global__ void k_fb_compute(SegArgs a, const uint4 *__restrict__ srec, uint32_t n, uint32_t bucket,
                             const uint32_t *__restrict__ cstart) {
  const uint32_t act_mask = (1u << a.act_bits) - 1;
  GlobalSink sink{&a, (uint64_t)bucket << a.clb};
  const int64_t lo = a.bucket_off[bucket];
  auto fetch = [&](int p) { return srec[p]; };
  const int lane = threadIdx.x & 31;
  const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = wg * 32; base < (int64_t)n; base += nw * 32)
    process_warp_tile<kExport>(a, sink, fetch, cstart, (int)base + lane, (int)n, lo, sink.slot_base, act_mask);
}
cudaError_t launch_fb_compute(bool exp, const SegArgs &a, const uint4 *srec, uint32_t n, uint32_t bucket,
                              const uint32_t *cstart, unsigned grid, cudaStream_t s) {
  if (exp) k_fb_compute<true><<<grid, 256, 0, s>>>(a, srec, n, bucket, cstart);
  else k_fb_compute<false><<<grid, 256, 0, s>>>(a, srec, n, bucket, cstart);
  return cudaGetLastError();
}

__global__ void k_fb_cases(SegArgs a, const uint4 *__restrict__ srec, uint32_t bucket,
                           const uint32_t *__restrict__ ccnt, const uint32_t *__restrict__ cstart, int ncl,
                           int write_cases) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t present = 0;
  if (c < ncl && write_cases) {
    const uint64_t slot = ((uint64_t)bucket << a.clb) + (uint64_t)c;
    if (slot < a.n_slots) {
      const uint32_t Lc = ccnt[c];
      a.len[slot] = Lc;
      if (a.cattr) a.cattr[slot] = (Lc && a.attr_in) ? a.attr_in[srec[cstart[c]].y] : 0;
      present = Lc ? 1u : 0u;
    }
  }
  present = __reduce_add_sync(kFull, present);
  if ((threadIdx.x & 31) == 0 && present) atomicAdd(a.n_cases, (unsigned long long)present);
}

__global__ void k_fill_u64(unsigned long long *p, int64_t n, unsigned long long v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

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
      const uint32_t c = r.x >> a.act_bits;
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
  const uint64_t slot = ((uint64_t)b << a.clb) + (r.x >> a.act_bits);
  if (!a.case_ok[slot]) return false;
  if (a.mode == PM4G_TW_EVENTS) {
    const int64_t t = rec_ts(r);
    return t >= a.t_lo && t <= a.t_hi;
  }
  return true;
}

__global__ void __launch_bounds__(256) k_filter_count(FilterArgs a) {
  for (uint32_t b = blockIdx.x; b < a.nb; b += gridDim.x) {
    const uint32_t lo = a.bucket_off[b], hi = a.bucket_off[b + 1];
    uint32_t k = 0;
    for (uint32_t i = lo + threadIdx.x; i < hi; i += blockDim.x) k += filter_keep(a, b, a.rec[i]) ? 1u : 0u;
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
    for (uint32_t t0 = lo; t0 < hi; t0 += blockDim.x) {
      const uint32_t i = t0 + threadIdx.x;
      uint4 r = make_uint4(0, 0, 0, 0);
      bool keep = false;
      if (i < hi) {
        r = a.rec[i];
        keep = filter_keep(a, b, r);
      }
      uint32_t tot;
      const uint32_t pre = block_exclusive_scan<256>(keep ? 1u : 0u, s_warp, tot);
      if (keep) a.out[out + pre] = r;
      out += tot;
    }
  }
}

}  // namespace pm4g
