// Segment pass: per bucket, order the events by (case, timestamp, row) on chip
// and derive every summary in the same pass (Section 3: the second formatting
// step adds each event's previous activity and timestamp; the DFG, performance
// DFG, start/end activities and the per-case variant features follow from
// consecutive events of a case).
//
// One persistent 32-warp CTA per SM takes buckets from a work counter (the
// register budget is 64 per thread, which the sort paths below respect). For a
// bucket it
//  1. loads the bucket's 16-byte records into registers, each warp a
//     contiguous run of them (a bucket larger than the on-chip capacity is
//     processed in case-slot ranges that fit, streaming the bucket once per
//     range);
//  2. counting-sorts them by case slot, stably: per-warp counts over the
//     warps' runs, then each record goes from registers straight to its
//     ordered position in shared memory, in record order, so each case keeps
//     the order the scatter wrote, which is row order for most cases;
//  3. flags every case whose events are not in (timestamp, row) order and
//     sorts only those, one warp per case (warp bitonic sort in registers of
//     up to 128 events; longer cases merge sorted 128-event chunks by rank);
//  4. walks the ordered positions 32 at a time per warp: writes the activity
//     sequence, counts start/end activities, and forms the directly-follows
//     pair (a_i, a_{i+1}) with duration ts_{i+1} - ts_i and aggregates it.
// (The variant step forms each case's sequence hash from the activity
// sequence written here.)
// Pair aggregation uses full-warp operations only: twice, the lanes holding
// the same edge as the first pending lane are reduced together (count, exact
// sum, min, max) and one lane updates the table; the remaining lanes update it
// one by one (the hardware serialises equal addresses). The table lives in
// shared memory (dense over A*A cells when that fits, otherwise open
// addressing on src*A+dst; misses go to global atomics) and is flushed once
// per CTA. Sums are exact: 32-bit low and middle words with every carry out of
// bit 63 added to the global high word. Minimum and maximum are pushed to
// global memory with fire-and-forget reductions only when they can improve:
// the table keeps float guards of the extremes this CTA already pushed,
// rounded outward, and a value the guard shows cannot win is not pushed.
//
// Buckets holding a case longer than kMaxCaseSmem go to the global-memory path
// at the end of this file (device radix sort, then the same per-position code).
#include "device_common.cuh"
#include "engine.h"
#include "kernels.h"
#include "sink.cuh"

namespace pm4g {

namespace {

struct GlobalSink {
  const SegArgs *a;
  uint64_t slot_base;
  __device__ __forceinline__ void edge_group(uint32_t key, uint32_t cnt, u128 sum, uint64_t mn, uint64_t mx) {
    global_edge_add(a->g, key, cnt, (uint64_t)sum, (uint64_t)(sum >> 64), mn, mx);
  }
  __device__ __forceinline__ void start(uint32_t act) { atomicAdd(&a->g_start[act], 1ull); }
  __device__ __forceinline__ void end(uint32_t act) { atomicAdd(&a->g_end[act], 1ull); }
};

// One warp handles 32 consecutive ordered positions p = base + lane of a
// bucket. fetch(p) returns the record at ordered position p; cstart[c] is the
// first ordered position of case slot c (cstart[ncl] = n). Outputs go to
// ordered position out_base + p.
template <bool kExport, class Sink, class Fetch>
__device__ __forceinline__ void process_warp_tile(const SegArgs &a, Sink &sink, const Fetch &fetch,
                                                  const uint32_t *cstart, int p, int n, int64_t out_base,
                                                  uint64_t slot_base, uint32_t act_mask) {
  const int lane = (int)lane_id();
  const bool valid = p < n;
  uint32_t c = 0xFFFFFFFFu, act = 0, cs = 0, ce = 0;
  int64_t ts = 0;
  uint4 r = make_uint4(0, 0, 0, 0);
  if (valid) {
    r = fetch(p);
    c = (r.x >> a.act_bits) & ((1u << a.clb) - 1);
    act = r.x & act_mask;
    ts = rec_ts(r);
    cs = cstart[c];
    ce = cstart[c + 1];
  }
  if (kExport) {
    if (valid) {
      const uint64_t slot = slot_base + c;
      if (a.act_s) a.act_s[out_base + p] = (uint16_t)act;
      if (a.ex_case) a.ex_case[out_base + p] = a.uniq ? a.uniq[slot] : (int32_t)((uint32_t)a.min_case + (uint32_t)slot);
      if (a.ex_ts) a.ex_ts[out_base + p] = ts;
      if (a.ex_row) a.ex_row[out_base + p] = (int64_t)r.y;
    }
    return;
  }
  const bool first = valid && (uint32_t)p == cs;
  const bool last = valid && (uint32_t)p + 1 == ce;
  if (valid) a.act_s[out_base + p] = (uint16_t)act;
  if (first) sink.start(act);
  if (last) sink.end(act);
  // the next event of the case: the next lane's, or one fetch for lane 31
  uint32_t nx = __shfl_down_sync(kFull, r.x, 1);
  uint32_t nz = __shfl_down_sync(kFull, r.z, 1);
  uint32_t nw = __shfl_down_sync(kFull, r.w, 1);
  const bool has_edge = valid && !last;
  if (lane == 31 && has_edge) {
    const uint4 r2 = fetch(p + 1);
    nx = r2.x;
    nz = r2.z;
    nw = r2.w;
  }
  const int64_t nts = (int64_t)(((uint64_t)nw << 32) | nz);
  aggregate_edges(sink, has_edge, act * a.n_act + (nx & act_mask), (uint64_t)nts - (uint64_t)ts);
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

// Cases of 129..kMaxCaseSmem events: each 128-event chunk is sorted in
// registers, then every element moves to its rank, which is its position in
// its own chunk plus the number of smaller elements in each other chunk
// (binary search; (timestamp, row) keys are unique because rows are). All
// ranks are computed before any index is overwritten.
constexpr int kLongPerLane = kMaxCaseSmem / 32;
__device__ __forceinline__ void sort_long_case(const uint4 *rec_s, uint16_t *idx_s, uint32_t s0, uint32_t L) {
  for (uint32_t c0 = 0; c0 < L; c0 += 128) sort_case<4>(rec_s, idx_s, s0 + c0, min(128u, L - c0));
  const int lane = (int)lane_id();
  uint32_t pk[kLongPerLane];  // index (low 16 bits) and its rank (high 16 bits)
#pragma unroll
  for (int e = 0; e < kLongPerLane; ++e) {
    const uint32_t i = (uint32_t)(lane + 32 * e);
    pk[e] = 0;
    if (i < L) {
      const uint32_t v = idx_s[s0 + i];
      const uint4 r = rec_s[v];
      const uint64_t key = ts_key(rec_ts(r));
      const uint32_t own = i >> 7;
      uint32_t rank = i & 127u;
      for (uint32_t j = 0; j * 128 < L; ++j) {
        if (j == own) continue;
        const uint16_t *chunk = idx_s + s0 + j * 128;
        uint32_t lo = 0, hi = min(128u, L - j * 128);
        while (lo < hi) {
          const uint32_t mid = (lo + hi) >> 1;
          const uint4 q = rec_s[chunk[mid]];
          if (kr_less(ts_key(rec_ts(q)), q.y, key, r.y)) lo = mid + 1;
          else hi = mid;
        }
        rank += lo;
      }
      pk[e] = v | (rank << 16);
    }
  }
  __syncwarp();
#pragma unroll
  for (int e = 0; e < kLongPerLane; ++e)
    if ((uint32_t)(lane + 32 * e) < L) idx_s[s0 + (pk[e] >> 16)] = (uint16_t)(pk[e] & 0xFFFFu);
  __syncwarp();
}

struct SegShared {
  uint4 *rec;
  uint16_t *idx;
  uint32_t *ccnt, *cstart;
  uint8_t *flg;  // per case: events out of (timestamp, row) order
};

// Processes n_r records of bucket b, all with case slots in [c_a, c_b); their
// ordered positions start at out_base in the bucketed log. The records are
// read from global memory (src) or, when from_smem, from S.rec, where a case
// range of an oversized bucket was compacted. Each warp holds a contiguous
// run of them in registers while they are counted, and then writes each one
// straight to its ordered position in S.rec, so every later step reads S.rec
// in order. Returns false (having written nothing) if a case is too long to
// sort on chip.
template <bool kExport>
__device__ bool process_range(const SegArgs &a, SmemSink &sink, const SegShared &S, uint16_t *hw, uint32_t *misc,
                              const uint4 *src, bool from_smem, uint32_t b, uint32_t n_r, uint32_t c_a,
                              uint32_t c_b, int64_t out_base, uint32_t act_mask, uint32_t &n_sorted) {
  const int ncl = 1 << a.clb;
  const int hws = (ncl + 1) & ~1;  // per-warp row of 16-bit counts, 4-byte aligned
  const uint32_t cmask = (uint32_t)ncl - 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // warp w owns records [w_lo, w_hi), chunk k of it is w_lo + 32k + lane
  const uint32_t per = ((n_r + kSegWarps - 1) / kSegWarps + 31) & ~31u;  // at most 32 * kSegChunks
  const uint32_t w_lo = min(n_r, (uint32_t)warp * per), w_hi = min(n_r, w_lo + per);
  uint4 r[kSegChunks];
#pragma unroll
  for (int k = 0; k < kSegChunks; ++k) {
    const uint32_t i = w_lo + 32u * k + lane;
    r[k] = make_uint4(0, 0, 0, 0);
    if (i < w_hi) r[k] = from_smem ? S.rec[i] : __ldcs(src + i);
  }
  for (int j = tid; j < kSegWarps * hws; j += kSegThreads) hw[j] = 0;
  for (int c = tid; c < ncl; c += kSegThreads) {
    S.flg[c] = 0;
  }
  __syncthreads();
  // stable counting sort by case slot
  uint16_t *myh = hw + warp * hws;
  // myh holds 16-bit counts, two per 32-bit word (no count reaches 2^16)
  uint32_t *myw = reinterpret_cast<uint32_t *>(myh);
  // each record's rank among the warp's earlier records of its case (two
  // 16-bit ranks per word), kept for the placement below
  uint32_t lr[(kSegChunks + 1) / 2];
#pragma unroll
  for (int k = 0; k < (kSegChunks + 1) / 2; ++k) lr[k] = 0;
#pragma unroll
  for (int k = 0; k < kSegChunks; ++k) {
    if (w_lo + 32u * k < w_hi) {
      const bool v = w_lo + 32u * k + lane < w_hi;
      const uint32_t c = v ? ((r[k].x >> a.act_bits) & cmask) : 0xFFFFFFFFu;
      uint32_t run;
      const uint32_t head = run_head(c, run);
      uint32_t base = 0;
      if (v && (uint32_t)lane == head)
        base = (atomicAdd(&myw[c >> 1], run << (16 * (c & 1))) >> (16 * (c & 1))) & 0xFFFFu;
      base = __shfl_sync(kFull, base, (int)head);
      lr[k >> 1] |= (base + ((uint32_t)lane - head)) << (16 * (k & 1));
    }
  }
  __syncthreads();
  {
    uint32_t tot = 0;
    if (tid < ncl)
      for (int w = 0; w < kSegWarps; ++w) tot += hw[w * hws + tid];
    uint32_t all;
    const uint32_t pre = block_exclusive_scan<kSegThreads>(tot, misc + 8, all);
    if (tid < ncl) {
      S.ccnt[tid] = tot;
      S.cstart[tid] = pre;
      uint32_t run = pre;
      for (int w = 0; w < kSegWarps; ++w) {
        const uint32_t t = hw[w * hws + tid];
        hw[w * hws + tid] = (uint16_t)run;
        run += t;
      }
    }
    if (tid == 0) S.cstart[ncl] = n_r;
    if (__syncthreads_or(tot > (uint32_t)kMaxCaseSmem)) return false;
  }
  // myh now holds where the warp's records of each case start
#pragma unroll
  for (int k = 0; k < kSegChunks; ++k) {
    if (w_lo + 32u * k + lane < w_hi) {
      const uint32_t c = (r[k].x >> a.act_bits) & cmask;
      S.rec[myh[c] + ((lr[k >> 1] >> (16 * (k & 1))) & 0xFFFFu)] = r[k];
    }
  }
  __syncthreads();
  // flag the cases whose events are out of (timestamp, row) order (S.flg was
  // cleared with the per-case sums at the start of the range)
  bool any = false;
  for (uint32_t p = tid + 1; p < n_r; p += kSegThreads) {
    const uint4 x = S.rec[p - 1], y = S.rec[p];
    const uint32_t cx = (x.x >> a.act_bits) & cmask, cy = (y.x >> a.act_bits) & cmask;
    if (cx == cy && !kr_less(ts_key(rec_ts(x)), x.y, ts_key(rec_ts(y)), y.y)) {
      S.flg[cy] = 1;
      any = true;
    }
  }
  const uint64_t slot_base = (uint64_t)b << a.clb;
  if (__syncthreads_or(any)) {
    // the flagged cases are ordered through the index S.idx (identity elsewhere)
    for (uint32_t p = tid; p < n_r; p += kSegThreads) S.idx[p] = (uint16_t)p;
    __syncthreads();
    for (uint32_t c = c_a + warp; c < c_b; c += kSegWarps) {
      if (!S.flg[c]) continue;
      const uint32_t s0 = S.cstart[c], L = S.ccnt[c];
      if (L <= 32) sort_case<1>(S.rec, S.idx, s0, L);
      else if (L <= 64) sort_case<2>(S.rec, S.idx, s0, L);
      else if (L <= 128) sort_case<4>(S.rec, S.idx, s0, L);
      else sort_long_case(S.rec, S.idx, s0, L);
      ++n_sorted;
    }
    __syncthreads();
    auto fetch = [&](int p) { return S.rec[S.idx[p]]; };
    for (uint32_t base = (uint32_t)warp * 32; base < n_r; base += kSegThreads)
      process_warp_tile<kExport>(a, sink, fetch, S.cstart, (int)(base + lane), (int)n_r, out_base, slot_base,
                                 act_mask);
  } else {
    auto fetch = [&](int p) { return S.rec[p]; };
    for (uint32_t base = (uint32_t)warp * 32; base < n_r; base += kSegThreads)
      process_warp_tile<kExport>(a, sink, fetch, S.cstart, (int)(base + lane), (int)n_r, out_base, slot_base,
                                 act_mask);
  }
  __syncthreads();
  // per-case outputs (the first event of a sorted case is found through S.idx)
  if (!kExport) {
    uint32_t present = 0;
    for (uint32_t c = c_a + tid; c < c_b; c += kSegThreads) {
      const uint64_t slot = slot_base + c;
      if (slot < a.n_slots) {
        const uint32_t Lc = S.ccnt[c];
        a.len[slot] = Lc;
        if (a.cattr) {
          const uint32_t q = S.cstart[c];
          a.cattr[slot] = (Lc && a.attr_in) ? a.attr_in[S.rec[S.flg[c] ? S.idx[q] : q].y] : 0;
        }
        present += Lc ? 1u : 0u;
      }
    }
    present = __reduce_add_sync(kFull, present);
    if (lane == 0 && present) atomicAdd(a.n_cases, (unsigned long long)present);
  }
  __syncthreads();
  return true;
}

}  // namespace

template <bool kExport>
__global__ void __launch_bounds__(kSegThreads, 1) k_segment(SegArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  // with the streaming pass launched before it, only a log that pass gave up
  // on (a case out of timestamp order) is left to this pass
  if (a.skip_ordered && !(*(volatile uint32_t *)a.err & kStDisorder)) return;
  const int ncl = 1 << a.clb;
  const int a_s = a.ep_smem ? (int)a.n_act : 0;
  const SegSmem L = seg_smem_layout(a.cap, ncl, a_s, a.tbl_slots, a.tbl_mode);
  SegShared S;
  S.rec = reinterpret_cast<uint4 *>(smem + L.rec);
  S.idx = reinterpret_cast<uint16_t *>(smem + L.hw);  // shares the per-warp counts' area (dead by the sort)
  S.ccnt = reinterpret_cast<uint32_t *>(smem + L.ccnt);
  S.cstart = reinterpret_cast<uint32_t *>(smem + L.cstart);
  S.flg = smem + L.flg;
  uint32_t *tl = reinterpret_cast<uint32_t *>(smem + L.tlo);
  uint32_t *tm = tl + a.tbl_slots;
  uint16_t *hw = reinterpret_cast<uint16_t *>(smem + L.hw);
  uint32_t *rng = reinterpret_cast<uint32_t *>(smem + L.rng);
  uint32_t *st = reinterpret_cast<uint32_t *>(smem + L.st);
  uint32_t *en = reinterpret_cast<uint32_t *>(smem + L.en);
  uint32_t *tkey = reinterpret_cast<uint32_t *>(smem + L.tkey);
  uint32_t *tcnt = reinterpret_cast<uint32_t *>(smem + L.tcnt);
  uint32_t *tminh = reinterpret_cast<uint32_t *>(smem + L.tminh);
  uint32_t *tmaxh = reinterpret_cast<uint32_t *>(smem + L.tmaxh);
  uint32_t *misc = reinterpret_cast<uint32_t *>(smem + L.misc);
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t act_mask = (1u << a.act_bits) - 1;
  const uint32_t cmask = (uint32_t)ncl - 1;

  if (!kExport) {
    for (int i = tid; i < a.tbl_slots; i += kSegThreads) {
      tcnt[i] = 0;
      tl[i] = 0;
      tm[i] = 0;
      tminh[i] = kGuardMinInit;
      tmaxh[i] = kGuardMaxInit;
      if (a.tbl_mode) tkey[i] = kEmptyKey;
    }
    for (int i = tid; i < a_s; i += kSegThreads) {
      st[i] = 0;
      en[i] = 0;
    }
  }
  SmemSink sink{tkey, tcnt, tminh, tmaxh, tl, tm, (uint32_t)(a.tbl_slots - 1),
                (uint32_t)__clz((uint32_t)a.tbl_slots) + 1u, a.tbl_mode,
                a_s ? st : nullptr, a_s ? en : nullptr, a.g, a.g_start, a.g_end};
  uint32_t n_sorted = 0;
  // Buckets are claimed one ahead (misc[0] and misc[1] alternate between the
  // current and the next claim): while a bucket is processed, lane 0 of the
  // last warp claims the next one and starts moving its records into L2.
  if (tid == 0) misc[0] = atomicAdd(a.work, 1u);
  __syncthreads();

  for (uint32_t it = 0;; ++it) {
    const uint32_t b = misc[it & 1];
    if (b >= a.nb) break;
    if (tid == kSegThreads - 32) {
      const uint32_t nx = atomicAdd(a.work, 1u);
      misc[(it & 1) ^ 1] = nx;
      if (nx < a.nb) prefetch_l2(a.rec + a.bucket_off[nx], (a.bucket_off[nx + 1] - a.bucket_off[nx]) * 16u);
    }
    const uint32_t lo = a.bucket_off[b];
    const uint32_t n = a.bucket_off[b + 1] - lo;
    const uint4 *src = a.rec + lo;
    bool ok = true;
    if (n <= (uint32_t)a.cap) {
      ok = process_range<kExport>(a, sink, S, hw, misc, src, false, b, n, 0, (uint32_t)ncl, (int64_t)lo, act_mask,
                                  n_sorted);
    } else {
      // too large for one pass: split the case slots into ranges that fit
      for (int c = tid; c < ncl; c += kSegThreads) S.ccnt[c] = 0;
      __syncthreads();
      for (uint32_t i = tid; i < n; i += kSegThreads) atomicAdd(&S.ccnt[(__ldcg(src + i).x >> a.act_bits) & cmask], 1u);
      __syncthreads();
      if (tid == 0) {
        uint32_t nr = 0, acc = 0, pos = 0;
        bool fits = true;
        rng[0] = 0;
        rng[ncl + 2] = 0;
        for (int c = 0; c < ncl; ++c) {
          const uint32_t v = S.ccnt[c];
          if (v > (uint32_t)a.cap || v > (uint32_t)kMaxCaseSmem) fits = false;
          if (acc + v > (uint32_t)a.cap) {
            rng[++nr] = (uint32_t)c;  // range nr-1 is [rng[nr-1], c)
            rng[ncl + 2 + nr] = pos;  // its first ordered position
            acc = 0;
          }
          acc += v;
          pos += v;
        }
        rng[++nr] = (uint32_t)ncl;
        misc[2] = fits ? nr : 0u;
      }
      __syncthreads();
      const uint32_t nr = misc[2];
      ok = nr > 0;
      for (uint32_t r = 0; r < nr && ok; ++r) {
        const uint32_t c_a = rng[r], c_b = rng[r + 1];
        const uint32_t pos_a = rng[ncl + 2 + r];
        uint32_t cnt = 0;
        for (uint32_t t0 = 0; t0 < n; t0 += kSegThreads) {
          const uint32_t i = t0 + tid;
          uint4 rv = make_uint4(0, 0, 0, 0);
          bool keep = false;
          if (i < n) {
            rv = __ldcg(src + i);
            const uint32_t c = (rv.x >> a.act_bits) & cmask;
            keep = c >= c_a && c < c_b;
          }
          uint32_t tot;
          const uint32_t pre = block_exclusive_scan<kSegThreads>(keep ? 1u : 0u, misc + 8, tot);
          if (keep) S.rec[cnt + pre] = rv;
          cnt += tot;
        }
        __syncthreads();
        ok = process_range<kExport>(a, sink, S, hw, misc, src, true, b, cnt, c_a, c_b, (int64_t)lo + pos_a,
                                    act_mask, n_sorted);
      }
    }
    if (!ok) {
      if (tid == 0) a.ovf[atomicAdd(a.n_ovf, 1u)] = b;
    }
    __syncthreads();
  }
  if (a.n_sorted && lane == 0 && n_sorted) atomicAdd(a.n_sorted, (unsigned long long)n_sorted);
  if (!kExport) {
    for (int s = tid; s < a.tbl_slots; s += kSegThreads) {
      const uint32_t cnt = tcnt[s];
      if (cnt) global_edge_group(a.g, a.tbl_mode ? tkey[s] : (uint32_t)s, cnt, tl[s] | ((uint64_t)tm[s] << 32), 0);
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
    e = cudaFuncSetAttribute(k_segment<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin_max());
    if (e != cudaSuccess) return e;
    k_segment<true><<<grid, kSegThreads, smem, s>>>(a);
  } else {
    e = cudaFuncSetAttribute(k_segment<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin_max());
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
                               int act_bits, uint32_t cmask, uint32_t *keys) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    keys[i] = (rec[perm[i]].x >> act_bits) & cmask;
}
__global__ void k_fb_gather(const uint4 *__restrict__ rec, const uint32_t *__restrict__ perm, uint32_t n,
                            uint4 *out) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = rec[perm[i]];
}
__global__ void k_fb_hist(const uint4 *__restrict__ srec, uint32_t n, int act_bits, uint32_t cmask, uint32_t *ccnt) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    atomicAdd(&ccnt[(srec[i].x >> act_bits) & cmask], 1u);
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

}  // namespace pm4g
