// Formatting kernels (Section 3, first formatting step: ordering by case
// identifier, timestamp and absolute index).
//
// The engine orders the log in two levels. Here, one scatter moves every event
// into the bucket of its case: a bucket holds 2^clb consecutive case slots
// (slot = case id - smallest case id) and is small enough for shared memory.
// The per-bucket ordering by (case, timestamp, row) then happens on chip in the
// segment pass. Offsets come from per-CTA bucket histograms (a CTA x bucket
// count matrix, prefixed per bucket over CTAs and scanned over buckets), so
// the scatter needs no global atomics: each CTA owns a private cursor per bucket
// in shared memory.
#include "device_common.cuh"
#include "engine.h"
#include "kernels.h"

namespace pm4g {

// ---------------------------------------------------------------------------
// Stats: per-block min/max of the case column (column reduction, Section 2.1).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_stats(const int32_t *__restrict__ case_id, int64_t n,
                                               int2 *__restrict__ partial) {
  int mn = INT_MAX, mx = INT_MIN;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (((uintptr_t)case_id & 15) == 0) {
    const int4 *v = reinterpret_cast<const int4 *>(case_id);
    const int64_t nv = n >> 2;
    for (int64_t i = tid; i < nv; i += stride) {
      int4 q = __ldcs(v + i);
      mn = min(mn, min(min(q.x, q.y), min(q.z, q.w)));
      mx = max(mx, max(max(q.x, q.y), max(q.z, q.w)));
    }
    for (int64_t i = (nv << 2) + tid; i < n; i += stride) {
      mn = min(mn, case_id[i]);
      mx = max(mx, case_id[i]);
    }
  } else {
    for (int64_t i = tid; i < n; i += stride) {
      mn = min(mn, case_id[i]);
      mx = max(mx, case_id[i]);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mn = min(mn, __shfl_xor_sync(kFull, mn, o));
    mx = max(mx, __shfl_xor_sync(kFull, mx, o));
  }
  __shared__ int2 s[8];
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = make_int2(mn, mx);
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      mn = min(mn, s[w].x);
      mx = max(mx, s[w].y);
    }
    partial[blockIdx.x] = make_int2(mn, mx);
  }
}

// Loads four consecutive int32 starting at i (i % 4 == 0) as one vector when the
// column is 16-byte aligned, else element by element; q.* beyond n are unset.
__device__ __forceinline__ int4 load4_i32(const int32_t *__restrict__ p, int64_t i, int64_t n, bool aligned) {
  if (aligned && i + 3 < n) return __ldcs(reinterpret_cast<const int4 *>(p + i));
  int4 q = make_int4(0, 0, 0, 0);
  if (i < n) q.x = p[i];
  if (i + 1 < n) q.y = p[i + 1];
  if (i + 2 < n) q.z = p[i + 2];
  if (i + 3 < n) q.w = p[i + 3];
  return q;
}

// An enclosing guess of the case id range is widened from the minimum and
// maximum of kRangeSamples rows spread evenly over the column, the first and
// last rows included (one block of 1024 threads).
__global__ void __launch_bounds__(1024) k_sample_range(const int32_t *__restrict__ case_id, int64_t n,
                                                       int2 *__restrict__ out) {
  int mn = INT_MAX, mx = INT_MIN;
  for (int k = threadIdx.x; k < kRangeSamples; k += blockDim.x) {
    const int v = case_id[(n - 1) * k / (kRangeSamples - 1)];
    mn = min(mn, v);
    mx = max(mx, v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mn = min(mn, __shfl_xor_sync(kFull, mn, o));
    mx = max(mx, __shfl_xor_sync(kFull, mx, o));
  }
  __shared__ int2 s[32];
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = make_int2(mn, mx);
  __syncthreads();
  if (threadIdx.x == 0) {
    int2 r = s[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = make_int2(min(r.x, s[w].x), max(r.y, s[w].y));
    *out = r;
  }
}

// ---------------------------------------------------------------------------
// Bucket histogram of one CTA's row chunk, for buckets [b_lo, b_lo + nbs).
// mat is CTA-major: mat[p * nb + b]. The same read checks every case id
// against the range the buckets were laid out for (range_err), so that a
// guessed range needs no reduction of its own.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_bucket_hist(FormatArgs a, uint32_t b_lo, uint32_t nbs) {
  extern __shared__ uint32_t s_h[];
  for (uint32_t b = threadIdx.x; b < nbs; b += blockDim.x) s_h[b] = 0;
  __syncthreads();
  const int64_t r0 = (int64_t)blockIdx.x * a.chunk;
  const int64_t r1 = min(a.n, r0 + a.chunk);
  const bool al = ((uintptr_t)a.case_id & 15) == 0;
  bool out = false;
  auto count4 = [&](int4 q, int64_t i) {
    const int32_t cc[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (i + k < r1) {
        const uint32_t slot = (uint32_t)cc[k] - (uint32_t)a.min_case;
        out |= slot > a.slot_hi;
        const uint32_t b = (slot >> a.clb) - b_lo;
        if (b < nbs) atomicAdd(&s_h[b], 1u);
      }
    }
  };
  // four 16-byte loads in flight per thread before their adds (one block per
  // SM: a single load a thread leaves the column read latency-bound)
  const int64_t step = (int64_t)blockDim.x * 4;
  int64_t i = r0 + (int64_t)threadIdx.x * 4;
  for (; i + 3 * step < r1; i += 4 * step) {
    int4 q[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) q[u] = load4_i32(a.case_id, i + u * step, r1, al);
#pragma unroll
    for (int u = 0; u < 4; ++u) count4(q[u], i + u * step);
  }
  for (; i < r1; i += step) count4(load4_i32(a.case_id, i, r1, al), i);
  if (__syncthreads_or(out) && threadIdx.x == 0 && a.range_err) atomicOr(a.range_err, 1u);
  uint32_t *row = a.mat + (int64_t)blockIdx.x * a.nb + b_lo;
  for (uint32_t b = threadIdx.x; b < nbs; b += blockDim.x) row[b] = s_h[b];
}

// Per bucket: exclusive prefix of the counts over CTAs (in place) and the
// bucket total. A block handles 32 buckets; its 8 warps split the CTA range so
// that no thread walks more than an eighth of it serially.
__global__ void __launch_bounds__(256) k_bucket_colprefix(uint32_t *__restrict__ mat, uint32_t nb, int p_ctas,
                                                          uint32_t *__restrict__ total) {
  __shared__ uint32_t s_part[8][33];
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t b = blockIdx.x * 32 + lane;
  const int per = (p_ctas + 7) / 8;
  const int p0 = min(p_ctas, (int)w * per), p1 = min(p_ctas, p0 + per);
  // the rows are independent loads: unrolled so that many are in flight
  uint32_t s = 0;
  if (b < nb) {
#pragma unroll 8
    for (int p = p0; p < p1; ++p) s += __ldcg(mat + (int64_t)p * nb + b);
  }
  s_part[w][lane] = s;
  __syncthreads();
  uint32_t acc = 0;
  for (uint32_t ww = 0; ww < w; ++ww) acc += s_part[ww][lane];
  if (b < nb) {
    constexpr int kU = 8;
    int p = p0;
    for (; p + kU <= p1; p += kU) {
      uint32_t v[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) v[u] = __ldcg(mat + (int64_t)(p + u) * nb + b);
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        mat[(int64_t)(p + u) * nb + b] = acc;
        acc += v[u];
      }
    }
    for (; p < p1; ++p) {
      uint32_t *q = mat + (int64_t)p * nb + b;
      const uint32_t v = *q;
      *q = acc;
      acc += v;
    }
    if (w == 7) total[b] = acc;
  }
}

// The same histogram for all nb buckets in one pass with 16-bit counters (two
// per shared word), for bucket counts that would need two passes with 32-bit
// ones. A counter passing 65535 inside one CTA's chunk is detected from the
// atomic's old value; that CTA then counts its chunk again straight into its
// global row (exact, slow, and only for chunks where one bucket holds more
// than 65535 events).
__global__ void __launch_bounds__(1024) k_bucket_hist16(FormatArgs a) {
  extern __shared__ uint32_t s_w[];  // (nb + 1) / 2 words of counters, then the overflow word
  const uint32_t nw = (a.nb + 1) / 2;
  uint32_t &s_ovf = s_w[nw];
  for (uint32_t w = threadIdx.x; w < nw; w += blockDim.x) s_w[w] = 0;
  if (threadIdx.x == 0) s_ovf = 0;
  __syncthreads();
  const int64_t r0 = (int64_t)blockIdx.x * a.chunk;
  const int64_t r1 = min(a.n, r0 + a.chunk);
  const bool al = ((uintptr_t)a.case_id & 15) == 0;
  bool ovf = false, out = false;
  auto count4 = [&](int4 q, int64_t i) {
    const int32_t cc[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (i + k < r1) {
        const uint32_t slot = (uint32_t)cc[k] - (uint32_t)a.min_case;
        out |= slot > a.slot_hi;
        const uint32_t b = slot >> a.clb;
        if (b < a.nb) {
          const uint32_t sh = (b & 1u) * 16u;
          const uint32_t old = atomicAdd(&s_w[b >> 1], 1u << sh);
          ovf |= ((old >> sh) & 0xFFFFu) == 0xFFFFu;
        }
      }
    }
  };
  // four 16-byte loads in flight per thread before their adds
  const int64_t step = (int64_t)blockDim.x * 4;
  int64_t i = r0 + (int64_t)threadIdx.x * 4;
  for (; i + 3 * step < r1; i += 4 * step) {
    int4 q[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) q[u] = load4_i32(a.case_id, i + u * step, r1, al);
#pragma unroll
    for (int u = 0; u < 4; ++u) count4(q[u], i + u * step);
  }
  for (; i < r1; i += step) count4(load4_i32(a.case_id, i, r1, al), i);
  if (ovf) s_ovf = 1;
  if (__syncthreads_or(out) && threadIdx.x == 0 && a.range_err) atomicOr(a.range_err, 1u);
  uint32_t *row = a.mat + (int64_t)blockIdx.x * a.nb;
  if (!s_ovf) {
    for (uint32_t b = threadIdx.x; b < a.nb; b += blockDim.x) row[b] = (s_w[b >> 1] >> ((b & 1u) * 16u)) & 0xFFFFu;
    return;
  }
  for (uint32_t b = threadIdx.x; b < a.nb; b += blockDim.x) row[b] = 0;
  __syncthreads();
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    const uint32_t b = ((uint32_t)a.case_id[i] - (uint32_t)a.min_case) >> a.clb;
    if (b < a.nb) atomicAdd(&row[b], 1u);
  }
}

// ---------------------------------------------------------------------------
// Scatter: every event of buckets [b_lo, b_lo + nbs) goes to its bucket as one
// 16-byte record. Activity codes outside [0, A) raise the error flag and are
// stored as 0 so that every later index stays in bounds.
//
// The scatter keeps row order inside each bucket for almost every case: CTAs
// own consecutive row chunks (their cursors start at the CTA-major prefix of
// the count matrix), a CTA walks its chunk in tiles with a barrier between
// tiles, sub-step k of a tile covers rows k*blockDim .. with consecutive rows
// on consecutive lanes, and a run of consecutive lanes hitting the same bucket
// reserves its slots with one atomic, in lane order. Only events of one case
// that fall in one tile on different warps, or on non-adjacent lanes of one
// warp, can swap. Order is an optimisation only: every
// record keeps its row, so the segment pass sorts any case that arrives out
// of order.
// The next tile's columns are prefetched into registers while the current
// tile is scattered.
// ---------------------------------------------------------------------------
constexpr int kScatterThreads = 1024;
constexpr int kScatterSub = 4;  // sub-steps per tile

__global__ void __launch_bounds__(kScatterThreads) k_bucket_scatter(FormatArgs a, uint32_t b_lo, uint32_t nbs) {
  extern __shared__ uint32_t s_cur[];
  {
    const uint32_t *row = a.mat + (int64_t)blockIdx.x * a.nb + b_lo;
    for (uint32_t b = threadIdx.x; b < nbs; b += blockDim.x) s_cur[b] = a.bucket_off[b_lo + b] + row[b];
  }
  __syncthreads();
  const int64_t r0 = (int64_t)blockIdx.x * a.chunk;
  const int64_t r1 = min(a.n, r0 + a.chunk);
  const int lane = threadIdx.x & 31;
  constexpr int64_t kTile = (int64_t)kScatterThreads * kScatterSub;
  int32_t nc[kScatterSub], na[kScatterSub];
  int64_t nt[kScatterSub];
#pragma unroll
  for (int k = 0; k < kScatterSub; ++k) {
    const int64_t i = r0 + k * kScatterThreads + threadIdx.x;
    nc[k] = i < r1 ? __ldcs(a.case_id + i) : 0;
    na[k] = i < r1 ? __ldcs(a.activity + i) : 0;
    nt[k] = i < r1 ? __ldcs(a.ts + i) : 0;
  }
  bool bad = false;
  const uint64_t pol = l2_evict_last_policy();
  for (int64_t base = r0; base < r1; base += kTile) {
    int32_t cc[kScatterSub], aa[kScatterSub];
    int64_t tt[kScatterSub];
#pragma unroll
    for (int k = 0; k < kScatterSub; ++k) {
      cc[k] = nc[k];
      aa[k] = na[k];
      tt[k] = nt[k];
    }
    if (base + kTile < r1) {
#pragma unroll
      for (int k = 0; k < kScatterSub; ++k) {
        const int64_t i = base + kTile + k * kScatterThreads + threadIdx.x;
        nc[k] = i < r1 ? __ldcs(a.case_id + i) : 0;
        na[k] = i < r1 ? __ldcs(a.activity + i) : 0;
        nt[k] = i < r1 ? __ldcs(a.ts + i) : 0;
      }
    }
#pragma unroll
    for (int k = 0; k < kScatterSub; ++k) {
      const int64_t i = base + k * kScatterThreads + threadIdx.x;
      const uint32_t slot = (uint32_t)cc[k] - (uint32_t)a.min_case;
      const uint32_t b = (slot >> a.clb) - b_lo;
      const bool in = i < r1 && b < nbs;
      uint32_t act = (uint32_t)aa[k];
      if (in && act >= (uint32_t)a.n_act) {
        bad = true;
        act = 0;
      }
      uint32_t run;
      const uint32_t head = run_head(in ? b : 0xFFFFFFFFu, run);
      uint32_t pos = 0;
      if (in && (uint32_t)lane == head) pos = atomicAdd(&s_cur[b], run);
      pos = __shfl_sync(kFull, pos, (int)head) + ((uint32_t)lane - head);
      // a half-written sector must stay in L2 until the next record of the
      // same bucket front fills it
      if (in) st_evict_last(a.rec + pos, make_rec(slot & kSlotLoMask, act, a.act_bits, (uint32_t)i, tt[k]), pol);
    }
    __syncthreads();
  }
  if (__any_sync(kFull, bad) && lane == 0) atomicOr(a.err_flags, 1u);
}

// ---------------------------------------------------------------------------
// Sparse case ids: dense renumbering by rank among the distinct ids.
// ---------------------------------------------------------------------------
__global__ void k_case_keys(const int32_t *__restrict__ case_id, int64_t n, uint32_t *__restrict__ keys,
                            uint32_t *__restrict__ vals) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    keys[i] = (uint32_t)case_id[i] ^ 0x80000000u;
    vals[i] = (uint32_t)i;
  }
}

__global__ void k_case_heads(const uint32_t *__restrict__ keys, int64_t n, uint32_t *__restrict__ head) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    head[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

__global__ void k_case_dense(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ rows,
                             const uint32_t *__restrict__ head, const uint32_t *__restrict__ head_excl, int64_t n,
                             int32_t *__restrict__ dense, int32_t *__restrict__ uniq) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t r = head_excl[i] + head[i] - 1;
    dense[rows[i]] = (int32_t)r;
    if (head[i]) uniq[r] = (int32_t)(keys[i] ^ 0x80000000u);
  }
}

}  // namespace pm4g

namespace pm4g {

// ---------------------------------------------------------------------------
// Bucket partition with coalesced writes (replaces the record-by-record
// scatter whenever the bucket count allows it). Scattered 16-byte stores run
// about 8x slower than streaming ones on this GPU, so a tile of kItems * kPartThreads
// events is first ordered by digit in shared memory and then written out as
// one contiguous run per digit, by a bulk copy of the tensor memory
// accelerator that overlaps the next tile.
//
// Level 1 reads the input columns; its digit is the coarse bucket
// slot >> (clb + fbits), and CTA p owns row chunk p (cursors from the CTA-major
// prefix of the coarse count matrix). With fbits = 0 the coarse bucket is the
// final bucket and level 1 is the only pass. Level 2 reads level 1's output;
// CTA C owns coarse bucket C and its digit is the final bucket inside it,
// (slot_lo >> clb) & (2^fbits - 1); its cursors are the final bucket offsets.
// Both levels keep row order within every digit: items of a tile are ranked by
// warp (warps own consecutive items), then by round, then by lane.
// ---------------------------------------------------------------------------
// kItems records a thread per tile: 8 (4,096-record tiles, two blocks per SM)
// or 4 (2,048-record tiles in about two thirds of the shared memory, three
// blocks per SM for more loads in flight).
template <int kLevel, int kItems>
__global__ void __launch_bounds__(kPartThreads, kItems == 4 ? 3 : 2) k_partition(PartArgs a) {
  constexpr int kTile = kPartThreads * kItems;
  extern __shared__ __align__(16) unsigned char sm[];
  const uint32_t nbins = a.nbins;
  uint4 *stg = reinterpret_cast<uint4 *>(sm);
  uint16_t *wh = reinterpret_cast<uint16_t *>(sm + (size_t)kTile * 16);
  uint32_t *pm = reinterpret_cast<uint32_t *>(sm + (size_t)kTile * 16 + part_wh_bytes(nbins));
  uint32_t *cur = pm + kPartWarps * nbins;  // next output index of every digit
  uint32_t *tst = cur + nbins;              // staged start of every digit, nbins + 1
  uint32_t *sw = tst + nbins + 1;           // block-scan scratch, 32 words
  uint32_t *dlt = sw + 32;                  // every digit's output position minus its staged position
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // item indices fit 32 bits (at most 2^31 - 1 events)
  uint32_t i0, i1;
  if (kLevel == 1) {
    i0 = (uint32_t)((int64_t)blockIdx.x * a.chunk);
    i1 = (uint32_t)min(a.n, (int64_t)i0 + a.chunk);
    for (uint32_t d = tid; d < nbins; d += kPartThreads) cur[d] = a.cur1[(int64_t)blockIdx.x * nbins + d];
  } else {
    // unit (C, j): the part of coarse bucket C that level 1 wrote from row
    // chunks [p0, p1); its records of final bucket b go after those that
    // chunks before p0 contributed to b (the CTA-major prefix in mat)
    const uint32_t C = blockIdx.x / a.splits, j = blockIdx.x % a.splits;
    const int p0 = (int)((int64_t)j * a.p_ctas / a.splits), p1 = (int)((int64_t)(j + 1) * a.p_ctas / a.splits);
    const uint32_t nc = (a.nb + (1u << a.fbits) - 1) >> a.fbits;
    const uint32_t b0 = C << a.fbits;
    i0 = a.cur1[(int64_t)p0 * nc + C];
    i1 = p1 < a.p_ctas ? a.cur1[(int64_t)p1 * nc + C] : a.bucket_off[min(a.nb, b0 + (1u << a.fbits))];
    for (uint32_t d = tid; d < nbins; d += kPartThreads)
      cur[d] = b0 + d < a.nb ? a.bucket_off[b0 + d] + a.mat[(int64_t)p0 * a.nb + b0 + d] : 0u;
  }
  for (uint32_t j = tid; j < kPartWarps * nbins; j += kPartThreads) {
    wh[j] = 0;
    pm[j] = 0;
  }
  __syncthreads();
  const uint32_t fmask = (1u << a.fbits) - 1;
  const int shift1 = a.clb + a.fbits;
  bool bad = false;
  uint16_t *myh = wh + warp * nbins;
  // The tile loop is software-pipelined: the loads of tile t + 1 are issued
  // before the runs of tile t are copied out, so both are in flight while
  // the warps go on to rank tile t + 1.
  // Level 1 holds the raw columns (case id, activity, timestamp) in rec until
  // the record is formed.
  uint4 rec[kItems];
  // Loading tile t + 1 also starts moving tile t + 2 into L2, so that the
  // loads of every tile after the first find their data there.
  auto prefetch_tile = [&](uint32_t base) {
    if (base >= i1 || warp != kPartWarps - 1 || lane > 2) return;
    const uint32_t e = min(i1, base + kTile);
    if (kLevel == 1) {
      if (lane == 0) prefetch_l2_inner(a.case_id + base, (size_t)(e - base) * 4);
      if (lane == 1) prefetch_l2_inner(a.activity + base, (size_t)(e - base) * 4);
      if (lane == 2) prefetch_l2_inner(a.ts + base, (size_t)(e - base) * 8);
    } else if (lane == 0) {
      prefetch_l2_inner(a.rec_in + base, (size_t)(e - base) * 16);
    }
  };
  auto load_tile = [&](uint32_t base) {
    prefetch_tile(base + kTile);
    const uint32_t wb = base + (uint32_t)warp * (32 * kItems) + lane;
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      const uint32_t i = wb + r * 32;
      if (i < i1) {
        if (kLevel == 1) {
          const uint64_t t = (uint64_t)__ldcs(a.ts + i);
          rec[r] = make_uint4((uint32_t)__ldcs(a.case_id + i), (uint32_t)__ldcs(a.activity + i), (uint32_t)t,
                              (uint32_t)(t >> 32));
        } else {
          rec[r] = __ldcs(a.rec_in + i);
        }
      }
    }
  };
  if (i0 < i1) load_tile(i0);
  for (uint32_t base = i0; base < i1; base += kTile) {
    uint32_t dg[kItems];
    const uint32_t wbase = base + (uint32_t)warp * (32 * kItems) + lane;
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      const uint32_t i = wbase + r * 32;
      dg[r] = 0xFFFFFFFFu;
      if (i < i1) {
        if (kLevel == 1) {
          const uint32_t slot = rec[r].x - (uint32_t)a.min_case;
          uint32_t act = rec[r].y;
          if (act >= (uint32_t)a.n_act) {
            bad = true;
            act = 0;
          }
          rec[r] = make_uint4(((slot & kSlotLoMask) << a.act_bits) | act, i, rec[r].z, rec[r].w);
          dg[r] = slot >> shift1;

        } else {
          dg[r] = ((rec[r].x >> a.act_bits) >> a.clb) & fmask;
        }
      }
    }
    // stable ranks: per-warp counts in item order (rounds, then lanes).
    // Each round finds the lanes that share a digit by OR-ing the lane bits
    // into a per-warp mask word of the digit (cheaper than a warp match when
    // most lanes differ); all of them read the digit's count, and the lowest
    // lane adds the group's size and clears the mask for the next round.
    uint32_t rk[kItems];
    uint32_t *pmw = pm + warp * nbins;
    const uint32_t lt = lanemask_lt(), bit = 1u << lane;
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      const uint32_t d = dg[r];
      const bool v = d != 0xFFFFFFFFu;
      if (v) atomicOr(&pmw[d], bit);
      __syncwarp();
      uint32_t peers = 0, bb = 0;
      if (v) {
        peers = pmw[d];
        bb = myh[d];
      }
      __syncwarp();
      if (v && (peers & lt) == 0) {
        myh[d] = (uint16_t)(bb + __popc(peers));
        pmw[d] = 0;
      }
      __syncwarp();
      rk[r] = bb + __popc(peers & lt);
    }
    __syncthreads();
    {
      uint32_t tot = 0;
      if ((uint32_t)tid < nbins)
        for (int w = 0; w < kPartWarps; ++w) tot += wh[w * nbins + tid];
      uint32_t all;
      const uint32_t pre = block_exclusive_scan<kPartThreads>(tot, sw, all);
      if ((uint32_t)tid < nbins) {
        tst[tid] = pre;
        dlt[tid] = cur[tid] - pre;
        uint32_t run = pre;
        for (int w = 0; w < kPartWarps; ++w) {
          const uint32_t t = wh[w * nbins + tid];
          wh[w * nbins + tid] = (uint16_t)run;
          run += t;
        }
      }
      if (tid == 0) tst[nbins] = all;
      // the previous tile's copies must be done reading the staging tile
      if ((uint32_t)tid < nbins) bulk_wait_read();
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      if (dg[r] != 0xFFFFFFFFu) {
        const uint32_t sp = myh[dg[r]] + rk[r];
        stg[sp] = rec[r];
        // one level only: the final bucketing, so the key words go out here
        if (kLevel == 1 && a.fbits == 0 && a.keys_out) a.keys_out[dlt[dg[r]] + sp] = rec[r].x;
      }
    }
    fence_smem_to_async();
    __syncthreads();
    if (kLevel == 2 && a.keys_out) {
      // the first word of every record, in final order, from the staged tile
      // (consecutive staged records of a digit go to consecutive positions)
      const uint32_t cnt = tst[nbins];
      for (uint32_t k = tid; k < cnt; k += kPartThreads) {
        const uint32_t x = stg[k].x;
        a.keys_out[dlt[((x >> a.act_bits) >> a.clb) & fmask] + k] = x;
      }
    }
    if (base + kTile < i1) load_tile(base + kTile);
    // each digit's run is one bulk copy, issued by the digit's thread; the
    // copies proceed while the next tile is loaded and ranked
    if ((uint32_t)tid < nbins) {
      const uint32_t s0 = tst[tid], cnt = tst[tid + 1] - s0, o = cur[tid];
      if (cnt) bulk_copy_s2g(a.rec_out + o, stg + s0, cnt * 16u);
      bulk_commit();
      cur[tid] = o + cnt;
    }
    // every warp clears its own counts for the next tile
    for (uint32_t j = lane; j < nbins; j += 32) myh[j] = 0;
    __syncwarp();
  }
  if ((uint32_t)tid < nbins) bulk_wait_all();
  if (kLevel == 1) {
    if (__any_sync(kFull, bad) && lane == 0) atomicOr(a.err_flags, 1u);
  }
}

template <int kLevel, int kItems>
static cudaError_t launch_part(const PartArgs &a, unsigned grid, cudaStream_t s) {
  const cudaError_t e =
      cudaFuncSetAttribute(k_partition<kLevel, kItems>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin_max());
  if (e != cudaSuccess) return e;
  k_partition<kLevel, kItems><<<grid, kPartThreads, part_smem_bytes(a.nbins, kItems), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_partition(int level, const PartArgs &a, unsigned grid, cudaStream_t s, int items) {
  if (level == 1) return items == 4 ? launch_part<1, 4>(a, grid, s) : launch_part<1, 8>(a, grid, s);
  return items == 4 ? launch_part<2, 4>(a, grid, s) : launch_part<2, 8>(a, grid, s);
}

// Coarse count matrix: mat1[p][C] = sum of mat[p][b] over the final buckets b
// of coarse bucket C.
// One warp per (p, C): the warp reads the 2^fbits counts coalesced and sums
// them with a warp reduction.
__global__ void k_coarse_counts(const uint32_t *__restrict__ mat, uint32_t nb, int p_ctas, int fbits, uint32_t nc,
                                uint32_t *__restrict__ mat1) {
  const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  if (k >= (int64_t)p_ctas * nc) return;  // warp-uniform
  const int64_t p = k / nc;
  const uint32_t C = (uint32_t)(k % nc);
  const uint32_t b0 = C << fbits, b1 = min(nb, b0 + (1u << fbits));
  uint32_t s = 0;
  for (uint32_t b = b0 + lane; b < b1; b += 32) s += __ldcg(mat + p * nb + b);
  s = __reduce_add_sync(0xFFFFFFFFu, s);
  if (lane == 0) mat1[p * nc + C] = s;
}

// Adds the coarse bucket's first position to every CTA's prefix.
__global__ void k_add_base(uint32_t *__restrict__ mat1, int p_ctas, uint32_t nc, const uint32_t *__restrict__ bucket_off,
                           int fbits) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (int64_t)p_ctas * nc) return;
  mat1[k] += bucket_off[(uint32_t)(k % nc) << fbits];
}

}  // namespace pm4g

