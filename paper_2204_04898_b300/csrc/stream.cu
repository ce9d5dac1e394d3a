// Streaming segment pass for logs whose cases' events come in timestamp
// order (Section 3: the directly-follows pairs, the performance DFG,
// start/end activities and the per-case variant features of the formatted
// log).
//
// When every case's events have non-decreasing timestamps in row order (as
// in a log whose rows are sorted by time, or grouped by case), the stable
// bucket partition delivers every case's events in (timestamp, row) order
// inside its bucket, interleaved with the other cases of the bucket. The formatting sort
// of Section 3 then reduces to grouping by case, and the grouping needs no
// reordering at all: one warp takes a bucket and
//  1. counts its cases from the first word of every record, which the
//     partition's final level also wrote to a compact array (4 bytes per
//     event), and forms every case's first formatted position (written out
//     as the log's case offsets);
//  2. streams the records once, 32 at a time, linking every event to the
//     previous event of its case:
//     - the lanes holding events of one case are found with one match of
//       the case slots (measured faster here than one ballot per slot bit);
//       an event's predecessor is the highest lower
//       lane of its case, read with a shuffle, or the case's last event of an
//       earlier chunk, kept in shared memory;
//     - the pair (previous activity, activity) with duration ts - ts_prev is
//       added to a shared edge table indexed by the edge's id (below), with
//       32-bit atomics and no probing;
//     - the case's highest lane in the chunk updates the case's state, so the
//       case state needs no atomics;
//     - the activity goes straight to its formatted position;
//  3. counts the end activities (a case's last event is the last one seen).
// (The variant step forms each case's sequence hash from the activities
// written here.)
// No block barrier is taken between buckets.
//
// Edge ids: the first lane to meet an edge claims an id for it in a global
// A x A map (compare-and-swap from "none" to "pending", then the id); ids
// below the shared table's size index it directly, and the id's key is kept
// so that the table can be flushed by key. A lane that finds the edge
// pending, or an id beyond the table, adds its pair to the global table
// directly. Sums are exact: 32-bit low and middle words in shared memory with
// every carry out of bit 63 added to the global high word; minimum and maximum
// are pushed to global memory (fire-and-forget) only when the duration can
// beat what this block already pushed, judged by float guards rounded outward
// (device_common.cuh).
#include "device_common.cuh"
#include "engine.h"
#include "kernels.h"
#include "sink.cuh"

namespace pm4g {

namespace {

constexpr uint32_t kIdNone = 0xFFFFFFFFu;     // no id claimed yet
constexpr uint32_t kIdPending = 0xFFFFFFFEu;  // being claimed
constexpr uint32_t kIdGlobal = 0xFFFFFFFDu;   // claimed beyond the shared table

// Per-warp case state in shared memory, one entry per case slot of a bucket.
struct StState {
  unsigned long long *lts;  // timestamp of the last event seen
  uint32_t *first;          // formatted position of the case's first event
  uint32_t *seen;           // events of the case counted (step 1), then streamed (step 2)
  uint32_t *lact;           // activity of the last event seen
};

__device__ __forceinline__ StState st_state(unsigned char *base, int ncl) {
  StState s;
  s.lts = reinterpret_cast<unsigned long long *>(base);
  s.first = reinterpret_cast<uint32_t *>(base + (size_t)ncl * 8);
  s.seen = s.first + ncl;
  s.lact = s.seen + ncl;
  return s;
}

struct EdgeTable {
  uint32_t *tcnt, *tl, *tm, *tminh, *tmaxh;  // shared, kStSlots each (tminh/tmaxh: float guards)
  uint32_t *emap, *key_of, *n_ids;           // global
  DfgTable g;

  // The edge's id, claiming one if the edge has none; kIdPending or
  // kIdGlobal (or any value >= kStSlots) sends the pair to the global table.
  // e: the map's entry as loaded earlier. L1 may have held a stale "none"
  // (the compare-and-swap below then returns the id) or a stale "pending"
  // (read again from L2); an id never changes once set.
  __device__ __forceinline__ uint32_t id_of(uint32_t key, uint32_t e) {
    if (e == kIdPending) e = __ldcg(emap + key);
    if (e == kIdNone) {
      e = atomicCAS(&emap[key], kIdNone, kIdPending);
      if (e == kIdNone) {
        const uint32_t id = atomicAdd(n_ids, 1u);
        if (id < (uint32_t)kStSlots) key_of[id] = key;
        __threadfence();  // the key is visible before the id is
        e = id < (uint32_t)kStSlots ? id : kIdGlobal;
        atomicExch(&emap[key], e);
      }
    }
    return e;
  }

  __device__ __forceinline__ void add(uint32_t key, uint64_t d, uint32_t e0) {
    const uint32_t e = id_of(key, e0);
    const uint32_t l = (uint32_t)d, h = (uint32_t)(d >> 32);
    if (e < (uint32_t)kStSlots) {
      atomicAdd(&tcnt[e], 1u);
      const uint32_t ol = atomicAdd(&tl[e], l);
      const uint32_t hm = h + (ol + l < ol ? 1u : 0u);  // wraps to 0 only for h = 2^32 - 1 with a carry
      const uint32_t om = atomicAdd(&tm[e], hm);
      const uint32_t top = (om + hm < om ? 1u : 0u) + (hm < h ? 1u : 0u);
      const bool pmn = __float_as_uint(__ull2float_rd(d)) < tminh[e];
      const bool pmx = __float_as_uint(__ull2float_ru(d)) > tmaxh[e];
      if (top || pmn || pmx) {
        const uint64_t i = g_index(g, key);
        if (i != ~0ull) {
          if (top) red_add_u64(&g.hi[i], top);
          if (pmn) red_min_u64(&g.mn[i], d);
          if (pmx) red_max_u64(&g.mx[i], d);
        }
        if (pmn) atomicMin(&tminh[e], guard_up(d));
        if (pmx) atomicMax(&tmaxh[e], guard_down(d));
      }
    } else {
      global_edge_add(g, key, 1, d, 0, d, d);
    }
  }
};

}  // namespace

// Blocks of at most 28 warps (73 registers a thread) for 256-slot buckets,
// whose per-warp case state lets no more fit (24 measured 1 % slower); 32
// warps (64 registers) for narrower buckets.
template <int kClb>
__global__ void __launch_bounds__(kClb >= 8 ? 896 : 1024, 1) k_stream_segment(SegArgs a, int n_warps) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (a.ran && blockIdx.x == 0 && threadIdx.x == 0) *a.ran = 1u;
  constexpr int ncl = 1 << kClb;
  constexpr int per = (ncl + 31) >> 5;  // case slots per lane in the per-bucket loops
  const int a_s = a.ep_smem ? (int)a.n_act : 0;
  const StSmem L = st_smem_layout(ncl, a_s, n_warps);
  EdgeTable T;
  T.tcnt = reinterpret_cast<uint32_t *>(smem + L.tcnt);
  T.tl = T.tcnt + kStSlots;
  T.tm = T.tl + kStSlots;
  T.tminh = T.tm + kStSlots;
  T.tmaxh = T.tminh + kStSlots;
  T.emap = a.emap;
  T.key_of = a.key_of;
  T.n_ids = a.n_ids;
  T.g = a.g;
  uint32_t *st = reinterpret_cast<uint32_t *>(smem + L.st);
  uint32_t *en = st + a_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < kStSlots; i += blockDim.x) {
    T.tcnt[i] = 0;
    T.tl[i] = 0;
    T.tm[i] = 0;
    T.tminh[i] = kGuardMinInit;
    T.tmaxh[i] = kGuardMaxInit;
  }
  for (int i = tid; i < a_s; i += blockDim.x) {
    st[i] = 0;
    en[i] = 0;
  }
  __syncthreads();
  const StState S = st_state(smem + L.warp0 + (size_t)warp * L.per_warp, ncl);
  const uint32_t act_mask = (1u << a.act_bits) - 1;
  constexpr uint32_t cmask = (uint32_t)ncl - 1;
  const uint32_t lt_mask = lanemask_lt();
  uint32_t present = 0;

  // buckets are claimed per warp (a whole-bucket L2 prefetch per warp would
  // put more bytes in flight than L2 holds; records are instead loaded into
  // registers two chunks ahead)
  bool disorder = false;  // this lane met an event earlier than its case's previous one
  for (;;) {
    uint32_t b = 0;
    // a case out of order anywhere: the sorting pass redoes the log
    if (lane == 0) b = (*(volatile uint32_t *)a.err & kStDisorder) ? a.nb : atomicAdd(a.work, 1u);
    b = __shfl_sync(kFull, b, 0);
    if (b >= a.nb) break;
    const uint32_t lo = a.bucket_off[b], n = a.bucket_off[b + 1] - lo;
    const uint64_t slot_base = (uint64_t)b << kClb;
    // the bucket's key words and its first records start moving into L2; the
    // records then follow in a window of 512-1024 records ahead of the warp
    // (a few KB per warp, so that all warps together stay well inside L2)
    if (lane == 0 && n) {
      prefetch_l2_inner(a.keys + lo, (size_t)n * 4);
      prefetch_l2(a.rec + lo, min(n, 1024u) * 16u);
    }
    // 1. case lengths and first positions
#pragma unroll
    for (int k = 0; k < per; ++k)
      if (lane * per + k < ncl) S.seen[lane * per + k] = 0;
    __syncwarp();
    {
      // eight independent loads in flight per lane before their adds
      constexpr int kU = 8;
      const uint32_t *kp = a.keys + lo;
      uint32_t i = lane;
      for (; i + 32 * (kU - 1) < n; i += 32 * kU) {
        uint32_t x[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) x[u] = __ldcs(kp + i + 32 * u);
#pragma unroll
        for (int u = 0; u < kU; ++u) atomicAdd(&S.seen[(x[u] >> a.act_bits) & cmask], 1u);
      }
      for (; i < n; i += 32) atomicAdd(&S.seen[(__ldcs(kp + i) >> a.act_bits) & cmask], 1u);
    }
    __syncwarp();
    {
      uint32_t cnt[per], sum = 0;
#pragma unroll
      for (int k = 0; k < per; ++k) {
        const int c = lane * per + k;
        cnt[k] = c < ncl ? S.seen[c] : 0u;
        sum += cnt[k];
      }
      uint32_t x = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
      }
      uint32_t run = lo + x - sum;
#pragma unroll
      for (int k = 0; k < per; ++k) {
        const int c = lane * per + k;
        if (c < ncl) {
          const uint64_t slot = slot_base + (uint64_t)c;
          if (slot < a.n_slots) {
            a.len[slot] = cnt[k];
            if (a.off_out) a.off_out[slot] = run;
          }
          S.first[c] = run;
          S.seen[c] = 0;
          run += cnt[k];
        }
      }
      if (a.off_out && lane == 0 && b == a.nb - 1) a.off_out[a.n_slots] = lo + n;  // the event count
    }
    __syncwarp();
    // 2. the records, 32 at a time
    const uint4 *src = a.rec + lo;
    uint4 r1 = make_uint4(0, 0, 0, 0), r2 = make_uint4(0, 0, 0, 0);
    if ((uint32_t)lane < n) r1 = __ldcs(src + lane);
    if (32u + lane < n) r2 = __ldcs(src + 32 + lane);
    // the previous chunk's pair, added to the edge table one chunk late so
    // that its edge-id load overlaps this chunk's work
    bool p_has = false;
    uint32_t p_key = 0, p_e = kIdNone;
    uint64_t p_d = 0;
    for (uint32_t base = 0; base < n; base += 32) {
      if ((base & 511u) == 0 && lane == 0 && base + 1024 < n)
        prefetch_l2(src + base + 1024, min(n - (base + 1024), 512u) * 16u);
      const bool valid = base + lane < n;
      const uint4 r = r1;
      r1 = r2;
      if (base + 64 + lane < n) r2 = __ldcs(src + base + 64 + lane);
      const uint32_t c = valid ? (r.x >> a.act_bits) & cmask : 0u;
      const uint32_t act = r.x & act_mask;
      const uint64_t ts = ((uint64_t)r.w << 32) | r.z;
      const uint32_t peers = __match_any_sync(kFull, valid ? c : 0xFFFFFFFFu);
      const uint32_t lower = peers & lt_mask;
      uint32_t seen = 0, first = 0;
      if (valid) {
        seen = S.seen[c];
        first = S.first[c];
      }
      const uint32_t pos = seen + __popc(lower);  // rank of the event in its case
      // the previous event of the case: the highest lower lane of the chunk,
      // else the last event of an earlier chunk
      const int from = lower ? 31 - __clz(lower) : lane;
      uint32_t pact = __shfl_sync(kFull, act, from);
      const uint32_t pz = __shfl_sync(kFull, r.z, from), pw = __shfl_sync(kFull, r.w, from);
      uint64_t pts = ((uint64_t)pw << 32) | pz;
      if (valid && !lower && seen) {
        pact = S.lact[c];
        pts = S.lts[c];
      }
      if (valid) {
        // a case's events stay inside its bucket's formatted range unless the
        // counted lengths disagree with the records (reported)
        if (first + pos < lo + n) a.act_s[first + pos] = (uint16_t)act;
        else atomicOr(a.err, 1u);
        if (pos == 0) {
          if (a_s) atomicAdd(&st[act], 1u);
          else atomicAdd(&a.g_start[act], 1ull);
          if (a.cattr) a.cattr[slot_base + c] = a.attr_in ? a.attr_in[r.y] : 0;
        }
      }
      const bool has = valid && pos > 0;
      if (has && (int64_t)ts < (int64_t)pts) disorder = true;
      const uint32_t key = pact * a.n_act + act;
      const uint32_t e = has ? T.emap[key] : kIdNone;  // used one chunk later
      if (p_has) T.add(p_key, p_d, p_e);
      p_has = has;
      p_key = key;
      p_d = ts - pts;
      p_e = e;
      if (valid && lane == 31 - __clz(peers)) {  // the case's last lane in this chunk
        S.seen[c] = pos + 1;
        S.lact[c] = act;
        S.lts[c] = ts;
      }
      __syncwarp();
    }
    if (p_has) T.add(p_key, p_d, p_e);
    if (__any_sync(kFull, disorder) && lane == 0) atomicOr(a.err, kStDisorder);
    // 3. per-case outputs; the end activity is the last event seen
#pragma unroll
    for (int k = 0; k < per; ++k) {
      const int c = lane * per + k;
      const uint64_t slot = slot_base + (uint64_t)c;
      if (c < ncl && slot < a.n_slots) {
        const uint32_t Lc = S.seen[c];
        if (Lc != a.len[slot]) atomicOr(a.err, 1u);
        if (Lc) {
          const uint32_t la = S.lact[c];
          if (a_s) atomicAdd(&en[la], 1u);
          else atomicAdd(&a.g_end[la], 1ull);
          ++present;
        }
      }
    }
    __syncwarp();
  }
  present = __reduce_add_sync(kFull, present);
  if (lane == 0 && present) atomicAdd(a.n_cases, (unsigned long long)present);
  __syncthreads();
  __threadfence();
  for (int s = tid; s < kStSlots; s += blockDim.x) {
    const uint32_t cnt = T.tcnt[s];
    if (cnt) global_edge_group(a.g, __ldcg(a.key_of + s), cnt, T.tl[s] | ((uint64_t)T.tm[s] << 32), 0);
  }
  for (int i = tid; i < a_s; i += blockDim.x) {
    if (st[i]) atomicAdd(&a.g_start[i], (unsigned long long)st[i]);
    if (en[i]) atomicAdd(&a.g_end[i], (unsigned long long)en[i]);
  }
}

__global__ void k_stream_undo(const uint32_t *err, DfgTable g, uint64_t cells, unsigned long long *ends,
                              uint32_t n_act, unsigned long long *n_cases, uint32_t *work) {
  if (!(*err & kStDisorder)) return;
  const uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, st = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = i0; i < cells; i += st) {
    g.cnt[i] = 0;
    g.lo[i] = 0;
    g.hi[i] = 0;
    g.mn[i] = ~0ull;
    g.mx[i] = 0;
  }
  for (uint64_t i = i0; i < 2 * (uint64_t)n_act; i += st) ends[i] = 0;
  if (i0 == 0) {
    *n_cases = 0;
    *work = 0;  // the sorting pass claims the buckets from the same counter
  }
}

cudaError_t launch_stream_undo(const SegArgs &a, uint32_t n_act, unsigned grid, cudaStream_t s) {
  k_stream_undo<<<grid, 256, 0, s>>>(a.err, a.g, (uint64_t)n_act * n_act, a.g_start, n_act, a.n_cases, a.work);
  return cudaGetLastError();
}

int stream_segment_warps(int clb, int a_s, size_t smem_optin) {
  const int ncl = 1 << clb;
  for (int w = (clb >= 8 ? 896 : kStMaxThreads) / 32; w >= 1; --w)
    if (st_smem_layout(ncl, a_s, w).total <= smem_optin) return w;
  return 0;
}

template <int kClb>
static cudaError_t launch_st(const SegArgs &a, int n_warps, unsigned grid, size_t smem, cudaStream_t s) {
  const cudaError_t e =
      cudaFuncSetAttribute(k_stream_segment<kClb>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin_max());
  if (e != cudaSuccess) return e;
  k_stream_segment<kClb><<<grid, n_warps * 32, smem, s>>>(a, n_warps);
  return cudaGetLastError();
}

cudaError_t launch_stream_segment(const SegArgs &a, int n_warps, unsigned grid, size_t smem, cudaStream_t s) {
  switch (a.clb) {
    case 0: return launch_st<0>(a, n_warps, grid, smem, s);
    case 1: return launch_st<1>(a, n_warps, grid, smem, s);
    case 2: return launch_st<2>(a, n_warps, grid, smem, s);
    case 3: return launch_st<3>(a, n_warps, grid, smem, s);
    case 4: return launch_st<4>(a, n_warps, grid, smem, s);
    case 5: return launch_st<5>(a, n_warps, grid, smem, s);
    case 6: return launch_st<6>(a, n_warps, grid, smem, s);
    case 7: return launch_st<7>(a, n_warps, grid, smem, s);
    case 8: return launch_st<8>(a, n_warps, grid, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pm4g
