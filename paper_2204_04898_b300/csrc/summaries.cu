// Summary kernels: DFG edge compaction, activity frequency, and the variant
// table (Section 3, variants.py: a double aggregation, events into cases and
// cases into variants).
//
// Variants: cases are grouped by a key made of their sequence hash and length
// in an open-addressing table; each group's representative is its smallest
// case slot. Every other member compares its full activity sequence with the
// representative's. A member that differs leaves the group and is grouped
// again in the next round with a freshly seeded hash, until no member differs,
// so the grouping is exact whatever the hash does. Groups are then ranked by
// (count descending, smallest case id ascending) with a stable radix sort of
// the representatives listed in ascending case order.
#include "device_common.cuh"
#include "engine.h"
#include "kernels.h"
#include "variants.h"

namespace pm4g {

__global__ void k_dfg_flags(const unsigned long long *__restrict__ cnt, int64_t cells, uint32_t *__restrict__ flags) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cells; i += (int64_t)gridDim.x * blockDim.x)
    flags[i] = cnt[i] ? 1u : 0u;
}

// Edges with a count, in (src, dst) order, with the mean duration formed from
// the exact sum (edge_mean: the host formula (double)sum / (double)count).
__global__ void k_dfg_compact(DfgTable g, int64_t cells, uint32_t n_act, const uint32_t *__restrict__ flags,
                              const uint32_t *__restrict__ pos, int32_t *src, int32_t *dst, unsigned long long *cnt,
                              unsigned long long *lo, unsigned long long *hi, unsigned long long *mn,
                              unsigned long long *mx, double *mean) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cells; i += (int64_t)gridDim.x * blockDim.x) {
    if (!flags[i]) continue;
    const uint32_t p = pos[i];
    const unsigned long long c = g.cnt[i], l = g.lo[i], h = g.hi[i];
    src[p] = (int32_t)(i / n_act);
    dst[p] = (int32_t)(i % n_act);
    cnt[p] = c;
    lo[p] = l;
    hi[p] = h;
    mn[p] = g.mn[i];
    mx[p] = g.mx[i];
    mean[p] = edge_mean(h, l, c);
  }
}

// ---- hashed global table (large alphabets) ----
__global__ void k_gkey_flags(const unsigned long long *__restrict__ gkey, uint64_t T, uint32_t *__restrict__ flags) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < T; i += (uint64_t)gridDim.x * blockDim.x)
    flags[i] = gkey[i] ? 1u : 0u;
}
// The occupied slots' keys (src * A + dst) and slot indices, in slot order.
__global__ void k_gkey_compact(const unsigned long long *__restrict__ gkey, uint64_t T,
                               const uint32_t *__restrict__ flags, const uint32_t *__restrict__ pos,
                               uint32_t *__restrict__ keys, uint32_t *__restrict__ slots) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < T; i += (uint64_t)gridDim.x * blockDim.x) {
    if (!flags[i]) continue;
    const uint32_t p = pos[i];
    keys[p] = (uint32_t)(gkey[i] - 1ull);
    slots[p] = (uint32_t)i;
  }
}
// Edge p (keys ascending) from its slot, with the mean as for the dense table.
__global__ void k_dfg_gather(DfgTable g, const uint32_t *__restrict__ keys, const uint32_t *__restrict__ slots,
                             uint32_t E, uint32_t n_act, int32_t *src, int32_t *dst, unsigned long long *cnt,
                             unsigned long long *lo, unsigned long long *hi, unsigned long long *mn,
                             unsigned long long *mx, double *mean) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < E; p += gridDim.x * blockDim.x) {
    const uint32_t k = keys[p], i = slots[p];
    const unsigned long long c = g.cnt[i], l = g.lo[i], h = g.hi[i];
    src[p] = (int32_t)(k / n_act);
    dst[p] = (int32_t)(k % n_act);
    cnt[p] = c;
    lo[p] = l;
    hi[p] = h;
    mn[p] = g.mn[i];
    mx[p] = g.mx[i];
    mean[p] = edge_mean(h, l, c);
  }
}
// Activity frequency from the listed edges: out-edges of each activity, plus
// its end count.
__global__ void k_freq_edges(const int32_t *__restrict__ src, const unsigned long long *__restrict__ cnt, uint32_t E,
                             unsigned long long *freq) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < E; p += gridDim.x * blockDim.x)
    atomicAdd(&freq[src[p]], cnt[p]);
}
__global__ void k_freq_end(const unsigned long long *__restrict__ end, uint32_t n_act, unsigned long long *freq) {
  for (uint32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < n_act; a += gridDim.x * blockDim.x) freq[a] += end[a];
}

// Activity frequency: every event is either followed by another event of its
// case (one out-edge) or is its case's last event, so freq(a) = sum over b of
// count(a, b) + end(a).
__global__ void k_freq(const unsigned long long *__restrict__ cnt, const unsigned long long *__restrict__ end,
                       uint32_t n_act, unsigned long long *__restrict__ freq) {
  const uint32_t a = blockIdx.x;
  unsigned long long s = 0;
  for (uint32_t b = threadIdx.x; b < n_act; b += blockDim.x) s += cnt[(uint64_t)a * n_act + b];
  __shared__ unsigned long long s_p[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
  if ((threadIdx.x & 31) == 0) s_p[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_p[w];
    freq[a] = t + end[a];
  }
}

// ---------------------------------------------------------------------------
// Variants
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool var_item(const VarArgs &a, const uint32_t *list, uint32_t n_list, uint64_t i,
                                         uint32_t &s) {
  if (list) {
    if (i >= n_list) return false;
    s = list[i];
    return true;
  }
  if (i >= a.n_slots) return false;
  s = (uint32_t)i;
  return a.len[s] != 0;
}

// Inserts item s (a case slot, or a list entry) with sequence hash h into the
// grouping table: finds or claims the slot of its key, counts it and keeps the
// smallest member.
__device__ __forceinline__ void var_insert_one(const VarArgs &a, uint32_t s, uint32_t L, uint64_t h,
                                               uint32_t round) {
  if (a.cls) h ^= fmix64(((uint64_t)a.cls[s] << 1) | 1u);  // keys of different classes differ
  const unsigned long long key = variant_key(h, L, a.bits);
  uint32_t g = (uint32_t)fmix64(key ^ round) & a.tmask;
  for (uint32_t it = 0; it <= a.tmask; ++it) {
    const unsigned long long k = *(volatile unsigned long long *)&a.tab[g].key;
    if (k == key) break;
    if (k == 0) {
      const unsigned long long old = atomicCAS(&a.tab[g].key, 0ull, key);
      if (old == 0 || old == key) break;
    }
    g = (g + 1) & a.tmask;
  }
  a.grp[s] = g;
  atomicAdd(&a.tab[g].cnt, 1u);
  atomicMax(&a.tab[g].nmin, ~s);
}

// First grouping round over all case slots, with the sequence hash (seed 0)
// formed on the way from the formatted activities. A warp takes 32
// consecutive case slots, whose events are contiguous in the formatted order,
// and walks them 32 events at a time, lane-dense. One OR-reduction per window
// gives the bits of the positions where a (non-empty) case starts; a lane's
// case is then the number of starts up to its position (a popcount, counted
// from the cases that started before the window). The terms of the walk are
// prefix-summed (a warp scan per window plus the running total of the windows
// before), and each case start records the prefix sum just before it: a
// case's hash is the difference between the next case's record (or the walk's
// total, for the last case) and its own, so the walk needs no segmented
// reduction. Each lane then inserts its own slot.
__global__ void __launch_bounds__(kHiThreads) k_var_hash_insert(VarArgs a) {
  // per warp: low and high words of the prefix sum before each of up to 32
  // cases, and each case's first position
  __shared__ uint32_t s_acc[kHiThreads / 32][96];
  const uint32_t lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
  uint32_t *gs_lo = s_acc[wb], *gs_hi = gs_lo + 32, *sstart = gs_lo + 64;
  const uint32_t le = 0xFFFFFFFFu >> (31 - lane), lt = lanemask_lt();
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t s0 = warp * 32; s0 < a.n_slots; s0 += n_warps * 32) {
    const uint64_t s = s0 + lane;
    const uint32_t L = s < a.n_slots ? a.len[s] : 0u;
    uint32_t incl = L;  // events of this warp's slots up to and including this lane's
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, incl, o);
      if ((int)lane >= o) incl += y;
    }
    const uint32_t excl = incl - L;
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    const uint32_t off0 = a.off[s0];  // first formatted position of the slots
    const uint32_t ne = __ballot_sync(kFull, L > 0);
    const uint32_t rank = __popc(ne & lt), n_ne = __popc(ne);  // among the non-empty slots
    if (L) sstart[rank] = excl;
    __syncwarp();
    // the activities of the next four windows are loaded ahead
    const int32_t *q = a.act_s + off0 + lane;
    int32_t q0 = lane < total ? __ldcs(q) : 0, q1 = 32 + lane < total ? __ldcs(q + 32) : 0;
    int32_t q2 = 64 + lane < total ? __ldcs(q + 64) : 0, q3 = 96 + lane < total ? __ldcs(q + 96) : 0;
    uint32_t before = 0;       // non-empty cases that start before the window
    uint32_t clo = 0, chi = 0;  // sums of the terms of the windows before
    for (uint32_t p0 = 0; p0 < total; p0 += 32) {
      const int32_t act = q0;
      q0 = q1;
      q1 = q2;
      q2 = q3;
      q3 = p0 + 128 + lane < total ? __ldcs(q + p0 + 128) : 0;
      const uint32_t bit = (L && excl >= p0 && excl - p0 < 32u) ? (1u << (excl - p0)) : 0u;
      const uint32_t starts = __reduce_or_sync(kFull, bit);
      const uint32_t p = p0 + lane;
      const uint32_t cr = before + __popc(starts & le) - 1;  // the case's rank (valid lanes)
      uint32_t tl = 0, th = 0;
      if (p < total) {
        const uint64_t t = event_hash((uint32_t)act, p - sstart[cr], 0);
        tl = (uint32_t)t;
        th = (uint32_t)(t >> 32);
      }
      uint32_t il = tl, ih = th;  // inclusive prefix sums within the window
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t yl = __shfl_up_sync(kFull, il, o), yh = __shfl_up_sync(kFull, ih, o);
        if ((int)lane >= o) {
          il += yl;
          ih += yh;
        }
      }
      if ((starts >> lane) & 1u) {
        gs_lo[cr] = clo + il - tl;
        gs_hi[cr] = chi + ih - th;
      }
      clo += __shfl_sync(kFull, il, 31);
      chi += __shfl_sync(kFull, ih, 31);
      before += __popc(starts);
    }
    __syncwarp();
    if (L) {
      const uint32_t nl = rank + 1 < n_ne ? gs_lo[rank + 1] : clo, nh = rank + 1 < n_ne ? gs_hi[rank + 1] : chi;
      var_insert_one(a, (uint32_t)s, L, ((uint64_t)(nh - gs_hi[rank]) << 32) | (nl - gs_lo[rank]), 0);
    }
    __syncwarp();
  }
}

__global__ void k_var_insert(VarArgs a, const uint32_t *list, uint32_t n_list, uint32_t round) {
  const uint64_t total = list ? (uint64_t)n_list : a.n_slots;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t s;
    if (!var_item(a, list, n_list, i, s)) continue;
    const uint32_t L = a.len[s];
    uint64_t h;
    if (round == 0 && a.hash) {
      h = a.hash[s];
    } else {
      h = 0;
      const int32_t *q = a.act_s + a.off[s];
      uint32_t hl = 0, hh = 0;  // same combination as the segment pass: two 32-bit sums
      for (uint32_t k = 0; k < L; ++k) {
        const uint64_t t = event_hash((uint32_t)q[k], k, round);
        hl += (uint32_t)t;
        hh += (uint32_t)(t >> 32);
      }
      h = ((uint64_t)hh << 32) | hl;
    }
    var_insert_one(a, s, L, h, round);
  }
}

// Each item is compared with its group's representative, event by event.
// The comparisons are shared out within the warp: each round, four 8-lane
// groups take the next four items that need one and read eight consecutive
// activities of both sequences per step, so a load instruction covers four
// contiguous 32-byte runs instead of 32 scattered words. An item that
// matches records its representative; one that does not leaves its group.
__global__ void k_var_verify(VarArgs a, const uint32_t *list, uint32_t n_list, uint32_t *bad_out,
                             uint32_t *n_bad) {
  const uint64_t total = list ? (uint64_t)n_list : a.n_slots;
  const int lane = threadIdx.x & 31, grp = lane >> 3, gl = lane & 7;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t w0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); w0 < total; w0 += stride) {
    uint32_t s = 0, g = 0, L = 0, xo = 0, yo = 0, rep = 0;
    const bool item = var_item(a, list, n_list, w0 + lane, s);
    bool same = true, need = false;
    if (item) {
      g = a.grp[s];
      rep = ~a.tab[g].nmin;
      if (rep != s) {
        L = a.len[s];
        same = a.len[rep] == L && (!a.cls || a.cls[rep] == a.cls[s]);
        need = same && L > 0;
        if (need) {
          xo = a.off[s];
          yo = a.off[rep];
        }
      }
    }
    uint32_t todo = __ballot_sync(kFull, need);
    while (todo) {
      const uint32_t before = todo;
      int src = -1;  // the item of this lane's group: the grp-th lowest pending lane
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (todo && j == grp) src = __ffs(todo) - 1;
        todo &= todo - 1;
      }
      const int sl = src < 0 ? 0 : src;
      const uint32_t Ls = __shfl_sync(kFull, L, sl), xs = __shfl_sync(kFull, xo, sl), ys = __shfl_sync(kFull, yo, sl);
      bool eq = true;
      if (src >= 0) {
#pragma unroll 4
        for (uint32_t k = gl; k < Ls; k += 8) eq &= a.act_s[xs + k] == a.act_s[ys + k];
      }
      const uint32_t ne = __ballot_sync(kFull, !eq);
      // the pending lanes of this round were taken by groups 0..3 in lane order
      if ((before >> lane) & 1u) {
        const int gi = __popc(before & lanemask_lt());
        if (gi < 4) same = ((ne >> (8 * gi)) & 0xFFu) == 0;
      }
    }
    if (item) {
      a.isbad[s] = same ? 0 : 1;
      if (same) {
        a.rep_of[s] = rep;
      } else {
        atomicSub(&a.tab[g].cnt, 1u);
        bad_out[atomicAdd(n_bad, 1u)] = s;
      }
    }
  }
}

// The group sizes, once every mismatch of the round has left its group: the
// representatives (never mismatched) read their slot's count.
__global__ void k_var_final(VarArgs a, const uint32_t *list, uint32_t n_list) {
  const uint64_t total = list ? (uint64_t)n_list : a.n_slots;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t s;
    if (!var_item(a, list, n_list, i, s)) continue;
    if (a.isbad[s] || a.rep_of[s] != s) continue;
    a.vcount[s] = a.tab[a.grp[s]].cnt;
  }
}

__global__ void k_rep_flags(VarArgs a, uint32_t *flags) {
  for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.n_slots; s += (uint64_t)gridDim.x * blockDim.x)
    flags[s] = (a.len[s] != 0 && a.rep_of[s] == (uint32_t)s) ? 1u : 0u;
}

__global__ void k_rep_compact(VarArgs a, const uint32_t *flags, const uint32_t *pos, uint32_t cmask,
                              uint32_t *rep_slots, uint32_t *keys, uint32_t *vals) {
  for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.n_slots; s += (uint64_t)gridDim.x * blockDim.x) {
    if (!flags[s]) continue;
    const uint32_t v = pos[s];
    rep_slots[v] = (uint32_t)s;
    keys[v] = (~a.vcount[s]) & cmask;
    vals[v] = v;
  }
}

__global__ void k_rank_scatter(const uint32_t *order, uint32_t V, uint32_t *rank_of) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < V; k += gridDim.x * blockDim.x) rank_of[order[k]] = k;
}

__global__ void k_case_variant(VarArgs a, const uint32_t *rep_pos, const uint32_t *rank_of, int32_t *cvar) {
  for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.n_slots; s += (uint64_t)gridDim.x * blockDim.x)
    if (a.len[s]) cvar[s] = (int32_t)rank_of[rep_pos[a.rep_of[s]]];
}

__global__ void k_present_flags(const uint32_t *len, uint64_t n_slots, uint32_t *flags) {
  for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_slots; s += (uint64_t)gridDim.x * blockDim.x)
    flags[s] = len[s] ? 1u : 0u;
}

__global__ void k_cases_out(const uint32_t *len, uint64_t n_slots, const uint32_t *pos, const int32_t *cvar,
                            int32_t min_case, const int32_t *uniq, int32_t *case_ids, int32_t *case_variant) {
  for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_slots; s += (uint64_t)gridDim.x * blockDim.x) {
    if (!len[s]) continue;
    const uint32_t p = pos[s];
    case_ids[p] = uniq ? uniq[s] : (int32_t)((uint32_t)min_case + (uint32_t)s);
    case_variant[p] = cvar[s];
  }
}

__global__ void k_var_out_head(VarArgs a, const uint32_t *order, const uint32_t *rep_slots, uint32_t k_out,
                               int32_t min_case, const int32_t *uniq, unsigned long long *o_count, int32_t *o_min,
                               uint32_t *o_len) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k_out; i += gridDim.x * blockDim.x) {
    const uint32_t rep = rep_slots[order[i]];
    o_count[i] = a.vcount[rep];
    o_min[i] = uniq ? uniq[rep] : (int32_t)((uint32_t)min_case + rep);
    o_len[i] = a.len[rep];
  }
}

__global__ void k_var_out_acts(VarArgs a, const uint32_t *order, const uint32_t *rep_slots, uint32_t k_out,
                               const uint32_t *o_off, int32_t *o_acts) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k_out; i += gridDim.x * blockDim.x) {
    const uint32_t rep = rep_slots[order[i]];
    const int32_t *q = a.act_s + a.off[rep];
    const uint32_t L = a.len[rep];
    int32_t *o = o_acts + o_off[i];
    for (uint32_t j = 0; j < L; ++j) o[j] = q[j];
  }
}

}  // namespace pm4g
