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

// The table slot of an item's key: the first slot along the key's probe
// sequence that holds the key's tag (the key's high word) or that this call
// claims, writing the tag and the item in one 64-bit word. Every item of one
// sequence follows the same probe sequence, and a slot changes only once
// (from empty to claimed), so all of them stop at the same slot; an item of
// another sequence whose tag happens to match stops there too and fails the
// sequence check. *claimer: the item that claimed the slot.
__device__ __forceinline__ uint32_t var_slot(const VarArgs &a, uint32_t s, uint32_t L, uint64_t h, uint32_t round,
                                             uint32_t &claimer) {
  if (a.cls) h ^= fmix64(((uint64_t)a.cls[s] << 1) | 1u);  // keys of different classes differ
  const unsigned long long key = variant_key(h, L, a.bits);
  uint32_t tag = (uint32_t)(key >> 32);
  if (tag == 0) tag = 1;  // 0 marks an empty slot
  const unsigned long long mine = ((unsigned long long)tag << 32) | s;
  uint32_t g = (uint32_t)fmix64(key ^ round) & a.tmask;
  for (uint32_t it = 0; it <= a.tmask; ++it) {
    unsigned long long k = *(volatile unsigned long long *)&a.tab[g].tagc;
    if (k == 0) {
      k = atomicCAS(&a.tab[g].tagc, 0ull, mine);
      if (k == 0) k = mine;
    }
    if ((uint32_t)(k >> 32) == tag) {
      claimer = (uint32_t)k;
      return g;
    }
    g = (g + 1) & a.tmask;
  }
  claimer = s;  // not reached: the table has more slots than items
  return g;
}

// Inserts item s (a case slot, or a list entry) with sequence hash h into the
// grouping table: finds or claims the slot of its key, counts it and keeps the
// smallest member (every member counts; the check against the group's
// representative follows).
__device__ __forceinline__ void var_insert_one(const VarArgs &a, uint32_t s, uint32_t L, uint64_t h,
                                               uint32_t round) {
  uint32_t claimer;
  const uint32_t g = var_slot(a, s, L, h, round, claimer);
  a.grp[s] = g;
  atomicAdd(&a.tab[g].cnt, 1u);
  atomicMax(&a.tab[g].nmin, ~s);
}

// Compares, for every lane in `todo`, the L activities at act_s[xo] with those
// at act_s[yo], clearing `same` on a difference. The comparisons are shared
// out within the warp: each round, four 8-lane groups take the next four
// pending lanes and read eight consecutive activities of both sequences per
// step, so a load instruction covers four contiguous 32-byte runs instead of
// 32 scattered words. All lanes of the warp call it.
__device__ __forceinline__ void warp_compare(const uint16_t *act_s, uint32_t todo, uint32_t L, uint32_t xo,
                                             uint32_t yo, bool &same) {
  const uint32_t lane = threadIdx.x & 31, grp = lane >> 3, gl = lane & 7;
  while (todo) {
    const uint32_t before = todo;
    int src = -1;  // the item of this lane's group: the grp-th lowest pending lane
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (todo && j == (int)grp) src = __ffs(todo) - 1;
      todo &= todo - 1;
    }
    const int sl = src < 0 ? 0 : src;
    const uint32_t Ls = __shfl_sync(kFull, L, sl), xs = __shfl_sync(kFull, xo, sl), ys = __shfl_sync(kFull, yo, sl);
    bool eq = true;
    if (src >= 0) {
#pragma unroll 4
      for (uint32_t k = gl; k < Ls; k += 8) eq &= act_s[xs + k] == act_s[ys + k];
    }
    const uint32_t ne = __ballot_sync(kFull, !eq);
    // the pending lanes of this round were taken by groups 0..3 in lane order
    if ((before >> lane) & 1u) {
      const int gi = __popc(before & lanemask_lt());
      if (gi < 4 && ((ne >> (8 * gi)) & 0xFFu) != 0) same = false;
    }
  }
}

// First-round sequence hash: a polynomial over the case's activities,
// H = sum_j g(a_j) r^j mod 2^64 (j the position in the case, g a table of
// mixed 64-bit words of the activity codes, r an odd constant). It only
// accelerates grouping (equality is always checked on the sequences), and
// unlike a sum of mixed (activity, position) terms it needs no position per
// event: a walk that sums g(a) r^w over walk positions w gets a case's H as
// (sum over the case) * r^-(its first position).
constexpr uint64_t kVarR = 0x9E3779B97F4A7C15ull;  // odd
__host__ __device__ constexpr uint64_t inv_odd(uint64_t r) {
  uint64_t x = r;  // r * r = 1 mod 8; each step doubles the correct low bits
  for (int i = 0; i < 6; ++i) x *= 2 - r * x;
  return x;
}
constexpr uint64_t kVarRinv = inv_odd(kVarR);
static_assert(kVarR * kVarRinv == 1ull, "inverse of the hash base");
__host__ __device__ constexpr uint64_t pow_u64(uint64_t b, uint64_t e) {
  uint64_t x = 1;
  for (; e; e >>= 1, b *= b)
    if (e & 1) x *= b;
  return x;
}

__global__ void k_var_gtab(unsigned long long *g, uint32_t n_act) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_act; i += gridDim.x * blockDim.x)
    g[i] = fmix64(((uint64_t)i << 1) ^ 0x632BE59BD9B4E019ull);
}

// First grouping round over all case slots, with the polynomial hash formed
// on the way from the formatted activities. A warp takes 32 consecutive case
// slots, whose events are contiguous in the formatted order, and walks them
// 128 events at a time, four consecutive events a lane (one 8-byte load of
// 16-bit activities; the walk starts at the 8-byte boundary at or before the
// slots' first event).
// Each lane sums g(a) r^(4 lane + j) over its four events; a warp scan of the
// lanes' sums, scaled by r^(window start), and the running total of the
// windows before give the prefix sums of the walk. Each case's lane fetches,
// with shuffles, the prefix sum just before its first event when the window
// holds it; a case's sum is the difference between the next case's record
// (or the walk's total, for the last case) and its own. Each lane then
// normalises its case's sum by r^-(first position) and inserts its slot.
// (Measured slower: lanes walking whole cases of their own, whose loads touch
// 32 lines at once; checking each case against its group's claimer inside
// this walk, which puts the check's chain of dependent random loads on the
// walk's warps; a per-event hash of (activity, position in case), which
// needs each event's case and position.)
__global__ void __launch_bounds__(kHiThreads) k_var_hash_insert(VarArgs a) {
  // per warp: the prefix sum before each of up to 32 cases
  __shared__ unsigned long long s_pre[kHiThreads / 32][32];
  const uint32_t lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
  unsigned long long *pre = s_pre[wb];
  const uint32_t lt = lanemask_lt();
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t stride = n_warps * 32;
  constexpr uint64_t kR128 = pow_u64(kVarR, 128);
  uint64_t rp[4];  // r^(4 lane + j)
  rp[0] = pow_u64(kVarR, 4 * lane);
#pragma unroll
  for (int j = 1; j < 4; ++j) rp[j] = rp[j - 1] * kVarR;
  // the next group's lengths and first position are loaded one group ahead
  uint64_t s0 = warp * 32;
  uint32_t L_next = s0 + lane < a.n_slots ? a.len[s0 + lane] : 0u;
  uint32_t off_next = s0 < a.n_slots ? a.off[s0] : 0u;
  for (; s0 < a.n_slots; s0 += stride) {
    const uint64_t s = s0 + lane;
    const uint32_t L = L_next, off0 = off_next;  // off0: first formatted position of the slots
    if (s0 + stride < a.n_slots) {
      L_next = s0 + stride + lane < a.n_slots ? a.len[s0 + stride + lane] : 0u;
      off_next = a.off[s0 + stride];
    }
    uint32_t incl = L;  // events of this warp's slots up to and including this lane's
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, incl, o);
      if ((int)lane >= o) incl += y;
    }
    const uint32_t excl = incl - L;
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    const uint32_t ne = __ballot_sync(kFull, L > 0);
    const uint32_t rank = __popc(ne & lt), n_ne = __popc(ne);  // among the non-empty slots
    // walk position w = formatted position - e0, with e0 a multiple of four
    const uint64_t e0 = off0 & ~3u;
    const uint32_t sh = off0 - (uint32_t)e0, tw = total + sh;
    const uint32_t my_ws = excl + sh;  // this slot's first event, in walk positions
    // the lane's four activities of the window at w0 (16 bits each, one
    // 8-byte load), loaded two windows ahead
    auto load4 = [&](uint32_t w0) {
      const uint32_t wl = w0 + 4 * lane;
      uint2 v = make_uint2(0, 0);
      if (wl < tw) {
        const uint64_t e = e0 + wl;
        if (e + 4 <= a.n_events) {
          v = __ldcs(reinterpret_cast<const uint2 *>(a.act_s + e));
        } else {
          v.x = a.act_s[e];
          if (e + 1 < a.n_events) v.x |= (uint32_t)a.act_s[e + 1] << 16;
          if (e + 2 < a.n_events) v.y = a.act_s[e + 2];
        }
      }
      return v;
    };
    uint2 v1 = load4(0), v2 = load4(128);
    uint64_t rw = 1;     // r^w0
    uint64_t done = 0;   // the walk's sum over the windows before
    for (uint32_t w0 = 0; w0 < tw; w0 += 128) {
      const uint32_t wl = w0 + 4 * lane;  // walk position of the lane's first event
      const uint2 v = v1;
      v1 = v2;
      v2 = load4(w0 + 256);
      const uint32_t act4[4] = {v.x & 0xFFFFu, v.x >> 16, v.y & 0xFFFFu, v.y >> 16};
      uint64_t ex[4], u = 0;  // the lane's sums before each of its events, and in all
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        ex[j] = u;
        const uint32_t w = wl + j;
        if (w >= sh && w < tw) u += (uint64_t)__ldg(a.gtab + act4[j]) * rp[j];
      }
      uint64_t inc = u;  // inclusive prefix sums of the lanes' sums
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(kFull, inc, o);
        if ((int)lane >= o) inc += y;
      }
      const uint64_t x = inc - u;
      // a case starting in this window reads the prefix sum before its first
      // event from the lane that holds it
      const uint32_t bi = my_ws - w0;
      const bool mine = L && my_ws >= w0 && bi < 128u;
      const int src = mine ? (int)(bi >> 2) : (int)lane;
      const uint64_t p0 = __shfl_sync(kFull, x + ex[0], src), p1 = __shfl_sync(kFull, x + ex[1], src);
      const uint64_t p2 = __shfl_sync(kFull, x + ex[2], src), p3 = __shfl_sync(kFull, x + ex[3], src);
      if (mine) {
        const uint32_t sub = bi & 3u;
        pre[rank] = done + rw * (sub == 0 ? p0 : sub == 1 ? p1 : sub == 2 ? p2 : p3);
      }
      done += rw * __shfl_sync(kFull, inc, 31);
      rw *= kR128;
    }
    __syncwarp();
    if (L) {
      const uint64_t nxt = rank + 1 < n_ne ? pre[rank + 1] : done;
      var_insert_one(a, (uint32_t)s, L, (nxt - pre[rank]) * pow_u64(kVarRinv, my_ws), 0);
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
      const uint16_t *q = a.act_s + a.off[s];
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

// Each item is compared with its group's representative, the smallest
// member, event by event (warp_compare). One that differs leaves its group.
__global__ void k_var_verify(VarArgs a, const uint32_t *list, uint32_t n_list, uint32_t *bad_out,
                             uint32_t *n_bad) {
  const uint64_t total = list ? (uint64_t)n_list : a.n_slots;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint32_t lane = threadIdx.x & 31;
  for (uint64_t w0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); w0 < total; w0 += stride) {
    uint32_t s = 0, g = 0, L = 0, xo = 0, yo = 0;
    const bool item = var_item(a, list, n_list, w0 + lane, s);
    bool same = true, need = false;
    if (item) {
      g = a.grp[s];
      const uint32_t rep = ~a.tab[g].nmin;
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
    warp_compare(a.act_s, __ballot_sync(kFull, need), L, xo, yo, same);
    if (item) {
      a.isbad[s] = same ? 0 : 1;
      if (!same) {
        atomicSub(&a.tab[g].cnt, 1u);
        bad_out[atomicAdd(n_bad, 1u)] = s;
      }
    }
  }
}

// Every item that stayed in its group records the group's representative
// (its smallest member), and each representative its group's size. With
// a.rep_flag, every slot of the round also gets its representative flag (a
// slot that left its group gets 0 here and its flag in a later round).
__global__ void k_var_final(VarArgs a, const uint32_t *list, uint32_t n_list) {
  const uint64_t total = list ? (uint64_t)n_list : a.n_slots;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t s;
    if (!var_item(a, list, n_list, i, s)) {
      if (a.rep_flag && !list) a.rep_flag[i] = 0;  // no case in the slot
      continue;
    }
    if (a.isbad[s]) {
      if (a.rep_flag) a.rep_flag[s] = 0;
      continue;
    }
    const uint32_t g = a.grp[s];
    const uint32_t rep = ~a.tab[g].nmin;
    a.rep_of[s] = rep;
    if (rep == s) a.vcount[s] = a.tab[g].cnt;
    if (a.rep_flag) a.rep_flag[s] = rep == s ? 1u : 0u;
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

// The top variants' sequences at o_acts[o_off[i]]; a sequence that would end
// beyond `cap` entries is not written (the caller then sizes a buffer from
// the offsets and calls again).
// One warp a variant, its lanes copying consecutive activities (coalesced
// writes, also when o_acts is mapped host memory).
__global__ void k_var_out_acts(VarArgs a, const uint32_t *order, const uint32_t *rep_slots, uint32_t k_out,
                               const uint32_t *o_off, int32_t *o_acts, uint64_t cap) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t i = w0; i < k_out; i += nw) {
    const uint32_t rep = rep_slots[order[i]];
    const uint16_t *q = a.act_s + a.off[rep];
    const uint32_t L = a.len[rep];
    if ((uint64_t)o_off[i] + L > cap) continue;
    int32_t *o = o_acts + o_off[i];
    for (uint32_t j = lane; j < L; j += 32) o[j] = q[j];
  }
}

}  // namespace pm4g
