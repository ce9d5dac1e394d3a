// Eventually-follows graph and temporal profile (Section 3, efg.py).
//
// A pair of events (i, j) of one case eventually follows when i comes before
// j in the case's (timestamp, row) order. Per activity pair (a, b): the
// number of such pairs, the exact sum of ts_j - ts_i (128-bit), the exact sum
// of their squares (192-bit), the mean (the rounded sum over the count, as for
// the DFG) and the population standard deviation sqrt(rn(n * S2 - S1^2) / n /
// n), where rn rounds the exact 256-bit numerator to the nearest double (ties
// to even) and every other step is one IEEE operation.
//
// The pass reads the formatted log (activities and timestamps in case order):
// one warp per case holds up to 32 of its events in registers and, for every
// event i, the lanes j > i add their pair to a dense A x A table of exact
// sums with 64-bit atomics (carries propagate to the next word at once). The
// frequent activity pairs would serialise those atomics at one L2 slice each,
// so the blocks share K copies of the table (block b uses copy b mod K; up to
// one per block within a memory budget), folded exactly into the first one
// afterwards. A flag/scan/compaction lists the pairs with their mean and
// deviation.

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "device_common.cuh"
#include "engine.h"
#include "kernels.h"

using namespace pm4g;

namespace pm4g {
namespace {

struct EfTable {
  unsigned long long *cnt, *s_lo, *s_hi, *q0, *q1, *q2;  // A x A cells each
};

// One pair of duration d into cell key.
__device__ __forceinline__ void ef_add(const EfTable &t, uint32_t key, uint64_t d) {
  atomicAdd(&t.cnt[key], 1ull);
  const unsigned long long o = atomicAdd(&t.s_lo[key], (unsigned long long)d);
  if (o + d < o) atomicAdd(&t.s_hi[key], 1ull);
  const uint64_t sq_lo = d * d, sq_hi = __umul64hi(d, d);  // d^2 < 2^128, so sq_hi <= 2^64 - 2
  const unsigned long long o0 = atomicAdd(&t.q0[key], (unsigned long long)sq_lo);
  const uint64_t up = sq_hi + (o0 + sq_lo < o0 ? 1u : 0u);
  if (up) {
    const unsigned long long o1 = atomicAdd(&t.q1[key], (unsigned long long)up);
    if (o1 + up < o1) atomicAdd(&t.q2[key], 1ull);
  }
}

// Cases are taken by warps from a counter, longest cases first is not needed:
// a warp walks its case's events in chunks of 32 (lanes hold a chunk of the
// later events; the earlier event is broadcast).
__global__ void __launch_bounds__(256) k_efg_pairs(const uint32_t *len, const uint32_t *off, uint64_t n_slots,
                                                   const uint16_t *act_s, const int64_t *ts_s, uint32_t A,
                                                   EfTable t0, uint64_t copy_stride, uint32_t n_copies,
                                                   unsigned long long *work) {
  const int lane = threadIdx.x & 31;
  const uint64_t sh = (uint64_t)(blockIdx.x % n_copies) * copy_stride;  // this block's copy of the table
  const EfTable t{t0.cnt + sh, t0.s_lo + sh, t0.s_hi + sh, t0.q0 + sh, t0.q1 + sh, t0.q2 + sh};
  for (;;) {
    unsigned long long s0 = 0;
    if (lane == 0) s0 = atomicAdd(work, 32ull);  // 32 slots per claim
    s0 = __shfl_sync(kFull, s0, 0);
    if (s0 >= n_slots) break;
    const uint64_t s1 = min((unsigned long long)n_slots, s0 + 32ull);
    for (uint64_t s = s0; s < s1; ++s) {
      const uint32_t L = len[s];
      if (L < 2) continue;
      const uint32_t o = off[s];
      for (uint32_t jb = 0; jb < L; jb += 32) {  // lanes: events jb + lane (the later ones)
        const uint32_t j = jb + (uint32_t)lane;
        const bool vj = j < L;
        const uint32_t b = vj ? (uint32_t)act_s[o + j] : 0u;
        const int64_t tj = vj ? ts_s[o + j] : 0;
        for (uint32_t ib = 0; ib < min(L, jb + 32); ib += 32) {  // earlier events in chunks
          const uint32_t i_me = ib + (uint32_t)lane;
          const uint32_t a_me = i_me < L ? (uint32_t)act_s[o + i_me] : 0u;
          const int64_t t_me = i_me < L ? ts_s[o + i_me] : 0;
          const uint32_t kmax = min(32u, min(L, jb + 32) - ib);
          for (uint32_t k = 0; k < kmax; ++k) {
            const uint32_t i = ib + k;
            const uint32_t a = __shfl_sync(kFull, a_me, (int)k);
            const int64_t ti = __shfl_sync(kFull, t_me, (int)k);
            if (vj && j > i) ef_add(t, a * A + b, (uint64_t)tj - (uint64_t)ti);
          }
        }
      }
    }
  }
}

// Adds copies 1..K-1 of the table into copy 0, exactly (carries between the
// words of each sum).
__global__ void k_efg_fold(EfTable t, uint64_t cells, uint64_t copy_stride, uint32_t n_copies) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < cells; k += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t c = t.cnt[k], slo = t.s_lo[k], shi = t.s_hi[k], q0 = t.q0[k], q1 = t.q1[k], q2 = t.q2[k];
    for (uint32_t r = 1; r < n_copies; ++r) {
      const uint64_t o = k + (uint64_t)r * copy_stride;
      c += t.cnt[o];
      const uint64_t a = t.s_lo[o];
      slo += a;
      shi += t.s_hi[o] + (slo < a ? 1u : 0u);
      const uint64_t b0 = t.q0[o], b1 = t.q1[o];
      q0 += b0;
      const uint64_t c0 = q0 < b0 ? 1u : 0u;
      const uint64_t s1 = q1 + b1;
      const uint64_t c1 = s1 < q1 ? 1u : 0u;
      q1 = s1 + c0;
      q2 += t.q2[o] + c1 + (q1 < s1 ? 1u : 0u);
    }
    t.cnt[k] = c;
    t.s_lo[k] = slo;
    t.s_hi[k] = shi;
    t.q0[k] = q0;
    t.q1[k] = q1;
    t.q2[k] = q2;
  }
}

__global__ void k_efg_flags(const unsigned long long *cnt, uint64_t cells, uint32_t *flags) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < cells; k += (uint64_t)gridDim.x * blockDim.x)
    flags[k] = cnt[k] ? 1u : 0u;
}

// 256-bit arithmetic for the variance numerator (four 64-bit limbs, low first).
struct W4 {
  uint64_t w[4];
};

__device__ __forceinline__ W4 mul_w3_u64(uint64_t x0, uint64_t x1, uint64_t x2, uint64_t m) {
  W4 r;
  uint64_t lo = x0 * m, hi = __umul64hi(x0, m);
  r.w[0] = lo;
  uint64_t c = hi;
  lo = x1 * m;
  hi = __umul64hi(x1, m);
  r.w[1] = lo + c;
  c = hi + (r.w[1] < lo ? 1u : 0u);
  lo = x2 * m;
  hi = __umul64hi(x2, m);
  r.w[2] = lo + c;
  r.w[3] = hi + (r.w[2] < lo ? 1u : 0u);
  return r;
}

__device__ __forceinline__ W4 square_w2(uint64_t lo, uint64_t hi) {  // (hi:lo)^2
  // (h 2^64 + l)^2 = h^2 2^128 + 2 h l 2^64 + l^2
  const uint64_t ll_lo = lo * lo, ll_hi = __umul64hi(lo, lo);
  const uint64_t hl_lo = hi * lo, hl_hi = __umul64hi(hi, lo);
  const uint64_t hh_lo = hi * hi, hh_hi = __umul64hi(hi, hi);
  // 2 h l as three words
  const uint64_t m0 = hl_lo << 1, m1 = (hl_hi << 1) | (hl_lo >> 63), m2 = hl_hi >> 63;
  W4 r;
  r.w[0] = ll_lo;
  uint64_t s = ll_hi + m0;
  uint64_t c = s < ll_hi ? 1u : 0u;
  r.w[1] = s;
  uint64_t s2 = hh_lo + m1;
  uint64_t c2 = s2 < hh_lo ? 1u : 0u;
  const uint64_t s3 = s2 + c;
  c2 += s3 < s2 ? 1u : 0u;
  r.w[2] = s3;
  r.w[3] = hh_hi + m2 + c2;
  return r;
}

__device__ __forceinline__ W4 sub_w4(const W4 &a, const W4 &b) {
  W4 r;
  uint64_t borrow = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint64_t d = a.w[k] - b.w[k];
    const uint64_t d2 = d - borrow;
    borrow = (a.w[k] < b.w[k] ? 1u : 0u) | (d < borrow ? 1u : 0u);
    r.w[k] = d2;
  }
  return r;
}

// Nearest double to a 256-bit integer, ties to even: the top 53 significant
// bits, rounded up when the dropped bits exceed half of the last kept one or
// equal it with the last kept bit odd.
__device__ __forceinline__ double w4_to_double_rn(const W4 &x) {
  int top = 3;
  while (top > 0 && x.w[top] == 0) --top;
  if (top == 0) return __ull2double_rn(x.w[0]);
  const int nb = 64 * top + (64 - __clzll((long long)x.w[top]));  // significant bits, > 64
  const int drop = nb - 53;                                         // > 11
  // the top 64 bits, left-aligned
  const int q = drop / 64, r = drop % 64;  // bit `drop` lies in word q at position r
  uint64_t top64;
  if (r == 0) top64 = x.w[q];
  else top64 = (x.w[q] >> r) | (q + 1 < 4 ? x.w[q + 1] << (64 - r) : 0ull);
  const uint64_t mant = top64 & ((1ull << 53) - 1);  // bits [drop, drop + 53)
  // dropped part: bits [0, drop); compare with half = bit drop - 1
  const int hb = drop - 1, hq = hb / 64, hr = hb % 64;
  const bool half_bit = (x.w[hq] >> hr) & 1u;
  bool below = false;  // any set bit under the half bit
  for (int k = 0; k < hq; ++k) below = below || x.w[k] != 0;
  below = below || (hr > 0 && (x.w[hq] & ((1ull << hr) - 1)) != 0);
  uint64_t m = mant;
  if (half_bit && (below || (m & 1u))) ++m;  // m may reach 2^53: still exact
  return scalbn(__ull2double_rn(m), drop);
}

__global__ void k_efg_compact(EfTable t, uint64_t cells, uint32_t A, const uint32_t *flags, const uint32_t *pos,
                              int32_t *src, int32_t *dst, unsigned long long *o_cnt, unsigned long long *o_slo,
                              unsigned long long *o_shi, unsigned long long *o_q0, unsigned long long *o_q1,
                              unsigned long long *o_q2, double *o_mean, double *o_sd) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < cells; k += (uint64_t)gridDim.x * blockDim.x) {
    if (!flags[k]) continue;
    const uint32_t p = pos[k];
    const uint64_t n = t.cnt[k], slo = t.s_lo[k], shi = t.s_hi[k], q0 = t.q0[k], q1 = t.q1[k], q2 = t.q2[k];
    src[p] = (int32_t)(k / A);
    dst[p] = (int32_t)(k % A);
    o_cnt[p] = n;
    o_slo[p] = slo;
    o_shi[p] = shi;
    o_q0[p] = q0;
    o_q1[p] = q1;
    o_q2[p] = q2;
    o_mean[p] = edge_mean(shi, slo, n);
    const W4 num = sub_w4(mul_w3_u64(q0, q1, q2, n), square_w2(slo, shi));
    const double dn = __ull2double_rn(n);
    o_sd[p] = sqrt(w4_to_double_rn(num) / dn / dn);
  }
}

}  // namespace
}  // namespace pm4g

int pm4g_efg(pm4g_log *L, pm4g_efg_t *out) {
  pm4g::ApiRange nvtx_range("pm4g_efg");
  if (!L || !out) {
    set_error("pm4g_efg: NULL argument");
    return PM4G_EINVAL;
  }
  memset(out, 0, sizeof(*out));
  Ctx *c = L->ctx;
  PM4G_CK(cudaSetDevice(c->device));
  const uint32_t A = (uint32_t)L->A;
  const uint64_t cells = (uint64_t)A * A;
  auto alloc_out = [&](size_t P) {
    out->n_pairs = (int64_t)P;
    const size_t m = std::max<size_t>(P, 1);
    out->src = (int32_t *)malloc(m * 4);
    out->dst = (int32_t *)malloc(m * 4);
    uint64_t **u[] = {&out->count, &out->sum_lo, &out->sum_hi, &out->sq0, &out->sq1, &out->sq2};
    bool ok = out->src && out->dst;
    for (auto p : u) ok = ((*p = (uint64_t *)malloc(m * 8)) != nullptr) && ok;
    out->mean = (double *)malloc(m * 8);
    out->stdev = (double *)malloc(m * 8);
    return ok && out->mean && out->stdev;
  };
  if (L->n == 0 || L->C == 0) {
    if (!alloc_out(0)) {
      pm4g_efg_free(out);
      return PM4G_ENOMEM;
    }
    return PM4G_OK;
  }
  PM4G_TRY(ensure_offsets(L));
  if (!L->ts_s.p) {  // timestamps in formatted order (shared with the drill-down index)
    PM4G_TRY(alloc_buf(c, L->ts_s, (size_t)L->n));
    const int st = run_export(L, nullptr, nullptr, L->ts_s.p, nullptr);
    if (st != PM4G_OK) {  // an unfilled array must not look formed to the next call
      free_buf(c, L->ts_s);
      return st;
    }
  }
  // copies of the table: at most one per block of the pair kernel, within
  // min(8 GB, an eighth of free memory); more copies spread the frequent
  // pairs' atomics further (on the 206.6M-event log, 12 MB a copy: 5 copies
  // 437 ms, 16 copies 316 ms, 64 copies 200 ms, 256 copies 154 ms, 699
  // copies 142 ms)
  const unsigned blocks = 8u * (unsigned)c->num_sms;
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  const uint64_t table_bytes = 48 * cells;
  const uint64_t budget = std::min<uint64_t>(8ull << 30, fr / 8);
  // the dense A x A table must fit at least once (large alphabets)
  if (table_bytes > std::max<uint64_t>(budget, fr / 2)) {
    set_error("pm4g_efg: the %d x %d activity-pair table (%llu bytes) does not fit the device", (int)A, (int)A,
              (unsigned long long)table_bytes);
    return PM4G_ENOMEM;
  }
  // (and one copy per 2^17 events, so a small log does not clear and fold
  // gigabytes of copies)
  const uint64_t by_work = std::max<uint64_t>(1, (uint64_t)L->n >> 17);
  const uint32_t K = (uint32_t)std::max<uint64_t>(
      1, std::min<uint64_t>(std::min<uint64_t>(blocks, by_work), budget / std::max<uint64_t>(table_bytes, 1)));
  Scratch S(c);
  unsigned long long *tab = S.get<unsigned long long>(6 * cells * K);
  unsigned long long *work = S.get<unsigned long long>(1);
  uint32_t *flags = S.get<uint32_t>(cells), *pos = S.get<uint32_t>(cells + 1);
  if (!tab || !work || !flags || !pos) {
    set_error("pm4g_efg: out of device memory");
    return PM4G_ENOMEM;
  }
  cudaStream_t s = c->stream;
  PM4G_CK(cudaMemsetAsync(tab, 0, 6 * cells * K * 8, s));
  PM4G_CK(cudaMemsetAsync(work, 0, 8, s));
  // layout: word w of copy r of cell k at tab[(w * K + r) * cells + k]
  const uint64_t cs = cells;  // stride between copies of one word
  EfTable t{tab, tab + cells * K, tab + 2 * cells * K, tab + 3 * cells * K, tab + 4 * cells * K, tab + 5 * cells * K};
  {
    KTime kt(c, "efg");
    k_efg_pairs<<<blocks, 256, 0, s>>>(L->len.p, L->off.p, L->R, L->act_s.p, L->ts_s.p, A, t, cs, K,
                                               work);
    PM4G_TRY(check_launch(c, "k_efg_pairs"));
    if (K > 1) {
      k_efg_fold<<<grid_for((int64_t)cells, 256, 65535), 256, 0, s>>>(t, cells, cs, K);
      PM4G_TRY(check_launch(c, "k_efg_fold"));
    }
    k_efg_flags<<<grid_for((int64_t)cells, 256, 65535), 256, 0, s>>>(t.cnt, cells, flags);
    PM4G_TRY(check_launch(c, "k_efg_flags"));
  }
  PM4G_TRY(scan_u32(c, flags, pos, (int64_t)cells));
  uint32_t P = 0;
  PM4G_TRY(d2h(c, &P, pos + cells, 4));
  int32_t *osrc = S.get<int32_t>(P), *odst = S.get<int32_t>(P);
  unsigned long long *o6 = S.get<unsigned long long>(6 * (size_t)P);
  double *o2 = S.get<double>(2 * (size_t)P);
  if (P && (!osrc || !odst || !o6 || !o2)) {
    set_error("pm4g_efg: out of device memory");
    return PM4G_ENOMEM;
  }
  if (P) {
    KTime kt(c, "efg");
    k_efg_compact<<<grid_for((int64_t)cells, 256, 65535), 256, 0, s>>>(
        t, cells, A, flags, pos, osrc, odst, o6, o6 + P, o6 + 2 * (size_t)P, o6 + 3 * (size_t)P,
        o6 + 4 * (size_t)P, o6 + 5 * (size_t)P, o2, o2 + P);
    PM4G_TRY(check_launch(c, "k_efg_compact"));
  }
  if (!alloc_out(P)) {
    pm4g_efg_free(out);
    return PM4G_ENOMEM;
  }
  if (P) {
    D2HBatch hb(c, (size_t)P * 72 + 16 * 11);
    hb.add(out->src, osrc, (size_t)P * 4);
    hb.add(out->dst, odst, (size_t)P * 4);
    uint64_t *dsts[] = {out->count, out->sum_lo, out->sum_hi, out->sq0, out->sq1, out->sq2};
    for (int k = 0; k < 6; ++k) hb.add(dsts[k], o6 + (size_t)k * P, (size_t)P * 8);
    hb.add(out->mean, o2, (size_t)P * 8);
    hb.add(out->stdev, o2 + P, (size_t)P * 8);
    const int st = hb.finish();
    if (st != PM4G_OK) {
      pm4g_efg_free(out);
      return st;
    }
  }
  return PM4G_OK;
}

int pm4g_efg_free(pm4g_efg_t *r) {
  if (!r) return PM4G_OK;
  void *p[] = {r->src, r->dst, r->count, r->sum_lo, r->sum_hi, r->sq0, r->sq1, r->sq2, r->mean, r->stdev};
  for (void *q : p) free(q);
  memset(r, 0, sizeof(*r));
  return PM4G_OK;
}
