// Device helpers shared by the engine's kernels: the bucketed event record,
// hashing for variant keys, warp-level reductions and the warp bitonic sort
// used to order each case's events by (timestamp, row).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pm4g {

typedef unsigned __int128 u128;

constexpr int kWarp = 32;
constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kSlotLoMask = 0xFFFFu;  // case-slot bits kept in a record

// ---------------------------------------------------------------------------
// Bucketed event record (16 bytes, one 128-bit store/load):
//   x = (slot_lo << act_bits) | activity   slot_lo: low 16 bits of the case slot;
//                                           its low clb bits are the slot within
//                                           the bucket
//   y = row                                 0-based row in the loaded columns
//   z, w = timestamp low / high 32 bits     signed int64
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 make_rec(uint32_t case_lo, uint32_t act, int act_bits, uint32_t row,
                                          int64_t ts) {
  uint64_t t = (uint64_t)ts;
  return make_uint4((case_lo << act_bits) | act, row, (uint32_t)t, (uint32_t)(t >> 32));
}
// 16-byte store that asks L2 to keep the line (a bucket front's sector is
// completed by a later store of the same CTA).
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void st_evict_last(uint4 *p, uint4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w), "l"(pol)
               : "memory");
}
// Asks the copy engine to bring [p, p + bytes) into L2 (a hint: nothing is
// written, and the range lies inside an allocation). p must be 16-byte
// aligned and bytes a multiple of 16; issued in 32 KB pieces.
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
  const char *c = static_cast<const char *>(p);
  for (uint32_t o = 0; o < bytes; o += 32768u) {
    const uint32_t sz = min(32768u, bytes - o);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(c + o), "r"(sz) : "memory");
  }
}
// Bulk copies from shared to global memory through the tensor memory
// accelerator (one thread per copy; both addresses and the size multiples of
// 16 bytes). Shared-memory writes a copy reads must be fenced to the async
// proxy (fence_smem_to_async by every writer, then a barrier) first.
__device__ __forceinline__ void bulk_copy_s2g(void *gdst, const void *ssrc, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst),
               "r"((uint32_t)__cvta_generic_to_shared(ssrc)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// this thread's committed copies have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// this thread's committed copies are complete (their writes are visible)
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// L2 prefetch of the 16-byte-aligned interior of [p, p + bytes): it never
// touches a byte outside the range, whatever the alignment of p.
__device__ __forceinline__ void prefetch_l2_inner(const void *p, size_t bytes) {
  const uintptr_t b = ((uintptr_t)p + 15) & ~(uintptr_t)15, e = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
  if (e > b) prefetch_l2(reinterpret_cast<const void *>(b), (uint32_t)(e - b));
}
__device__ __forceinline__ int64_t rec_ts(uint4 r) {
  return (int64_t)(((uint64_t)r.w << 32) | (uint64_t)r.z);
}
// Order-preserving map of a signed timestamp to an unsigned key.
__device__ __forceinline__ uint64_t ts_key(int64_t ts) { return (uint64_t)ts ^ 0x8000000000000000ULL; }

// ---------------------------------------------------------------------------
// Hashing. fmix64 and fmix32 are the finalizers of MurmurHash3 (Austin
// Appleby, public domain). A case's variant hash sums, over its events, a
// 64-bit term of (activity, position in case, seed): its low words and its
// high words each in a 32-bit wrap-around sum. The two words of a term are
// two independent 32-bit mixes, so a term costs two fmix32 rather than a
// 64-bit multiply chain. The sum is order-sensitive through the position, and
// any thread can add any event's term. It only accelerates grouping; equality
// of sequences is always verified.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t fmix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdULL;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ULL;
  k ^= k >> 33;
  return k;
}
__host__ __device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}
__host__ __device__ __forceinline__ uint64_t event_hash(uint32_t act, uint32_t pos, uint64_t seed) {
  const uint32_t s0 = (uint32_t)seed * 0x9E3779B9u, s1 = (uint32_t)(seed >> 32) ^ 0x7F4A7C15u;
  const uint32_t lo = fmix32(act * 0x9E3779B1u + pos * 0x85EBCA77u + s0 + 0x632BE59Bu);
  const uint32_t hi = fmix32((act ^ 0x5BD1E995u) * 0xC2B2AE3Du + pos * 0x27D4EB2Fu + (s0 ^ s1) + 0x165667B1u);
  return ((uint64_t)hi << 32) | lo;
}
// Grouping key of a case from its sequence hash and length; never 0 (0 marks
// an empty table slot). bits < 64 truncates it (tests force collisions).
__host__ __device__ __forceinline__ uint64_t variant_key(uint64_t h, uint32_t len, int bits) {
  uint64_t k = fmix64(h ^ fmix64((uint64_t)len * 0xD6E8FEB86659FD93ULL + 1));
  if (bits > 0 && bits < 64) k &= ((1ULL << bits) - 1);
  return k == 0 ? 1 : k;
}

// ---------------------------------------------------------------------------
// Mean of a performance-DFG edge: the exact 128-bit duration sum converted to
// double with round-to-nearest-even (IEEE 754), divided by the count (also
// converted), so that it equals (double)sum / (double)count computed on the
// host. The conversion keeps the top 53 significant bits and rounds on the
// bits below them: above half up, below half down, exactly half to even.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double u128_to_double_rn(uint64_t hi, uint64_t lo) {
  if (hi == 0) return __ull2double_rn(lo);
  const int nbits = 128 - __clzll((long long)hi);  // 65..128 significant bits
  const int shift = nbits - 53;                    // 12..75 low bits dropped
  uint64_t mant;     // the top 53 bits
  bool above, half;  // dropped bits compared with half of the last kept bit
  if (shift < 64) {
    mant = (hi << (64 - shift)) | (lo >> shift);
    const uint64_t rem = lo & ((1ull << shift) - 1), h = 1ull << (shift - 1);
    above = rem > h;
    half = rem == h;
  } else {
    const int s2 = shift - 64;  // 0..11 dropped bits of hi, then all of lo
    mant = hi >> s2;
    if (s2 == 0) {
      above = lo > (1ull << 63);
      half = lo == (1ull << 63);
    } else {
      const uint64_t remh = hi & ((1ull << s2) - 1), hh = 1ull << (s2 - 1);
      above = remh > hh || (remh == hh && lo != 0);
      half = remh == hh && lo == 0;
    }
  }
  if (above || (half && (mant & 1ull))) ++mant;
  int e = shift;
  if (mant >> 53) {  // rounding carried into a 54th bit
    mant >>= 1;
    ++e;
  }
  // mant < 2^53 converts exactly; scaling by 2^e (e <= 76) is exact
  return (double)mant * __longlong_as_double((long long)(1023 + e) << 52);
}
__device__ __forceinline__ double edge_mean(uint64_t sum_hi, uint64_t sum_lo, uint64_t count) {
  return u128_to_double_rn(sum_hi, sum_lo) / __ull2double_rn(count);
}

// Fire-and-forget 64-bit global minimum / maximum (no value comes back, so
// the issuing warp does not wait for the memory system).
__device__ __forceinline__ void red_min_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("red.relaxed.gpu.global.min.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void red_max_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("red.relaxed.gpu.global.max.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void red_add_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Guards of the extremes a block has pushed to global memory, kept as the bit
// patterns of non-negative floats (which order like their bits). A minimum
// guard holds a value rounded up from one already pushed, so a duration whose
// downward-rounded float is at or above it cannot lower the global minimum; a
// maximum guard holds a value rounded down, so a duration whose upward-rounded
// float is at or below it cannot raise the global maximum. Only durations
// within a float's relative precision of the pushed extreme, or beyond it,
// are pushed.
__device__ __forceinline__ uint32_t guard_up(uint64_t v) { return __float_as_uint(__ull2float_ru(v)); }
__device__ __forceinline__ uint32_t guard_down(uint64_t v) { return __float_as_uint(__ull2float_rd(v)); }
constexpr uint32_t kGuardMinInit = 0x7F800000u;  // +infinity: nothing pushed yet
constexpr uint32_t kGuardMaxInit = 0u;           // 0.0f: the global maxima start at 0, so 0 needs no push

// ---------------------------------------------------------------------------
// Warp helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Ranks lanes by runs of equal keys on consecutive lanes (inactive lanes pass
// key = ~0): returns the lane of this lane's run head and the run length (valid
// on the head). A key repeated on non-adjacent lanes forms separate runs.
__device__ __forceinline__ uint32_t run_head(uint32_t key, uint32_t &run_len) {
  const uint32_t lane = lane_id();
  const uint32_t prev = __shfl_up_sync(kFull, key, 1);
  const uint32_t heads = __ballot_sync(kFull, lane == 0 || prev != key);
  const uint32_t head = 31 - __clz(heads & (0xFFFFFFFFu >> (31 - lane)));
  const uint32_t above = heads & ~(0xFFFFFFFFu >> (31 - lane));  // heads after this lane
  const uint32_t next = above ? (uint32_t)(__ffs(above) - 1) : 32u;
  run_len = next - lane;
  return head;
}

// ---------------------------------------------------------------------------
// Warp bitonic sort of up to 32*E (key, row, payload) triples held in
// registers, blocked layout: lane l holds elements l*E .. l*E+E-1. Sorted
// ascending by (key, row). Pads must use key = ~0, row = ~0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool kr_less(uint64_t ka, uint32_t ra, uint64_t kb, uint32_t rb) {
  return ka < kb || (ka == kb && ra < rb);
}

template <int E>
__device__ __forceinline__ void warp_bitonic_sort(uint64_t (&key)[E], uint32_t (&row)[E], uint32_t (&pay)[E]) {
  constexpr int N = 32 * E;
  const int lane = (int)lane_id();
#pragma unroll
  for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j < E) {
        // partner inside this lane
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int ei = e ^ j;
          if (ei > e) {
            const int i = lane * E + e;
            const bool asc = (i & k) == 0;
            const bool sw = asc ? kr_less(key[ei], row[ei], key[e], row[e]) : kr_less(key[e], row[e], key[ei], row[ei]);
            if (sw) {
              uint64_t tk = key[e]; key[e] = key[ei]; key[ei] = tk;
              uint32_t tr = row[e]; row[e] = row[ei]; row[ei] = tr;
              uint32_t tp = pay[e]; pay[e] = pay[ei]; pay[ei] = tp;
            }
          }
        }
      } else {
        const int lm = j / E;  // partner lane distance
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int i = lane * E + e;
          const uint64_t ok = __shfl_xor_sync(kFull, key[e], lm);
          const uint32_t orow = __shfl_xor_sync(kFull, row[e], lm);
          const uint32_t opay = __shfl_xor_sync(kFull, pay[e], lm);
          const bool lower = (lane & lm) == 0;     // this element has the lower index
          const bool asc = (i & k) == 0;
          const bool other_less = kr_less(ok, orow, key[e], row[e]);
          // lower index keeps the min when ascending, the max when descending
          const bool take = (lower == asc) ? other_less : !other_less;
          if (take) {
            key[e] = ok;
            row[e] = orow;
            pay[e] = opay;
          }
        }
      }
    }
  }
}

// Block-wide exclusive scan of one value per thread (NT threads); returns the
// thread's exclusive prefix and writes the block total. s_warp holds 32 words.
template <int NT>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *s_warp, uint32_t &total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < NT / 32 ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(kFull, t, o);
      if (lane >= o) t += y;
    }
    if (lane < NT / 32) s_warp[lane] = t;
  }
  __syncthreads();
  total = s_warp[NT / 32 - 1];
  const uint32_t before = w > 0 ? s_warp[w - 1] : 0;
  const uint32_t r = before + x - v;
  __syncthreads();
  return r;
}

}  // namespace pm4g
