// Kernel argument blocks and launch declarations shared between the .cu files.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pm4g {

struct FormatArgs {
  const int32_t *case_id;
  const int32_t *activity;
  const int64_t *ts;
  int64_t n;
  int64_t chunk;     // rows per CTA (multiple of 4)
  int32_t min_case;  // slot = case id - min_case
  int clb;           // log2(case slots per bucket)
  int act_bits;
  int32_t n_act;
  uint32_t nb;       // number of buckets
  uint32_t *mat;     // CTA-major bucket counts [ctas * nb]
  const uint32_t *bucket_off;
  uint4 *rec;
  uint32_t *err_flags;
  // bucket histogram only: the largest slot a case id may take under
  // min_case, and the word that is set when some id falls outside
  // [min_case, min_case + slot_hi] (null: the range is known to hold all ids)
  uint32_t slot_hi;
  uint32_t *range_err;
};

// Bucket partition (format.cu)
constexpr int kPartThreads = 512;
constexpr int kPartWarps = kPartThreads / 32;
constexpr uint32_t kPartMaxBins = 512;
static_assert(kPartMaxBins <= (uint32_t)kPartThreads, "one thread per digit");

struct PartArgs {
  const int32_t *case_id;
  const int32_t *activity;
  const int64_t *ts;
  int64_t n;
  int64_t chunk;
  int32_t min_case;
  int32_t n_act;
  int act_bits;
  int clb;
  int fbits;
  uint32_t nbins;
  const uint4 *rec_in;
  const uint32_t *bucket_off;
  uint32_t nb;
  const uint32_t *cur1;      // level 1 cursors: CTA-major coarse prefixes plus coarse starts
  const uint32_t *mat;       // level 2: CTA-major prefixes of the final-bucket counts
  int p_ctas;                // row chunks of level 1
  int splits;                // level 2: units per coarse bucket
  uint4 *rec_out;
  uint32_t *err_flags;
  uint32_t *keys_out;        // optional: the final level also writes every record's first word here
};

__host__ __device__ inline size_t part_wh_bytes(uint32_t nbins) { return ((size_t)kPartWarps * nbins * 2 + 15) / 16 * 16; }
// staging tile (items records a thread), per-warp 16-bit counts, per-warp
// peer masks, cursors, staged starts, block-scan scratch and each digit's
// output-minus-staged offset
__host__ __device__ inline size_t part_smem_bytes_hd(uint32_t nbins, int items) {
  return (size_t)kPartThreads * items * 16 + part_wh_bytes(nbins) + (size_t)kPartWarps * nbins * 4 +
         (size_t)(3 * nbins + 1 + 32) * 4;
}
inline size_t part_smem_bytes(uint32_t nbins, int items) { return part_smem_bytes_hd(nbins, items); }
// items: records a thread takes per tile, 8 or 4
cudaError_t launch_partition(int level, const PartArgs &a, unsigned grid, cudaStream_t s, int items);
__global__ void k_coarse_counts(const uint32_t *mat, uint32_t nb, int p_ctas, int fbits, uint32_t nc, uint32_t *mat1);
__global__ void k_add_base(uint32_t *mat1, int p_ctas, uint32_t nc, const uint32_t *bucket_off, int fbits);

__global__ void k_stats(const int32_t *case_id, int64_t n, int2 *partial);
constexpr int kRangeSamples = 4096;
__global__ void k_sample_range(const int32_t *case_id, int64_t n, int2 *out);
__global__ void k_bucket_hist(FormatArgs a, uint32_t b_lo, uint32_t nbs);
__global__ void k_bucket_hist16(FormatArgs a);
__global__ void k_bucket_colprefix(uint32_t *mat, uint32_t nb, int p_ctas, uint32_t *total);
__global__ void k_bucket_scatter(FormatArgs a, uint32_t b_lo, uint32_t nbs);
__global__ void k_case_keys(const int32_t *case_id, int64_t n, uint32_t *keys, uint32_t *vals);
__global__ void k_case_heads(const uint32_t *keys, int64_t n, uint32_t *head);
__global__ void k_case_dense(const uint32_t *keys, const uint32_t *rows, const uint32_t *head,
                             const uint32_t *head_excl, int64_t n, int32_t *dense, int32_t *uniq);

// Global DFG table: dense over the A*A cells (key = src*A + dst indexes it),
// or, when key is set, open addressing over mask + 1 slots whose key array
// holds key + 1 (0 marks an empty slot); err (hashed only) gets bit 0 if a
// pair finds the table full.
struct DfgTable {
  unsigned long long *cnt, *lo, *hi, *mn, *mx;
  unsigned long long *key = nullptr;
  uint64_t mask = 0;
  uint32_t *err = nullptr;
};

struct SegArgs {
  const uint4 *rec;
  const uint32_t *bucket_off;
  uint32_t nb;
  int clb;
  int act_bits;
  uint32_t n_act;
  uint64_t n_slots;
  int cap;        // events a bucket may hold in shared memory
  int ep_smem;    // 1: start/end counts privatised in shared memory
  int tbl_mode;   // 0: dense shared table over A*A cells, 1: hashed shared table
  int tbl_slots;  // shared table slots (power of two in hashed mode)
  uint32_t *work; // bucket work counter
  uint16_t *act_s;
  uint32_t *len;
  const int32_t *attr_in;
  int32_t *cattr;
  DfgTable g;
  unsigned long long *g_start, *g_end;
  uint32_t *ovf;
  uint32_t *n_ovf;
  unsigned long long *n_cases;
  unsigned long long *n_sorted;  // optional: windows/cases that needed sorting
  // export mode (formatted log in sorted order)
  int32_t *ex_case;
  int64_t *ex_ts;
  int64_t *ex_row;
  int32_t min_case;
  const int32_t *uniq;
  int skip_ordered;  // sorting pass: do nothing unless the streaming pass found a case out of order
  // streaming pass: bit 0 set when case lengths disagree with the records;
  // kStDisorder when a case's events are not in timestamp order in its
  // bucket (the pass then stops early; the sorting pass redoes the log)
  uint32_t *err;
  const uint32_t *keys;         // streaming pass: first word of every bucketed record (bucket order)
  // streaming pass: edge ids (emap, A * A, ~0 = none yet), the key of every
  // id (key_of, kStSlots) and the id counter; ids below kStSlots index the
  // shared edge table directly
  uint32_t *emap, *key_of, *n_ids;
  // streaming pass, optional: every case slot's first formatted position
  // (n_slots + 1 entries, the last = the event count), and a word set to 1
  // when the pass ran (its outputs count only without kStDisorder)
  uint32_t *off_out, *ran;
};
constexpr uint32_t kStDisorder = 4u;

// Streaming segment pass (stream.cu): one warp per bucket, for logs whose
// cases' events are in timestamp order in row order (it checks this itself). Shared memory: an edge table of
// kStSlots slots indexed by edge id (count, low and middle sum words, high
// words of the pushed minimum and maximum), the endpoint counts, then per
// warp the case state of its bucket (last timestamp, first position, events
// seen, last activity: 20 bytes per case slot).
constexpr int kStMaxThreads = 1024;
constexpr int kStSlots = 4096;
struct StSmem {
  size_t tcnt, st, warp0, per_warp, total;
};
__host__ __device__ inline StSmem st_smem_layout(int ncl, int a_s, int n_warps) {
  StSmem L;
  L.tcnt = 0;
  L.st = (size_t)kStSlots * 20;
  L.warp0 = (L.st + (size_t)a_s * 8 + 15) / 16 * 16;
  L.per_warp = ((size_t)ncl * 20 + 15) / 16 * 16;
  L.total = L.warp0 + (size_t)n_warps * L.per_warp;
  return L;
}
// warps per block whose layout fits smem_optin (0: none)
int stream_segment_warps(int clb, int a_s, size_t smem_optin);
cudaError_t launch_stream_segment(const SegArgs &a, int n_warps, unsigned grid, size_t smem, cudaStream_t s);
// After a streaming pass that found a case out of order: clears what it added
// to the global edge table (dense), the endpoint counts, the case counter and
// the bucket counter, so that the sorting pass starts from zero (returns at
// once otherwise).
cudaError_t launch_stream_undo(const SegArgs &a, uint32_t n_act, unsigned grid, cudaStream_t s);

struct SegSmem {
  size_t rec, tlo, hw, rng, flg, ccnt, cstart, st, en, tkey, tcnt, tminh, tmaxh, misc, total;
};

constexpr int kSegThreads = 1024;
constexpr int kSegWarps = kSegThreads / 32;
constexpr int kSegChunks = 8;  // records a thread holds in registers: capacity <= kSegThreads * kSegChunks

__host__ __device__ inline size_t seg_align(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Shared-memory layout of the segment kernel: cap records of 16 bytes, the
// per-warp case counts (whose area the ordered index of sorted cases, 2 bytes
// per record, reuses once the counts are spent), per-case arrays, endpoint
// counts and the edge table (key, count, 64-bit sum, high words of the pushed
// minimum and maximum).
__host__ __device__ inline SegSmem seg_smem_layout(int cap, int ncl, int a_s, int tbl_slots, int tbl_mode) {
  SegSmem L;
  size_t o = 0;
  L.rec = o;
  o += (size_t)cap * 16;
  L.tlo = o;
  o += (size_t)tbl_slots * 8;
  L.hw = o;
  const size_t hw_bytes = (size_t)kSegWarps * ((ncl + 1) & ~1) * 2, idx_bytes = (size_t)cap * 2;
  o += seg_align(hw_bytes > idx_bytes ? hw_bytes : idx_bytes, 16);
  L.rng = o;
  o += (size_t)(2 * ncl + 4) * 4;
  L.flg = o;
  o += seg_align((size_t)ncl, 16);
  L.ccnt = o;
  o += (size_t)(ncl + 1) * 4;
  L.cstart = o;
  o += (size_t)(ncl + 1) * 4;
  L.st = o;
  o += (size_t)a_s * 4;
  L.en = o;
  o += (size_t)a_s * 4;
  L.tkey = o;
  o += (size_t)(tbl_mode ? tbl_slots : 0) * 4;
  L.tcnt = o;
  o += (size_t)tbl_slots * 4;
  L.tminh = o;
  o += (size_t)tbl_slots * 4;
  L.tmaxh = o;
  o += (size_t)tbl_slots * 4;
  L.misc = seg_align(o, 16);
  o = L.misc + 256;
  L.total = seg_align(o, 16);
  return L;
}

constexpr int kMaxCaseSmem = 512;  // longest case sorted on chip

// Host launchers (the kernels are templates on the export mode).
cudaError_t launch_segment(bool exp, const SegArgs &a, unsigned grid, size_t smem, cudaStream_t s);
cudaError_t launch_fb_compute(bool exp, const SegArgs &a, const uint4 *srec, uint32_t n, uint32_t bucket,
                              const uint32_t *cstart, unsigned grid, cudaStream_t s);

// Global-memory path for one bucket whose records were sorted by
// (case slot, timestamp, row) into srec.
__global__ void k_fb_hist(const uint4 *srec, uint32_t n, int act_bits, uint32_t cmask, uint32_t *ccnt);
__global__ void k_fb_cases(SegArgs a, const uint4 *srec, uint32_t bucket, const uint32_t *ccnt,
                           const uint32_t *cstart, int ncl, int write_cases);
__global__ void k_fb_keys_row(const uint4 *rec, uint32_t n, uint32_t *keys, uint32_t *vals);
__global__ void k_fb_keys_ts(const uint4 *rec, const uint32_t *perm, uint32_t n, uint64_t *keys);
__global__ void k_fb_keys_case(const uint4 *rec, const uint32_t *perm, uint32_t n, int act_bits, uint32_t cmask,
                               uint32_t *keys);
__global__ void k_fb_gather(const uint4 *rec, const uint32_t *perm, uint32_t n, uint4 *out);
__global__ void k_fill_u64(unsigned long long *p, int64_t n, unsigned long long v);

// Filter kernels (one CTA per bucket, records streamed from global memory).
struct FilterArgs {
  const uint4 *rec;
  const uint32_t *bucket_off;
  uint32_t nb;
  int clb;
  int act_bits;
  uint64_t n_slots;
  int64_t *first_ts;  // per slot
  int64_t *last_ts;   // per slot
  const int32_t *cattr;
  const int32_t *attr_set;  // sorted, device
  int32_t n_attr;
  int64_t t_lo, t_hi;
  int32_t mode;
  uint8_t *case_ok;  // per slot
  const uint32_t *row_keep;  // optional, one bit per original row: replaces case_ok and the window
  const uint32_t *len;      // optional, per slot: whole-case predicates count kept events from it
  uint32_t *kept;    // per bucket
  const uint32_t *new_off;
  uint4 *out;
  uint32_t *keys_out;  // optional: the first word of every written record (the streaming pass's case counts)
};
__global__ void k_case_span(FilterArgs a);
__global__ void k_case_ok(FilterArgs a);
__global__ void k_filter_count(FilterArgs a);
__global__ void k_filter_write(FilterArgs a);

// Case filters on derived results: one thread per case slot.
struct CaseFilterArgs {
  uint64_t n_slots;
  const uint32_t *len, *off;     // per slot: events, first formatted position
  const uint16_t *act_s;         // activities in formatted order
  const int64_t *first_ts, *last_ts;
  const int32_t *cvar;           // per slot variant id (only with variants)
  int64_t min_events, max_events, min_duration, max_duration;  // negative: absent
  const uint32_t *start_bits, *end_bits, *act_bits;            // activity bitmaps, NULL: absent
  const int32_t *variants;       // sorted variant ids
  int32_t n_variants;            // 0: absent
  int32_t exclude;
  uint8_t *case_ok;
};
__global__ void k_case_filter(CaseFilterArgs a);
// Paths filter: first formatted position of every case, then the kept rows.
__global__ void k_mark_case_starts(const uint32_t *len, const uint32_t *off, uint64_t n_slots, uint8_t *start);
__global__ void k_path_keep(uint64_t n, const uint16_t *act_s, const uint8_t *start, const int64_t *row_s,
                            const uint64_t *keys, int32_t n_keys, uint32_t n_act, int32_t exclude,
                            uint32_t *row_keep);

// Summaries (summaries.cu)
__global__ void k_dfg_flags(const unsigned long long *cnt, int64_t cells, uint32_t *flags);
__global__ void k_dfg_compact(DfgTable g, int64_t cells, uint32_t n_act, const uint32_t *flags,
                              const uint32_t *pos, int32_t *src, int32_t *dst, unsigned long long *cnt,
                              unsigned long long *lo, unsigned long long *hi, unsigned long long *mn,
                              unsigned long long *mx, double *mean);
__global__ void k_freq(const unsigned long long *cnt, const unsigned long long *end, uint32_t n_act,
                       unsigned long long *freq);
__global__ void k_gkey_flags(const unsigned long long *gkey, uint64_t T, uint32_t *flags);
__global__ void k_gkey_compact(const unsigned long long *gkey, uint64_t T, const uint32_t *flags, const uint32_t *pos,
                               uint32_t *keys, uint32_t *slots);
__global__ void k_dfg_gather(DfgTable g, const uint32_t *keys, const uint32_t *slots, uint32_t E, uint32_t n_act,
                             int32_t *src, int32_t *dst, unsigned long long *cnt, unsigned long long *lo,
                             unsigned long long *hi, unsigned long long *mn, unsigned long long *mx, double *mean);
__global__ void k_freq_edges(const int32_t *src, const unsigned long long *cnt, uint32_t E, unsigned long long *freq);
__global__ void k_freq_end(const unsigned long long *end, uint32_t n_act, unsigned long long *freq);

}  // namespace pm4g
