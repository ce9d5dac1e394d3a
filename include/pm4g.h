/*
 * pm4g.h - C ABI of a B300-native engine for the process-mining summaries of a
 * columnar event log.
 *
 * Paper: A. Berti, M. Phan Nghia, W.M.P. van der Aalst, "PM4Py-GPU: a
 * High-Performance General-Purpose Library for Process Mining", arXiv
 * 2204.04898. The calls follow the paper's usage (Section 3, Listing 1): a log
 * is ingested and formatted once (ordering by case, timestamp and absolute
 * index), then queried for the frequency/performance directly-follows graph,
 * start/end activities and variants, and drilled down with timestamp and
 * attribute filters.
 *
 * Conventions
 *  - Every function returns an int status: PM4G_OK (0) or a negative code.
 *    No C++ exception crosses this boundary. pm4g_last_error() returns a
 *    message for the calling thread's most recent failure.
 *  - A query or filter that returns PM4G_ENOMEM leaves its log usable and
 *    holding no memory of the failed attempt; the same call may be retried
 *    (with more memory free) and then gives the results it would have given.
 *  - A context (pm4g_ctx) binds one CUDA device and one stream; all work of
 *    the context and of its logs runs in order on that stream. A context is
 *    used by one thread at a time.
 *  - Input columns are owned by the caller. Host inputs are copied. Device
 *    inputs are read only until pm4g_load_log returns.
 *  - Log handles and result arrays are owned by the library. Result arrays are
 *    host memory (malloc) released by the matching *_free call.
 *  - Limits: 0 <= n_events <= 2^31 - 1; 1 <= n_activities <= 65536. Up to
 *    4096 activities the directly-follows pairs are aggregated into a table
 *    dense over the A x A pairs; above that, into an open-addressing table
 *    of twice as many slots as the log can have distinct pairs (Section 3:
 *    the DFG of large alphabets goes to a hashed global table). Results are
 *    the same either way. pm4g_efg needs its dense A x A table (48 bytes a
 *    cell) to fit the device, and pm4g_dfg_noalloc keeps its own limits.
 *
 * Outputs are exact: counts and duration sums/min/max are integers (durations
 * are unsigned 64-bit nanosecond differences, sums 128-bit); the mean duration
 * is (double)sum / (double)count, formed once from the exact sum.
 */
#ifndef PM4G_H
#define PM4G_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes */
#define PM4G_OK 0
#define PM4G_EINVAL (-1)   /* null pointer, negative size, bad mode or option */
#define PM4G_ERANGE (-2)   /* an activity code outside [0, n_activities); results larger than caller buffers */
#define PM4G_ENOMEM (-3)   /* the allocator returned NULL */
#define PM4G_ECUDA (-4)    /* a CUDA runtime call failed */
#define PM4G_ETIMEOUT (-5) /* a bounded device wait gave up */

/* pm4g_load_log flags: where the input columns live */
#define PM4G_HOST_PTRS 0x1u
#define PM4G_DEVICE_PTRS 0x2u

/* pm4g_variants flags */
#define PM4G_VARIANTS_CASES 0x1u /* also return case_ids[] and case_variant[] */

/* Time-window modes of pm4g_filter (Section 3, timestamp.py) */
#define PM4G_TW_NONE 0
#define PM4G_TW_EVENTS 1
#define PM4G_TW_CASES_CONTAINED 2
#define PM4G_TW_CASES_INTERSECTING 3

/* Context options (pm4g_ctx_set_option) */
#define PM4G_OPT_TIMING 1            /* 1 = time every kernel launch with CUDA events;
                                        2 = time only the dominant kernels (segment,
                                        partition, batch_dfg, efg, filter), whose
                                        events then cost the host little; 0 = off */
#define PM4G_OPT_TEST_HASH_BITS 2    /* test only: keep this many bits (1..63) of the
                                        variant key, forcing the collision path; 0 = off */
#define PM4G_OPT_TEST_BUCKET_CAP 3   /* test only: events a bucket may hold in shared
                                        memory (>= 32); smaller values force the
                                        global-memory path; 0 = default */
/* Launch choices of pm4g_load_log's single-log pass (results never depend on
 * them; 0 = the library's default; set by the autotuner): */
#define PM4G_OPT_EDGE_TABLE 7         /* global edge table: 0 = dense up to 4096 activities,
                                        hashed above; 1 = hashed at any alphabet size */
#define PM4G_OPT_LOAD_CLB 8           /* log2 of the case slots of a bucket, 1..8 */
#define PM4G_OPT_LOAD_SPLITS 9        /* units each coarse bucket's second partition level is
                                        cut into, 1..64 */
#define PM4G_OPT_STREAM_WARPS 10      /* most warps per block of the streaming segment pass,
                                        1..32; the pass takes fewer where its shared memory
                                        (or, at 256-slot buckets, its 28-warp register
                                        budget) does not allow that many */
#define PM4G_OPT_STREAM_OFF 11        /* 1 = the sorting segment pass for every log (also those
                                        whose cases come in timestamp order) */
#define PM4G_OPT_PART1_ITEMS 12       /* records a thread stages per tile in the first partition
                                        level: 8 (default; 4,096-record tiles, 2 blocks an SM)
                                        or 4 (2,048-record tiles, 3 blocks an SM) */
#define PM4G_OPT_PART2_ITEMS 13       /* the same for the second partition level: 4 (default)
                                        or 8 */
#define PM4G_OPT_PART_FBITS 14        /* log2 of the final buckets in a coarse bucket of the
                                        first partition level, 1..9, when above the smallest
                                        that keeps the coarse buckets within one pass (fewer,
                                        larger coarse buckets); 0 = that smallest */
/* Launch choices of pm4g_batch_dfg (0 = default; results never depend on them;
 * an autotuner picks them by timing, see paper_2204_04898_b300/autotune.py): */
#define PM4G_OPT_BATCH_CHUNK 4       /* cases a warp takes at once: 8, 16 (default) or 32 */
#define PM4G_OPT_BATCH_STAGES 5      /* groups a batch of >= 64 views into caller-owned
                                        arrays is pipelined in: 1..16 (default 4) */
#define PM4G_OPT_BATCH_ITEMS_PER_SM 6 /* work items per SM a batch's events are cut
                                        into: 1..32 (default 4) */

typedef struct pm4g_ctx pm4g_ctx;
typedef struct pm4g_log pm4g_log;

/* Device-memory hook. alloc returns device memory of `bytes` bytes usable on
 * `stream` (a cudaStream_t), aligned to at least 16 bytes, or NULL on failure
 * (memory that is not aligned is given back and the call fails with
 * PM4G_ENOMEM); free releases it in stream order. `user` is passed through. */
typedef struct {
  void *(*alloc)(size_t bytes, void *stream, void *user);
  void (*free)(void *ptr, size_t bytes, void *stream, void *user);
  void *user;
} pm4g_allocator;

/* Creates a context on CUDA device `device`. cuda_stream is a cudaStream_t to
 * run on (borrowed, not destroyed), or NULL for a stream the context owns.
 * alloc may be NULL: stream-ordered cudaMallocAsync is used, and freed blocks
 * (rounded up to size classes) are kept by the context for reuse, up to half
 * the device memory, until an allocation fails or the context is destroyed;
 * the device's default memory pool is then also set to keep what is freed
 * into it for this process (its release threshold, a per-process setting).
 * *out is set only on success. */
int pm4g_ctx_create(pm4g_ctx **out, int device, void *cuda_stream, const pm4g_allocator *alloc);

/* Destroys a context. Its logs must have been freed. NULL is accepted. */
int pm4g_ctx_destroy(pm4g_ctx *ctx);

/* Sets one PM4G_OPT_* option. */
int pm4g_ctx_set_option(pm4g_ctx *ctx, int option, int64_t value);

/* Kernel timing (when PM4G_OPT_TIMING is on): for kernel `name` (see
 * pm4g_kernel_names), the number of launches and their total device time in
 * milliseconds since the last reset, measured with CUDA events on the context
 * stream. Synchronizes the stream. Unknown names give 0 launches. The name
 * "launches" gives the number of kernels the context launched since the last
 * reset (counted whether or not timing is on). */
int pm4g_ctx_timing(pm4g_ctx *ctx, const char *name, int64_t *launches, double *total_ms);
int pm4g_ctx_timing_reset(pm4g_ctx *ctx);

/* Comma-separated names of the engine's kernels (static string). */
const char *pm4g_kernel_names(void);

/* Ingests and formats a log (Section 3: the log is ordered by case identifier,
 * timestamp and absolute row index; each event's predecessor in its case and
 * a per-case table are derived). Columns have n_events entries:
 *   case_id   int32  case identifier (any int32 values)
 *   activity  int32  activity code in [0, n_activities)
 *   ts_ns     int64  timestamp (any int64 values; nanoseconds by convention)
 *   case_attr int32  optional case attribute (NULL: none); a case's value is
 *                    its value at the case's first event
 * flags is PM4G_HOST_PTRS or PM4G_DEVICE_PTRS. The frequency/performance DFG
 * and endpoints are computed during this call; variants on first request.
 * Errors: EINVAL, ERANGE (nothing is kept), ENOMEM, ECUDA. */
int pm4g_load_log(pm4g_ctx *ctx, const int32_t *case_id, const int32_t *activity,
                  const int64_t *ts_ns, const int32_t *case_attr, int64_t n_events,
                  int32_t n_activities, uint32_t flags, pm4g_log **out);

/* Number of events and of cases (distinct case ids) of a log. */
int pm4g_log_info(const pm4g_log *log, int64_t *n_events, int64_t *n_cases);
/* The n_activities the log was loaded with. */
int pm4g_log_activities(const pm4g_log *log, int32_t *n_activities);

/* Releases a log and its device memory. NULL is accepted. */
int pm4g_log_free(pm4g_log *log);

/* The formatted log (Section 3, format.py): every event in (case id,
 * timestamp, row) order. Each output is a host array of n_events entries, or
 * NULL to skip it. row is the event's 0-based row in the originally loaded
 * columns (a filtered log keeps those rows). */
int pm4g_log_export(pm4g_log *log, int32_t *case_id, int32_t *activity, int64_t *ts_ns,
                    int64_t *row);

/* Frequency DFG (Section 3, dfg.py): edges (src, dst) with count > 0,
 * ascending by (src, dst). An edge counts consecutive events of one case. */
typedef struct {
  int64_t n_edges;
  int32_t *src;
  int32_t *dst;
  uint64_t *count;
} pm4g_dfg_t;
int pm4g_dfg(pm4g_log *log, pm4g_dfg_t *out);
int pm4g_dfg_free(pm4g_dfg_t *res);

/* Performance DFG (Section 3, dfg.py): the frequency DFG plus, per edge, the
 * exact sum (sum_lo + 2^64 * sum_hi), minimum and maximum of the durations
 * ts(next) - ts(prev) as unsigned 64-bit values, and mean = (double)sum /
 * (double)count. */
typedef struct {
  int64_t n_edges;
  int32_t *src;
  int32_t *dst;
  uint64_t *count;
  uint64_t *sum_lo;
  uint64_t *sum_hi;
  uint64_t *min;
  uint64_t *max;
  double *mean;
} pm4g_perf_dfg_t;
int pm4g_perf_dfg(pm4g_log *log, pm4g_perf_dfg_t *out);
int pm4g_perf_dfg_free(pm4g_perf_dfg_t *res);

/* Start and end activity counts (Section 3, start_end_activities.py) and
 * activity frequency (Section 3, event-level aggregation). Caller-provided
 * host arrays of n_activities entries; freq may be NULL. */
int pm4g_start_end(pm4g_log *log, uint64_t *start, uint64_t *end, uint64_t *freq);

/* Variants (Section 3, variants.py): a case's variant is its exact activity
 * sequence. Variants are ranked by count descending, then by smallest case id;
 * the rank is the variant id. top_k < 0 returns all, otherwise the first
 * min(top_k, n_variants). With PM4G_VARIANTS_CASES, case_ids (ascending) and
 * case_variant (variant id of each case) are returned for all n_cases cases. */
typedef struct {
  int64_t n_variants; /* total V */
  int64_t n_out;      /* variants returned */
  uint64_t *count;    /* [n_out] */
  int32_t *min_case;  /* [n_out] smallest case id with the variant */
  int64_t *off;       /* [n_out + 1] CSR offsets into acts */
  int32_t *acts;      /* [off[n_out]] activity sequences */
  int64_t n_cases;    /* entries of case_ids / case_variant (0 without the flag) */
  int32_t *case_ids;
  int32_t *case_variant;
} pm4g_variants_t;
int pm4g_variants(pm4g_log *log, int64_t top_k, uint32_t flags, pm4g_variants_t *out);
int pm4g_variants_free(pm4g_variants_t *res);

/* Drill-down filter (Section 3, timestamp.py and attributes.py; Section 1,
 * drill-down). A case is kept iff n_attr == 0 or its attribute value (at its
 * first event) is in attr_set[0..n_attr). Then the closed window [t_lo, t_hi]
 * applies: EVENTS keeps the events inside it; CASES_CONTAINED keeps cases whose
 * first and last timestamps are inside; CASES_INTERSECTING keeps cases whose
 * span overlaps it; NONE ignores it. The result is a new log (still ordered,
 * original rows kept) owned by the caller, to be freed with pm4g_log_free.
 * attr_set is a host array. A log loaded without case_attr accepts only
 * n_attr == 0. */
typedef struct {
  const int32_t *attr_set;
  int32_t n_attr;
  int64_t t_lo;
  int64_t t_hi;
  int32_t mode;
} pm4g_filter_spec;
int pm4g_filter(pm4g_log *log, const pm4g_filter_spec *spec, pm4g_log **out);

/* Filters on derived results (Section 3: the directly-follows, case and
 * variant levels; the cases, variants, endpoints and paths-filtering modules).
 * Each returns a new log (still ordered, original rows kept) owned by the
 * caller, to be freed with pm4g_log_free; sets are host arrays (repeats
 * allowed). Errors: PM4G_EINVAL for a NULL log/out, a negative set size with
 * or a NULL set of positive size, or an activity code outside [0, A) in a set
 * (variant ids outside [0, n_variants) match no case); PM4G_ENOMEM; PM4G_ECUDA.
 *
 * pm4g_filter_paths keeps the events that have a previous event in their case
 * and whose pair (previous activity, activity) is one of the n_pairs pairs
 * (src[k], dst[k]); with exclude != 0, exactly the other events. The first
 * paths filter of a log forms the original row of every formatted position
 * and keeps it on the log (8 bytes per event) for later paths filters, until
 * the log is freed: the log's device footprint grows by that much.
 *
 * pm4g_filter_cases keeps the cases for which every given criterion holds (a
 * negative bound or an empty set is absent): number of events in [min_events,
 * max_events]; throughput time, the last timestamp minus the first as an
 * unsigned 64-bit difference, in [min_duration, max_duration]; first activity
 * in start_set; last activity in end_set; at least one event with an activity
 * in act_set; variant id (the rank of pm4g_variants: count descending, then
 * smallest case id) in variant_set. With exclude != 0, exactly the other
 * cases. */
int pm4g_filter_paths(pm4g_log *log, const int32_t *src, const int32_t *dst, int32_t n_pairs, int32_t exclude,
                      pm4g_log **out);
typedef struct {
  int64_t min_events, max_events;
  int64_t min_duration, max_duration;
  const int32_t *start_set;
  int32_t n_start;
  const int32_t *end_set;
  int32_t n_end;
  const int32_t *act_set;
  int32_t n_act;
  const int32_t *variant_set;
  int32_t n_variant;
  int32_t exclude;
} pm4g_case_filter;
int pm4g_filter_cases(pm4g_log *log, const pm4g_case_filter *spec, pm4g_log **out);

/* Eventually-follows graph and temporal profile (Section 3, efg.py). A pair
 * of events (i, j) of one case eventually follows when i comes before j in the
 * case's (timestamp, row) order. For every activity pair (src, dst) with at
 * least one such pair, ascending by (src, dst): count; the exact sum of
 * ts_j - ts_i as sum_lo/sum_hi; the exact sum of their squares as sq0 (low
 * word), sq1, sq2; mean = the sum rounded to double over the count (as for
 * the DFG); stdev = the population standard deviation sqrt(v / n / n) with v
 * the exact integer n * S2 - S1^2 rounded to the nearest double (ties to even)
 * and n = (double)count, each step one IEEE operation. Library-allocated
 * arrays, released with pm4g_efg_free. Errors: PM4G_EINVAL (NULL), PM4G_ENOMEM,
 * PM4G_ECUDA. */
typedef struct {
  int64_t n_pairs;
  int32_t *src, *dst;
  uint64_t *count, *sum_lo, *sum_hi, *sq0, *sq1, *sq2;
  double *mean, *stdev;
} pm4g_efg_t;
int pm4g_efg(pm4g_log *log, pm4g_efg_t *out);
int pm4g_efg_free(pm4g_efg_t *res);

/* Batched drill-down (Section 1, drill-down; Section 3, filters then the
 * frequency and performance DFG): for each of n_sub sub-logs, the results that
 * pm4g_filter(log, spec_i) followed by pm4g_perf_dfg and pm4g_start_end on the
 * sub-log would give, computed in one pass over the resident log without
 * forming the sub-logs.
 *   Sub-log i: attribute values attr_vals[attr_off[i] .. attr_off[i+1]) (any
 *   order, repeats allowed; none = no attribute filter), window [t_lo[i],
 *   t_hi[i]] and mode[i] (PM4G_TW_*), as in pm4g_filter_spec. All spec arrays
 *   are host arrays; attr_off has n_sub + 1 entries, attr_off[0] = 0 and
 *   non-decreasing. A log loaded without case_attr accepts only empty lists.
 * Results (host arrays owned by the library, freed with pm4g_batch_dfg_free):
 *   n_events[i], n_cases[i]: size of sub-log i;
 *   edge_off[n_sub + 1]: sub-log i's edges are rows edge_off[i] ..
 *   edge_off[i+1] of src, dst, count, sum_lo, sum_hi, min, max, mean, in
 *   ascending (src, dst) order, with pm4g_perf_dfg's meaning;
 *   start, end, freq: n_sub x n_activities, row i for sub-log i.
 * Errors: PM4G_EINVAL for a malformed spec (n_sub < 0, bad offsets or mode,
 * attribute lists on a log without case_attr), PM4G_ENOMEM, PM4G_ECUDA. */
typedef struct {
  int32_t n_sub;
  const int64_t *attr_off;
  const int32_t *attr_vals;
  const int64_t *t_lo;
  const int64_t *t_hi;
  const int32_t *mode;
  int64_t var_top_k; /* variants per sub-log: 0 none, < 0 all, else the first var_top_k */
} pm4g_batch_spec;
typedef struct {
  int32_t n_sub;
  int32_t n_activities;
  int64_t *n_events;  /* [n_sub] */
  int64_t *n_cases;   /* [n_sub] */
  int64_t *edge_off;  /* [n_sub + 1] */
  int32_t *src;
  int32_t *dst;
  uint64_t *count;
  uint64_t *sum_lo;
  uint64_t *sum_hi;
  uint64_t *min;
  uint64_t *max;
  double *mean;
  uint64_t *start;    /* [n_sub * n_activities] */
  uint64_t *end;
  uint64_t *freq;
  /* Variants of each sub-log (pm4g_variants' order and meaning) when
   * spec->var_top_k != 0: sub-log i has n_variants[i] variants, of which rows
   * var_off[i] .. var_off[i+1] are returned; row r has var_count[r] cases, the
   * smallest case id var_min_case[r] and the activity sequence
   * var_acts[var_seq_off[r] .. var_seq_off[r+1]). */
  int64_t *n_variants;   /* [n_sub] */
  int64_t *var_off;      /* [n_sub + 1] */
  uint64_t *var_count;
  int32_t *var_min_case;
  int64_t *var_seq_off;  /* [rows + 1] */
  int32_t *var_acts;
  int64_t var_capacity;  /* pm4g_batch_dfg_into: rows var_count/var_min_case hold (var_seq_off one more) */
  int64_t acts_capacity; /* pm4g_batch_dfg_into: entries var_acts holds */
} pm4g_batch_dfg_t;
int pm4g_batch_dfg(pm4g_log *log, const pm4g_batch_spec *spec, pm4g_batch_dfg_t *out);
int pm4g_batch_dfg_free(pm4g_batch_dfg_t *res);
/* The same results written into caller-owned host arrays, which may be
 * page-locked and reused from call to call (no allocation, one copy from the
 * device): every pointer of out must be set, n_events/n_cases to n_sub
 * entries, edge_off to n_sub + 1, start/end/freq to n_sub * n_activities and
 * the eight edge arrays to edge_capacity entries (their pointers may be NULL
 * when edge_capacity is 0); with variants, n_variants to n_sub, var_off to
 * n_sub + 1 and the variant arrays to out->var_capacity / acts_capacity. n_sub
 * and n_activities are filled in. If the batch has more edges than
 * edge_capacity, or more variant rows or activities than the variant
 * capacities, the call returns PM4G_ERANGE with the sizes written
 * (edge_off[n_sub] = edges needed, var_off[n_sub] = rows needed, var_seq_off
 * unchanged and acts_capacity set to the activities needed); the overflowing
 * arrays then hold no complete result. Never free out with
 * pm4g_batch_dfg_free. */
int pm4g_batch_dfg_into(pm4g_log *log, const pm4g_batch_spec *spec, pm4g_batch_dfg_t *out, int64_t edge_capacity);

/* Allocation-free frequency/performance DFG and start/end counts of a small
 * log. The paper has no counterpart: this serves callers that cannot allocate
 * device memory when they need the summary (code running under CUDA graph
 * capture, serving processes with a fixed memory budget, hosts whose device
 * memory belongs to another framework's pool).
 *   case_id, activity, ts_ns: device columns of n_events entries
 *     (0 <= n_events <= 262144; max case id - min case id < 262144; no case
 *     longer than 512 events; activity in [0, n_activities), n_activities <=
 *     2048).
 *   Errors: an event count or alphabet outside these limits, a NULL pointer,
 *     or case ids spanning more values return PM4G_EINVAL before any output
 *     is written (beyond the cleared initial values); an activity outside
 *     [0, n_activities) returns PM4G_ERANGE with the outputs cleared only.
 *     A case of more than 512 events returns PM4G_EINVAL after the other
 *     cases' pairs have been added: the outputs are then partly written and
 *     undefined, and must be discarded.
 *   count, sum_lo, sum_hi, min, max: device arrays of n_activities^2 cells,
 *     cell src * n_activities + dst, written by the call (cells without a
 *     pair: count 0, min UINT64_MAX, max 0). start, end: device arrays of
 *     n_activities entries.
 *   cuda_stream: the cudaStream_t to run on (NULL: the legacy default stream).
 * The only working memory is a fixed array inside the library (about 7 MB per
 * GPU that loads it, held until the process exits); the call allocates nothing
 * and returns after the stream has finished its work. All calls share that
 * array: calls that overlap on the GPU race and must be serialised by the
 * caller. The first call on a device looks up the array's device address with
 * that device current; make it before any stream capture. */
int pm4g_dfg_noalloc(const int32_t *case_id, const int32_t *activity, const int64_t *ts_ns,
                     int64_t n_events, int32_t n_activities, void *cuda_stream, uint64_t *count,
                     uint64_t *sum_lo, uint64_t *sum_hi, uint64_t *min, uint64_t *max,
                     uint64_t *start, uint64_t *end);

/* The capturable form of pm4g_dfg_noalloc: no host synchronisation, no
 * allocation and launch shapes that do not depend on the log, so a CUDA graph
 * captured around one call replays for any log of up to 262,144 events copied
 * into the same input arrays. The event count is read from device memory
 * (*n_events_dev); everything is enqueued on cuda_stream and the call returns
 * at once. Input errors come back in *status_dev (device memory, written last):
 * bit 0 an activity outside [0, n_activities), bit 1 a case of more than 512
 * events, bit 2 case ids spanning more than 262,144 values, bit 3 an event
 * count outside [0, 262,144]; with bit 0, 2 or 3 set the outputs hold only
 * their initial values (zero; minima all ones). Host-side argument errors
 * return EINVAL at once. The scratch array and the limits are those of
 * pm4g_dfg_noalloc, and so is the rule on overlapping calls; make one call
 * (of either form) on the device before a stream capture begins. */
int pm4g_dfg_noalloc_async(const int32_t *case_id, const int32_t *activity, const int64_t *ts_ns,
                           const int64_t *n_events_dev, int32_t n_activities, void *cuda_stream, uint64_t *count,
                           uint64_t *sum_lo, uint64_t *sum_hi, uint64_t *min, uint64_t *max, uint64_t *start,
                           uint64_t *end, uint32_t *status_dev);

/* Message of the calling thread's last failure ("" if none). */
const char *pm4g_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PM4G_H */
