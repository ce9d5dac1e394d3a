// CPU oracle for the process-mining summaries of a columnar event log.
//
// TEST INFRASTRUCTURE. This file is a plain, slow, single-threaded statement of
// what the engine computes, written from the paper's definitions. It is linked
// or executed only by the tests, by the smoke check and by the benchmark's CPU
// baseline leg; the engine never calls it and shares no code with it.
//
// Paper: Berti, Phan Nghia, van der Aalst, "PM4Py-GPU: a High-Performance
// General-Purpose Library for Process Mining" (arXiv 2204.04898).
//
// Readings of the paper used here (where it is silent or ambiguous):
//  * Ordering (Section 3, the first formatting step): events are ordered by case
//    identifier, then timestamp, then the event's absolute row index. Case ids
//    compare as signed int32, timestamps as signed int64, rows ascending.
//  * A case is a maximal run of equal case ids in that order; cases appear in
//    ascending case id order.
//  * Directly-follows pairs (Section 3, the directly-follows level and the
//    second formatting step, which adds each event's previous activity and
//    timestamp): consecutive events (i, j) of one case. The duration is
//    ts_j - ts_i as an unsigned 64-bit value (exact, since ts_j >= ts_i).
//  * Performance DFG aggregate (Section 3, dfg.py, aggregate unnamed): per edge
//    the count, the exact sum of durations (128-bit), the minimum, the maximum,
//    and mean = (double)sum / (double)count, formed once from the exact sum.
//  * Start/end activities (Section 3, start_end_activities.py): the activity of
//    each case's first and last event; activity frequency (Section 3, event-level
//    aggregation example): occurrences per activity.
//  * Variants (Section 3, variant level and variants.py): a case's variant is its
//    exact activity sequence. Variants are ordered by count descending, then by
//    the smallest case id having the variant; the variant id is the rank.
//  * Filters (Section 3, timestamp.py and attributes.py): the case attribute is
//    its value at the case's first event; a case is kept iff the attribute set is
//    empty or holds that value. Time windows are closed [t_lo, t_hi]: EVENTS keeps
//    the events inside the window, CASES_CONTAINED keeps whole cases whose first
//    and last timestamps are inside, CASES_INTERSECTING keeps whole cases whose
//    span overlaps the window. The result keeps the original rows.
//  * Filters on derived results (Section 3, the directly-follows, case and
//    variant levels; cases_df.py, variants.py, start_end_activities.py and
//    dfg.py's paths filtering). Paths: an event is kept iff it has a previous
//    event in its case and the pair (previous activity, its activity) is one of
//    the given pairs; with exclude, exactly the other events are kept. Cases: a
//    case is kept iff every given criterion holds (an absent one holds): number
//    of events in [min_events, max_events]; throughput time (last timestamp
//    minus first, as an unsigned 64-bit difference) in [min_duration,
//    max_duration]; first activity in the start set; last activity in the end
//    set; at least one event whose activity is in the activity set; variant id
//    (the rank above) in the variant set. With exclude, exactly the other cases
//    are kept. Either way the result is the kept rows, ascending.
//  * Eventually-follows graph and temporal profile (Section 3, efg.py): a pair
//    of events (i, j) of one case eventually follows when i comes before j in
//    the case's order (i < j as positions; a pair needs two distinct events).
//    Per activity pair (a, b) with at least one such pair: the count, the exact
//    sum of ts_j - ts_i (128-bit) and the exact sum of their squares (192-bit);
//    mean = (double)sum / (double)count as for the DFG; the standard deviation
//    is the population one, sqrt(var) with var = rn(count * sumsq - sum^2) /
//    (double)count / (double)count, where rn rounds the exact non-negative
//    integer to the nearest double (ties to even) and every other step is one
//    IEEE operation.
//
// Status codes: 0 ok, -1 invalid argument, -2 activity code outside [0, A).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <tuple>
#include <utility>
#include <vector>

namespace {

typedef unsigned __int128 u128;

struct EdgeAgg {
  uint64_t count = 0;
  u128 sum = 0;
  uint64_t min = ~0ULL;
  uint64_t max = 0;
};

struct VariantAgg {
  uint64_t count = 0;
  int32_t min_case = 0;
};

struct Result {
  int64_t n_events = 0;
  int32_t n_activities = 0;
  std::vector<int64_t> sorted_rows;  // rows in (case, ts, row) order
  std::vector<int32_t> case_ids;     // ascending
  std::vector<int64_t> case_off;     // n_cases + 1 offsets into sorted_rows
  std::vector<std::pair<std::pair<int32_t, int32_t>, EdgeAgg>> edges;  // ascending (src, dst)
  std::vector<uint64_t> start, end, freq;
  std::vector<uint64_t> var_count;
  std::vector<int32_t> var_min_case;
  std::vector<std::vector<int32_t>> var_seq;
  std::vector<int32_t> case_variant;  // per case, aligned with case_ids
};

int validate(const int32_t *case_id, const int32_t *act, const int64_t *ts, int64_t n, int32_t A) {
  if (n < 0 || A <= 0) return -1;
  if (n > 0 && (!case_id || !act || !ts)) return -1;
  for (int64_t r = 0; r < n; ++r)
    if (act[r] < 0 || act[r] >= A) return -2;
  return 0;
}

// Section 3, formatting step 1: order by (case id, timestamp, absolute row).
std::vector<int64_t> sort_rows(const int32_t *case_id, const int64_t *ts, int64_t n) {
  std::vector<int64_t> rows(n);
  for (int64_t r = 0; r < n; ++r) rows[r] = r;
  std::sort(rows.begin(), rows.end(), [&](int64_t a, int64_t b) {
    return std::make_tuple(case_id[a], ts[a], a) < std::make_tuple(case_id[b], ts[b], b);
  });
  return rows;
}

void summarize(const int32_t *case_id, const int32_t *act, const int64_t *ts, int64_t n, int32_t A,
               Result &R) {
  R.n_events = n;
  R.n_activities = A;
  R.sorted_rows = sort_rows(case_id, ts, n);
  const std::vector<int64_t> &s = R.sorted_rows;

  // Cases: maximal runs of equal case ids in sorted order.
  for (int64_t i = 0; i < n; ++i) {
    if (i == 0 || case_id[s[i]] != case_id[s[i - 1]]) {
      R.case_ids.push_back(case_id[s[i]]);
      R.case_off.push_back(i);
    }
  }
  R.case_off.push_back(n);
  const int64_t C = (int64_t)R.case_ids.size();

  // Directly-follows pairs and their durations (Section 3, directly-follows level).
  std::map<std::pair<int32_t, int32_t>, EdgeAgg> dfg;
  R.start.assign(A, 0);
  R.end.assign(A, 0);
  R.freq.assign(A, 0);
  for (int64_t c = 0; c < C; ++c) {
    const int64_t b = R.case_off[c], e = R.case_off[c + 1];
    R.start[act[s[b]]] += 1;
    R.end[act[s[e - 1]]] += 1;
    for (int64_t i = b; i < e; ++i) R.freq[act[s[i]]] += 1;
    for (int64_t i = b; i + 1 < e; ++i) {
      const int64_t x = s[i], y = s[i + 1];
      const uint64_t delta = (uint64_t)ts[y] - (uint64_t)ts[x];
      EdgeAgg &g = dfg[std::make_pair(act[x], act[y])];
      g.count += 1;
      g.sum += (u128)delta;
      g.min = std::min(g.min, delta);
      g.max = std::max(g.max, delta);
    }
  }
  R.edges.assign(dfg.begin(), dfg.end());

  // Variants: exact activity sequences (Section 3, variant level).
  std::map<std::vector<int32_t>, VariantAgg> var;
  std::vector<std::vector<int32_t>> case_seq(C);
  for (int64_t c = 0; c < C; ++c) {
    std::vector<int32_t> seq;
    for (int64_t i = R.case_off[c]; i < R.case_off[c + 1]; ++i) seq.push_back(act[s[i]]);
    auto it = var.find(seq);
    if (it == var.end()) {
      VariantAgg v;
      v.count = 1;
      v.min_case = R.case_ids[c];
      var.emplace(seq, v);
    } else {
      it->second.count += 1;
      it->second.min_case = std::min(it->second.min_case, R.case_ids[c]);
    }
    case_seq[c] = std::move(seq);
  }
  std::vector<std::pair<std::vector<int32_t>, VariantAgg>> vv(var.begin(), var.end());
  std::sort(vv.begin(), vv.end(), [](const auto &a, const auto &b) {
    if (a.second.count != b.second.count) return a.second.count > b.second.count;
    return a.second.min_case < b.second.min_case;
  });
  std::map<std::vector<int32_t>, int32_t> rank;
  for (size_t k = 0; k < vv.size(); ++k) {
    R.var_count.push_back(vv[k].second.count);
    R.var_min_case.push_back(vv[k].second.min_case);
    R.var_seq.push_back(vv[k].first);
    rank[vv[k].first] = (int32_t)k;
  }
  R.case_variant.resize(C);
  for (int64_t c = 0; c < C; ++c) R.case_variant[c] = rank[case_seq[c]];
}

}  // namespace

extern "C" {

// Computes every summary of the log (Section 3). Returns a status code; on
// success *out holds a result handle to be released with oracle_free.
int oracle_summarize(const int32_t *case_id, const int32_t *act, const int64_t *ts, int64_t n,
                     int32_t n_activities, void **out) {
  if (!out) return -1;
  *out = nullptr;
  int st = validate(case_id, act, ts, n, n_activities);
  if (st != 0) return st;
  Result *R = new Result();
  summarize(case_id, act, ts, n, n_activities, *R);
  *out = R;
  return 0;
}

void oracle_free(void *h) { delete static_cast<Result *>(h); }

int64_t oracle_n_events(void *h) { return static_cast<Result *>(h)->n_events; }
int64_t oracle_n_cases(void *h) { return (int64_t) static_cast<Result *>(h)->case_ids.size(); }
int64_t oracle_n_edges(void *h) { return (int64_t) static_cast<Result *>(h)->edges.size(); }
int64_t oracle_n_variants(void *h) { return (int64_t) static_cast<Result *>(h)->var_count.size(); }

// Rows in (case, timestamp, row) order: the formatted log of Section 3.
void oracle_sorted_rows(void *h, int64_t *rows) {
  const Result *R = static_cast<Result *>(h);
  std::copy(R->sorted_rows.begin(), R->sorted_rows.end(), rows);
}

// Frequency and performance DFG, edges ascending by (src, dst).
void oracle_edges(void *h, int32_t *src, int32_t *dst, uint64_t *count, uint64_t *sum_lo,
                  uint64_t *sum_hi, uint64_t *mn, uint64_t *mx, double *mean) {
  const Result *R = static_cast<Result *>(h);
  for (size_t k = 0; k < R->edges.size(); ++k) {
    const auto &e = R->edges[k];
    src[k] = e.first.first;
    dst[k] = e.first.second;
    count[k] = e.second.count;
    sum_lo[k] = (uint64_t)e.second.sum;
    sum_hi[k] = (uint64_t)(e.second.sum >> 64);
    mn[k] = e.second.min;
    mx[k] = e.second.max;
    mean[k] = (double)e.second.sum / (double)e.second.count;
  }
}

// Start, end and frequency counts per activity code (arrays of n_activities).
void oracle_endpoints(void *h, uint64_t *start, uint64_t *end, uint64_t *freq) {
  const Result *R = static_cast<Result *>(h);
  std::copy(R->start.begin(), R->start.end(), start);
  std::copy(R->end.begin(), R->end.end(), end);
  std::copy(R->freq.begin(), R->freq.end(), freq);
}

// Number of activity codes over all variant sequences (CSR payload length).
int64_t oracle_n_variant_acts(void *h) {
  const Result *R = static_cast<Result *>(h);
  int64_t t = 0;
  for (const auto &s : R->var_seq) t += (int64_t)s.size();
  return t;
}

// Variants in rank order: count, smallest case id, CSR offsets and activities.
void oracle_variants(void *h, uint64_t *count, int32_t *min_case, int64_t *off, int32_t *acts) {
  const Result *R = static_cast<Result *>(h);
  int64_t o = 0;
  for (size_t k = 0; k < R->var_seq.size(); ++k) {
    count[k] = R->var_count[k];
    min_case[k] = R->var_min_case[k];
    off[k] = o;
    for (int32_t a : R->var_seq[k]) acts[o++] = a;
  }
  off[R->var_seq.size()] = o;
}

// Per case (ascending case id): id, number of events, variant id.
void oracle_cases(void *h, int32_t *case_ids, int64_t *case_len, int32_t *case_variant) {
  const Result *R = static_cast<Result *>(h);
  for (size_t c = 0; c < R->case_ids.size(); ++c) {
    case_ids[c] = R->case_ids[c];
    case_len[c] = R->case_off[c + 1] - R->case_off[c];
    case_variant[c] = R->case_variant[c];
  }
}

// Drill-down filter (Section 3, timestamp.py and attributes.py). Writes the kept
// rows, ascending, to rows_out (capacity n) and returns their number, or a
// negative status. mode: 0 none, 1 events, 2 cases contained, 3 cases
// intersecting. attr may be NULL only when n_attr == 0.
int64_t oracle_filter(const int32_t *case_id, const int32_t *act, const int64_t *ts,
                      const int32_t *attr, int64_t n, int32_t n_activities, const int32_t *attr_set,
                      int32_t n_attr, int64_t t_lo, int64_t t_hi, int32_t mode, int64_t *rows_out) {
  int st = validate(case_id, act, ts, n, n_activities);
  if (st != 0) return st;
  if (mode < 0 || mode > 3 || n_attr < 0 || (n_attr > 0 && (!attr || !attr_set))) return -1;
  std::vector<int64_t> s = sort_rows(case_id, ts, n);
  std::vector<char> keep(n, 0);
  int64_t b = 0;
  while (b < n) {
    int64_t e = b + 1;
    while (e < n && case_id[s[e]] == case_id[s[b]]) ++e;
    bool case_ok = true;
    if (n_attr > 0) {
      const int32_t v = attr[s[b]];
      case_ok = std::find(attr_set, attr_set + n_attr, v) != attr_set + n_attr;
    }
    const int64_t first = ts[s[b]], last = ts[s[e - 1]];
    if (case_ok && mode == 2) case_ok = first >= t_lo && last <= t_hi;
    if (case_ok && mode == 3) case_ok = first <= t_hi && last >= t_lo;
    for (int64_t i = b; i < e; ++i) {
      bool k = case_ok;
      if (k && mode == 1) k = ts[s[i]] >= t_lo && ts[s[i]] <= t_hi;
      keep[s[i]] = k ? 1 : 0;
    }
    b = e;
  }
  int64_t m = 0;
  for (int64_t r = 0; r < n; ++r)
    if (keep[r]) rows_out[m++] = r;
  return m;
}

// Paths filter (Section 3, the directly-follows level; dfg.py paths filtering).
// Writes the kept rows, ascending, to rows_out (capacity n) and returns their
// number, or a negative status.
int64_t oracle_filter_paths(const int32_t *case_id, const int32_t *act, const int64_t *ts, int64_t n,
                            int32_t n_activities, const int32_t *src, const int32_t *dst, int32_t n_pairs,
                            int32_t exclude, int64_t *rows_out) {
  int st = validate(case_id, act, ts, n, n_activities);
  if (st != 0) return st;
  if (n_pairs < 0 || (n_pairs > 0 && (!src || !dst))) return -1;
  std::vector<std::pair<int32_t, int32_t>> pairs;
  for (int32_t k = 0; k < n_pairs; ++k) pairs.emplace_back(src[k], dst[k]);
  std::vector<int64_t> s = sort_rows(case_id, ts, n);
  std::vector<char> keep(n, 0);
  for (int64_t i = 0; i < n; ++i) {
    bool match = false;
    if (i > 0 && case_id[s[i - 1]] == case_id[s[i]]) {
      const std::pair<int32_t, int32_t> p(act[s[i - 1]], act[s[i]]);
      match = std::find(pairs.begin(), pairs.end(), p) != pairs.end();
    }
    keep[s[i]] = (match != (exclude != 0)) ? 1 : 0;
  }
  int64_t m = 0;
  for (int64_t r = 0; r < n; ++r)
    if (keep[r]) rows_out[m++] = r;
  return m;
}

// Case filters (Section 3, the case and variant levels). Bounds are inclusive
// and a negative bound is absent; an empty set is absent. Writes the kept rows,
// ascending, to rows_out (capacity n) and returns their number, or a negative
// status.
int64_t oracle_filter_cases(const int32_t *case_id, const int32_t *act, const int64_t *ts, int64_t n,
                            int32_t n_activities, int64_t min_events, int64_t max_events,
                            int64_t min_duration, int64_t max_duration, const int32_t *start_set,
                            int32_t n_start, const int32_t *end_set, int32_t n_end, const int32_t *act_set,
                            int32_t n_act, const int32_t *variant_set, int32_t n_variant, int32_t exclude,
                            int64_t *rows_out) {
  int st = validate(case_id, act, ts, n, n_activities);
  if (st != 0) return st;
  if (n_start < 0 || n_end < 0 || n_act < 0 || n_variant < 0 || (n_start > 0 && !start_set) ||
      (n_end > 0 && !end_set) || (n_act > 0 && !act_set) || (n_variant > 0 && !variant_set))
    return -1;
  Result R;
  summarize(case_id, act, ts, n, n_activities, R);
  const std::vector<int64_t> &s = R.sorted_rows;
  auto in = [](const int32_t *set, int32_t m, int32_t v) { return std::find(set, set + m, v) != set + m; };
  std::vector<char> keep(n, 0);
  for (size_t c = 0; c < R.case_ids.size(); ++c) {
    const int64_t b = R.case_off[c], e = R.case_off[c + 1];
    const int64_t len = e - b;
    const uint64_t dur = (uint64_t)ts[s[e - 1]] - (uint64_t)ts[s[b]];
    bool ok = true;
    if (min_events >= 0 && len < min_events) ok = false;
    if (max_events >= 0 && len > max_events) ok = false;
    if (min_duration >= 0 && dur < (uint64_t)min_duration) ok = false;
    if (max_duration >= 0 && dur > (uint64_t)max_duration) ok = false;
    if (n_start > 0 && !in(start_set, n_start, act[s[b]])) ok = false;
    if (n_end > 0 && !in(end_set, n_end, act[s[e - 1]])) ok = false;
    if (n_act > 0) {
      bool any = false;
      for (int64_t i = b; i < e; ++i) any = any || in(act_set, n_act, act[s[i]]);
      if (!any) ok = false;
    }
    if (n_variant > 0 && !in(variant_set, n_variant, R.case_variant[c])) ok = false;
    if (exclude) ok = !ok;
    for (int64_t i = b; i < e; ++i) keep[s[i]] = ok ? 1 : 0;
  }
  int64_t m = 0;
  for (int64_t r = 0; r < n; ++r)
    if (keep[r]) rows_out[m++] = r;
  return m;
}

// Unsigned integers of four 64-bit limbs (little end first), for the exact
// variance numerator of the temporal profile.
struct U256 {
  uint64_t w[4] = {0, 0, 0, 0};
};

U256 mul_u64_by(const uint64_t *x, int nx, uint64_t m) {  // x (nx limbs) times m
  U256 r;
  u128 carry = 0;
  for (int k = 0; k < 4; ++k) {
    const u128 p = (k < nx ? (u128)x[k] * m : 0) + carry;
    r.w[k] = (uint64_t)p;
    carry = p >> 64;
  }
  return r;
}

U256 square_u128(u128 v) {  // v * v, exactly
  const uint64_t lo = (uint64_t)v, hi = (uint64_t)(v >> 64);
  const uint64_t x[2] = {lo, hi};
  U256 a = mul_u64_by(x, 2, lo), b = mul_u64_by(x, 2, hi);
  U256 r;  // a + (b << 64)
  u128 carry = 0;
  for (int k = 0; k < 4; ++k) {
    const u128 t = (u128)a.w[k] + (k >= 1 ? b.w[k - 1] : 0) + carry;
    r.w[k] = (uint64_t)t;
    carry = t >> 64;
  }
  return r;
}

U256 sub_u256(const U256 &a, const U256 &b) {  // a - b, a >= b
  U256 r;
  uint64_t borrow = 0;
  for (int k = 0; k < 4; ++k) {
    const uint64_t d = a.w[k] - b.w[k] - borrow;
    borrow = (a.w[k] < b.w[k] || (a.w[k] == b.w[k] && borrow)) ? 1 : 0;
    r.w[k] = d;
  }
  return r;
}

// The nearest double to x, ties to even (the top 53 significant bits, then
// the round bit and the sticky bits below it).
double u256_to_double(const U256 &x) {
  int top = -1;
  for (int k = 3; k >= 0 && top < 0; --k)
    for (int b = 63; b >= 0; --b)
      if ((x.w[k] >> b) & 1) {
        top = 64 * k + b;
        break;
      }
  if (top < 0) return 0.0;
  auto bit = [&](int i) -> uint64_t { return i < 0 ? 0 : (x.w[i / 64] >> (i % 64)) & 1; };
  if (top < 53) {
    double v = 0;
    for (int i = top; i >= 0; --i) v = v * 2 + (double)bit(i);
    return v;
  }
  uint64_t mant = 0;
  for (int i = top; i > top - 53; --i) mant = (mant << 1) | bit(i);
  const int rpos = top - 53;
  const uint64_t round = bit(rpos);
  bool sticky = false;
  for (int i = rpos - 1; i >= 0 && !sticky; --i) sticky = bit(i) != 0;
  if (round && (sticky || (mant & 1))) ++mant;  // may carry into bit 53: still exact below
  return std::ldexp((double)mant, rpos + 1);
}

struct EfAgg {
  uint64_t count = 0;
  u128 sum = 0;
  U256 sq;  // sum of squared durations (at most 192 bits)
};

// Eventually-follows graph and temporal profile (Section 3, efg.py). Returns a
// handle (released with oracle_free_efg) and the number of activity pairs in
// *n_pairs, or NULL on a bad argument or activity code.
void *oracle_efg(const int32_t *case_id, const int32_t *act, const int64_t *ts, int64_t n, int32_t n_activities,
                 int64_t *n_pairs) {
  if (validate(case_id, act, ts, n, n_activities) != 0 || !n_pairs) return nullptr;
  std::vector<int64_t> s = sort_rows(case_id, ts, n);
  auto *M = new std::map<std::pair<int32_t, int32_t>, EfAgg>();
  int64_t b = 0;
  while (b < n) {
    int64_t e = b + 1;
    while (e < n && case_id[s[e]] == case_id[s[b]]) ++e;
    for (int64_t i = b; i < e; ++i)
      for (int64_t j = i + 1; j < e; ++j) {
        const uint64_t d = (uint64_t)ts[s[j]] - (uint64_t)ts[s[i]];
        EfAgg &g = (*M)[std::make_pair(act[s[i]], act[s[j]])];
        g.count += 1;
        g.sum += (u128)d;
        const u128 d2 = (u128)d * d;
        u128 carry = 0;
        const uint64_t add[4] = {(uint64_t)d2, (uint64_t)(d2 >> 64), 0, 0};
        for (int k = 0; k < 4; ++k) {
          const u128 t = (u128)g.sq.w[k] + add[k] + carry;
          g.sq.w[k] = (uint64_t)t;
          carry = t >> 64;
        }
      }
    b = e;
  }
  *n_pairs = (int64_t)M->size();
  return M;
}

// The pairs ascending by (a, b): counts, sums (low, high words), sums of
// squares (three words, low first), means and standard deviations.
void oracle_efg_pairs(void *h, int32_t *src, int32_t *dst, uint64_t *count, uint64_t *sum_lo, uint64_t *sum_hi,
                      uint64_t *sq0, uint64_t *sq1, uint64_t *sq2, double *mean, double *stdev) {
  const auto *M = static_cast<std::map<std::pair<int32_t, int32_t>, EfAgg> *>(h);
  size_t k = 0;
  for (const auto &kv : *M) {
    const EfAgg &g = kv.second;
    src[k] = kv.first.first;
    dst[k] = kv.first.second;
    count[k] = g.count;
    sum_lo[k] = (uint64_t)g.sum;
    sum_hi[k] = (uint64_t)(g.sum >> 64);
    sq0[k] = g.sq.w[0];
    sq1[k] = g.sq.w[1];
    sq2[k] = g.sq.w[2];
    mean[k] = (double)g.sum / (double)g.count;
    const U256 num = sub_u256(mul_u64_by(g.sq.w, 3, g.count), square_u128(g.sum));
    const double var = u256_to_double(num) / (double)g.count / (double)g.count;
    stdev[k] = std::sqrt(var);
    ++k;
  }
}

void oracle_free_efg(void *h) { delete static_cast<std::map<std::pair<int32_t, int32_t>, EfAgg> *>(h); }

}  // extern "C"
