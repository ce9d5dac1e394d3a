// Seeded synthetic event-log generator.
//
// Produces columnar event logs (case id int32, activity code int32, timestamp
// int64 ns, optional int32 case attribute) with the shapes of the public logs
// the paper measures on (Section 4, Table 1: case lengths of about 4 to 57
// events, tens of activities, hundreds to tens of thousands of variants),
// pushed to larger sizes. It holds none of the summaries' arithmetic: it only
// draws random logs. Both the CPU oracle and the CUDA engine consume its
// output, unchanged.
//
// Randomness: xoshiro256** (Blackman & Vigna) seeded through SplitMix64. Every
// case draws from its own generator seeded by (seed, case index), so the output
// does not depend on how many threads generate it.
//
// Build: g++ -O2 -std=c++17 -shared -fPIC -pthread synth.cpp -o libpm4g_synth.so

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

inline uint64_t splitmix64(uint64_t &x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

struct Xoshiro256ss {
  uint64_t s[4];
  explicit Xoshiro256ss(uint64_t seed) {
    uint64_t x = seed;
    for (auto &v : s) v = splitmix64(x);
  }
  static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
  uint64_t next() {
    const uint64_t r = rotl(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return r;
  }
  // uniform in [0, 1) with 53 random bits
  double uniform() { return (double)(next() >> 11) * 0x1.0p-53; }
  // uniform in (0, 1]
  double uniform_pos() { return ((double)(next() >> 11) + 1.0) * 0x1.0p-53; }
  uint64_t below(uint64_t n) {  // unbiased integer in [0, n) (Lemire)
    unsigned __int128 m = (unsigned __int128)next() * n;
    uint64_t l = (uint64_t)m;
    if (l < n) {
      uint64_t t = (0 - n) % n;
      while (l < t) {
        m = (unsigned __int128)next() * n;
        l = (uint64_t)m;
      }
    }
    return (uint64_t)(m >> 64);
  }
  double normal() {  // Box-Muller, one value per call
    double u1 = uniform_pos(), u2 = uniform();
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  }
  double gamma(double a) {  // Marsaglia-Tsang; a < 1 boosted via U^(1/a)
    if (a < 1.0) return gamma(a + 1.0) * std::pow(uniform_pos(), 1.0 / a);
    const double d = a - 1.0 / 3.0, c = 1.0 / std::sqrt(9.0 * d);
    for (;;) {
      double x, v;
      do {
        x = normal();
        v = 1.0 + c * x;
      } while (v <= 0.0);
      v = v * v * v;
      double u = uniform_pos();
      if (u < 1.0 - 0.0331 * x * x * x * x) return d * v;
      if (std::log(u) < 0.5 * x * x + d * (1.0 - v + std::log(v))) return d * v;
    }
  }
};

uint64_t case_seed(uint64_t seed, uint64_t idx) {
  uint64_t a = seed ^ 0x5851F42D4C957F2DULL, b = idx * 0xD1342543DE82EF95ULL + 0x2545F4914F6CDD1DULL;
  return splitmix64(a) ^ splitmix64(b);
}

}  // namespace

extern "C" {

// Length laws
enum { SYN_LEN_GEOMETRIC = 0, SYN_LEN_LOGNORMAL = 1, SYN_LEN_FIXED = 2 };
// Activity models
enum { SYN_ACT_DIRICHLET_MARKOV = 0, SYN_ACT_ZIPF_RESTART = 1, SYN_ACT_SPARSE_CHAIN = 2 };
// Gap laws
enum { SYN_GAP_EXPONENTIAL = 0, SYN_GAP_PARETO = 1 };
// Row orders
enum { SYN_ROWS_SHUFFLED = 0, SYN_ROWS_TS_SORTED = 1, SYN_ROWS_CASE_ORDER = 2 };

typedef struct {
  uint64_t seed;
  int64_t n_cases;
  int32_t n_activities;
  int32_t len_law;
  double len_p;        // geometric success probability
  double len_median;   // lognormal median
  double len_sigma;    // lognormal sigma
  int32_t len_cap;     // upper clamp for the length (>= 1)
  int32_t act_model;
  double dirichlet_alpha;
  double zipf_s;
  double restart_p;    // probability of drawing the next activity from pi
  int32_t max_succ;    // sparse chain: successors per activity drawn in 1..max_succ
  int32_t gap_law;
  double gap_mean_ns;  // exponential mean
  double pareto_alpha;
  double pareto_xm_ns;
  double p_zero_gap;   // probability of a zero gap (duplicate timestamp)
  double gap_cap_ns;   // upper clamp for one gap
  double start_span_ns;
  int32_t row_order;
  int32_t n_attr_values;  // 0 = no case attribute; else U[0, n_attr_values)
  int32_t n_threads;      // 0 = hardware concurrency
} synth_params;

}  // extern "C"

namespace {

struct Model {
  int A = 0;
  std::vector<double> pi_cdf;              // first-activity distribution
  std::vector<std::vector<int>> succ;      // per activity: successor list
  std::vector<std::vector<double>> cdf;    // per activity: cumulative weights
  double restart = 0.0;
};

int sample_cdf(const std::vector<double> &c, double u) {
  // first index with c[i] > u*c.back()
  double t = u * c.back();
  auto it = std::upper_bound(c.begin(), c.end(), t);
  if (it == c.end()) --it;
  return (int)(it - c.begin());
}

std::vector<double> cumulative(const std::vector<double> &w) {
  std::vector<double> c(w.size());
  double s = 0;
  for (size_t i = 0; i < w.size(); ++i) c[i] = (s += w[i]);
  return c;
}

Model build_model(const synth_params &p) {
  Model m;
  m.A = p.n_activities;
  const int A = m.A;
  Xoshiro256ss rng(case_seed(p.seed, 0xFFFFFFFFFFFFULL));
  std::vector<double> zipf(A);
  for (int i = 0; i < A; ++i) zipf[i] = std::pow((double)(i + 1), -p.zipf_s);
  m.succ.resize(A);
  m.cdf.resize(A);
  if (p.act_model == SYN_ACT_DIRICHLET_MARKOV) {
    std::vector<double> w(A);
    for (int i = 0; i < A; ++i) w[i] = rng.gamma(p.dirichlet_alpha);
    m.pi_cdf = cumulative(w);
    for (int a = 0; a < A; ++a) {
      for (int i = 0; i < A; ++i) w[i] = rng.gamma(p.dirichlet_alpha);
      m.succ[a].resize(A);
      for (int i = 0; i < A; ++i) m.succ[a][i] = i;
      m.cdf[a] = cumulative(w);
    }
  } else if (p.act_model == SYN_ACT_ZIPF_RESTART) {
    m.pi_cdf = cumulative(zipf);
    double zs = m.pi_cdf.back();
    std::vector<double> w(A);
    for (int a = 0; a < A; ++a) {
      double s = 0;
      for (int i = 0; i < A; ++i) s += (w[i] = zipf[i] * rng.gamma(p.dirichlet_alpha));
      for (int i = 0; i < A; ++i) w[i] = (1.0 - p.restart_p) * (w[i] / s) + p.restart_p * (zipf[i] / zs);
      m.succ[a].resize(A);
      for (int i = 0; i < A; ++i) m.succ[a][i] = i;
      m.cdf[a] = cumulative(w);
    }
  } else {  // sparse chain
    m.pi_cdf = cumulative(zipf);
    for (int a = 0; a < A; ++a) {
      int k = 1 + (int)rng.below((uint64_t)std::max(1, p.max_succ));
      k = std::min(k, A);
      // draw k distinct targets proportionally to zipf weights
      std::vector<double> rem = zipf;
      std::vector<int> tg;
      for (int j = 0; j < k; ++j) {
        auto c = cumulative(rem);
        int t = sample_cdf(c, rng.uniform());
        tg.push_back(t);
        rem[t] = 0.0;
      }
      std::vector<double> w(k);
      for (int j = 0; j < k; ++j) w[j] = rng.gamma(p.dirichlet_alpha);
      m.succ[a] = tg;
      m.cdf[a] = cumulative(w);
    }
  }
  m.restart = (p.act_model == SYN_ACT_ZIPF_RESTART) ? 0.0 : 0.0;  // restart already mixed into rows
  return m;
}

int32_t draw_length(const synth_params &p, Xoshiro256ss &r) {
  double L;
  if (p.len_law == SYN_LEN_GEOMETRIC) {
    L = 1.0 + std::floor(std::log(r.uniform_pos()) / std::log1p(-p.len_p));
  } else if (p.len_law == SYN_LEN_LOGNORMAL) {
    L = std::nearbyint(std::exp(std::log(p.len_median) + p.len_sigma * r.normal()));
  } else {
    L = p.len_median;
  }
  if (!(L >= 1.0)) L = 1.0;
  if (L > (double)p.len_cap) L = (double)p.len_cap;
  return (int32_t)L;
}

int64_t draw_gap(const synth_params &p, Xoshiro256ss &r) {
  double g;
  if (p.gap_law == SYN_GAP_EXPONENTIAL) {
    g = -std::log(r.uniform_pos()) * p.gap_mean_ns;
  } else {
    if (r.uniform() < p.p_zero_gap) return 0;
    g = p.pareto_xm_ns * std::pow(r.uniform_pos(), -1.0 / p.pareto_alpha);
  }
  if (g > p.gap_cap_ns) g = p.gap_cap_ns;
  return (int64_t)std::nearbyint(g);
}

template <class F>
void parallel_for(int64_t n, int nt, F f) {
  if (nt <= 1 || n < 4096) {
    f(0, n, 0);
    return;
  }
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t) {
    int64_t lo = n * t / nt, hi = n * (t + 1) / nt;
    th.emplace_back([=]() { f(lo, hi, t); });
  }
  for (auto &x : th) x.join();
}

int threads_of(const synth_params &p) {
  int nt = p.n_threads > 0 ? p.n_threads : (int)std::thread::hardware_concurrency();
  return std::max(1, std::min(nt, 64));
}

// Stable LSD radix sort of (key, index) pairs by key (unsigned), parallel over
// threads with per-thread digit histograms. Returns the permutation.
void stable_sort_by_key(std::vector<uint64_t> &key, std::vector<uint32_t> &idx, int nt) {
  const int64_t n = (int64_t)key.size();
  uint64_t mx = 0;
  for (int64_t i = 0; i < n; ++i) mx = std::max(mx, key[i]);
  int bits = 0;
  while (bits < 64 && (mx >> bits)) ++bits;
  const int D = 11, B = 1 << D;
  std::vector<uint64_t> k2(n);
  std::vector<uint32_t> i2(n);
  std::vector<int64_t> hist((size_t)nt * B);
  for (int sh = 0; sh < bits; sh += D) {
    std::fill(hist.begin(), hist.end(), 0);
    parallel_for(n, nt, [&](int64_t lo, int64_t hi, int t) {
      int64_t *h = &hist[(size_t)t * B];
      for (int64_t i = lo; i < hi; ++i) h[(key[i] >> sh) & (B - 1)]++;
    });
    // exclusive prefix over (digit, thread)
    int64_t run = 0;
    for (int d = 0; d < B; ++d)
      for (int t = 0; t < nt; ++t) {
        int64_t c = hist[(size_t)t * B + d];
        hist[(size_t)t * B + d] = run;
        run += c;
      }
    parallel_for(n, nt, [&](int64_t lo, int64_t hi, int t) {
      int64_t *h = &hist[(size_t)t * B];
      for (int64_t i = lo; i < hi; ++i) {
        int64_t pos = h[(key[i] >> sh) & (B - 1)]++;
        k2[pos] = key[i];
        i2[pos] = idx[i];
      }
    });
    key.swap(k2);
    idx.swap(i2);
  }
}

}  // namespace

extern "C" {

// Number of events the parameters produce (draws only the case lengths).
int64_t synth_count(const synth_params *p) {
  if (!p || p->n_cases < 0 || p->n_activities <= 0) return -1;
  const int nt = threads_of(*p);
  std::vector<int64_t> part(nt, 0);
  parallel_for(p->n_cases, nt, [&](int64_t lo, int64_t hi, int t) {
    int64_t s = 0;
    for (int64_t c = lo; c < hi; ++c) {
      Xoshiro256ss r(case_seed(p->seed, (uint64_t)c));
      s += draw_length(*p, r);
    }
    part[t] = s;
  });
  int64_t n = 0;
  for (auto v : part) n += v;
  return n;
}

// Fills the columns (each of length synth_count(p)). case_attr may be NULL.
// Returns the number of events, or -1 on bad arguments.
int64_t synth_fill(const synth_params *p, int32_t *case_id, int32_t *activity, int64_t *ts_ns,
                   int32_t *case_attr) {
  if (!p || !case_id || !activity || !ts_ns) return -1;
  const int64_t C = p->n_cases;
  const int nt = threads_of(*p);
  Model m = build_model(*p);

  // per-case lengths and offsets in generation order
  std::vector<int32_t> len(C);
  parallel_for(C, nt, [&](int64_t lo, int64_t hi, int) {
    for (int64_t c = lo; c < hi; ++c) {
      Xoshiro256ss r(case_seed(p->seed, (uint64_t)c));
      len[c] = draw_length(*p, r);
    }
  });
  std::vector<int64_t> off(C + 1, 0);
  for (int64_t c = 0; c < C; ++c) off[c + 1] = off[c] + len[c];
  const int64_t N = off[C];

  // case ids: a seeded random permutation of [0, C); case attribute per case
  std::vector<int32_t> cid(C);
  for (int64_t c = 0; c < C; ++c) cid[c] = (int32_t)c;
  {
    Xoshiro256ss r(case_seed(p->seed, 0xC0FFEE000000ULL));
    for (int64_t i = C - 1; i > 0; --i) std::swap(cid[i], cid[r.below((uint64_t)i + 1)]);
  }
  std::vector<int32_t> cattr;
  if (p->n_attr_values > 0) {
    cattr.resize(C);
    Xoshiro256ss r(case_seed(p->seed, 0xA77A000000ULL));
    for (int64_t c = 0; c < C; ++c) cattr[c] = (int32_t)r.below((uint64_t)p->n_attr_values);
  }

  // events in generation order
  std::vector<int32_t> g_act(N);
  std::vector<int64_t> g_ts(N);
  parallel_for(C, nt, [&](int64_t lo, int64_t hi, int) {
    for (int64_t c = lo; c < hi; ++c) {
      Xoshiro256ss r(case_seed(p->seed, (uint64_t)c));
      (void)draw_length(*p, r);  // same draw as above
      int64_t t = (int64_t)std::floor(r.uniform() * p->start_span_ns);
      int a = sample_cdf(m.pi_cdf, r.uniform());
      for (int64_t k = off[c]; k < off[c + 1]; ++k) {
        if (k > off[c]) {
          t += draw_gap(*p, r);
          int j = sample_cdf(m.cdf[a], r.uniform());
          a = m.succ[a][j];
        }
        g_act[k] = a;
        g_ts[k] = t;
      }
    }
  });

  // row order
  std::vector<uint32_t> perm(N);
  for (int64_t i = 0; i < N; ++i) perm[i] = (uint32_t)i;
  if (p->row_order == SYN_ROWS_SHUFFLED) {
    Xoshiro256ss r(case_seed(p->seed, 0x5AFF1E000000ULL));
    for (int64_t i = N - 1; i > 0; --i) std::swap(perm[i], perm[r.below((uint64_t)i + 1)]);
  } else if (p->row_order == SYN_ROWS_TS_SORTED) {
    std::vector<uint64_t> key(N);
    for (int64_t i = 0; i < N; ++i) key[i] = (uint64_t)g_ts[i] ^ 0x8000000000000000ULL;
    stable_sort_by_key(key, perm, nt);
  }
  // case index of each generated event
  std::vector<int32_t> g_case(N);
  parallel_for(C, nt, [&](int64_t lo, int64_t hi, int) {
    for (int64_t c = lo; c < hi; ++c)
      for (int64_t k = off[c]; k < off[c + 1]; ++k) g_case[k] = (int32_t)c;
  });
  parallel_for(N, nt, [&](int64_t lo, int64_t hi, int) {
    for (int64_t i = lo; i < hi; ++i) {
      const uint32_t g = perm[i];
      const int32_t c = g_case[g];
      case_id[i] = cid[c];
      activity[i] = g_act[g];
      ts_ns[i] = g_ts[g];
      if (case_attr) case_attr[i] = cattr.empty() ? 0 : cattr[c];
    }
  });
  return N;
}

}  // extern "C"
