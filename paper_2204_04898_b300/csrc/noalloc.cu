// Allocation-free DFG for small logs (pm4g_dfg_noalloc).
//
// Some callers cannot allocate device memory at the moment they need a
// summary: code running while a CUDA graph is being captured (allocation
// calls are not capturable there), serving processes that reserve a fixed
// memory budget up front and must not grow it per request, and hosts whose
// device memory belongs to another framework's pool. This entry point serves
// them: it computes the frequency and performance directly-follows graph and
// the start/end counts of a log of at most kNoAllocMaxEvents events from device
// columns into caller-provided device arrays, and its only working memory is
// the fixed array below, which every GPU that loads this library holds until
// the process exits.
//
// The array is shared by all calls on a device and keeps the last call's
// contents; each call clears what must start at zero. Calls that overlap on
// the GPU (concurrent streams or threads) race on it and must be serialised by
// the caller. The device address of the array is looked up once per device, on
// the first call made with that device current; make that first call before
// any stream capture, since the lookup is a runtime call.
#include <climits>
#include <mutex>

#include "device_common.cuh"
#include "engine.h"

namespace pm4g {
namespace {

constexpr int64_t kNoAllocMaxEvents = 1 << 18;  // events per call
constexpr int64_t kNoAllocMaxSlots = 1 << 18;   // max case id - min case id + 1
constexpr int kNoAllocMaxCase = 512;            // events of one case

// Layout of the scratch array (bytes)
constexpr size_t kRecOff = 0;                                       // uint4 [kNoAllocMaxEvents]
constexpr size_t kCntOff = kRecOff + 16 * (size_t)kNoAllocMaxEvents;  // uint32 [kNoAllocMaxSlots]
constexpr size_t kCurOff = kCntOff + 4 * (size_t)kNoAllocMaxSlots;    // uint32 [kNoAllocMaxSlots]
constexpr size_t kMiscOff = kCurOff + 4 * (size_t)kNoAllocMaxSlots;   // int32 min, int32 max, uint32 status
constexpr size_t kScratchBytes = kMiscOff + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct NaArgs {
  const int32_t *case_id;
  const int32_t *activity;
  const int64_t *ts;
  int64_t n;
  const int64_t *n_dev;  // the capturable form: the event count in device memory (else NULL)
  uint32_t n_act;
  unsigned char *scratch;
  unsigned long long *count, *sum_lo, *sum_hi, *mn, *mx, *start, *end;
};

__device__ __forceinline__ int32_t *na_minmax(const NaArgs &a) { return (int32_t *)(a.scratch + kMiscOff); }
__device__ __forceinline__ uint32_t *na_status(const NaArgs &a) { return (uint32_t *)(a.scratch + kMiscOff + 8); }

// Status bits of a call
constexpr uint32_t kNaBadActivity = 1, kNaLongCase = 2, kNaWideSpan = 4, kNaBadCount = 8;

// The events of the call: the host's count, or in the capturable form the
// device's (0 when it is out of range; the status then says so).
__device__ __forceinline__ int64_t na_n(const NaArgs &a) {
  if (!a.n_dev) return a.n;
  const int64_t n = *a.n_dev;
  return (n < 0 || n > kNoAllocMaxEvents) ? 0 : n;
}

// In the capturable form the host does not read the case-id range: every
// kernel after the range check takes it from the scratch array, and does no
// work once the status holds an input error (so no index leaves its array).
constexpr uint32_t kNaFromDevice = 0xFFFFFFFFu;
__device__ __forceinline__ bool na_span(const NaArgs &a, uint32_t R_in, int32_t min_in, uint32_t &R,
                                        int32_t &min_case) {
  if (R_in != kNaFromDevice) {
    R = R_in;
    min_case = min_in;
    return true;
  }
  if (*(volatile uint32_t *)na_status(a) & (kNaBadActivity | kNaWideSpan | kNaBadCount)) return false;
  const int32_t mn = na_minmax(a)[0], mx = na_minmax(a)[1];
  if (na_n(a) == 0 || mx < mn) return false;
  R = (uint32_t)((int64_t)mx - (int64_t)mn + 1);
  min_case = mn;
  return true;
}

__global__ void k_na_init(NaArgs a) {
  const int64_t cells = (int64_t)a.n_act * a.n_act;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cells; i += (int64_t)gridDim.x * blockDim.x) {
    a.count[i] = 0;
    a.sum_lo[i] = 0;
    a.sum_hi[i] = 0;
    a.mn[i] = ~0ull;
    a.mx[i] = 0;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n_act; i += (int64_t)gridDim.x * blockDim.x) {
    a.start[i] = 0;
    a.end[i] = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    na_minmax(a)[0] = INT_MAX;
    na_minmax(a)[1] = INT_MIN;
    *na_status(a) = (a.n_dev && (*a.n_dev < 0 || *a.n_dev > kNoAllocMaxEvents)) ? kNaBadCount : 0u;
  }
}

// case id range and activity range check
__global__ void k_na_minmax(NaArgs a) {
  int mn = INT_MAX, mx = INT_MIN;
  bool bad = false;
  const int64_t n = na_n(a);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    mn = min(mn, a.case_id[i]);
    mx = max(mx, a.case_id[i]);
    bad |= (uint32_t)a.activity[i] >= a.n_act;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mn = min(mn, __shfl_xor_sync(kFull, mn, o));
    mx = max(mx, __shfl_xor_sync(kFull, mx, o));
  }
  bad = __any_sync(kFull, bad);
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&na_minmax(a)[0], mn);
    atomicMax(&na_minmax(a)[1], mx);
    if (bad) atomicOr(na_status(a), 1u);
  }
}

// The range check's verdict in the capturable form (one thread; the kernels
// after it read the status it leaves).
__global__ void k_na_span_check(NaArgs a) {
  const int32_t mn = na_minmax(a)[0], mx = na_minmax(a)[1];
  if (na_n(a) > 0 && mx >= mn && (int64_t)mx - (int64_t)mn + 1 > kNoAllocMaxSlots) atomicOr(na_status(a), kNaWideSpan);
}

__global__ void k_na_zero(NaArgs a, uint32_t R_in) {
  uint32_t R;
  int32_t min_case;
  if (!na_span(a, R_in, 0, R, min_case)) return;
  uint32_t *cnt = (uint32_t *)(a.scratch + kCntOff);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < R; i += gridDim.x * blockDim.x) cnt[i] = 0;
}

__global__ void k_na_count(NaArgs a, uint32_t R_in, int32_t min_in) {
  uint32_t R;
  int32_t min_case;
  if (!na_span(a, R_in, min_in, R, min_case)) return;
  uint32_t *cnt = (uint32_t *)(a.scratch + kCntOff);
  const int64_t n = na_n(a);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[(uint32_t)a.case_id[i] - (uint32_t)min_case], 1u);
}

// Exclusive scan of the case counts into the placement cursors (one CTA).
__global__ void __launch_bounds__(1024) k_na_scan(NaArgs a, uint32_t R_in) {
  __shared__ uint32_t s_warp[32];
  uint32_t R;
  int32_t min_case;
  if (!na_span(a, R_in, 0, R, min_case)) return;
  const uint32_t *cnt = (const uint32_t *)(a.scratch + kCntOff);
  uint32_t *cur = (uint32_t *)(a.scratch + kCurOff);
  uint32_t carry = 0;
  for (uint32_t base = 0; base < R; base += 1024) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t v = i < R ? cnt[i] : 0;
    uint32_t tot;
    const uint32_t pre = block_exclusive_scan<1024>(v, s_warp, tot);
    if (i < R) cur[i] = carry + pre;
    carry += tot;
  }
}

__global__ void k_na_place(NaArgs a, uint32_t R_in, int32_t min_in) {
  uint32_t R;
  int32_t min_case;
  if (!na_span(a, R_in, min_in, R, min_case)) return;
  uint4 *rec = (uint4 *)(a.scratch + kRecOff);
  uint32_t *cur = (uint32_t *)(a.scratch + kCurOff);
  const int64_t n = na_n(a);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t pos = atomicAdd(&cur[(uint32_t)a.case_id[i] - (uint32_t)min_case], 1u);
    const uint64_t t = (uint64_t)a.ts[i];
    rec[pos] = make_uint4((uint32_t)a.activity[i], (uint32_t)i, (uint32_t)t, (uint32_t)(t >> 32));
  }
}

__device__ __forceinline__ void na_edge(const NaArgs &a, uint32_t src, uint32_t dst, uint64_t d) {
  const uint32_t key = src * a.n_act + dst;
  atomicAdd(&a.count[key], 1ull);
  const unsigned long long old = atomicAdd(&a.sum_lo[key], (unsigned long long)d);
  if (old + d < old) atomicAdd(&a.sum_hi[key], 1ull);
  atomicMin(&a.mn[key], (unsigned long long)d);
  atomicMax(&a.mx[key], (unsigned long long)d);
}

// One warp per case: order its events by (timestamp, row) and add its
// directly-follows pairs and endpoints to the outputs.
template <int E>
__device__ __forceinline__ void na_case(const NaArgs &a, const uint4 *rec, uint32_t s0, uint32_t L) {
  uint64_t key[E];
  uint32_t row[E], act[E];
  const int lane = (int)lane_id();
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t i = (uint32_t)(lane * E + e);
    if (i < L) {
      const uint4 r = rec[s0 + i];
      key[e] = ts_key((int64_t)(((uint64_t)r.w << 32) | r.z));
      row[e] = r.y;
      act[e] = r.x;
    } else {
      key[e] = ~0ull;
      row[e] = ~0u;
      act[e] = 0;
    }
  }
  warp_bitonic_sort<E>(key, row, act);
  const uint64_t nk = __shfl_down_sync(kFull, key[0], 1);
  const uint32_t na = __shfl_down_sync(kFull, act[0], 1);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t i = (uint32_t)(lane * E + e);
    if (i == 0) atomicAdd(&a.start[act[e]], 1ull);
    if (i + 1 == L) atomicAdd(&a.end[act[e]], 1ull);
    if (i + 1 < L) {
      const uint64_t k2 = e + 1 < E ? key[e + 1 < E ? e + 1 : e] : nk;
      const uint32_t a2 = e + 1 < E ? act[e + 1 < E ? e + 1 : e] : na;
      na_edge(a, act[e], a2, k2 - key[e]);
    }
  }
}

__global__ void k_na_cases(NaArgs a, uint32_t R_in) {
  uint32_t R;
  int32_t min_case;
  if (!na_span(a, R_in, 0, R, min_case)) return;
  const uint4 *rec = (const uint4 *)(a.scratch + kRecOff);
  const uint32_t *cnt = (const uint32_t *)(a.scratch + kCntOff);
  const uint32_t *cur = (const uint32_t *)(a.scratch + kCurOff);  // now the end of every case
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = warp; s < R; s += nw) {
    const uint32_t L = cnt[s];
    if (L == 0) continue;
    const uint32_t s0 = cur[s] - L;
    if (L <= 32) na_case<1>(a, rec, s0, L);
    else if (L <= 64) na_case<2>(a, rec, s0, L);
    else if (L <= 128) na_case<4>(a, rec, s0, L);
    else if (L <= 256) na_case<8>(a, rec, s0, L);
    else if (L <= (uint32_t)kNoAllocMaxCase) na_case<16>(a, rec, s0, L);
    else if (lane_id() == 0) atomicOr(na_status(a), kNaLongCase);
  }
}

__global__ void k_na_status_out(NaArgs a, uint32_t *status_out) { *status_out = *na_status(a); }

std::mutex g_na_mu;
void *g_na_addr[256] = {};

// Device address of the scratch array on `device` (looked up once per device,
// with that device current).
int na_scratch(int device, unsigned char **out) {
  if (device < 0 || device >= 256) {
    set_error("pm4g_dfg_noalloc: device %d out of range", device);
    return PM4G_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_na_mu);
  if (!g_na_addr[device]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error("pm4g_dfg_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return PM4G_ECUDA;
    }
    g_na_addr[device] = p;
  }
  *out = (unsigned char *)g_na_addr[device];
  return PM4G_OK;
}

#define NA_CK(call)                                                                       \
  do {                                                                                    \
    const cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                              \
      set_error("pm4g_dfg_noalloc: %s failed: %s", #call, cudaGetErrorString(e_));        \
      return PM4G_ECUDA;                                                                  \
    }                                                                                     \
  } while (0)

}  // namespace
}  // namespace pm4g

using namespace pm4g;

int pm4g_dfg_noalloc(const int32_t *case_id, const int32_t *activity, const int64_t *ts_ns, int64_t n_events,
                     int32_t n_activities, void *cuda_stream, uint64_t *count, uint64_t *sum_lo, uint64_t *sum_hi,
                     uint64_t *min, uint64_t *max, uint64_t *start, uint64_t *end) {
  pm4g::ApiRange nvtx_range("pm4g_dfg_noalloc");
  if (n_events < 0 || n_events > kNoAllocMaxEvents) {
    set_error("pm4g_dfg_noalloc: n_events %lld outside [0, %lld]", (long long)n_events,
              (long long)kNoAllocMaxEvents);
    return PM4G_EINVAL;
  }
  if (n_activities < 1 || n_activities > 2048) {
    set_error("pm4g_dfg_noalloc: n_activities %d outside [1, 2048]", n_activities);
    return PM4G_EINVAL;
  }
  if (!count || !sum_lo || !sum_hi || !min || !max || !start || !end ||
      (n_events > 0 && (!case_id || !activity || !ts_ns))) {
    set_error("pm4g_dfg_noalloc: NULL pointer");
    return PM4G_EINVAL;
  }
  int device = 0;
  NA_CK(cudaGetDevice(&device));
  unsigned char *scratch = nullptr;
  const int st = na_scratch(device, &scratch);
  if (st != PM4G_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  NaArgs a{case_id, activity, ts_ns, n_events, nullptr, (uint32_t)n_activities, scratch,
           (unsigned long long *)count, (unsigned long long *)sum_lo, (unsigned long long *)sum_hi,
           (unsigned long long *)min, (unsigned long long *)max, (unsigned long long *)start,
           (unsigned long long *)end};
  const int64_t cells = (int64_t)n_activities * n_activities;
  k_na_init<<<(unsigned)std::min<int64_t>((cells + 255) / 256 + 1, 4096), 256, 0, s>>>(a);
  NA_CK(cudaGetLastError());
  if (n_events == 0) {
    NA_CK(cudaStreamSynchronize(s));
    return PM4G_OK;
  }
  const unsigned g = (unsigned)std::min<int64_t>((n_events + 255) / 256, 1024);
  k_na_minmax<<<g, 256, 0, s>>>(a);
  NA_CK(cudaGetLastError());
  int32_t h[3] = {0, 0, 0};  // min, max, status (host stack; nothing is allocated)
  NA_CK(cudaMemcpyAsync(h, scratch + kMiscOff, sizeof(h), cudaMemcpyDeviceToHost, s));
  NA_CK(cudaStreamSynchronize(s));
  if (h[2] & 1) {
    set_error("pm4g_dfg_noalloc: activity code outside [0, %d)", n_activities);
    return PM4G_ERANGE;
  }
  const int64_t R = (int64_t)h[1] - (int64_t)h[0] + 1;
  if (R > kNoAllocMaxSlots) {
    set_error("pm4g_dfg_noalloc: case ids span %lld values, more than %lld", (long long)R,
              (long long)kNoAllocMaxSlots);
    return PM4G_EINVAL;
  }
  const uint32_t r = (uint32_t)R;
  k_na_zero<<<(r + 255) / 256, 256, 0, s>>>(a, r);
  k_na_count<<<g, 256, 0, s>>>(a, r, h[0]);
  k_na_scan<<<1, 1024, 0, s>>>(a, r);
  k_na_place<<<g, 256, 0, s>>>(a, r, h[0]);
  k_na_cases<<<(unsigned)std::min<int64_t>((R * 32 + 255) / 256, 4096), 256, 0, s>>>(a, r);
  NA_CK(cudaGetLastError());
  uint32_t status = 0;
  NA_CK(cudaMemcpyAsync(&status, scratch + kMiscOff + 8, sizeof(status), cudaMemcpyDeviceToHost, s));
  NA_CK(cudaStreamSynchronize(s));
  if (status & 2) {
    set_error("pm4g_dfg_noalloc: a case has more than %d events", kNoAllocMaxCase);
    return PM4G_EINVAL;
  }
  return PM4G_OK;
}

int pm4g_dfg_noalloc_async(const int32_t *case_id, const int32_t *activity, const int64_t *ts_ns,
                           const int64_t *n_events_dev, int32_t n_activities, void *cuda_stream, uint64_t *count,
                           uint64_t *sum_lo, uint64_t *sum_hi, uint64_t *min, uint64_t *max, uint64_t *start,
                           uint64_t *end, uint32_t *status_dev) {
  pm4g::ApiRange nvtx_range("pm4g_dfg_noalloc_async");
  if (n_activities < 1 || n_activities > 2048) {
    set_error("pm4g_dfg_noalloc_async: n_activities %d outside [1, 2048]", n_activities);
    return PM4G_EINVAL;
  }
  if (!case_id || !activity || !ts_ns || !n_events_dev || !count || !sum_lo || !sum_hi || !min || !max || !start ||
      !end || !status_dev) {
    set_error("pm4g_dfg_noalloc_async: NULL pointer");
    return PM4G_EINVAL;
  }
  int device = 0;
  NA_CK(cudaGetDevice(&device));
  unsigned char *scratch = nullptr;
  const int st = na_scratch(device, &scratch);
  if (st != PM4G_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  NaArgs a{case_id, activity, ts_ns, 0, n_events_dev, (uint32_t)n_activities, scratch,
           (unsigned long long *)count, (unsigned long long *)sum_lo, (unsigned long long *)sum_hi,
           (unsigned long long *)min, (unsigned long long *)max, (unsigned long long *)start,
           (unsigned long long *)end};
  // Fixed launch shapes, sized for the largest call: the same launches serve
  // every event count, so a captured graph replays for any log that fits.
  const int64_t cells = (int64_t)n_activities * n_activities;
  const unsigned g = (unsigned)(kNoAllocMaxEvents / 256);
  k_na_init<<<(unsigned)std::min<int64_t>((cells + 255) / 256 + 1, 4096), 256, 0, s>>>(a);
  k_na_minmax<<<g, 256, 0, s>>>(a);
  k_na_span_check<<<1, 1, 0, s>>>(a);
  k_na_zero<<<(unsigned)(kNoAllocMaxSlots / 256), 256, 0, s>>>(a, kNaFromDevice);
  k_na_count<<<g, 256, 0, s>>>(a, kNaFromDevice, 0);
  k_na_scan<<<1, 1024, 0, s>>>(a, kNaFromDevice);
  k_na_place<<<g, 256, 0, s>>>(a, kNaFromDevice, 0);
  k_na_cases<<<4096, 256, 0, s>>>(a, kNaFromDevice);
  k_na_status_out<<<1, 1, 0, s>>>(a, status_dev);
  NA_CK(cudaGetLastError());
  return PM4G_OK;
}
