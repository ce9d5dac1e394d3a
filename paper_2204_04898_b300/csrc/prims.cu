// Device-wide primitives: exclusive scan of uint32 and a stable LSD radix sort
// of (key, value) pairs. Both are reduce-then-scan designs with fixed tiles,
// so results are deterministic and the radix sort is stable: a tile's digit
// offsets come from a digit-major scan of per-tile histograms, and ranks inside
// a tile come from per-warp match/popc ranking in item order.
#include "device_common.cuh"
#include "engine.h"

namespace pm4g {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *__restrict__ in, int64_t n,
                                                              uint32_t *__restrict__ tile_sums) {
  __shared__ uint32_t s_warp[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) s += in[base + k];
  uint32_t total;
  block_exclusive_scan<kScanThreads>(s, s_warp, total);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const uint32_t *__restrict__ in, int64_t n,
                                                             const uint32_t *__restrict__ tile_off,
                                                             uint32_t *__restrict__ out) {
  __shared__ uint32_t s_warp[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = base + k < n ? in[base + k] : 0;
    s += v[k];
  }
  uint32_t total;
  uint32_t pre = block_exclusive_scan<kScanThreads>(s, s_warp, total) + (tile_off ? tile_off[blockIdx.x] : 0);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = pre;
    pre += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) out[n] = pre;
}

// ---------------- radix sort ----------------
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsRounds = 16;
constexpr int kRsTile = kRsThreads * kRsRounds;  // 4096 items
constexpr int kRsBins = 256;

template <class K>
__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const K *__restrict__ keys, int64_t n, int shift,
                                                        uint32_t *__restrict__ hist, int64_t n_tiles) {
  __shared__ uint32_t s_h[kRsBins];
  s_h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRsTile;
  for (int k = threadIdx.x; k < kRsTile; k += kRsThreads) {
    const int64_t i = base + k;
    if (i < n) atomicAdd(&s_h[(uint32_t)(keys[i] >> shift) & 0xFF], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = s_h[threadIdx.x];
}

template <class K>
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const K *__restrict__ keys_in,
                                                           const uint32_t *__restrict__ vals_in, int64_t n,
                                                           int shift, const uint32_t *__restrict__ offs,
                                                           int64_t n_tiles, K *__restrict__ keys_out,
                                                           uint32_t *__restrict__ vals_out) {
  __shared__ uint32_t s_wh[kRsWarps * (kRsBins + 1)];
  __shared__ uint32_t s_off[kRsBins];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = threadIdx.x; k < kRsWarps * (kRsBins + 1); k += kRsThreads) s_wh[k] = 0;
  s_off[threadIdx.x] = offs[(int64_t)threadIdx.x * n_tiles + blockIdx.x];
  __syncthreads();
  const int64_t wbase = (int64_t)blockIdx.x * kRsTile + (int64_t)w * 32 * kRsRounds;
  K key[kRsRounds];
  uint32_t val[kRsRounds];
  uint32_t rank[kRsRounds];
  uint32_t dig[kRsRounds];
  uint32_t *wh = s_wh + w * (kRsBins + 1);
#pragma unroll
  for (int r = 0; r < kRsRounds; ++r) {
    const int64_t i = wbase + r * 32 + lane;
    const bool valid = i < n;
    key[r] = valid ? keys_in[i] : (K)0;
    val[r] = valid ? vals_in[i] : 0u;
    const uint32_t d = valid ? ((uint32_t)(key[r] >> shift) & 0xFF) : (uint32_t)kRsBins;
    dig[r] = d;
    const uint32_t peers = __match_any_sync(kFull, d);
    const int leader = __ffs(peers) - 1;
    uint32_t b = 0;
    if (lane == leader) {
      b = wh[d];
      wh[d] = b + __popc(peers);
    }
    b = __shfl_sync(kFull, b, leader);
    rank[r] = b + __popc(peers & lanemask_lt());
    __syncwarp();
  }
  __syncthreads();
  {  // exclusive prefix over warps, per digit
    const int d = threadIdx.x;
    uint32_t acc = 0;
    for (int ww = 0; ww < kRsWarps; ++ww) {
      uint32_t t = s_wh[ww * (kRsBins + 1) + d];
      s_wh[ww * (kRsBins + 1) + d] = acc;
      acc += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRsRounds; ++r) {
    const int64_t i = wbase + r * 32 + lane;
    if (i < n) {
      const uint32_t d = dig[r];
      const uint32_t pos = s_off[d] + wh[d] + rank[r];
      keys_out[pos] = key[r];
      vals_out[pos] = val[r];
    }
  }
}

__global__ void k_iota(uint32_t *out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (uint32_t)i;
}

template <class K>
int radix_sort_impl(Ctx *c, K *keys, uint32_t *vals, K *keys_tmp, uint32_t *vals_tmp, int64_t n, int begin_bit,
                    int end_bit, const char *name) {
  if (n <= 1 || end_bit <= begin_bit) return PM4G_OK;
  const int64_t tiles = (n + kRsTile - 1) / kRsTile;
  Scratch s(c);
  uint32_t *hist = s.get<uint32_t>(tiles * kRsBins);
  uint32_t *offs = s.get<uint32_t>(tiles * kRsBins + 1);
  if (!hist || !offs) {
    set_error("radix sort: out of device memory");
    return PM4G_ENOMEM;
  }
  K *ka = keys, *kb = keys_tmp;
  uint32_t *va = vals, *vb = vals_tmp;
  int passes = 0;
  for (int sh = begin_bit; sh < end_bit; sh += 8) {
    {
      KTime t(c, name);
      k_rs_hist<K><<<(unsigned)tiles, kRsThreads, 0, c->stream>>>(ka, n, sh, hist, tiles);
      PM4G_TRY(check_launch(c, "k_rs_hist"));
    }
    PM4G_TRY(scan_u32(c, hist, offs, tiles * kRsBins));
    {
      KTime t(c, name);
      k_rs_scatter<K><<<(unsigned)tiles, kRsThreads, 0, c->stream>>>(ka, va, n, sh, offs, tiles, kb, vb);
      PM4G_TRY(check_launch(c, "k_rs_scatter"));
    }
    std::swap(ka, kb);
    std::swap(va, vb);
    ++passes;
  }
  if (passes & 1) {
    PM4G_CK(cudaMemcpyAsync(keys, ka, n * sizeof(K), cudaMemcpyDeviceToDevice, c->stream));
    PM4G_CK(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, c->stream));
  }
  return PM4G_OK;
}

}  // namespace

int scan_u32(Ctx *c, const uint32_t *in, uint32_t *out, int64_t n) {
  if (n <= 0) {
    PM4G_CK(cudaMemsetAsync(out, 0, sizeof(uint32_t), c->stream));
    return PM4G_OK;
  }
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles == 1) {
    KTime t(c, "scan");
    k_scan_tiles<<<1, kScanThreads, 0, c->stream>>>(in, n, nullptr, out);
    return check_launch(c, "k_scan_tiles");
  }
  Scratch s(c);
  uint32_t *sums = s.get<uint32_t>(tiles);
  uint32_t *offs = s.get<uint32_t>(tiles + 1);
  if (!sums || !offs) {
    set_error("scan: out of device memory");
    return PM4G_ENOMEM;
  }
  {
    KTime t(c, "scan");
    k_scan_reduce<<<(unsigned)tiles, kScanThreads, 0, c->stream>>>(in, n, sums);
    PM4G_TRY(check_launch(c, "k_scan_reduce"));
  }
  PM4G_TRY(scan_u32(c, sums, offs, tiles));
  KTime t(c, "scan");
  k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, c->stream>>>(in, n, offs, out);
  return check_launch(c, "k_scan_tiles");
}

int radix_sort_u32(Ctx *c, uint32_t *keys, uint32_t *vals, uint32_t *keys_tmp, uint32_t *vals_tmp, int64_t n,
                   int begin_bit, int end_bit) {
  return radix_sort_impl<uint32_t>(c, keys, vals, keys_tmp, vals_tmp, n, begin_bit, end_bit, "radix_sort");
}

int radix_sort_u64(Ctx *c, uint64_t *keys, uint32_t *vals, uint64_t *keys_tmp, uint32_t *vals_tmp, int64_t n,
                   int begin_bit, int end_bit) {
  return radix_sort_impl<uint64_t>(c, keys, vals, keys_tmp, vals_tmp, n, begin_bit, end_bit, "radix_sort");
}

int iota_u32(Ctx *c, uint32_t *out, int64_t n) {
  if (n <= 0) return PM4G_OK;
  k_iota<<<grid_for(n, 256, 4096), 256, 0, c->stream>>>(out, n);
  return check_launch(c, "k_iota");
}

}  // namespace pm4g
