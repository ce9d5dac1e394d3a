// Host-side engine internals: context, device buffers, kernel timing, status
// handling and the declarations shared by the .cu files.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "../../include/pm4g.h"

namespace pm4g {

void set_error(const char *fmt, ...);

#define PM4G_CK(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      ::pm4g::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                     \
      return PM4G_ECUDA;                                                               \
    }                                                                                  \
  } while (0)

#define PM4G_TRY(expr)           \
  do {                           \
    int st_ = (expr);            \
    if (st_ != PM4G_OK) return st_; \
  } while (0)

// Records a CUDA event pair around every launch when timing is on.
struct TimingRec {
  std::string name;
  cudaEvent_t a, b;
};

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool has_alloc = false;
  pm4g_allocator alloc{};
  int num_sms = 148;
  int smem_optin = 227 * 1024;
  // options
  bool timing = false;
  int test_hash_bits = 0;
  int test_bucket_cap = 0;
  // timing
  std::vector<TimingRec> pending;
  std::vector<cudaEvent_t> free_events;
  std::map<std::string, std::pair<int64_t, double>> totals;
  int64_t live_logs = 0;
  int64_t launches = 0;  // kernels launched by this context
  // pinned host staging for device-to-host results
  void *pin = nullptr;
  size_t pin_bytes = 0;
  // device blocks freed by this context, kept for reuse in stream order
  // (rounded size -> blocks); every kernel of the context runs on its stream
  std::multimap<size_t, void *> cache;
  size_t cached_bytes = 0;
  size_t cache_limit = 0;
};

// Device memory through the context's allocator (stream ordered).
void *dalloc(Ctx *c, size_t bytes);
void dfree(Ctx *c, void *p, size_t bytes);

// A device array owned by a log or a scope.
template <class T>
struct DBuf {
  T *p = nullptr;
  size_t n = 0;
};

// Scope holding temporary device buffers, released in stream order.
struct Scratch {
  Ctx *c;
  std::vector<std::pair<void *, size_t>> bufs;
  explicit Scratch(Ctx *ctx) : c(ctx) {}
  ~Scratch() {
    for (auto &b : bufs) dfree(c, b.first, b.second);
  }
  template <class T>
  T *get(size_t n) {
    size_t bytes = (n ? n : 1) * sizeof(T);
    void *p = dalloc(c, bytes);
    if (p) bufs.push_back({p, bytes});
    return (T *)p;
  }
};

// Kernel timing scope: begin/end events on the context stream.
struct KTime {
  Ctx *c;
  const char *name;
  cudaEvent_t a = nullptr, b = nullptr;
  KTime(Ctx *ctx, const char *nm);
  ~KTime();
};

int check_launch(Ctx *c, const char *what);

// ---- primitives (prims.cu) ----
// Exclusive scan of n uint32 values; out must hold n + 1 entries, out[n] = total.
int scan_u32(Ctx *c, const uint32_t *in, uint32_t *out, int64_t n);
// Stable LSD radix sort of (key, value) pairs by key bits [begin_bit, end_bit).
// Sorts in place using the given temporaries of the same length.
int radix_sort_u32(Ctx *c, uint32_t *keys, uint32_t *vals, uint32_t *keys_tmp, uint32_t *vals_tmp,
                   int64_t n, int begin_bit, int end_bit);
int radix_sort_u64(Ctx *c, uint64_t *keys, uint32_t *vals, uint64_t *keys_tmp, uint32_t *vals_tmp,
                   int64_t n, int begin_bit, int end_bit);
// Stream compaction helpers
int iota_u32(Ctx *c, uint32_t *out, int64_t n);

inline int bits_for(uint64_t maxval) {  // bits to represent values in [0, maxval]
  int b = 0;
  while (b < 64 && (maxval >> b)) ++b;
  return b;
}

inline unsigned grid_for(int64_t n, int per_block, unsigned cap = 1u << 20) {
  int64_t g = (n + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > (int64_t)cap) g = cap;
  return (unsigned)g;
}

}  // namespace pm4g
