// Variant-table kernel arguments and declarations.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pm4g {

// One slot of the grouping table (16 bytes, one sector): the key's tag (its
// high word, never 0) and the item that claimed the slot in one word, the
// member count, and the bitwise complement of the smallest member (so that
// an all-zero slot is empty and atomicMax keeps the smallest member).
struct __align__(16) VarSlot {
  unsigned long long tagc;  // tag << 32 | claiming item
  uint32_t cnt;
  uint32_t nmin;
};

struct VarArgs {
  uint64_t n_slots;
  const uint32_t *len;     // per case slot, 0 = no case
  const uint64_t *hash;    // per case slot, sequence hash (seed 0); NULL: formed from act_s in round 0
  const uint32_t *off;     // per case slot, first position in the ordered log
  const uint16_t *act_s;   // activity of every event in (case, ts, row) order (16-byte aligned)
  uint64_t n_events;       // length of act_s
  int bits;                // key truncation (tests only), 0 = full key
  VarSlot *tab;
  uint32_t tmask;
  uint32_t *grp;
  uint32_t *rep_of;
  uint32_t *vcount;
  uint8_t *isbad;
  const uint32_t *cls;     // optional class of each slot (batched sub-logs): a variant never spans two classes
  uint32_t *rep_flag;      // optional: 1 at every representative, 0 at every other slot (k_var_final)
  const unsigned long long *gtab;  // first round without a.hash: the hash's word of every activity (k_var_gtab)
};

// Groups the items of `a` (slots with len > 0, or the whole list) by exact
// sequence: fills a.rep_of (smallest slot of the item's group) and a.vcount
// (group size, at the representative). n_items bounds the present slots.
// With rep_pos (and a.rep_flag), also the exclusive prefix of the
// representative flags over the n_slots slots (n_slots + 1 entries) and
// their number (*n_reps).
struct Ctx;
int group_variants(Ctx *c, VarArgs a, uint64_t n_items, uint32_t *rep_pos = nullptr, uint32_t *n_reps = nullptr);

// First round over all slots with the hash formed from act_s (a.hash NULL).
constexpr int kHiThreads = 256;
__global__ void k_var_gtab(unsigned long long *g, uint32_t n_act);
__global__ void k_var_hash_insert(VarArgs a);
__global__ void k_var_insert(VarArgs a, const uint32_t *list, uint32_t n_list, uint32_t round);
__global__ void k_var_verify(VarArgs a, const uint32_t *list, uint32_t n_list, uint32_t *bad_out, uint32_t *n_bad);
__global__ void k_var_final(VarArgs a, const uint32_t *list, uint32_t n_list);
__global__ void k_rep_flags(VarArgs a, uint32_t *flags);
__global__ void k_rep_compact(VarArgs a, const uint32_t *flags, const uint32_t *pos, uint32_t cmask,
                              uint32_t *rep_slots, uint32_t *keys, uint32_t *vals);
__global__ void k_rank_scatter(const uint32_t *order, uint32_t V, uint32_t *rank_of);
__global__ void k_case_variant(VarArgs a, const uint32_t *rep_pos, const uint32_t *rank_of, int32_t *cvar);
__global__ void k_present_flags(const uint32_t *len, uint64_t n_slots, uint32_t *flags);
__global__ void k_cases_out(const uint32_t *len, uint64_t n_slots, const uint32_t *pos, const int32_t *cvar,
                            int32_t min_case, const int32_t *uniq, int32_t *case_ids, int32_t *case_variant);
__global__ void k_var_out_head(VarArgs a, const uint32_t *order, const uint32_t *rep_slots, uint32_t k_out,
                               int32_t min_case, const int32_t *uniq, unsigned long long *o_count, int32_t *o_min,
                               uint32_t *o_len);
__global__ void k_var_out_acts(VarArgs a, const uint32_t *order, const uint32_t *rep_slots, uint32_t k_out,
                               const uint32_t *o_off, int32_t *o_acts, uint64_t cap);

}  // namespace pm4g
