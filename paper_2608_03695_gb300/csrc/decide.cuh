// Generic move-decision kernels.  For each node v of a work list the
// neighbour weights are aggregated per key (community or sub-community
// label), every distinct key is scored by the policy, and the best candidate
// (largest key, ties to the smallest label) is handed to the policy.
//
// Three tiers by degree, all grid-stride over a device-resident list whose
// length is read on the device:
//   warp   deg <= 32   one warp per node; lanes holding equal keys are grouped
//                      with __match_any_sync and summed in shared memory;
//   block  deg <= 1024 one block per node, shared-memory open-addressing table;
//   global otherwise   one block per node, table in global scratch (2*deg
//                      slots rounded up to a power of two, offset per node).
//
// Policy interface (all __device__):
//   bool begin(v)                      node takes part (uniform per node)
//   void skip(v)                       record "no move" for a non-participant
//   bool edge(v, e, key&, w&)          entry e contributes w to key
//   Cand cand(v, key, W)               score of moving v to key (INT32_MAX = not allowed)
//   int32_t own_key(v)                 the key whose weight finish() needs (-1 none)
//   void finish(v, best, W_best, W_own)
#pragma once
#include "level.h"

namespace mslice {

constexpr int WARP_TIER_MAX = 32;
constexpr int BLOCK_TIER_MAX = 1024;
constexpr int BLOCK_TIER_SLOTS = 2048;
constexpr int BLOCK_TIER_THREADS = 128;
constexpr int GLOBAL_TIER_THREADS = 256;
constexpr int DECIDE_WARP_THREADS = 256;

__device__ __forceinline__ uint32_t small_hash(int32_t key, int bits) {
  return ((uint32_t)key * 2654435769u) >> (32 - bits);
}

template <class Pol>
__global__ void __launch_bounds__(DECIDE_WARP_THREADS) k_decide_warp(Pol pol, const int32_t* list, const int32_t* count_ptr) {
  constexpr int WARPS = DECIDE_WARP_THREADS / 32;
  __shared__ long long sw[WARPS][32];
  const int count = *count_ptr;
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  for (int idx = blockIdx.x * WARPS + wi; idx < count; idx += gridDim.x * WARPS) {
    const int32_t v = list[idx];
    if (!pol.begin(v)) {
      if (lane == 0) pol.skip(v);
      continue;
    }
    const int64_t beg = pol.g.rowptr[v];
    const int deg = (int)(pol.g.rowptr[v + 1] - beg);
    int32_t key = -1;
    long long w = 0;
    const bool valid = lane < deg && pol.edge(v, beg + lane, key, w);
    sw[wi][lane] = 0;
    __syncwarp();
    const unsigned peers = __match_any_sync(0xffffffffu, valid ? key : -1);
    const int leader = __ffs(peers) - 1;
    if (valid) atomicAdd((ull*)&sw[wi][leader], (ull)w);
    __syncwarp();
    const bool lead = valid && leader == lane;
    const long long Wk = lead ? sw[wi][lane] : 0;
    Cand c{0, INT32_MAX};
    if (lead) c = pol.cand(v, key, Wk);
    const Cand best = warp_best(c);
    const int32_t own = pol.own_key(v);
    const unsigned mo = __ballot_sync(0xffffffffu, lead && key == own);
    const unsigned mb = __ballot_sync(0xffffffffu, lead && key == best.label);
    const long long Wown = mo ? sw[wi][__ffs(mo) - 1] : 0;
    const long long Wb = mb ? sw[wi][__ffs(mb) - 1] : 0;
    if (lane == 0) pol.finish(v, best, Wb, Wown);
    __syncwarp();
  }
}

template <int SLOTS_BITS>
__device__ __forceinline__ void table_add(int32_t* hk, long long* hv, int32_t key, long long w) {
  constexpr uint32_t mask = (1u << SLOTS_BITS) - 1u;
  uint32_t i = small_hash(key, SLOTS_BITS);
  for (uint32_t p = 0; p <= mask; ++p) {
    const int32_t prev = atomicCAS(&hk[i], -1, key);
    if (prev == -1 || prev == key) {
      atomicAdd((ull*)&hv[i], (ull)w);
      return;
    }
    i = (i + 1) & mask;
  }
}

__device__ __forceinline__ void gtable_add(int32_t* hk, long long* hv, int bits, int32_t key, long long w,
                                           unsigned* status) {
  const uint32_t mask = (1u << bits) - 1u;
  uint32_t i = small_hash(key, bits);
  for (uint32_t p = 0; p <= mask; ++p) {
    const int32_t prev = atomicCAS(&hk[i], -1, key);
    if (prev == -1 || prev == key) {
      atomicAdd((ull*)&hv[i], (ull)w);
      return;
    }
    i = (i + 1) & mask;
  }
  atomicOr(status, ERR_HASH_FULL);
}

__device__ __forceinline__ long long table_get(const int32_t* hk, const long long* hv, int bits, int32_t key) {
  if (key < 0) return 0;
  const uint32_t mask = (1u << bits) - 1u;
  uint32_t i = small_hash(key, bits);
  for (uint32_t p = 0; p <= mask; ++p) {
    const int32_t k = hk[i];
    if (k == key) return hv[i];
    if (k == -1) return 0;
    i = (i + 1) & mask;
  }
  return 0;
}

template <class Pol>
__global__ void __launch_bounds__(BLOCK_TIER_THREADS) k_decide_block(Pol pol, const int32_t* list, const int32_t* count_ptr) {
  constexpr int BITS = 11;
  static_assert((1 << BITS) == BLOCK_TIER_SLOTS, "slots");
  __shared__ int32_t hk[BLOCK_TIER_SLOTS];
  __shared__ long long hv[BLOCK_TIER_SLOTS];
  __shared__ Cand red[BLOCK_TIER_THREADS / 32];
  const int count = *count_ptr;
  for (int idx = blockIdx.x; idx < count; idx += gridDim.x) {
    const int32_t v = list[idx];
    if (!pol.begin(v)) {
      if (threadIdx.x == 0) pol.skip(v);
      continue;
    }
    for (int i = threadIdx.x; i < BLOCK_TIER_SLOTS; i += BLOCK_TIER_THREADS) {
      hk[i] = -1;
      hv[i] = 0;
    }
    __syncthreads();
    const int64_t beg = pol.g.rowptr[v], end = pol.g.rowptr[v + 1];
    for (int64_t e = beg + threadIdx.x; e < end; e += BLOCK_TIER_THREADS) {
      int32_t key;
      long long w;
      if (pol.edge(v, e, key, w)) table_add<BITS>(hk, hv, key, w);
    }
    __syncthreads();
    Cand c{0, INT32_MAX};
    for (int i = threadIdx.x; i < BLOCK_TIER_SLOTS; i += BLOCK_TIER_THREADS) {
      const int32_t k = hk[i];
      if (k >= 0) {
        const Cand x = pol.cand(v, k, hv[i]);
        if (better(x, c)) c = x;
      }
    }
    const Cand best = block_best<BLOCK_TIER_THREADS / 32>(c, red);
    if (threadIdx.x == 0) {
      const long long Wb = best.label != INT32_MAX ? table_get(hk, hv, BITS, best.label) : 0;
      const long long Wown = table_get(hk, hv, BITS, pol.own_key(v));
      pol.finish(v, best, Wb, Wown);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int table_bits_for_degree(int64_t deg) {
  int bits = 1;
  while ((1ll << bits) < 2 * deg) ++bits;
  return bits;
}

template <class Pol>
__global__ void __launch_bounds__(GLOBAL_TIER_THREADS) k_decide_global(Pol pol, const int32_t* list, const int32_t* count_ptr,
                                int32_t* gkeys, long long* gvals, const int64_t* goff, unsigned* status) {
  __shared__ Cand red[GLOBAL_TIER_THREADS / 32];
  const int count = *count_ptr;
  for (int idx = blockIdx.x; idx < count; idx += gridDim.x) {
    const int32_t v = list[idx];
    if (!pol.begin(v)) {
      if (threadIdx.x == 0) pol.skip(v);
      continue;
    }
    const int64_t beg = pol.g.rowptr[v], end = pol.g.rowptr[v + 1];
    const int bits = table_bits_for_degree(end - beg);
    const int64_t S = 1ll << bits;
    int32_t* hk = gkeys + goff[v];
    long long* hv = gvals + goff[v];
    for (int64_t i = threadIdx.x; i < S; i += GLOBAL_TIER_THREADS) {
      hk[i] = -1;
      hv[i] = 0;
    }
    __syncthreads();
    for (int64_t e = beg + threadIdx.x; e < end; e += GLOBAL_TIER_THREADS) {
      int32_t key;
      long long w;
      if (pol.edge(v, e, key, w)) gtable_add(hk, hv, bits, key, w, status);
    }
    __syncthreads();
    Cand c{0, INT32_MAX};
    for (int64_t i = threadIdx.x; i < S; i += GLOBAL_TIER_THREADS) {
      const int32_t k = hk[i];
      if (k >= 0) {
        const Cand x = pol.cand(v, k, hv[i]);
        if (better(x, c)) c = x;
      }
    }
    const Cand best = block_best<GLOBAL_TIER_THREADS / 32>(c, red);
    if (threadIdx.x == 0) {
      const long long Wb = best.label != INT32_MAX ? table_get(hk, hv, bits, best.label) : 0;
      const long long Wown = table_get(hk, hv, bits, pol.own_key(v));
      pol.finish(v, best, Wb, Wown);
    }
    __syncthreads();
  }
}

}  // namespace mslice
