// Device-side building blocks shared by the mslice kernels (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mslice {

typedef __int128 i128;
typedef unsigned __int128 u128;
typedef unsigned long long ull;

constexpr int P_BITS = 64;           // quantisation exponent of the null coefficient
constexpr int32_t NO_MOVE = -1;      // decision: stay
constexpr int32_t TO_EMPTY = -2;     // decision: move to an empty community
constexpr ull EMPTY_KEY = ~0ull;     // free hash slot

// Error bits of the device status word.
constexpr unsigned ERR_HASH_FULL = 1u;   // a probe sequence exceeded the table
constexpr unsigned ERR_BAD_INPUT = 2u;   // validation of a snapshot failed
constexpr unsigned ERR_INTERNAL = 4u;    // an internal consistency check failed
constexpr unsigned ERR_BOUNDS = 8u;      // checked builds: an index or table bound was violated

// Checked builds (-DMSLICE_CHECKED=1) test indices and table capacities on
// the hot paths and record violations in the status word instead of making
// the access; the tests run them against the oracle.
#ifndef MSLICE_CHECKED
#define MSLICE_CHECKED 0
#endif

// SplitMix64 output finaliser (Steele, Lea & Flood, OOPSLA 2014), written from
// its published definition.  Drives the vertex classes of the schedule.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

// Class of node v in round r of level lvl, iteration it; tag 0 = local
// moving, 1 = refinement.  The chain folds one counter per step.
// The schedule's counter-based hash of (seed, tag, iteration, level, round,
// node); its value mod K is the node's class, and tag 2 gives the draw of
// the randomised refinement.
__host__ __device__ __forceinline__ uint64_t class_hash(uint64_t seed, uint64_t tag, uint64_t it, uint64_t lvl,
                                                        uint64_t r, uint64_t v) {
  return mix64(seed ^ mix64(tag ^ mix64(it ^ mix64(lvl ^ mix64(r ^ mix64(v))))));
}

__host__ __device__ __forceinline__ int vertex_class(uint64_t seed, uint64_t tag, uint64_t it, uint64_t lvl,
                                                     uint64_t r, uint64_t v, int K) {
  return (int)(class_hash(seed, tag, it, lvl, r, v) % (uint64_t)K);
}

// -------------------------------------------------------------------------
// Open-addressing hash keyed by a 64-bit key with an int64 payload, one
// 16-byte slot per entry so a probe touches one sector.  Linear probing over
// an arbitrary capacity (Lemire's multiply-high range reduction), bounded
// probe length; payload updates are integer atomics, so the stored values do
// not depend on the order of the updates.
struct alignas(16) Slot {
  ull key;
  long long val;
};

// The table is cut into one region per null slice s (the low 32 bits of a
// key): keys (c, s) live in slots [region[s], region[s+1]), and probing wraps
// inside the region.  A region is sized for the level-0 nodes of its slice,
// so the keys a sub-round touches, which belong to the few snapshots its
// nodes are drawn from at any moment, stay in a small part of the table
// (L2-resident) instead of spreading over all of it.
//
// Narrow tables hold 8-byte slots {community, sum}: inside a region the
// snapshot is implied, and a sum fits 32 bits when every null slice's mass
// (the largest sum it can reach) is below 2^32.  They take half the bytes of
// the 16-byte {key, sum} slots and put four slots in a sector.
struct alignas(8) Slot8 {
  uint32_t key;  // community, EMPTY_KEY8 when free
  uint32_t val;
};
constexpr uint32_t EMPTY_KEY8 = 0xffffffffu;

struct HashView {
  Slot* slots;                       // 16-byte slots, or (narrow) Slot8 storage
  uint64_t cap;                      // slots over all regions
  unsigned* status;
  ull* used = nullptr;               // optional: regions past half their capacity since the last clear
  const uint64_t* region = nullptr;  // R + 1 slot offsets
  ull* region_used = nullptr;        // optional with `used`: slots taken per region since the last clear
  int32_t nregions = 0;
  int32_t narrow = 0;
};

__device__ __forceinline__ ull pack_cs(int32_t c, int32_t s) {
  return ((ull)(uint32_t)c << 32) | (uint32_t)s;
}

__device__ __forceinline__ Slot8* slots8(const HashView& h) { return reinterpret_cast<Slot8*>(h.slots); }

// Region of a key: its first slot and its size.
__device__ __forceinline__ void hash_region(const HashView& h, ull key, uint64_t& base, uint64_t& size) {
  const uint32_t s = (uint32_t)key;
  base = __ldg(&h.region[s]);
  size = __ldg(&h.region[s + 1]) - base;
}

// Home slot inside the region: one multiplicative mixing step (Fibonacci
// hashing) and a multiply-high range reduction; slot positions never affect
// results.  Narrow tables hash the community alone (the region fixes the
// snapshot).
__device__ __forceinline__ uint64_t hash_home(ull key, uint64_t base, uint64_t size) {
  return base + __umul64hi((key ^ (key >> 29)) * 0x9E3779B97F4A7C15ULL, size);
}

__device__ __forceinline__ uint64_t hash_home8(uint32_t c, uint64_t base, uint64_t size) {
  return base + __umul64hi((ull)c * 0x9E3779B97F4A7C15ULL, size);
}

__device__ __forceinline__ uint64_t hash_next(uint64_t i, uint64_t base, uint64_t size) {
  return (i + 1 == base + size) ? base : i + 1;
}

// Counts a freshly taken slot against its region (rebuild trigger).
__device__ __forceinline__ void hash_took_slot(const HashView& h, ull key, uint64_t size) {
  if (!h.used) return;
  // count the region once, when its taken slots pass half of it
  const ull taken = atomicAdd(&h.region_used[(uint32_t)key], 1ull) + 1;
  if (2 * taken > size && 2 * (taken - 1) <= size) atomicAdd(h.used, 1ull);
}

__device__ __forceinline__ void hash_add(const HashView& h, ull key, long long delta) {
  uint64_t base, size;
  hash_region(h, key, base, size);
  if (h.narrow) {
    Slot8* sl = slots8(h);
    const uint32_t c = (uint32_t)(key >> 32);
    uint64_t i = hash_home8(c, base, size);
    for (uint64_t probe = 0; probe < size; ++probe) {
      const uint32_t k = sl[i].key;
      if (k == c) {
        atomicAdd(&sl[i].val, (uint32_t)delta);
        return;
      }
      if (k == EMPTY_KEY8) {
        const uint32_t prev = atomicCAS(&sl[i].key, EMPTY_KEY8, c);
        if (prev == EMPTY_KEY8 || prev == c) {
          atomicAdd(&sl[i].val, (uint32_t)delta);
          if (prev == EMPTY_KEY8) hash_took_slot(h, key, size);
          return;
        }
      }
      i = hash_next(i, base, size);
    }
    atomicOr(h.status, ERR_HASH_FULL);
    return;
  }
  uint64_t i = hash_home(key, base, size);
  for (uint64_t probe = 0; probe < size; ++probe) {
    ull k = h.slots[i].key;
    if (k == key) {
      atomicAdd((ull*)&h.slots[i].val, (ull)delta);
      return;
    }
    if (k == EMPTY_KEY) {
      ull prev = atomicCAS(&h.slots[i].key, EMPTY_KEY, key);
      if (prev == EMPTY_KEY || prev == key) {
        atomicAdd((ull*)&h.slots[i].val, (ull)delta);
        if (prev == EMPTY_KEY) hash_took_slot(h, key, size);
        return;
      }
    }
    i = hash_next(i, base, size);
  }
  atomicOr(h.status, ERR_HASH_FULL);
}

// A narrow slot as a 16-byte one: key = the community (EMPTY_KEY when free).
__device__ __forceinline__ Slot widen(const Slot8& x) {
  return Slot{x.key == EMPTY_KEY8 ? EMPTY_KEY : (ull)x.key, (long long)x.val};
}

// Read-only lookup (0 when absent).  Only valid while no thread inserts.
__device__ __forceinline__ long long hash_get(const HashView& h, ull key) {
  uint64_t base, size;
  hash_region(h, key, base, size);
  if (h.narrow) {
    const Slot8* sl = slots8(h);
    const uint32_t c = (uint32_t)(key >> 32);
    uint64_t i = hash_home8(c, base, size);
    for (uint64_t probe = 0; probe < size; ++probe) {
      const Slot8 x = sl[i];
      if (x.key == c) return (long long)x.val;
      if (x.key == EMPTY_KEY8) return 0;
      i = hash_next(i, base, size);
    }
    return 0;
  }
  uint64_t i = hash_home(key, base, size);
  for (uint64_t probe = 0; probe < size; ++probe) {
    const Slot s = h.slots[i];
    if (s.key == key) return s.val;
    if (s.key == EMPTY_KEY) return 0;
    i = hash_next(i, base, size);
  }
  return 0;
}

// Lookup continuing from an already loaded home slot `first` (narrow: as
// widen() gives it).
__device__ __forceinline__ long long hash_get_from(const HashView& h, ull key, const Slot& first) {
  if (h.narrow) {
    const uint32_t c = (uint32_t)(key >> 32);
    if (first.key == (ull)c) return first.val;
    if (first.key == EMPTY_KEY) return 0;
    uint64_t base, size;
    hash_region(h, key, base, size);
    const Slot8* sl = slots8(h);
    uint64_t i = hash_home8(c, base, size);
    for (uint64_t probe = 1; probe < size; ++probe) {
      i = hash_next(i, base, size);
      const Slot8 x = sl[i];
      if (x.key == c) return (long long)x.val;
      if (x.key == EMPTY_KEY8) return 0;
    }
    return 0;
  }
  if (first.key == key) return first.val;
  if (first.key == EMPTY_KEY) return 0;
  uint64_t base, size;
  hash_region(h, key, base, size);
  uint64_t i = hash_home(key, base, size);
  for (uint64_t probe = 1; probe < size; ++probe) {
    i = hash_next(i, base, size);
    const Slot s = h.slots[i];
    if (s.key == key) return s.val;
    if (s.key == EMPTY_KEY) return 0;
  }
  return 0;
}

__device__ __forceinline__ Slot hash_first(const HashView& h, ull key) {
  uint64_t base, size;
  hash_region(h, key, base, size);
  if (h.narrow) return widen(slots8(h)[hash_home8((uint32_t)(key >> 32), base, size)]);
  return h.slots[hash_home(key, base, size)];
}

// Region holding slot i (binary search over the offsets).
__device__ __forceinline__ int32_t hash_region_of(const HashView& h, uint64_t i) {
  int32_t lo = 0, hi = h.nregions - 1;
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (__ldg(&h.region[mid]) <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// -------------------------------------------------------------------------
// Table of per-(label, snapshot) sums (Sigma_{c,s}, K_{R,s}).  Dense rows of
// T entries when labels x T fits the memory budget (one indexed load per
// lookup, no hashing), the hash above otherwise.
struct SigStore {
  long long* d = nullptr;  // dense: rows x T, zero = absent
  int64_t rows = 0;
  int32_t T = 1;
  HashView h{};
};

__device__ __forceinline__ long long ss_get(const SigStore& st, int32_t c, int32_t s) {
  if (st.d) return st.d[(int64_t)c * st.T + s];
  return hash_get(st.h, pack_cs(c, s));
}

__device__ __forceinline__ void ss_add(const SigStore& st, int32_t c, int32_t s, long long x) {
  if (st.d)
    atomicAdd((ull*)&st.d[(int64_t)c * st.T + s], (ull)x);
  else
    hash_add(st.h, pack_cs(c, s), x);
}

// First load of a lookup (issued early), and its resolution.
__device__ __forceinline__ Slot ss_first(const SigStore& st, int32_t c, int32_t s) {
  if (st.d) return Slot{pack_cs(c, s), st.d[(int64_t)c * st.T + s]};
  return hash_first(st.h, pack_cs(c, s));
}

__device__ __forceinline__ long long ss_resolve(const SigStore& st, int32_t c, int32_t s, const Slot& first) {
  if (st.d) return first.val;
  return hash_get_from(st.h, pack_cs(c, s), first);
}

// The same lookups with the table kind fixed at compile time (the decision
// kernels are instantiated for both kinds, keeping register use low).
template <bool DENSE>
__device__ __forceinline__ long long sst_get(const SigStore& st, int32_t c, int32_t s) {
  if constexpr (DENSE)
    return st.d[(int64_t)c * st.T + s];
  else
    return hash_get(st.h, pack_cs(c, s));
}

template <bool DENSE>
__device__ __forceinline__ Slot sst_first(const SigStore& st, int32_t c, int32_t s) {
  if constexpr (DENSE)
    return Slot{0, st.d[(int64_t)c * st.T + s]};
  else
    return hash_first(st.h, pack_cs(c, s));
}

template <bool DENSE>
__device__ __forceinline__ long long sst_resolve(const SigStore& st, int32_t c, int32_t s, const Slot& first) {
  if constexpr (DENSE)
    return first.val;
  else
    return hash_get_from(st.h, pack_cs(c, s), first);
}

// Enumeration of the non-zero entries: index i in [0, ss_span).
__device__ __forceinline__ uint64_t ss_span(const SigStore& st) {
  return st.d ? (uint64_t)st.rows * (uint64_t)st.T : st.h.cap;
}

__device__ __forceinline__ bool ss_entry(const SigStore& st, uint64_t i, int32_t& c, int32_t& s, long long& v) {
  if (st.d) {
    v = st.d[i];
    if (v == 0) return false;
    c = (int32_t)(i / (uint64_t)st.T);
    s = (int32_t)(i % (uint64_t)st.T);
    return true;
  }
  if (st.h.narrow) {
    const Slot8 x = slots8(st.h)[i];
    if (x.key == EMPTY_KEY8 || x.val == 0) return false;
    c = (int32_t)x.key;
    s = hash_region_of(st.h, i);
    v = (long long)x.val;
    return true;
  }
  const Slot sl = st.h.slots[i];
  if (sl.key == EMPTY_KEY || sl.val == 0) return false;
  c = (int32_t)(sl.key >> 32);
  s = (int32_t)(sl.key & 0xffffffffu);
  v = sl.val;
  return true;
}

// -------------------------------------------------------------------------
// Unsigned 128-bit accumulation into two 64-bit words with carry propagation.
// Exact as long as the true sum stays below 2^128.
__device__ __forceinline__ void atomic_add_u128(ull* lohi, u128 x) {
  ull lo = (ull)x, hi = (ull)(x >> 64);
  ull old = atomicAdd(&lohi[0], lo);
  if (old + lo < old) hi += 1;
  if (hi) atomicAdd(&lohi[1], hi);
}

// u128 -> double, round to nearest even.  The top 64 significant bits are
// converted by the hardware's correctly rounded u64 conversion with every
// lower bit folded into the least significant one (a sticky bit); since the
// u64 holds 11 bits below the double's rounding position, the sticky bit
// decides ties exactly as an infinitely precise conversion would.
__device__ __forceinline__ double u128_to_double(u128 x) {
  ull hi = (ull)(x >> 64), lo = (ull)x;
  if (hi == 0) return __ull2double_rn(lo);
  int lz = __clzll((long long)hi);
  u128 y = x << lz;
  ull top = (ull)(y >> 64);
  ull rest = (ull)y;
  top |= (rest != 0) ? 1ull : 0ull;
  return ldexp(__ull2double_rn(top), 64 - lz);
}

// -------------------------------------------------------------------------
// Candidate of a move decision: larger key wins, ties go to the smaller label.
struct Cand {
  i128 G;
  int32_t label;  // INT32_MAX = none
};

__device__ __forceinline__ bool better(const Cand& a, const Cand& b) {
  if (a.label == INT32_MAX) return false;
  if (b.label == INT32_MAX) return true;
  if (a.G != b.G) return a.G > b.G;
  return a.label < b.label;
}

__device__ __forceinline__ Cand shfl_cand(const Cand& c, int src) {
  Cand o;
  ull lo = (ull)(u128)c.G, hi = (ull)((u128)c.G >> 64);
  lo = __shfl_sync(0xffffffffu, lo, src);
  hi = __shfl_sync(0xffffffffu, hi, src);
  o.G = (i128)(((u128)hi << 64) | lo);
  o.label = __shfl_sync(0xffffffffu, c.label, src);
  return o;
}

__device__ __forceinline__ Cand shfl_xor_cand(const Cand& c, int m) {
  Cand o;
  ull lo = (ull)(u128)c.G, hi = (ull)((u128)c.G >> 64);
  lo = __shfl_xor_sync(0xffffffffu, lo, m);
  hi = __shfl_xor_sync(0xffffffffu, hi, m);
  o.G = (i128)(((u128)hi << 64) | lo);
  o.label = __shfl_xor_sync(0xffffffffu, c.label, m);
  return o;
}

__device__ __forceinline__ Cand warp_best(Cand c) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    Cand o = shfl_xor_cand(c, m);
    if (better(o, c)) c = o;
  }
  return c;
}

template <int WARPS>
__device__ __forceinline__ Cand block_best(Cand c, Cand* sm) {
  c = warp_best(c);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sm[w] = c;
  __syncthreads();
  if (w == 0) {
    Cand x = lane < WARPS ? sm[lane] : Cand{0, INT32_MAX};
    x = warp_best(x);
    if (lane == 0) sm[0] = x;
  }
  __syncthreads();
  Cand r = sm[0];
  __syncthreads();
  return r;
}

// Sum of one u128 per lane over the warp (every lane gets it).
__device__ __forceinline__ u128 warp_sum_u128(u128 x) {
  ull lo = (ull)x, hi = (ull)(x >> 64);
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    const ull l2 = __shfl_xor_sync(0xffffffffu, lo, m), h2 = __shfl_xor_sync(0xffffffffu, hi, m);
    const ull nl = lo + l2;
    hi += h2 + (nl < lo ? 1ull : 0ull);
    lo = nl;
  }
  return ((u128)hi << 64) | lo;
}

template <class T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) x += __shfl_xor_sync(0xffffffffu, x, m);
  return x;
}

}  // namespace mslice
