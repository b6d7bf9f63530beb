// Generic move-decision kernels.  For each node v of a work list the
// neighbour weights are aggregated per key (community or sub-community
// label) in a small open-addressing table, every distinct key is scored by
// the policy, and the best candidate (largest key, ties to the smallest
// label) is handed to the policy together with the key of staying.
//
// The work is latency-bound (row pointer -> entries -> neighbour labels ->
// per-community table), so the kernels aim at many independent loads in
// flight: small groups of lanes per low-degree node, all entry loads of a
// lane issued before any insert, scoring restricted to the node's distinct
// candidates, and the next node's row bounds fetched while the current node
// is scored.  Adjacency entries are read with
// evict-first loads so the label and community tables stay in L2.
//
// Five tiers by degree, all grid-stride over a device-resident list whose
// length is read on the device (no host round trip):
//   tier 0  deg <= 16    4-lane groups, eight nodes per warp, 32-slot tables
//   tier 1  deg <= 32    8-lane groups, four nodes per warp, 64-slot tables
//   tier 2  deg <= 256   one warp per node, 512-slot table
//   tier 3  deg <= 1024  one 256-thread block per node, shared table of
//                        2*deg slots rounded up to a power of two
//   tier 4  larger       one block per node, table of up to 8192 slots in
//                        dynamic shared memory (degree <= 4096), global
//                        scratch above
//
// Policy interface (all __device__):
//   bool begin(v)                      node takes part (uniform per node)
//   VCtx vctx(v)                       per-node values computed once (and
//                                      loads issued early for finish())
//   void skip(v)                       record "no move" for a non-participant
//   bool edge(v, vc, e, key&, w&)      entry e contributes w to key
//   Probe probe(v, vc, key)            first table load(s) for scoring key
//   Cand cand(v, vc, key, W, probe)    score of moving to key (INT32_MAX = not allowed)
//   int32_t own_key(v)                 the node's current key (-1 none)
//   i128 own(v, vc, W_own)             score of staying
//   void finish(v, best, W_best, G_own, vc)
//   static constexpr int MIN_BLOCKS    resident blocks per SM the group tiers aim for
// and, for the block tiers' slice-parallel scoring of aggregated nodes:
//   int64_t slice_count(v)             entries of v's (snapshot, strength) list (0 at level 0)
//   u128 null_part(v, vc, key, self, t, nt)  the null sum over entries t, t+nt, ...
//   Cand cand_ns(v, vc, key, W, ns)    cand() from a complete null sum
//   bool own_walks_slices()            own() walks the list (else it is cheap)
//   i128 own_ns(v, vc, W_own, ns)      own() from a complete null sum
#pragma once
#include <cstdlib>

#include "internal.h"
#include "level.h"

namespace mslice {

// Tuning parameter (compile-time): minimum resident blocks per SM for the
// group kernels, which caps their registers (occupancy matters more than
// per-warp parallelism for these latency-bound loops).
#ifndef MSLICE_GROUP_MIN_BLOCKS
#define MSLICE_GROUP_MIN_BLOCKS 4
#endif
// The same for policies on dense community tables (aggregated levels), whose
// scoring code needs more registers: at 4 blocks (64 registers) their group
// kernels spill ~280 bytes; 3 blocks cut the spills to ~100 bytes and the
// power-law solve's local moving by ~1.7% (measured; 2 blocks: no spills,
// no further gain).
#ifndef MSLICE_DENSE_MIN_BLOCKS
#define MSLICE_DENSE_MIN_BLOCKS 3
#endif
// entries loaded per lane per round by the warp-per-node tier
// tier 2: lanes per node (32: a warp per node, 512-slot tables; 16: two
// nodes per warp, 256-slot tables, so degrees up to 128)
#ifndef MSLICE_T2_LANES
#define MSLICE_T2_LANES 32
#endif
#ifndef MSLICE_T2_EPL
#define MSLICE_T2_EPL (MSLICE_T2_LANES == 32 ? 2 : 4)
#endif
constexpr int T2_BITS = MSLICE_T2_LANES == 32 ? 9 : 8;

constexpr int NTIERS = 5;
// Largest degree each of tiers 0-3 can take (their table capacities); the
// cuts in use may be lower (TierCuts), the rest go to the next tier.
constexpr int TIER_MAX[NTIERS - 1] = {16, 32, (1 << T2_BITS) / 2, 1024};

// Degree cuts between the tiers: tier t takes degrees in (t[t-1], t[t]].
// Which tier decides a node never changes its decision, only the speed.
struct TierCuts {
  int32_t t[NTIERS - 1] = {16, 32, (1 << T2_BITS) / 2, 1024};
};
constexpr int TIER3_BITS = 11;  // 2 * 1024 slots
// Tier 4's shared-memory table: 2^13 slots (degrees up to 4096) in 104 KB of
// dynamic shared memory, with room for 2^12 listed candidates.
constexpr int TIER4_SMEM_BITS = 13;
constexpr int TIER4_SMEM_SLOTS = 1 << TIER4_SMEM_BITS;
constexpr size_t TIER4_SMEM_BYTES =
    (size_t)TIER4_SMEM_SLOTS * (sizeof(long long) + sizeof(int32_t)) + (size_t)(TIER4_SMEM_SLOTS / 2) * sizeof(uint16_t);
constexpr int BLOCK_THREADS = 256;
constexpr int GROUP_THREADS = 256;

__host__ __device__ __forceinline__ int degree_tier(int64_t d, const TierCuts& c) {
  return d <= c.t[0] ? 0 : (d <= c.t[1] ? 1 : (d <= c.t[2] ? 2 : (d <= c.t[3] ? 3 : 4)));
}

// Aggregated nodes carry a list of (snapshot, strength) entries, and scoring
// one candidate walks that list once (the null term sums over snapshots).
// On long sequences late-level nodes hold thousands of entries, so a node
// whose (degree + 1) * entries reaches SLICE_WORK_BLOCK is decided by a
// block-per-node tier, whose threads then split each candidate's walk
// (slice_parallel) instead of taking one candidate each.
constexpr int64_t SLICE_WORK_BLOCK = 4096;

__host__ __device__ __forceinline__ int work_tier(int64_t d, int64_t nslices, const TierCuts& c) {
  const int t = degree_tier(d, c);
  if (t < NTIERS - 2 && nslices > 1 && (d + 1) * nslices >= SLICE_WORK_BLOCK) return NTIERS - 2;
  return t;
}

// Block-per-node scoring takes a candidate per thread unless splitting each
// candidate's slice walk over the block is cheaper: ceil(n/B) * ns
// sequential entries against n * (ceil(ns/B) + 3) (the 3: a reduction).
__device__ __forceinline__ bool slice_parallel(int64_t n, int64_t ns, int B) {
  return ns > 1 && ((n + B - 1) / B) * ns > n * ((ns + B - 1) / B + 3);
}

// Sum of one u128 per thread over the block (every thread gets it); sm holds
// 2 words per warp.
template <int WARPS>
__device__ __forceinline__ u128 block_sum_u128(u128 x, ull* sm) {
  ull lo = (ull)x, hi = (ull)(x >> 64);
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    const ull l2 = __shfl_xor_sync(0xffffffffu, lo, m), h2 = __shfl_xor_sync(0xffffffffu, hi, m);
    const ull nl = lo + l2;
    hi += h2 + (nl < lo ? 1ull : 0ull);
    lo = nl;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    sm[2 * w] = lo;
    sm[2 * w + 1] = hi;
  }
  __syncthreads();
  u128 t = 0;
#pragma unroll
  for (int k = 0; k < WARPS; ++k) t += ((u128)sm[2 * k + 1] << 64) | sm[2 * k];
  __syncthreads();
  return t;
}

__device__ __forceinline__ uint32_t small_hash(int32_t key, int bits) {
  return ((uint32_t)key * 2654435769u) >> (32 - bits);
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

__device__ __forceinline__ Cand shfl_xor_cand_m(const Cand& c, int m, unsigned mask) {
  Cand o;
  ull lo = (ull)(u128)c.G, hi = (ull)((u128)c.G >> 64);
  lo = __shfl_xor_sync(mask, lo, m);
  hi = __shfl_xor_sync(mask, hi, m);
  o.G = (i128)(((u128)hi << 64) | lo);
  o.label = __shfl_xor_sync(mask, c.label, m);
  return o;
}

template <int G>
__device__ __forceinline__ Cand group_best(Cand c, unsigned mask) {
#pragma unroll
  for (int m = G / 2; m >= 1; m >>= 1) {
    const Cand o = shfl_xor_cand_m(c, m, mask);
    if (better(o, c)) c = o;
  }
  return c;
}

// Insert-or-add that reports the slot and whether this call claimed it.
__device__ __forceinline__ int table_add_slot(int32_t* hk, long long* hv, int bits, int32_t key, long long w,
                                              bool& fresh) {
  const uint32_t mask = (1u << bits) - 1u;
  uint32_t i = small_hash(key, bits);
  for (uint32_t p = 0; p <= mask; ++p) {
    const int32_t prev = atomicCAS(&hk[i], -1, key);
    if (prev == -1 || prev == key) {
      atomicAdd((ull*)&hv[i], (ull)w);
      fresh = prev == -1;
      return (int)i;
    }
    i = (i + 1) & mask;
  }
  fresh = false;
  return -1;
}

// Tiers 0-2: G lanes per node, entries loaded EPL per lane at a time
// (deg <= 2^BITS / 2), 2^BITS table slots per group in shared memory.  The distinct keys of a node are
// listed as their slots are claimed, so scoring touches only real
// candidates and only those slots are reset afterwards (the table is cleared
// once per block, not once per node).
// Work is claimed in runs of consecutive list entries from a per-tier
// counter (queue), a warp at a time, so the nodes in flight form a narrow
// window of the node-ordered list and their gathers (neighbour labels, the
// snapshots' community-table regions) stay in L2.  A static grid-stride walk
// let the blocks drift apart over a launch (per-node cost varies widely),
// spreading the nodes in flight over many snapshots.
template <int G>
struct GroupClaim {
  static constexpr int NPG = G == 32 ? 4 : (G == 8 ? 8 : 4);  // nodes per group per claim
  static constexpr int SIZE = (32 / G) * NPG;                 // list entries per warp claim
};

template <class Pol, int G, int BITS, int EPL>
__global__ void __launch_bounds__(GROUP_THREADS, Pol::MIN_BLOCKS)
    k_decide_groups(Pol pol, const int32_t* list, const int32_t* count_ptr, int32_t* queue) {
  constexpr int WARPS = GROUP_THREADS / 32, GPW = 32 / G, SLOTS = 1 << BITS, MAXC = SLOTS / 2;
  constexpr bool ONE_CHUNK = MAXC <= G * EPL;  // every row fits one load round
  constexpr int NG = WARPS * GPW;
  __shared__ int32_t hk[NG][SLOTS];
  __shared__ long long hv[NG][SLOTS];
  __shared__ uint16_t cl[NG][MAXC];
  __shared__ int32_t ncand[NG];
  const int count = *count_ptr;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int gl = lane % G, gi = lane / G, gx = w * GPW + gi;
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (gi * G));
  int32_t* K = hk[gx];
  long long* V = hv[gx];
  uint16_t* CL = cl[gx];
#pragma unroll
  for (int i = gl; i < SLOTS; i += G) {
    K[i] = -1;
    V[i] = 0;
  }
  if (gl == 0) ncand[gx] = 0;
  __syncwarp(gmask);
  // claims of claim_size entries: group gi takes entries base + k * GPW +
  // gi, k < npg; the next claim is taken one claim ahead (its first node's
  // row bounds are prefetched like any next node's).  queue == nullptr: the
  // claims are dealt to the warps round-robin instead (short lists, where
  // the atomics would cost more than they save)
  // (round-robin runs are one node per group, the finest dealing: a short
  // list gives each warp few runs, and coarse runs would leave the warps
  // that drew one run more working alone at the end)
  const int npg = queue ? GroupClaim<G>::NPG : 1;
  const int claim_size = GPW * npg;
  const int warp_id = blockIdx.x * WARPS + w, warps = gridDim.x * WARPS;
  int ticket = warp_id;
  auto claim = [&]() -> int {
    int b = 0;
    if (queue) {
      if (lane == 0) b = atomicAdd(queue, claim_size);
      b = __shfl_sync(0xffffffffu, b, 0);
    } else {
      b = ticket * claim_size;
      ticket += warps;
    }
    return b;
  };
  int base = claim();
  if (base >= count) return;  // uniform per warp
  int nbase = claim();
  int k = 0;
  int idx = base + gi;
  bool have = idx < count;
  int32_t v = have ? list[idx] : 0;
  int64_t beg = have ? pol.g.rowptr[v] : 0, end = have ? pol.g.rowptr[v + 1] : 0;
  for (;;) {
    const bool next_claim = k + 1 == npg;  // uniform per warp
    const int nb = next_claim ? nbase : base;
    const int nidx = nb + (next_claim ? 0 : k + 1) * GPW + gi;
    const bool more = nidx < count;
    const int32_t nv = more ? list[nidx] : 0;
    int64_t nbeg = 0, nend = 0;
    if (!have) {
      // past the end of the list inside the last claim
    } else if (pol.begin(v)) {
      const typename Pol::VCtx vc = pol.vctx(v);
      // one load round: all of a lane's entries (and gathers) in flight
      // before any insert
      auto load_insert = [&](int64_t base) {
        int32_t keys[EPL];
        long long ws[EPL];
        bool ok[EPL];
#pragma unroll
        for (int j = 0; j < EPL; ++j) {
          const int64_t e = base + j * G + gl;
          ok[j] = e < end && pol.edge(v, vc, e, keys[j], ws[j]);
        }
#pragma unroll
        for (int j = 0; j < EPL; ++j) {
          if (ok[j]) {
            bool fresh;
            const int slot = table_add_slot(K, V, BITS, keys[j], ws[j], fresh);
#if MSLICE_CHECKED
            if (slot < 0) atomicOr(pol.g.chk, ERR_BOUNDS);
#endif
            if (fresh) CL[atomicAdd(&ncand[gx], 1)] = (uint16_t)slot;
          }
        }
      };
      if constexpr (ONE_CHUNK) {
        load_insert(beg);
      } else {
        for (int64_t base = beg; base < end; base += G * EPL) load_insert(base);
      }
      if (more) {
        nbeg = pol.g.rowptr[nv];
        nend = pol.g.rowptr[nv + 1];
      }
      __syncwarp(gmask);
      const int n = ncand[gx];
      const int32_t own = pol.own_key(v);
      Cand c{0, INT32_MAX};
      for (int j = gl; j < n; j += G) {
        const int slot = CL[j];
        const int32_t key = K[slot];
        if (key != own) {
          const Cand x = pol.cand(v, vc, key, V[slot], pol.probe(v, vc, key));
          if (better(x, c)) c = x;
        }
      }
      i128 Gown = 0;
      if (gl == 0) Gown = pol.own(v, vc, table_get(K, V, BITS, own));
      c = group_best<G>(c, gmask);
      if (gl == 0) {
        const long long Wb = c.label != INT32_MAX ? table_get(K, V, BITS, c.label) : 0;
        pol.finish(v, c, Wb, Gown, vc);
      }
      __syncwarp(gmask);
      for (int j = gl; j < n; j += G) {
        const int slot = CL[j];
        K[slot] = -1;
        V[slot] = 0;
      }
      if (gl == 0) ncand[gx] = 0;
      __syncwarp(gmask);
    } else {
      if (gl == 0) pol.skip(v);
      if (more) {
        nbeg = pol.g.rowptr[nv];
        nend = pol.g.rowptr[nv + 1];
      }
    }
    if (!have && more) {
      nbeg = pol.g.rowptr[nv];
      nend = pol.g.rowptr[nv + 1];
    }
    if (next_claim) {
      if (nbase >= count) break;  // uniform per warp
      base = nbase;
      nbase = claim();
      k = 0;
    } else {
      ++k;
    }
    idx = nidx;
    have = more;
    v = nv;
    beg = nbeg;
    end = nend;
  }
}

__device__ __forceinline__ int table_bits_for_degree(int64_t deg) {
  int bits = 1;
  while ((1ll << bits) < 2 * deg) ++bits;
  return bits;
}

template <class Pol>
__device__ __forceinline__ Cand score_range(const Pol& pol, int32_t v, const typename Pol::VCtx& vc, int32_t own,
                                            const int32_t* hk, const long long* hv, int64_t S) {
  Cand c{0, INT32_MAX};
  for (int64_t i = threadIdx.x; i < S; i += blockDim.x) {
    const int32_t k = hk[i];
    if (k >= 0 && k != own) {
      const Cand x = pol.cand(v, vc, k, hv[i], pol.probe(v, vc, k));
      if (better(x, c)) c = x;
    }
  }
  return c;
}

// One node decided by the whole block with its table in shared memory
// (hk/hv of at least 2^bits slots, all free on entry and left free; cl: room
// for 2^bits / 2 slot numbers; ncand: a shared counter, 0 on entry and left
// 0).  The node's distinct keys are listed as their slots are claimed.
template <class Pol, int NT = BLOCK_THREADS>
__device__ __forceinline__ void block_decide_node(const Pol& pol, int32_t v, int32_t* hk, long long* hv, uint16_t* cl,
                                                  int32_t* ncand, Cand* red, ull* usm, i128* own_sm) {
  const typename Pol::VCtx vc = pol.vctx(v);
  const int64_t beg = pol.g.rowptr[v], end = pol.g.rowptr[v + 1];
  const int bits = table_bits_for_degree(end - beg);
  for (int64_t e = beg + threadIdx.x; e < end; e += NT) {
    int32_t key;
    long long w;
    if (pol.edge(v, vc, e, key, w)) {
      bool fresh;
      const int slot = table_add_slot(hk, hv, bits, key, w, fresh);
#if MSLICE_CHECKED
      if (slot < 0) atomicOr(pol.g.chk, ERR_BOUNDS);
#endif
      if (fresh) cl[atomicAdd(ncand, 1)] = (uint16_t)slot;
    }
  }
  __syncthreads();
  const int n = *ncand;
  const int32_t own = pol.own_key(v);
  if (slice_parallel(n, pol.slice_count(v), NT)) {
    // every thread walks a share of the slice list for each candidate in
    // turn; thread 0 keeps the best
    Cand c{0, INT32_MAX};
    for (int j = 0; j < n; ++j) {
      const int slot = cl[j];
      const int32_t k = hk[slot];
      if (k == own) continue;
      const u128 ns =
          block_sum_u128<NT / 32>(pol.null_part(v, vc, k, false, threadIdx.x, NT), usm);
      if (threadIdx.x == 0) {
        const Cand x = pol.cand_ns(v, vc, k, hv[slot], ns);
        if (better(x, c)) c = x;
      }
    }
    i128 Go = 0;
    if (pol.own_walks_slices()) {
      const u128 ns =
          block_sum_u128<NT / 32>(pol.null_part(v, vc, own, true, threadIdx.x, NT), usm);
      if (threadIdx.x == 0) Go = pol.own_ns(v, vc, table_get(hk, hv, bits, own), ns);
    } else if (threadIdx.x == 0) {
      Go = pol.own(v, vc, table_get(hk, hv, bits, own));
    }
    if (threadIdx.x == 0) {
      const long long Wb = c.label != INT32_MAX ? table_get(hk, hv, bits, c.label) : 0;
      pol.finish(v, c, Wb, Go, vc);
    }
  } else {
    Cand c{0, INT32_MAX};
    for (int j = threadIdx.x; j < n; j += NT) {
      const int slot = cl[j];
      const int32_t k = hk[slot];
      if (k != own) {
        const Cand x = pol.cand(v, vc, k, hv[slot], pol.probe(v, vc, k));
        if (better(x, c)) c = x;
      }
    }
    if (threadIdx.x == 0) *own_sm = pol.own(v, vc, table_get(hk, hv, bits, own));
    const Cand best = block_best<NT / 32>(c, red);
    if (threadIdx.x == 0) {
      const long long Wb = best.label != INT32_MAX ? table_get(hk, hv, bits, best.label) : 0;
      pol.finish(v, best, Wb, *own_sm, vc);
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += NT) {
    const int slot = cl[j];
    hk[slot] = -1;
    hv[slot] = 0;
  }
  if (threadIdx.x == 0) *ncand = 0;
  __syncthreads();
}

// Tier 3: one block per node, shared table of 2*deg (rounded up) slots.
// Claims one node at a time from the tier's counter (thread 0), broadcast
// through shared memory; -1 once the list is exhausted.  queue == nullptr:
// nodes dealt to the blocks round-robin (*slot starts at -1).
__device__ __forceinline__ int block_claim(int32_t* queue, int count, int32_t* slot) {
  __syncthreads();  // every thread has read the previous claim
  if (threadIdx.x == 0) {
    const int i = queue ? atomicAdd(queue, 1) : (*slot < 0 ? (int)blockIdx.x : *slot + (int)gridDim.x);
    *slot = i < count ? i : -(1 << 30);
  }
  __syncthreads();
  return *slot < 0 ? -1 : *slot;
}

template <class Pol>
__global__ void __launch_bounds__(BLOCK_THREADS)
    k_decide_block(Pol pol, const int32_t* list, const int32_t* count_ptr, int32_t* queue) {
  constexpr int SLOTS = 1 << TIER3_BITS;
  __shared__ int32_t hk[SLOTS];
  __shared__ long long hv[SLOTS];
  __shared__ uint16_t cl[SLOTS / 2];
  __shared__ int32_t ncand;
  __shared__ Cand red[BLOCK_THREADS / 32];
  __shared__ ull usm[2 * (BLOCK_THREADS / 32)];
  __shared__ i128 own_sm;
  const int count = *count_ptr;
  for (int i = threadIdx.x; i < SLOTS; i += BLOCK_THREADS) {
    hk[i] = -1;
    hv[i] = 0;
  }
  __shared__ int32_t claim;
  if (threadIdx.x == 0) {
    ncand = 0;
    claim = -1;
  }
  for (int idx; (idx = block_claim(queue, count, &claim)) >= 0;) {
    const int32_t v = list[idx];
    if (!pol.begin(v)) {
      if (threadIdx.x == 0) pol.skip(v);
      continue;
    }
    block_decide_node(pol, v, hk, hv, cl, &ncand, red, usm, &own_sm);
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

// Tier 4: one block of NT threads per node.  A node whose table fits
// 2^TIER4_SMEM_BITS slots (degree up to 4096) keeps it in dynamic shared
// memory (one block per SM), as tier 3 does; a larger one uses global
// scratch at goff[v].
template <class Pol, int NT>
__global__ void __launch_bounds__(NT) k_decide_global(Pol pol, const int32_t* list, const int32_t* count_ptr,
                                                                 int32_t* gkeys, long long* gvals, const int64_t* goff,
                                                                 unsigned* status, bool use_smem, int32_t* queue) {
  extern __shared__ __align__(16) unsigned char t4_smem[];
  long long* shv = reinterpret_cast<long long*>(t4_smem);
  int32_t* shk = reinterpret_cast<int32_t*>(t4_smem + TIER4_SMEM_SLOTS * sizeof(long long));
  uint16_t* scl = reinterpret_cast<uint16_t*>(t4_smem + TIER4_SMEM_SLOTS * (sizeof(long long) + sizeof(int32_t)));
  __shared__ int32_t ncand;
  __shared__ Cand red[NT / 32];
  __shared__ ull usm[2 * (NT / 32)];
  __shared__ i128 own_sm;
  const int count = *count_ptr;
  if (use_smem)
    for (int i = threadIdx.x; i < TIER4_SMEM_SLOTS; i += NT) {
      shk[i] = -1;
      shv[i] = 0;
    }
  __shared__ int32_t claim;
  if (threadIdx.x == 0) {
    ncand = 0;
    claim = -1;
  }
  for (int idx; (idx = block_claim(queue, count, &claim)) >= 0;) {
    const int32_t v = list[idx];
    if (!pol.begin(v)) {
      if (threadIdx.x == 0) pol.skip(v);
      continue;
    }
    if (use_smem && table_bits_for_degree(pol.g.rowptr[v + 1] - pol.g.rowptr[v]) <= TIER4_SMEM_BITS) {
      block_decide_node<Pol, NT>(pol, v, shk, shv, scl, &ncand, red, usm, &own_sm);
      continue;
    }
    const typename Pol::VCtx vc = pol.vctx(v);
    const int64_t beg = pol.g.rowptr[v], end = pol.g.rowptr[v + 1];
    const int bits = table_bits_for_degree(end - beg);
    const int64_t S = 1ll << bits;
    int32_t* hk = gkeys + goff[v];
    long long* hv = gvals + goff[v];
    for (int64_t i = threadIdx.x; i < S; i += NT) {
      hk[i] = -1;
      hv[i] = 0;
    }
    __syncthreads();
    for (int64_t e = beg + threadIdx.x; e < end; e += NT) {
      int32_t key;
      long long w;
      if (pol.edge(v, vc, e, key, w)) gtable_add(hk, hv, bits, key, w, status);
    }
    __syncthreads();
    const int32_t own = pol.own_key(v);
    if (slice_parallel(end - beg, pol.slice_count(v), NT)) {
      // (the degree bounds the candidates) the block splits each
      // candidate's slice walk; thread 0 keeps the best
      Cand c{0, INT32_MAX};
      for (int64_t i = 0; i < S; ++i) {
        const int32_t k = hk[i];
        if (k < 0 || k == own) continue;
        const u128 ns =
            block_sum_u128<NT / 32>(pol.null_part(v, vc, k, false, threadIdx.x, NT), usm);
        if (threadIdx.x == 0) {
          const Cand x = pol.cand_ns(v, vc, k, hv[i], ns);
          if (better(x, c)) c = x;
        }
      }
      i128 Go = 0;
      if (pol.own_walks_slices()) {
        const u128 ns =
            block_sum_u128<NT / 32>(pol.null_part(v, vc, own, true, threadIdx.x, NT), usm);
        if (threadIdx.x == 0) Go = pol.own_ns(v, vc, table_get(hk, hv, bits, own), ns);
      } else if (threadIdx.x == 0) {
        Go = pol.own(v, vc, table_get(hk, hv, bits, own));
      }
      if (threadIdx.x == 0) {
        const long long Wb = c.label != INT32_MAX ? table_get(hk, hv, bits, c.label) : 0;
        pol.finish(v, c, Wb, Go, vc);
      }
    } else {
      if (threadIdx.x == 0) own_sm = pol.own(v, vc, table_get(hk, hv, bits, own));
      const Cand best = block_best<NT / 32>(score_range(pol, v, vc, own, hk, hv, S), red);
      if (threadIdx.x == 0) {
        const long long Wb = best.label != INT32_MAX ? table_get(hk, hv, bits, best.label) : 0;
        pol.finish(v, best, Wb, own_sm, vc);
      }
    }
    __syncthreads();
  }
}

// Nodes a tier must hold at a level before its kernels claim work from a
// counter (at the T=64, n=10^6 workload's level 0 every tier but the top one
// does; the T=16, n=10^5 workload's lists are dealt round-robin, where the
// counter's atomics cost more than they saved).
constexpr int32_t DYN_CLAIM_MIN[NTIERS] = {1 << 22, 1 << 22, 1 << 21, 1 << 16, 1 << 16};

// The tier lists of one sub-round (device pointers; counts on device).
struct TierSegs {
  const int32_t* list[NTIERS];
  const int32_t* count[NTIERS];
  int32_t* queue = nullptr;  // NTIERS work counters of the decision kernels (zeroed by decide_all)
};

constexpr int64_t T4_WIDE_BELOW = 1 << 22;

template <class Pol, int NT>
void launch_tier4(Ctx& c, cudaStream_t st, const Pol& pol, const TierSegs& sg, int32_t* gkeys, long long* gvals,
                  const int64_t* goff, bool smem, int32_t* queue) {
  static bool smem_set = false;  // per instantiation: the dynamic shared memory limit, set once
  if (smem && !smem_set) {
    check_cuda(cudaFuncSetAttribute(k_decide_global<Pol, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)TIER4_SMEM_BYTES), "tier-4 shared memory");
    smem_set = true;
  }
  // with the shared table, one block per SM: its 104 KB leave room for the
  // other tiers' blocks, which run concurrently
  launch_on(c, st, k_decide_global<Pol, NT>, dim3(smem ? 152 : 152 * 2048 / NT), dim3(NT),
            smem ? TIER4_SMEM_BYTES : 0, pol, sg.list[4], sg.count[4], gkeys, gvals, goff, c.d_status, smem, queue);
}

// Launches the tiers of one sub-round; tier_cnt (host) skips tiers that are
// empty at this level.  Grids are fixed multiples of the 152 SMs.
template <class Pol>
void decide_all(Ctx& c, const Pol& pol, const TierSegs& sg, const int32_t* tier_cnt, int32_t* gkeys,
                long long* gvals, const int64_t* goff) {
  // The tiers decide disjoint node sets with separate scratch, so they may
  // run concurrently: heaviest first, each on its own side stream (their few
  // long rows then overlap the group tiers instead of trailing them).
  // dynamic claims only for tiers with many nodes at this level (each warp
  // or block then takes many claims, and balancing the concurrent tiers pays
  // for the atomics); short lists are dealt round-robin
  int32_t* q[NTIERS];
  bool any_dyn = false;
  for (int t = 0; t < NTIERS; ++t) {
    q[t] = tier_cnt[t] >= DYN_CLAIM_MIN[t] ? sg.queue + t : nullptr;
    any_dyn = any_dyn || q[t];
  }
  if (any_dyn) check_cuda(cudaMemsetAsync(sg.queue, 0, NTIERS * sizeof(int32_t), c.stream), "memset");
  StreamFan* f = c.fan;
  cudaStream_t st[NTIERS] = {c.stream, c.stream, c.stream, c.stream, c.stream};
  bool used[StreamFan::kSide] = {false, false, false, false};
  if (f) {
    int busy = 0;
    for (int t = 0; t < NTIERS; ++t) busy += tier_cnt[t] > 0;
    if (busy > 1) {
      check_cuda(cudaEventRecord(f->fork, c.stream), "event");
      // tiers 4, 3, 2, 1 on side streams 0..3; tier 0 on the context's stream
      for (int t = NTIERS - 1; t >= 1; --t)
        if (tier_cnt[t] > 0) {
          const int k = NTIERS - 1 - t;
          check_cuda(cudaStreamWaitEvent(f->side[k], f->fork, 0), "event");
          st[t] = f->side[k];
          used[k] = true;
        }
    }
  }
  if (tier_cnt[4] > 0) {
    // MSLICE_TIER4_SHARED=0: every tier-4 node uses global scratch
    static const bool smem = [] {
      const char* e = std::getenv("MSLICE_TIER4_SHARED");
      return !(e && e[0] == '0');
    }();
    // 32 warps per tier-4 block where the group tiers hold few nodes (coarse
    // levels, where the hubs are the whole sub-round), 16 beside long group
    // tiers, whose blocks share the SMs
    const int64_t group_nodes = (int64_t)tier_cnt[0] + tier_cnt[1] + tier_cnt[2];
    if (group_nodes < T4_WIDE_BELOW)
      launch_tier4<Pol, 1024>(c, st[4], pol, sg, gkeys, gvals, goff, smem, q[4]);
    else
      launch_tier4<Pol, 512>(c, st[4], pol, sg, gkeys, gvals, goff, smem, q[4]);
  }
  if (tier_cnt[3] > 0)
    launch_on(c, st[3], k_decide_block<Pol>, dim3(152 * 4), dim3(BLOCK_THREADS), 0, pol, sg.list[3], sg.count[3],
              q[3]);
  if (tier_cnt[2] > 0)
    launch_on(c, st[2], k_decide_groups<Pol, MSLICE_T2_LANES, T2_BITS, MSLICE_T2_EPL>, dim3(152 * 4), dim3(GROUP_THREADS), 0, pol,
              sg.list[2], sg.count[2], q[2]);
  if (tier_cnt[1] > 0)
    launch_on(c, st[1], k_decide_groups<Pol, 8, 6, 4>, dim3(152 * 4), dim3(GROUP_THREADS), 0, pol, sg.list[1],
              sg.count[1], q[1]);
  if (tier_cnt[0] > 0)
    launch_on(c, st[0], k_decide_groups<Pol, 4, 5, 4>, dim3(152 * 4), dim3(GROUP_THREADS), 0, pol, sg.list[0],
              sg.count[0], q[0]);
  for (int k = 0; k < StreamFan::kSide; ++k)
    if (used[k]) {
      check_cuda(cudaEventRecord(f->join[k], f->side[k]), "event");
      check_cuda(cudaStreamWaitEvent(c.stream, f->join[k], 0), "event");
    }
}

}  // namespace mslice
