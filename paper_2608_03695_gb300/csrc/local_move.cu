// Local moving (the Louvain/Leiden move phase, Sec. 3.2) of multislice
// modularity (Eq. multislice-modularity) under the synchronous schedule:
// in round r every node draws a class in [0, K) from the counter-based hash;
// in sub-round q the nodes of class q decide against the state at the start
// of the sub-round, then every decision is applied at once.
//
// Exact move key of node v for community c (c\v: v excluded):
//   G(v,c) = 2^64 W(v,c\v) - od * sum_s Lambda_s k_{v,s} Sigma_{c\v,s}
// with W in units of 1/od (intra-snapshot weight w counts od*w, a coupling
// entry counts on) and Lambda_s = floor(gn 2^64 / (gd 2m_s)).  G is 2^64*od
// times the modularity gain up to a per-node constant, with gamma/2m_s
// quantised to Lambda_s/2^64.  Best = largest key, ties to the smallest
// label; a node that is not alone may also move to an empty community
// (key 0, losing ties); it moves only on a strict improvement; a node alone
// in its community joins another singleton community only if that label is
// smaller (otherwise two neighbouring singletons could swap forever).
//
// Global null model (plain modularity of the supra-graph, Eq. modularity):
// one null slice per instance, strengths k' = od*k + on*(coupling edges),
// Lambda' = floor(gn 2^64 / (gd 2M')), 2M' = od*2mu, and the null term's
// scale od becomes 1 (Omega::nd):  G(v,c) = 2^64 W(v,c\v) - Lambda' k'_v
// Sigma'_{c\v}.
//
// Sigma_{c,s} lives in a hash keyed (c, s) and is kept exact by the integer
// atomics of every move; it is rebuilt from the labels only at the start of
// a level and when tombstone keys fill half of the table.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "../../include/mslice.h"
#include "decide.cuh"
#include "solver.h"

namespace cg = cooperative_groups;

namespace mslice {

namespace {

constexpr int APPLY_THREADS = 256;
constexpr int GRAPH_FROM_ROUND = 4;
// Levels of at most this many nodes replay round graphs in single solves too
// (their rounds are launch-bound).
constexpr int64_t GRAPH_MAX_NODES = 0;
constexpr int EMPTY_THREADS = 512;

unsigned fixed_grid(int per_sm) { return 152u * (unsigned)per_sm; }

// Tier of every node by degree, and by slice work at aggregated levels
// (sptr non-null: see work_tier).
__global__ void k_tier(const int64_t* rowptr, const int64_t* sptr, int32_t N, TierCuts cuts, uint8_t* tier,
                       int32_t* cnt, int64_t* gsize) {
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < N; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = base + threadIdx.x;
    int t = -1;
    if (v < N) {
      const int64_t d = rowptr[v + 1] - rowptr[v];
      t = work_tier(d, sptr ? sptr[v + 1] - sptr[v] : 0, cuts);
      tier[v] = (uint8_t)t;
      int64_t S = 0;
      if (t == NTIERS - 1) {
        S = 2;
        while (S < 2 * d) S <<= 1;
      }
      gsize[v] = S;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, t);
    if (t >= 0 && lane == __ffs(peers) - 1) atomicAdd(&cnt[t], __popc(peers));
  }
}

// Buckets the nodes of this round by (class, tier): row q of `lists` holds
// class q, tier t at [tier_off[t], tier_off[t] + count).  Order inside a
// bucket does not matter: decisions read only the sub-round snapshot.
struct TierOff {
  int32_t off[NTIERS];
};

// Bucketing in node order, in three steps over chunks of BUCKET_CHUNK
// consecutive nodes: count every chunk's nodes per (class, tier) segment,
// scan the counts of each segment over the chunks, then write every chunk's
// nodes at its offsets.  The lists come out in ascending node order, so the
// nodes a decision kernel holds in flight at any moment (a window of the
// list) are close in node order and their gathers (neighbour labels in the
// same snapshots, the snapshots' community-table regions) stay in L2.  A
// chunk is one block; ranks inside a chunk come from shared-memory atomics
// (order inside a chunk does not matter).
constexpr int BUCKET_THREADS = 256;
constexpr int BUCKET_ITEMS = 16;
constexpr int64_t BUCKET_CHUNK = (int64_t)BUCKET_THREADS * BUCKET_ITEMS;
constexpr int BUCKET_MAX_SEGS = 64 * NTIERS;  // segments (K * NTIERS) for K <= 64
constexpr uint16_t BUCKET_FROZEN = 0xffff;    // segment of a node of a converged instance

__device__ __forceinline__ int bucket_seg(const LevelDev& g, const uint8_t* tier, uint64_t seed, uint64_t tag,
                                          uint64_t it, uint64_t lvl, uint64_t r, int K, const int32_t* active,
                                          int64_t v) {
  if (active && !active[node_inst(g, (int32_t)v)]) return BUCKET_FROZEN;  // converged instance: frozen
  return vertex_class(seed, tag, it, lvl, r, local_id(g, (int32_t)v), K) * NTIERS + tier[v];
}

// Step 1: segment of every node (seg, one byte) and counts[s * nchunks + chunk].
__global__ void __launch_bounds__(BUCKET_THREADS)
    k_bucket_count(LevelDev g, const uint8_t* tier, uint64_t seed, uint64_t tag, uint64_t it, uint64_t lvl, uint64_t r,
                   int K, const int32_t* active, const int32_t* r_dev, uint16_t* seg, int32_t* counts,
                   int64_t nchunks) {
  __shared__ int32_t cnt[BUCKET_MAX_SEGS];
  if (r_dev) r = (uint64_t)*r_dev;  // a graph replay reads its round here
  const int nseg = K * NTIERS;
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    for (int i = threadIdx.x; i < nseg; i += BUCKET_THREADS) cnt[i] = 0;
    __syncthreads();
    for (int k = 0; k < BUCKET_ITEMS; ++k) {
      const int64_t v = ch * BUCKET_CHUNK + (int64_t)k * BUCKET_THREADS + threadIdx.x;
      if (v >= g.N) break;
      const int sg = bucket_seg(g, tier, seed, tag, it, lvl, r, K, active, v);
      seg[v] = (uint16_t)sg;
      if (sg < nseg) atomicAdd(&cnt[sg], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nseg; i += BUCKET_THREADS) counts[(int64_t)i * nchunks + ch] = cnt[i];
    __syncthreads();
  }
}

// Step 2: one block per segment turns its counts into exclusive offsets over
// the chunks and stores the segment's size in cursors[s].
__global__ void __launch_bounds__(1024) k_bucket_scan(int32_t* counts, int64_t nchunks, int32_t* cursors) {
  __shared__ int32_t part[32];
  __shared__ int32_t carry;
  const int s = blockIdx.x;
  int32_t* c = counts + (int64_t)s * nchunks;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nchunks; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const int32_t x = i < nchunks ? c[i] : 0;
    int32_t incl = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += y;
    }
    if (lane == 31) part[w] = incl;
    __syncthreads();
    if (w == 0) {
      const int32_t p = lane < (int)(blockDim.x >> 5) ? part[lane] : 0;
      int32_t pi = p;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, pi, d);
        if (lane >= d) pi += y;
      }
      part[lane] = pi - p;
    }
    __syncthreads();
    if (i < nchunks) c[i] = carry + part[w] + incl - x;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += part[w] + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) cursors[s] = carry;
}

// Step 3: every chunk writes its nodes at its offsets.
__global__ void __launch_bounds__(BUCKET_THREADS)
    k_bucket_write(int32_t N, const uint16_t* seg, const int32_t* counts, int64_t nchunks, int K, int32_t* lists,
                   int64_t row_stride, TierOff tier_off) {
  __shared__ int32_t pos[BUCKET_MAX_SEGS];
  const int nseg = K * NTIERS;
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    for (int i = threadIdx.x; i < nseg; i += BUCKET_THREADS) pos[i] = counts[(int64_t)i * nchunks + ch];
    __syncthreads();
    for (int k = 0; k < BUCKET_ITEMS; ++k) {
      const int64_t v = ch * BUCKET_CHUNK + (int64_t)k * BUCKET_THREADS + threadIdx.x;
      if (v >= N) break;
      const int sg = seg[v];
      if (sg >= nseg) continue;
      const int q = sg / NTIERS, t = sg % NTIERS;
      lists[(int64_t)q * row_stride + tier_off.off[t] + atomicAdd(&pos[sg], 1)] = (int32_t)v;
    }
    __syncthreads();
  }
}

__global__ void k_hash_clear(HashView h) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  if (h.narrow) {
    Slot8* sl = slots8(h);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < h.cap; i += stride)
      sl[i] = Slot8{EMPTY_KEY8, 0};
  } else {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < h.cap; i += stride)
      h.slots[i] = Slot{EMPTY_KEY, 0};
  }
}

// Aggregated levels: one warp per node, the lanes sharing its list.
__global__ void k_sigma_insert_warp(LevelDev g, const int32_t* labels, SigStore h, int32_t* size) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = (((int64_t)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5); v < g.N; v += warps) {
    const int32_t c = labels[v];
    if (size && lane == 0) atomicAdd(&size[c], 1);
    int64_t b, e;
    slice_range(g, (int32_t)v, b, e);
    for (int64_t j = b + lane; j < e; j += 32) {
      int32_t s;
      long long k;
      slice_entry(g, (int32_t)v, j, s, k);
      ss_add(h, c, s, k);
    }
  }
}

__global__ void k_sigma_insert(LevelDev g, const int32_t* labels, SigStore h, int32_t* size) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.N; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = labels[v];
    if (size) atomicAdd(&size[c], 1);
    int64_t b, e;
    slice_range(g, (int32_t)v, b, e);
    for (int64_t j = b; j < e; ++j) {
      int32_t s;
      long long k;
      slice_entry(g, (int32_t)v, j, s, k);
      ss_add(h, c, s, k);
    }
  }
}

// sum_s Lambda_s k_{v,s} (X_s - self*k_{v,s}) with X_s = table(c, s).
// (od is applied by the caller.)
template <bool DENSE>
__device__ __forceinline__ u128 null_sum(const LevelDev& g, const u128* lam, const SigStore& h, int32_t v, int32_t c,
                                         bool self) {
  int64_t b, e;
  slice_range(g, v, b, e);
  u128 t = 0;
  for (int64_t j = b; j < e; ++j) {
    int32_t s;
    long long k;
    slice_entry(g, v, j, s, k);
    long long x = sst_get<DENSE>(h, c, s);
    if (self) x -= k;
    t += lam[s] * (u128)(ull)k * (u128)(ull)x;
  }
  return t;
}

template <bool DENSE>
struct LMPolicy {
  static constexpr int MIN_BLOCKS = DENSE ? MSLICE_DENSE_MIN_BLOCKS : MSLICE_GROUP_MIN_BLOCKS;
  LevelDev g;
  const int32_t* labels;
  const int32_t* size;
  SigStore sig;
  const u128* lam;
  int32_t* target;

  typedef Slot Probe;
  // Per node: own community and its size; at level 0 the node's snapshot s,
  // strength k and A = nd * Lambda_s * k (nd: od, or 1 for the global null
  // model), so a candidate costs one probe and
  // one 128x64-bit product.
  struct VCtx {
    int32_t a, size_a, s;
    bool single;
    long long k;
    Omega om;
    u128 A;
  };

  __device__ bool begin(int32_t) const { return true; }
  __device__ VCtx vctx(int32_t v) const {
    VCtx c;
    c.a = labels[v];
    c.size_a = size[c.a];
    c.single = g.is0 != 0;
    c.s = 0;
    c.k = 0;
    c.A = 0;
    c.om = node_omega(g, v);
    if (c.single) {
      c.k = g.k0[v];
      c.s = node_slice0(g, v);
      if (c.k > 0) c.A = (u128)(ull)null_scale(g, c.om) * lam[c.s] * (u128)(ull)c.k;
    }
    return c;
  }
  __device__ void skip(int32_t v) const { target[v] = NO_MOVE; }
  __device__ bool edge(int32_t, const VCtx& vc, int64_t e, int32_t& key, long long& w) const {
    int32_t u;
    if (!edge_at(g, e, u, w, vc.om)) return false;
    key = labels[u];
    return true;
  }
  __device__ int32_t own_key(int32_t v) const { return labels[v]; }
  __device__ i128 key_of(int32_t v, const VCtx& vc, int32_t c, long long W, bool self) const {
    const u128 ns = null_sum<DENSE>(g, lam, sig, v, c, self);
    return (((i128)W) << P_BITS) - (i128)((u128)(ull)null_scale(g, vc.om) * ns);
  }
  __device__ Probe probe(int32_t, const VCtx& vc, int32_t c) const {
    if (vc.single && vc.k > 0) return sst_first<DENSE>(sig, c, vc.s);
    return Slot{EMPTY_KEY, 0};
  }
  __device__ Cand cand(int32_t v, const VCtx& vc, int32_t c, long long W, const Probe& pr) const {
    if (vc.single) {
      const long long x = vc.k > 0 ? sst_resolve<DENSE>(sig, c, vc.s, pr) : 0;
      return Cand{(((i128)W) << P_BITS) - (i128)(vc.A * (u128)(ull)x), c};
    }
    return Cand{key_of(v, vc, c, W, false), c};
  }
  __device__ i128 own(int32_t v, const VCtx& vc, long long Wown) const {
    if (vc.single) {
      const long long x = vc.k > 0 ? sst_get<DENSE>(sig, vc.a, vc.s) - vc.k : 0;
      return (((i128)Wown) << P_BITS) - (i128)(vc.A * (u128)(ull)x);
    }
    return key_of(v, vc, vc.a, Wown, true);
  }
  // slice-parallel scoring (block tiers, aggregated levels)
  __device__ int64_t slice_count(int32_t v) const { return g.is0 ? 0 : g.sptr[v + 1] - g.sptr[v]; }
  __device__ bool own_walks_slices() const { return true; }
  __device__ u128 null_part(int32_t v, const VCtx&, int32_t c, bool self, int t, int nt) const {
    int64_t b, e;
    slice_range(g, v, b, e);
    u128 acc = 0;
    for (int64_t j = b + t; j < e; j += nt) {
      int32_t s;
      long long k;
      slice_entry(g, v, j, s, k);
      long long x = sst_get<DENSE>(sig, c, s);
      if (self) x -= k;
      acc += lam[s] * (u128)(ull)k * (u128)(ull)x;
    }
    return acc;
  }
  __device__ Cand cand_ns(int32_t, const VCtx& vc, int32_t c, long long W, const u128& ns) const {
    return Cand{(((i128)W) << P_BITS) - (i128)((u128)(ull)null_scale(g, vc.om) * ns), c};
  }
  __device__ i128 own_ns(int32_t, const VCtx& vc, long long Wown, const u128& ns) const {
    return (((i128)Wown) << P_BITS) - (i128)((u128)(ull)null_scale(g, vc.om) * ns);
  }
  __device__ void finish(int32_t v, const Cand& best, long long, const i128& Ga, const VCtx& vc) const {
    const int32_t a = vc.a;
    const bool has = best.label != INT32_MAX;
    const i128 Gmax = (has && best.G > Ga) ? best.G : Ga;
    int32_t t = NO_MOVE;
    if (vc.size_a > 1 && Gmax < 0) {
      t = TO_EMPTY;
    } else if (has && best.G > Ga) {
      if (!(vc.size_a == 1 && best.label > a && size[best.label] == 1)) t = best.label;
    }
    target[v] = t;
  }
};

typedef TierSegs Segs;

__device__ __forceinline__ bool seg_item(const Segs& sg, int64_t idx, int32_t& v) {
#pragma unroll
  for (int t = 0; t < NTIERS; ++t) {
    const int cnt = *sg.count[t];
    if (idx < cnt) {
      v = sg.list[t][idx];
      return true;
    }
    idx -= cnt;
  }
  return false;
}

__device__ __forceinline__ int seg_total(const Segs& sg) {
  int t = 0;
#pragma unroll
  for (int i = 0; i < NTIERS; ++i) t += *sg.count[i];
  return t;
}

// Applies the sub-round's decisions: labels, community sizes and Sigma, and
// resets each applied decision.  Moves to an empty community only leave here
// (their label is assigned by k_empty_pass).
// End of a round of the device-side loop: accounts the round (acc: rounds
// run, moves, moves of this round), advances the round index and lets the
// loop go on while nodes moved, rounds remain, no hash region has passed half
// its slots (the host then rebuilds the table) and no error was raised.
__global__ void k_round_control(cudaGraphConditionalHandle h, int32_t* r_dev, int32_t r_end, const int32_t* counters,
                                const ull* sig_used, const unsigned* status, long long* acc) {
  const long long moved = (long long)(((unsigned long long)(uint32_t)counters[1] << 32) | (uint32_t)counters[0]);
  acc[0] += 1;
  acc[1] += moved;
  acc[2] = moved;
  const int32_t r = *r_dev + 1;
  *r_dev = r;
  const bool go = moved > 0 && r < r_end && (sig_used == nullptr || *sig_used == 0) && *status == 0;
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

// lm_active[i] stays 1 only for instances that moved in the round; clears
// the flags for the next round.
__global__ void k_round_freeze(int32_t* lm_active, int32_t* inst_moved, int32_t B) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < B) {
    if (!inst_moved[i]) lm_active[i] = 0;
    inst_moved[i] = 0;
  }
}

// A mover's (snapshot, strength) list moves between the two communities'
// rows; a long list (more than 32 entries, late levels of long sequences) is
// walked by the whole warp, a short one by its own thread.  The warp stays
// converged: every lane runs every iteration of the grid-stride loop.
__device__ __forceinline__ void move_slices(const LevelDev& g, SigStore& sig, int32_t v, int32_t a, int32_t t,
                                            int64_t b, int64_t e, int64_t from, int64_t step) {
  for (int64_t j = b + from; j < e; j += step) {
    int32_t s;
    long long k;
    slice_entry(g, v, j, s, k);
    ss_add(sig, a, s, -k);
    if (t >= 0) ss_add(sig, t, s, k);
  }
}

__global__ void k_lm_apply(LevelDev g, Segs sg, int32_t* labels, int32_t* size, SigStore sig, int32_t* target,
                           int32_t* counters, int32_t* inst_moved) {
  const int total = seg_total(sg);
  const int lane = threadIdx.x & 31;
  int local = 0, local_empty = 0;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < total;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t idx = base + lane;
    int32_t v = 0, t = NO_MOVE, a = 0;
    int64_t b = 0, e = 0;
    if (idx < total && seg_item(sg, idx, v)) t = target[v];
#if MSLICE_CHECKED
    if (t != NO_MOVE && (t >= g.N || (t < 0 && t != TO_EMPTY))) {
      atomicOr(g.chk, ERR_BOUNDS);
      t = NO_MOVE;
    }
#endif
    if (t != NO_MOVE) {
      if (inst_moved) inst_moved[node_inst(g, v)] = 1;
      a = labels[v];
      atomicSub(&size[a], 1);
      slice_range(g, v, b, e);
      if (e - b <= 32) move_slices(g, sig, v, a, t, b, e, 0, 1);
    }
    unsigned wide = __ballot_sync(0xffffffffu, t != NO_MOVE && e - b > 32);
    while (wide) {
      const int src = __ffs(wide) - 1;
      wide &= wide - 1;
      const int32_t vs = __shfl_sync(0xffffffffu, v, src), as = __shfl_sync(0xffffffffu, a, src),
                    ts = __shfl_sync(0xffffffffu, t, src);
      const int64_t bs = __shfl_sync(0xffffffffu, b, src), es = __shfl_sync(0xffffffffu, e, src);
      move_slices(g, sig, vs, as, ts, bs, es, lane, 32);
    }
    if (t >= 0) {
      atomicAdd(&size[t], 1);
      labels[v] = t;
      target[v] = NO_MOVE;
      local++;
    } else if (t == TO_EMPTY) {
      local_empty++;
    }
  }
  local = warp_sum(local);
  local_empty = warp_sum(local_empty);
  if ((threadIdx.x & 31) == 0) {
    if (local) atomicAdd((ull*)counters, (ull)local);
    if (local_empty) atomicAdd(&counters[2], local_empty);
  }
}

template <class T>
__device__ __forceinline__ T block_scan_excl(T x, T* sm, T& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T incl = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) sm[w] = incl;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    const T a = lane < nw ? sm[lane] : T(0);
    T ai = a;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const T y = __shfl_up_sync(0xffffffffu, ai, d);
      if (lane >= d) ai += y;
    }
    if (lane < nw) sm[lane] = ai - a;
    if (lane == nw - 1) sm[32] = ai;
  }
  __syncthreads();
  const T r = incl - x + sm[w];
  total = sm[32];
  __syncthreads();
  return r;
}

// Moves to an empty community (one cooperative launch; returns at once when
// the sub-round has none).  Within each instance, in ascending node order,
// the movers take the ascending labels of that instance that are free once
// every other move is applied and the movers have left.
//   blk:      2*gridDim.x ints (per-chunk counts)
//   freelist: all free labels in ascending order; mrank: movers' global ranks
//   icnt:     4*B + 2 ints (per-instance counts, then their prefixes); zero
//             on entry and left zero on exit
__global__ void __launch_bounds__(EMPTY_THREADS) k_empty_pass(LevelDev g, int32_t B, int32_t* target, int32_t* labels,
                                                              int32_t* size, SigStore sig, int32_t* counters,
                                                              int32_t* blk, int32_t* freelist, int32_t* mrank,
                                                              int32_t* icnt) {
  const int n_empty = counters[2];
  if (n_empty == 0) return;
  __shared__ int32_t sm[33];
  cg::grid_group grid = cg::this_grid();
  const int64_t N = g.N, nb = gridDim.x;
  const int64_t chunk = (N + nb - 1) / nb;
  const int64_t lo = min(N, (int64_t)blockIdx.x * chunk), hi = min(N, lo + chunk);
  int32_t* fcnt = icnt;           // free labels per instance
  int32_t* mcnt = icnt + B;       // movers per instance
  int32_t* fbase = icnt + 2 * B;  // exclusive prefixes (B + 1 each)
  int32_t* mbase = icnt + 3 * B + 1;
  int cf = 0, ce = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const bool f = size[i] == 0, m = target[i] == TO_EMPTY;
    cf += f;
    ce += m;
    if (B > 1) {
      if (f) atomicAdd(&fcnt[node_inst(g, (int32_t)i)], 1);
      if (m) atomicAdd(&mcnt[node_inst(g, (int32_t)i)], 1);
    }
  }
  int tf, te;
  block_scan_excl(cf, sm, tf);
  block_scan_excl(ce, sm, te);
  if (threadIdx.x == 0) {
    blk[blockIdx.x] = tf;
    blk[nb + blockIdx.x] = te;
  }
  grid.sync();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int32_t a = 0, b = 0;
    for (int32_t i = 0; i < B; ++i) {
      fbase[i] = a;
      mbase[i] = b;
      if (B > 1) {
        a += fcnt[i];
        b += mcnt[i];
      }
    }
    fbase[B] = a;
    mbase[B] = b;
  }
  int pf = 0, pe = 0;
  for (int b = threadIdx.x; b < blockIdx.x; b += blockDim.x) {
    pf += blk[b];
    pe += blk[nb + b];
  }
  int tot_pf, tot_pe;
  block_scan_excl(pf, sm, tot_pf);
  block_scan_excl(pe, sm, tot_pe);
  pf = tot_pf;
  pe = tot_pe;
  for (int64_t base = lo; base < hi; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const int f = (i < hi && size[i] == 0) ? 1 : 0;
    const int m = (i < hi && target[i] == TO_EMPTY) ? 1 : 0;
    int totf, totm;
    const int rf = block_scan_excl(f, sm, totf);
    const int rm = block_scan_excl(m, sm, totm);
    if (f) freelist[pf + rf] = (int32_t)i;
    if (m) mrank[i] = pe + rm;
    pf += totf;
    pe += totm;
  }
  grid.sync();
  for (int64_t v = lo + threadIdx.x; v < hi; v += blockDim.x) {
    if (target[v] != TO_EMPTY) continue;
    const int32_t inst = B > 1 ? node_inst(g, (int32_t)v) : 0;
    const int32_t L = freelist[fbase[inst] + (mrank[v] - mbase[inst])];
    labels[v] = L;
    size[L] = 1;
    int64_t b, en;
    slice_range(g, (int32_t)v, b, en);
    for (int64_t j = b; j < en; ++j) {
      int32_t s;
      long long k;
      slice_entry(g, (int32_t)v, j, s, k);
      ss_add(sig, L, s, k);
    }
    target[v] = NO_MOVE;
  }
  grid.sync();
  if (blockIdx.x == 0) {
    for (int32_t i = threadIdx.x; i < 4 * B + 2; i += blockDim.x) icnt[i] = 0;
    if (threadIdx.x == 0) {
      atomicAdd((ull*)counters, (ull)n_empty);
      counters[2] = 0;
    }
  }
}

}  // namespace

LevelDev level0_view(const SupraGraph& G, long long on, long long od) {
  LevelDev d;
  d.N = (int32_t)G.N;
  d.n = (int32_t)(G.n > 0 ? G.n : 1);
  d.is0 = 1;
  d.rowptr = G.rowptr;
  d.adj0 = G.adj;
  d.k0 = G.k;
  d.on = on;
  d.od = od;
  return d;
}

LevelDev level0_view(const SupraGraph& G, const Solver& S) {
  LevelDev d = level0_view(G, S.p.on, S.p.od);
  if (G.B > 1) {
    d.slice0 = G.slice0;
    d.inst = G.inst0;
    d.inst_off = G.inst_off0;
    d.on_i = S.on_d;
    d.od_i = S.od_d;
  }
  if (S.cw_d) {
    d.cw = S.cw_d;
    d.ncw = G.ncw;
  }
  if (S.p.cpm) d.k0 = S.kn;  // CPM: every node weighs 1, snapshots as null slices
  if (S.p.global_null) {
    // one null slice per instance: the instance id (batches) or 0 (v / N)
    d.global_null = 1;
    d.k0 = S.kn;
    if (G.B > 1)
      d.slice0 = G.inst0;
    else
      d.n = (int32_t)(G.N > 0 ? G.N : 1);
  }
  return d;
}

void solver_alloc(Solver& S) {
  Ctx& c = *S.c;
  const int64_t N = S.N0 > 0 ? S.N0 : 1;
  S.target = c.ws->get<int32_t>("s_target", N);
  S.size = c.ws->get<int32_t>("s_size", N);
  S.tmp32a = c.ws->get<int32_t>("s_tmpa", N + 1);
  S.tmp32b = c.ws->get<int32_t>("s_tmpb", N + 1);
  S.freelist = c.ws->get<int32_t>("s_free", N + 1);
  S.tier = c.ws->get<uint8_t>("s_tier", N);
  S.cls = c.ws->get<uint8_t>("s_cls", N);
  S.bseg = c.ws->get<uint16_t>("s_bseg", N);
  S.bcounts = c.ws->get<int32_t>("s_bcounts", (size_t)S.p.K * NTIERS * ((N + BUCKET_CHUNK - 1) / BUCKET_CHUNK));
  S.lists = c.ws->get<int32_t>("s_lists", (size_t)N * S.p.K);
  S.cursors = c.ws->get<int32_t>("s_cursors", NTIERS * S.p.K + NTIERS);
  S.counters = c.ws->get<int32_t>("s_counters", 8);
  S.sig_used = c.ws->get<ull>("s_sig_used", 1);
  S.goff = c.ws->get<int64_t>("s_goff", N + 1);
  S.R = c.ws->get<int32_t>("s_R", N);
  S.sizeR = c.ws->get<int32_t>("s_sizeR", N);
  S.Wc = c.ws->get<long long>("s_Wc", N);
  S.Wout = c.ws->get<long long>("s_Wout", N);
  S.Wsel = c.ws->get<long long>("s_Wsel", N);
  S.rhs = c.ws->get<ull>("s_rhs", 2 * N);
  S.elig = c.ws->get<uint8_t>("s_elig", N);
  S.wc = c.ws->get<uint8_t>("s_wc", N);
  int max_blocks = 0;
  check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&max_blocks, k_empty_pass, EMPTY_THREADS, 0), "occupancy");
  int dev = 0, sms = 0;
  check_cuda(cudaGetDevice(&dev), "device");
  check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "attribute");
  S.empty_grid = std::max(1, std::min(max_blocks, 2) * sms);
  S.empty_blk = c.ws->get<int32_t>("s_empty_blk", 2 * S.empty_grid);
  S.round_dev = c.ws->get<int32_t>("s_round", 1);
  S.loop_acc = c.ws->get<long long>("s_loop_acc", 3);
  S.wqueue = c.ws->get<int32_t>("s_wqueue", NTIERS);
  S.lm_active = c.ws->get<int32_t>("s_lm_active", S.B);
  S.inst_moved = c.ws->get<int32_t>("s_inst_moved", S.B);
  check_cuda(cudaMemsetAsync(S.inst_moved, 0, S.B * sizeof(int32_t), c.stream), "memset");
  S.inst_cnt = c.ws->get<int32_t>("s_inst_cnt", 4 * (size_t)S.B + 2);
  check_cuda(cudaMemsetAsync(S.inst_cnt, 0, (4 * (size_t)S.B + 2) * sizeof(int32_t), c.stream), "memset");
  fill_i32(c, S.target, NO_MOVE, N);
  check_cuda(cudaMemsetAsync(S.counters, 0, 8 * sizeof(int32_t), c.stream), "memset");
}

void prepare_level(Solver& S, const Level& L) {
  Ctx& c = *S.c;
  const int32_t N = L.d.N;
  configure_stores(S, N);
  int32_t* cnt = S.cursors;  // reused: tier counts
  check_cuda(cudaMemsetAsync(cnt, 0, NTIERS * sizeof(int32_t), c.stream), "memset");
  int64_t* gsize = reinterpret_cast<int64_t*>(c.ws->get<int64_t>("s_gsize", (size_t)(N > 0 ? N : 1)));
  if (N > 0)
    launch(c, k_tier, dim3(grid_for(N, 256) < 4096 ? grid_for(N, 256) : 4096), dim3(256), 0, L.d.rowptr,
           (const int64_t*)(L.d.is0 ? nullptr : L.d.sptr), N, S.p.cuts, S.tier, cnt, gsize);
  int64_t* gtotal = c.ws->get<int64_t>("s_gtotal", 1);
  scan_excl(c, gsize, S.goff, N, gtotal);
  check_cuda(cudaMemcpyAsync(S.goff + N, gtotal, sizeof(int64_t), cudaMemcpyDeviceToDevice, c.stream), "copy");
  struct {
    int32_t cnt[NTIERS];
    int32_t pad;
    int64_t gt;
  } hb;
  check_cuda(cudaMemcpyAsync(&hb.cnt, cnt, NTIERS * sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream), "copy");
  check_cuda(cudaMemcpyAsync(&hb.gt, gtotal, sizeof(int64_t), cudaMemcpyDeviceToHost, c.stream), "copy");
  sync(c);
  int32_t off = 0;
  for (int t = 0; t < NTIERS; ++t) {
    S.tier_cnt[t] = hb.cnt[t];
    S.tier_off[t] = off;
    off += hb.cnt[t];
  }
  if (hb.gt > S.gcap) {
    S.gcap = hb.gt;
    S.gkeys = c.ws->get<int32_t>("s_gkeys", S.gcap);
    S.gvals = c.ws->get<long long>("s_gvals", S.gcap);
    if (S.p.theta_num > 0) S.gwts = c.ws->get<ull>("s_gwts", S.gcap);
  }
}

// Level-0 nodes of every null slice: the snapshot's n (Q_MS and CPM, whose
// null slices are the snapshots) or the instance's n*T (the global model,
// one null slice per instance).
static std::vector<int64_t> null_slice_nodes(const Solver& S) {
  const SupraGraph& G = *S.G0;
  std::vector<int64_t> out(S.Tn > 0 ? S.Tn : 1, 0);
  for (int32_t i = 0; i < G.B; ++i) {
    const InstInfo& in = G.inst[i];
    if (S.p.global_null) {
      if (i < (int32_t)out.size()) out[i] = in.n * in.T;
    } else {
      for (int32_t s = in.soff; s < in.soff + in.T && s < (int32_t)out.size(); ++s) out[s] = in.n;
    }
  }
  return out;
}

// Largest mass of a null slice, the bound on every sum its table keys hold:
// 2m_s (Q_MS), the node count n (CPM, whose strengths are 1) or the
// instance's 2M' in units of 1/omega_den (the global model).
static int64_t null_slice_mass_max(const Solver& S) {
  const SupraGraph& G = *S.G0;
  int64_t mx = 0;
  for (int32_t i = 0; i < G.B; ++i) {
    const InstInfo& in = G.inst[i];
    if (S.p.cpm) {
      mx = std::max<int64_t>(mx, in.n);
    } else if (S.p.global_null) {
      u128 sum2m = 0;
      for (int32_t s = in.soff; s < in.soff + in.T; ++s) sum2m += (u128)(ull)G.two_m_host[s];
      const u128 m = (u128)(ull)S.od_h[i] * sum2m + (u128)(ull)S.csum_h[i];
      mx = m >= ((u128)1 << 62) ? INT64_MAX : std::max<int64_t>(mx, (int64_t)m);
      if (mx == INT64_MAX) break;
    } else {
      for (int32_t s = in.soff; s < in.soff + in.T; ++s) mx = std::max<int64_t>(mx, G.two_m_host[s]);
    }
  }
  return mx;
}

void configure_stores(Solver& S, int64_t N) {
  Ctx& c = *S.c;
  const int64_t T = S.Tn;
  S.sig = SigStore{};
  S.kr = SigStore{};
  S.sig.T = S.kr.T = (int32_t)T;
  const int64_t need = (N > 0 ? N : 1) * T;
  int64_t limit = DENSE_LIMIT;
  if (const char* e = std::getenv("MSLICE_DENSE_LIMIT")) limit = std::atoll(e);
  if (need <= limit) {
    if (need > S.dense_cap) {
      S.sig_d = c.ws->get<long long>("s_sig_d", need);
      S.kr_d = c.ws->get<long long>("s_kr_d", need);
      S.dense_cap = need;
    }
    S.sig.d = S.sig_d;
    S.kr.d = S.kr_d;
    S.sig.rows = S.kr.rows = (N > 0 ? N : 1);
    return;
  }
  if (S.region_T != T) {
    // hash tables keyed by (label, null slice), one region per null slice
    // sized for its level-0 nodes: at most one live key per (node, slice)
    // entry of that slice plus the keys one round of moves creates; a
    // rebuild is triggered once a region has taken half of its slots
    const std::vector<int64_t> ns = null_slice_nodes(S);
    S.region_h.assign(ns.size() + 1, 0);
    for (size_t s = 0; s < ns.size(); ++s)
      S.region_h[s + 1] = S.region_h[s] + (uint64_t)(2 * ns[s] + 2 * ((ns[s] + S.p.K - 1) / S.p.K) + 64);
    const uint64_t cap = S.region_h.back();
    uint64_t* region = c.ws->get<uint64_t>("s_region", S.region_h.size());
    check_cuda(cudaMemcpyAsync(region, S.region_h.data(), S.region_h.size() * sizeof(uint64_t),
                               cudaMemcpyHostToDevice, c.stream), "copy");
    ull* rused = S.sig_used ? c.ws->get<ull>("s_region_used", ns.size()) : nullptr;
    if (rused) check_cuda(cudaMemsetAsync(rused, 0, ns.size() * sizeof(ull), c.stream), "memset");
    S.sig_h = HashView{c.ws->get<Slot>("s_sig", cap), cap, c.d_status, S.sig_used, region, rused};
    S.kr_h = HashView{c.ws->get<Slot>("s_kr", cap), cap, c.d_status, nullptr, region, nullptr};
    S.region_T = T;
  }
  // 8-byte slots when no null slice's mass reaches 2^32 (no sum can)
  bool narrow = null_slice_mass_max(S) < ((int64_t)1 << 32);
  if (const char* e = std::getenv("MSLICE_WIDE_SLOTS")) narrow = narrow && std::atoi(e) == 0;
  S.sig_h.narrow = S.kr_h.narrow = narrow ? 1 : 0;
  S.sig_h.nregions = S.kr_h.nregions = (int32_t)(S.region_h.size() - 1);
  S.sig.h = S.sig_h;
  S.kr.h = S.kr_h;
}

// Empties a store (dense rows zeroed, hash slots freed).
void clear_store(Solver& S, const SigStore& st) {
  Ctx& c = *S.c;
  if (st.d)
    check_cuda(cudaMemsetAsync(st.d, 0, (size_t)st.rows * st.T * sizeof(long long), c.stream), "memset");
  else
    launch(c, k_hash_clear, dim3(fixed_grid(8)), dim3(256), 0, st.h);
}

// Sigma (and, optionally, the community sizes) from the labels.
static void rebuild_sigma(Solver& S, const Level& L, const int32_t* labels, bool sizes) {
  Ctx& c = *S.c;
  const int32_t N = L.d.N;
  if (sizes) check_cuda(cudaMemsetAsync(S.size, 0, (N > 0 ? N : 1) * sizeof(int32_t), c.stream), "memset");
  if (S.sig_used) check_cuda(cudaMemsetAsync(S.sig_used, 0, sizeof(ull), c.stream), "memset");
  if (!S.sig.d && S.sig.h.region_used)
    check_cuda(cudaMemsetAsync(S.sig.h.region_used, 0, (S.region_h.size() - 1) * sizeof(ull), c.stream), "memset");
  clear_store(S, S.sig);
  if (N > 0)
    if (L.d.is0)
      launch(c, k_sigma_insert, dim3(grid_for(N, 256)), dim3(256), 0, L.d, labels, S.sig, sizes ? S.size : nullptr);
    else
      launch(c, k_sigma_insert_warp, dim3(fixed_grid(8)), dim3(256), 0, L.d, labels, S.sig, sizes ? S.size : nullptr);
}

void sigma_rebuild(Solver& S, const Level& L, const int32_t* labels) { rebuild_sigma(S, L, labels, false); }

TierSegs bucket_segments(Solver& S, int q) {
  TierSegs sg;
  for (int t = 0; t < NTIERS; ++t) {
    sg.list[t] = S.lists + (int64_t)q * S.N0 + S.tier_off[t];
    sg.count[t] = S.cursors + NTIERS * q + t;
  }
  sg.queue = S.wqueue;
  return sg;
}

void bucket(Solver& S, const Level& L, uint64_t tag, int it, int lvl, int r, const int32_t* active,
            const int32_t* r_dev) {
  Ctx& c = *S.c;
  TierOff to;
  for (int t = 0; t < NTIERS; ++t) to.off[t] = S.tier_off[t];
  const int64_t N = L.d.N;
  if (N == 0) {
    check_cuda(cudaMemsetAsync(S.cursors, 0, NTIERS * S.p.K * sizeof(int32_t), c.stream), "memset");
    return;
  }
  const int64_t nchunks = (N + BUCKET_CHUNK - 1) / BUCKET_CHUNK;
  const unsigned grid = (unsigned)std::min<int64_t>(nchunks, fixed_grid(16));
  launch(c, k_bucket_count, dim3(grid), dim3(BUCKET_THREADS), 0, L.d, (const uint8_t*)S.tier, S.p.seed, tag,
         (uint64_t)it, (uint64_t)lvl, (uint64_t)r, S.p.K, active, r_dev, S.bseg, S.bcounts, nchunks);
  launch(c, k_bucket_scan, dim3(S.p.K * NTIERS), dim3(1024), 0, S.bcounts, nchunks, S.cursors);
  launch(c, k_bucket_write, dim3(grid), dim3(BUCKET_THREADS), 0, L.d.N, (const uint16_t*)S.bseg,
         (const int32_t*)S.bcounts, nchunks, S.p.K, S.lists, (int64_t)S.N0, to);
}

// Chooses the degree cuts of the decision tiers for this solve: every
// candidate decides the K sub-rounds of round r twice (decisions only,
// nothing is applied, so the state is untouched) and the candidate with the
// fastest pass is kept.  Decisions do not depend on the tier that makes
// them, so neither does the result.
template <class Decide>
static void autotune_cuts(Solver& S, const Level& L, int it, int r, const int32_t* active, Decide&& decide) {
  Ctx& c = *S.c;
  // (cut 2 in units of the tier-2 capacity: T2 = TIER_MAX[2])
  constexpr int T2 = TIER_MAX[2];
  static const TierCuts kCand[] = {{{16, 32, T2, 1024}}, {{12, 32, T2, 1024}}, {{16, 24, T2, 1024}},
                                   {{16, 32, T2, 512}},  {{12, 24, T2, 512}},  {{16, 32, T2 * 3 / 4, 1024}}};
  cudaEvent_t e0, e1;
  check_cuda(cudaEventCreate(&e0), "event");
  check_cuda(cudaEventCreate(&e1), "event");
  float best = 0;
  TierCuts chosen = kCand[0];
  // the first pass warms the caches and is not counted
  for (int k = -1; k < (int)(sizeof(kCand) / sizeof(kCand[0])); ++k) {
    S.p.cuts = kCand[k < 0 ? 0 : k];
    prepare_level(S, L);
    bucket(S, L, 0, it, 0, r, active, nullptr);
    float ms = 0;
    for (int rep = 0; rep < 2; ++rep) {
      check_cuda(cudaEventRecord(e0, c.stream), "event");
      for (int q = 0; q < S.p.K; ++q) decide(bucket_segments(S, q));
      check_cuda(cudaEventRecord(e1, c.stream), "event");
      check_cuda(cudaEventSynchronize(e1), "event");
      float x = 0;
      check_cuda(cudaEventElapsedTime(&x, e0, e1), "event time");
      ms = rep == 0 ? x : std::min(ms, x);
    }
    if (k >= 0 && (k == 0 || ms < best)) {
      best = ms;
      chosen = kCand[k];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  S.p.cuts = chosen;
  S.p.autotune = false;
  prepare_level(S, L);
  fill_i32(c, S.target, NO_MOVE, L.d.N);
}

// Builds a graph holding one conditional WHILE node and captures body(h) on
// the context's stream into its body graph (h: the loop's condition, set by
// the body's last kernel).  Returns the executable graph, or nullptr (and
// leaves the stream usable) when the loop cannot be built.  kernels: the
// kernels one pass of the body runs.
template <class Body>
static cudaGraphExec_t capture_loop(Ctx& c, Body&& body, int64_t& kernels) {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  kernels = 0;
  if (cudaGraphCreate(&graph, 0) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  cudaGraphConditionalHandle h{};
  bool ok = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault) == cudaSuccess;
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  ok = ok && cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np) == cudaSuccess;
  ok = ok && cudaStreamBeginCaptureToGraph(c.stream, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    const int64_t before = c.launches, before_host = c.host_launches;
    c.capturing = true;
    try {
      body(h);
    } catch (const Error&) {
      ok = false;
    }
    c.capturing = false;
    cudaGraph_t captured = nullptr;
    if (cudaStreamEndCapture(c.stream, &captured) != cudaSuccess) ok = false;
    kernels = c.launches - before;
    c.launches = before;
    c.host_launches = before_host;
  }
  if (ok && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) exec = nullptr;
  if (!ok) exec = nullptr;
  cudaGraphDestroy(graph);
  cudaGetLastError();
  return exec;
}

MoveOut local_move(Solver& S, const Level& L, int32_t* labels, int it, int lvl, int max_rounds) {
  Ctx& c = *S.c;
  MoveOut out;
  const int32_t N = L.d.N;
  if (N == 0) {
    // an empty level runs one round that moves nothing
    if (max_rounds > 0) {
      out.rounds = 1;
      S.lm_rounds++;
    }
    return out;
  }
  // community sizes and Sigma of the level's initial labels (refinement
  // reads Sigma even when no round runs)
  rebuild_sigma(S, L, labels, true);
  if (max_rounds <= 0) return out;
  LMPolicy<true> pol;
  pol.g = L.d;
  pol.labels = labels;
  pol.size = S.size;
  pol.sig = S.sig;
  pol.lam = S.lam;
  pol.target = S.target;
  LMPolicy<false> polh;
  polh.g = pol.g;
  polh.labels = pol.labels;
  polh.size = pol.size;
  polh.sig = pol.sig;
  polh.lam = pol.lam;
  polh.target = pol.target;
  auto decide = [&](const TierSegs& sg) {
    if (S.sig.d)
      decide_all(c, pol, sg, S.tier_cnt, S.gkeys, S.gvals, S.goff);
    else
      decide_all(c, polh, sg, S.tier_cnt, S.gkeys, S.gvals, S.goff);
  };
  // Batch: an instance whose round moved nothing is at a fixed point of
  // this level (its decisions read only its own state, which no longer
  // changes), so it is left out of the remaining rounds.
  const bool batch = S.B > 1;
  if (batch)
    check_cuda(cudaMemcpyAsync(S.lm_active, S.inst_active, S.B * sizeof(int32_t), cudaMemcpyDeviceToDevice, c.stream),
               "copy");
  const int32_t* active = batch ? S.lm_active : S.inst_active;
  // One round: buckets, K sub-rounds of decisions, applies and moves to
  // empty communities, then its end:
  //   HOST  the moved count, the table fill and the status word copied to
  //         the pinned buffer (the host decides whether another round runs);
  //   LOOP  k_round_control decides on the device and sets the condition of
  //         the enclosing graph loop (r_dev holds the round).
  enum class RoundEnd { HOST, LOOP };
  auto round_body = [&](int r, const int32_t* r_dev, bool prof, RoundEnd end, cudaGraphConditionalHandle h) {
    check_cuda(cudaMemsetAsync(S.counters, 0, 3 * sizeof(int32_t), c.stream), "memset");
    bucket(S, L, 0, it, lvl, r, active, r_dev);
    for (int q = 0; q < S.p.K; ++q) {
      const Segs sg = bucket_segments(S, q);
      if (prof) {
        cudaEvent_t e0, e1;
        check_cuda(cudaEventCreate(&e0), "event");
        check_cuda(cudaEventCreate(&e1), "event");
        check_cuda(cudaEventRecord(e0, c.stream), "event");
        decide(sg);
        check_cuda(cudaEventRecord(e1, c.stream), "event");
        c.prof_spans->push_back({e0, e1});
      } else {
        decide(sg);
      }
      launch(c, k_lm_apply, dim3(fixed_grid(4)), dim3(APPLY_THREADS), 0, L.d, sg, labels, S.size, S.sig, S.target,
             S.counters, batch ? S.inst_moved : nullptr);
      launch_coop(c, k_empty_pass, dim3(S.empty_grid), dim3(EMPTY_THREADS), 0, L.d, S.B, S.target, labels, S.size,
                  S.sig, S.counters, S.empty_blk, S.freelist, S.tmp32b, S.inst_cnt);
    }
    if (batch)
      launch(c, k_round_freeze, dim3(grid_for(S.B, 256)), dim3(256), 0, S.lm_active, S.inst_moved, S.B);
    if (end == RoundEnd::LOOP) {
      launch(c, k_round_control, dim3(1), dim3(1), 0, h, S.round_dev, (int32_t)max_rounds,
             (const int32_t*)S.counters, (const ull*)(S.sig.d ? nullptr : S.sig_used), (const unsigned*)c.d_status,
             S.loop_acc);
      return;
    }
    check_cuda(cudaMemcpyAsync(c.pinned, S.counters, sizeof(int64_t), cudaMemcpyDeviceToHost, c.stream), "copy");
    check_cuda(cudaMemcpyAsync(static_cast<char*>(c.pinned) + 8, S.sig_used, sizeof(ull), cudaMemcpyDeviceToHost,
                               c.stream), "copy");
    check_cuda(cudaMemcpyAsync(static_cast<char*>(c.pinned) + 16, c.d_status, sizeof(unsigned),
                               cudaMemcpyDeviceToHost, c.stream), "copy");
  };
  // A level still moving after GRAPH_FROM_ROUND rounds runs its remaining
  // rounds as one graph launch: a device-side loop (a conditional WHILE node)
  // around one captured round, whose last kernel decides whether another
  // round runs, so the host syncs once per level (or per table rebuild)
  // instead of once per round.  Capture and instantiation cost more than
  // they save on levels that settle sooner.  Not while profiling or tracing,
  // nor on a level whose tier cuts are still being tuned.  Batches use it;
  // single solves on request (MSLICE_GRAPHS=1; MSLICE_NO_GRAPHS=1 turns it
  // off everywhere), see the design notes for the measurements.
  int64_t graph_max_nodes = GRAPH_MAX_NODES;
  if (const char* e = std::getenv("MSLICE_GRAPH_MAX_NODES")) graph_max_nodes = std::atoll(e);
  const bool want =
      (batch || N <= graph_max_nodes || std::getenv("MSLICE_GRAPHS")) && !std::getenv("MSLICE_NO_GRAPHS");
  const bool graphs = want && c.stream != nullptr && !c.profile && !c.trace && !(S.p.autotune && lvl == 0);
  cudaGraphExec_t exec = nullptr;
  int64_t loop_kernels = 0;
  bool graph_failed = false;
  bool rebuild = false;
  int r = 0;
  while (r < max_rounds) {
    if (rebuild) rebuild_sigma(S, L, labels, false);
    // tuning waits for round 2, when the partition looks like the later rounds'
    if (S.p.autotune && lvl == 0 && r == 2) autotune_cuts(S, L, it, r, active, decide);
    if (graphs && r >= GRAPH_FROM_ROUND && !graph_failed) {
      if (!exec) {
        exec = capture_loop(c, [&](cudaGraphConditionalHandle h) { round_body(0, S.round_dev, false, RoundEnd::LOOP, h); },
                            loop_kernels);
        if (!exec) graph_failed = true;
      }
      if (exec) {
        struct LoopIn {
          int32_t r;
          int32_t pad;
          long long acc[3];
        };
        LoopIn* in = static_cast<LoopIn*>(c.pinned);
        in->r = r;
        in->acc[0] = in->acc[1] = in->acc[2] = 0;
        check_cuda(cudaMemcpyAsync(S.round_dev, &in->r, sizeof(int32_t), cudaMemcpyHostToDevice, c.stream), "copy");
        check_cuda(cudaMemcpyAsync(S.loop_acc, in->acc, 3 * sizeof(long long), cudaMemcpyHostToDevice, c.stream),
                   "copy");
        {
          CoopOrder order(c.stream);
          check_cuda(cudaGraphLaunch(exec, c.stream), "graph launch");
        }
        c.host_launches++;
        struct {
          long long acc[3];  // rounds run, moves, moves of the last round
          ull used;
          unsigned status;
        } lb;
        check_cuda(cudaMemcpyAsync(c.pinned, S.loop_acc, 3 * sizeof(long long), cudaMemcpyDeviceToHost, c.stream),
                   "copy");
        check_cuda(cudaMemcpyAsync(static_cast<char*>(c.pinned) + 24, S.sig_used, sizeof(ull),
                                   cudaMemcpyDeviceToHost, c.stream), "copy");
        check_cuda(cudaMemcpyAsync(static_cast<char*>(c.pinned) + 32, c.d_status, sizeof(unsigned),
                                   cudaMemcpyDeviceToHost, c.stream), "copy");
        sync(c);
        std::memcpy(&lb, c.pinned, sizeof(lb));
        const int64_t ran = lb.acc[0];
        c.launches += ran * loop_kernels;
        S.lm_rounds += ran;
        S.lm_edges += ran * L.nnz_eff;
        out.rounds += ran;
        out.moves += lb.acc[1];
        r += (int)ran;
        if (lb.status) {
          cudaGraphExecDestroy(exec);
          exec = nullptr;
          check_status(c, "local moving");
        }
        if (ran < 1) fail(MSLICE_ECUDA, "device round loop ran no round");
        if (lb.acc[2] == 0) break;
        if (r >= max_rounds) {
          out.capped = true;
          break;
        }
        rebuild = !S.sig.d && lb.used > 0;  // a region has taken half of its slots
        continue;
      }
    }
    S.lm_rounds++;
    S.lm_edges += L.nnz_eff;
    const bool prof = c.profile && lvl == 0;
    if (prof) c.prof_bytes += 12 * L.nnz_eff + 40 * (int64_t)N;
    round_body(r, nullptr, prof, RoundEnd::HOST, cudaGraphConditionalHandle{});
    sync(c);
    struct {
      int64_t moved;
      ull used;
      unsigned status;
    } rb;
    std::memcpy(&rb, c.pinned, sizeof(rb));
    if (rb.status) {
      if (exec) cudaGraphExecDestroy(exec);
      exec = nullptr;
      check_status(c, "local moving");
    }
    rebuild = !S.sig.d && rb.used > 0;  // a region has taken half of its slots
    out.rounds++;
    out.moves += rb.moved;
    ++r;
    if (rb.moved == 0) break;
    if (r == max_rounds) out.capped = true;
  }
  if (exec) cudaGraphExecDestroy(exec);
  S.lm_moves += out.moves;
  return out;
}

}  // namespace mslice
