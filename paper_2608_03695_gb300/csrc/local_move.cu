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
#include "decide.cuh"
#include "solver.h"

namespace mslice {

namespace {

constexpr int APPLY_THREADS = 256;

unsigned fixed_grid(int per_sm) { return 152u * (unsigned)per_sm; }

__global__ void k_tier(const int64_t* rowptr, int32_t N, uint8_t* tier, int32_t* cnt, int64_t* gsize) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = rowptr[v + 1] - rowptr[v];
    const int t = d <= WARP_TIER_MAX ? 0 : (d <= BLOCK_TIER_MAX ? 1 : 2);
    tier[v] = (uint8_t)t;
    int64_t S = 0;
    if (t == 2) {
      S = 2;
      while (S < 2 * d) S <<= 1;
    }
    gsize[v] = S;
    atomicAdd(&cnt[t], 1);
  }
}

// Buckets the nodes of this round by (class, tier): row q of `lists` holds
// class q, tier t at [tier_off[t], tier_off[t] + count).  Order inside a
// bucket does not matter: decisions read only the sub-round snapshot.
__global__ void k_bucket(int32_t N, const uint8_t* tier, uint64_t seed, uint64_t tag, uint64_t it, uint64_t lvl,
                         uint64_t r, int K, int32_t* lists, int64_t row_stride, int3 tier_off, int32_t* cursors) {
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < N; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = base + threadIdx.x;
    const bool ok = v < N;
    int seg = -1;
    if (ok) seg = vertex_class(seed, tag, it, lvl, r, (uint64_t)v, K) * 3 + tier[v];
    const unsigned peers = __match_any_sync(0xffffffffu, seg);
    const int leader = __ffs(peers) - 1;
    int pos = 0;
    if (ok && lane == leader) pos = atomicAdd(&cursors[seg], __popc(peers));
    pos = __shfl_sync(peers, pos, leader);
    if (ok) {
      const int q = seg / 3, t = seg % 3;
      const int off = t == 0 ? tier_off.x : (t == 1 ? tier_off.y : tier_off.z);
      lists[(int64_t)q * row_stride + off + pos + __popc(peers & ((1u << lane) - 1u))] = (int32_t)v;
    }
  }
}

__global__ void k_hash_clear(Slot* slots, uint64_t cap) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += (uint64_t)gridDim.x * blockDim.x)
    slots[i] = Slot{EMPTY_KEY, 0};
}

__global__ void k_sigma_insert(LevelDev g, const int32_t* labels, HashView h, int32_t* size) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.N; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = labels[v];
    if (size) atomicAdd(&size[c], 1);
    int64_t b, e;
    slice_range(g, (int32_t)v, b, e);
    for (int64_t j = b; j < e; ++j) {
      int32_t s;
      long long k;
      slice_entry(g, (int32_t)v, j, s, k);
      hash_add(h, pack_cs(c, s), k);
    }
  }
}

// sum_s Lambda_s k_{v,s} (X_s - self*k_{v,s}) with X_s = table(c, s).
__device__ __forceinline__ u128 null_sum(const LevelDev& g, const u128* lam, const HashView& h, int32_t v, int32_t c,
                                         bool self) {
  int64_t b, e;
  slice_range(g, v, b, e);
  u128 t = 0;
  for (int64_t j = b; j < e; ++j) {
    int32_t s;
    long long k;
    slice_entry(g, v, j, s, k);
    long long x = hash_get(h, pack_cs(c, s));
    if (self) x -= k;
    t += lam[s] * (u128)(ull)k * (u128)(ull)x;
  }
  return t;
}

struct LMPolicy {
  LevelDev g;
  const int32_t* labels;
  const int32_t* size;
  HashView sig;
  const u128* lam;
  int32_t* target;
  long long od;

  __device__ bool begin(int32_t) const { return true; }
  __device__ void skip(int32_t v) const { target[v] = NO_MOVE; }
  __device__ bool edge(int32_t, int64_t e, int32_t& key, long long& w) const {
    int32_t u;
    if (!edge_at(g, e, u, w)) return false;
    key = labels[u];
    return true;
  }
  __device__ int32_t own_key(int32_t v) const { return labels[v]; }
  __device__ i128 key_of(int32_t v, int32_t c, long long W, bool self) const {
    const u128 ns = null_sum(g, lam, sig, v, c, self);
    return (((i128)W) << P_BITS) - (i128)((u128)(ull)od * ns);
  }
  __device__ Cand cand(int32_t v, int32_t c, long long W) const {
    if (c == labels[v]) return Cand{0, INT32_MAX};
    return Cand{key_of(v, c, W, false), c};
  }
  __device__ void finish(int32_t v, const Cand& best, long long, long long Wown) const {
    const int32_t a = labels[v];
    const i128 Ga = key_of(v, a, Wown, true);
    const bool has = best.label != INT32_MAX;
    const i128 Gmax = (has && best.G > Ga) ? best.G : Ga;
    int32_t t = NO_MOVE;
    if (size[a] > 1 && Gmax < 0) {
      t = TO_EMPTY;
    } else if (has && best.G > Ga) {
      if (!(size[a] == 1 && size[best.label] == 1 && best.label > a)) t = best.label;
    }
    target[v] = t;
  }
};

struct Segs {
  const int32_t* list[3];
  const int32_t* count[3];
};

__device__ __forceinline__ bool seg_item(const Segs& sg, int64_t idx, int32_t& v) {
  for (int t = 0; t < 3; ++t) {
    const int cnt = *sg.count[t];
    if (idx < cnt) {
      v = sg.list[t][idx];
      return true;
    }
    idx -= cnt;
  }
  return false;
}

__device__ __forceinline__ int seg_total(const Segs& sg) { return *sg.count[0] + *sg.count[1] + *sg.count[2]; }

// Applies the sub-round's decisions: labels, community sizes and Sigma.
// Moves to an empty community only leave here (the label is assigned below).
__global__ void k_lm_apply(LevelDev g, Segs sg, int32_t* labels, int32_t* size, HashView sig, int32_t* target,
                           int32_t* counters) {
  const int total = seg_total(sg);
  int local = 0, local_empty = 0;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int32_t v;
    if (!seg_item(sg, idx, v)) break;
    const int32_t t = target[v];
    if (t == NO_MOVE) continue;
    const int32_t a = labels[v];
    atomicSub(&size[a], 1);
    int64_t b, e;
    slice_range(g, v, b, e);
    for (int64_t j = b; j < e; ++j) {
      int32_t s;
      long long k;
      slice_entry(g, v, j, s, k);
      hash_add(sig, pack_cs(a, s), -k);
      if (t >= 0) hash_add(sig, pack_cs(t, s), k);
    }
    if (t >= 0) {
      atomicAdd(&size[t], 1);
      labels[v] = t;
      local++;
    } else {
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

__global__ void k_free_flags(const int32_t* size, int32_t N, int32_t* flag, const int32_t* n_empty) {
  if (*n_empty == 0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = size[i] == 0 ? 1 : 0;
}

__global__ void k_free_scatter(const int32_t* size, const int32_t* rank, int32_t N, int32_t* freelist,
                               const int32_t* n_empty) {
  if (*n_empty == 0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    if (size[i] == 0) freelist[rank[i]] = (int32_t)i;
}

__global__ void k_empty_flags(const int32_t* target, int32_t N, int32_t* flag, const int32_t* n_empty) {
  if (*n_empty == 0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = target[i] == TO_EMPTY ? 1 : 0;
}

// Moves to an empty community: in ascending node order, the ascending labels
// that are free once every other move is applied and the movers have left.
__global__ void k_empty_assign(LevelDev g, const int32_t* target, const int32_t* rank, const int32_t* freelist,
                               int32_t* labels, int32_t* size, HashView sig, int32_t* counters) {
  if (counters[2] == 0) return;
  int local = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.N; v += (int64_t)gridDim.x * blockDim.x) {
    if (target[v] != TO_EMPTY) continue;
    const int32_t L = freelist[rank[v]];
    labels[v] = L;
    size[L] = 1;
    int64_t b, e;
    slice_range(g, (int32_t)v, b, e);
    for (int64_t j = b; j < e; ++j) {
      int32_t s;
      long long k;
      slice_entry(g, (int32_t)v, j, s, k);
      hash_add(sig, pack_cs(L, s), k);
    }
    local++;
  }
  local = warp_sum(local);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd((ull*)counters, (ull)local);
}

__global__ void k_reset_targets(Segs sg, int32_t* target, int32_t* counters) {
  const int total = seg_total(sg);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int32_t v;
    if (seg_item(sg, idx, v)) target[v] = NO_MOVE;
  }
}

__global__ void k_zero_empty(int32_t* counters) { counters[2] = 0; }

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

void solver_alloc(Solver& S) {
  Ctx& c = *S.c;
  const int64_t N = S.N0 > 0 ? S.N0 : 1;
  S.target = c.ws->get<int32_t>("s_target", N);
  S.size = c.ws->get<int32_t>("s_size", N);
  S.tmp32a = c.ws->get<int32_t>("s_tmpa", N + 1);
  S.tmp32b = c.ws->get<int32_t>("s_tmpb", N + 1);
  S.freelist = c.ws->get<int32_t>("s_free", N);
  S.tier = c.ws->get<uint8_t>("s_tier", N);
  S.lists = c.ws->get<int32_t>("s_lists", (size_t)N * S.p.K);
  S.cursors = c.ws->get<int32_t>("s_cursors", 3 * S.p.K + 3);
  S.counters = c.ws->get<int32_t>("s_counters", 8);
  S.goff = c.ws->get<int64_t>("s_goff", N + 1);
  S.R = c.ws->get<int32_t>("s_R", N);
  S.sizeR = c.ws->get<int32_t>("s_sizeR", N);
  S.Wc = c.ws->get<long long>("s_Wc", N);
  S.Wout = c.ws->get<long long>("s_Wout", N);
  S.Wsel = c.ws->get<long long>("s_Wsel", N);
  S.rhs = c.ws->get<ull>("s_rhs", 2 * N);
  S.elig = c.ws->get<uint8_t>("s_elig", N);
  S.wc = c.ws->get<uint8_t>("s_wc", N);
  // hash tables keyed by (label, snapshot): at most one live key per
  // (node, snapshot) entry plus the keys created by moves of one round
  const uint64_t cap = (uint64_t)(2 * N + 2 * ((N + S.p.K - 1) / S.p.K) + 64);
  S.sig = HashView{c.ws->get<Slot>("s_sig", cap), cap, c.d_status};
  S.kr = HashView{c.ws->get<Slot>("s_kr", cap), cap, c.d_status};
  fill_i32(c, S.target, NO_MOVE, N);
  check_cuda(cudaMemsetAsync(S.counters, 0, 8 * sizeof(int32_t), c.stream), "memset");
}

void prepare_level(Solver& S, const Level& L) {
  Ctx& c = *S.c;
  const int32_t N = L.d.N;
  int32_t* cnt = S.cursors;  // reused: 3 tier counts
  check_cuda(cudaMemsetAsync(cnt, 0, 3 * sizeof(int32_t), c.stream), "memset");
  int64_t* gsize = reinterpret_cast<int64_t*>(c.ws->get<int64_t>("s_gsize", (size_t)(N > 0 ? N : 1)));
  if (N > 0)
    launch(c, k_tier, dim3(grid_for(N, 256) < 4096 ? grid_for(N, 256) : 4096), dim3(256), 0, L.d.rowptr, N, S.tier,
           cnt, gsize);
  int64_t* gtotal = c.ws->get<int64_t>("s_gtotal", 1);
  scan_excl(c, gsize, S.goff, N, gtotal);
  check_cuda(cudaMemcpyAsync(S.goff + N, gtotal, sizeof(int64_t), cudaMemcpyDeviceToDevice, c.stream), "copy");
  struct {
    int32_t cnt[3];
    int32_t pad;
    int64_t gt;
  } hb;
  check_cuda(cudaMemcpyAsync(&hb.cnt, cnt, 3 * sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream), "copy");
  check_cuda(cudaMemcpyAsync(&hb.gt, gtotal, sizeof(int64_t), cudaMemcpyDeviceToHost, c.stream), "copy");
  sync(c);
  S.tier_cnt[0] = hb.cnt[0];
  S.tier_cnt[1] = hb.cnt[1];
  S.tier_cnt[2] = hb.cnt[2];
  S.tier_off[0] = 0;
  S.tier_off[1] = hb.cnt[0];
  S.tier_off[2] = hb.cnt[0] + hb.cnt[1];
  if (hb.gt > S.gcap) {
    S.gcap = hb.gt;
    S.gkeys = c.ws->get<int32_t>("s_gkeys", S.gcap);
    S.gvals = c.ws->get<long long>("s_gvals", S.gcap);
  }
}

void sigma_rebuild(Solver& S, const Level& L, const int32_t* labels) {
  Ctx& c = *S.c;
  launch(c, k_hash_clear, dim3(fixed_grid(8)), dim3(256), 0, S.sig.slots, S.sig.cap);
  if (L.d.N > 0)
    launch(c, k_sigma_insert, dim3(grid_for(L.d.N, 256)), dim3(256), 0, L.d, labels, S.sig, (int32_t*)nullptr);
}

// Buckets and returns the device segments of class q for every tier.
static Segs bucket_segments(Solver& S, int q) {
  Segs sg;
  for (int t = 0; t < 3; ++t) {
    sg.list[t] = S.lists + (int64_t)q * S.N0 + S.tier_off[t];
    sg.count[t] = S.cursors + 3 * q + t;
  }
  return sg;
}

void bucket(Solver& S, const Level& L, uint64_t tag, int it, int lvl, int r) {
  Ctx& c = *S.c;
  check_cuda(cudaMemsetAsync(S.cursors, 0, 3 * S.p.K * sizeof(int32_t), c.stream), "memset");
  if (L.d.N > 0)
    launch(c, k_bucket, dim3(grid_for(L.d.N, 256)), dim3(256), 0, L.d.N, (const uint8_t*)S.tier, S.p.seed, tag,
           (uint64_t)it, (uint64_t)lvl, (uint64_t)r, S.p.K, S.lists, (int64_t)S.N0,
           make_int3(S.tier_off[0], S.tier_off[1], S.tier_off[2]), S.cursors);
}

template <class Pol>
void decide_all(Solver& S, const Pol& pol, const Segs& sg) {
  Ctx& c = *S.c;
  if (S.tier_cnt[0] > 0)
    launch(c, k_decide_warp<Pol>, dim3(fixed_grid(8)), dim3(DECIDE_WARP_THREADS), 0, pol, sg.list[0], sg.count[0]);
  if (S.tier_cnt[1] > 0)
    launch(c, k_decide_block<Pol>, dim3(fixed_grid(8)), dim3(BLOCK_TIER_THREADS), 0, pol, sg.list[1], sg.count[1]);
  if (S.tier_cnt[2] > 0)
    launch(c, k_decide_global<Pol>, dim3(fixed_grid(4)), dim3(GLOBAL_TIER_THREADS), 0, pol, sg.list[2], sg.count[2],
           S.gkeys, S.gvals, (const int64_t*)S.goff, c.d_status);
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
  if (max_rounds <= 0) {
    // no round: refinement still reads Sigma of the given labels
    check_cuda(cudaMemsetAsync(S.size, 0, N * sizeof(int32_t), c.stream), "memset");
    launch(c, k_hash_clear, dim3(fixed_grid(8)), dim3(256), 0, S.sig.slots, S.sig.cap);
    launch(c, k_sigma_insert, dim3(grid_for(N, 256)), dim3(256), 0, L.d, (const int32_t*)labels, S.sig, S.size);
    return out;
  }
  LMPolicy pol;
  pol.g = L.d;
  pol.labels = labels;
  pol.size = S.size;
  pol.sig = S.sig;
  pol.lam = S.lam;
  pol.target = S.target;
  pol.od = S.p.od;
  for (int r = 0; r < max_rounds; ++r) {
    // community sizes and Sigma from the labels
    check_cuda(cudaMemsetAsync(S.size, 0, N * sizeof(int32_t), c.stream), "memset");
    launch(c, k_hash_clear, dim3(fixed_grid(8)), dim3(256), 0, S.sig.slots, S.sig.cap);
    launch(c, k_sigma_insert, dim3(grid_for(N, 256)), dim3(256), 0, L.d, (const int32_t*)labels, S.sig, S.size);
    check_cuda(cudaMemsetAsync(S.counters, 0, 3 * sizeof(int32_t), c.stream), "memset");
    bucket(S, L, 0, it, lvl, r);
    S.lm_rounds++;
    S.lm_edges += L.nnz_eff;
    if (c.profile) c.prof_bytes += 12 * L.nnz_eff + 40 * (int64_t)N;
    for (int q = 0; q < S.p.K; ++q) {
      const Segs sg = bucket_segments(S, q);
      if (c.profile) {
        cudaEvent_t e0, e1;
        check_cuda(cudaEventCreate(&e0), "event");
        check_cuda(cudaEventCreate(&e1), "event");
        check_cuda(cudaEventRecord(e0, c.stream), "event");
        decide_all(S, pol, sg);
        check_cuda(cudaEventRecord(e1, c.stream), "event");
        c.prof_spans->push_back({e0, e1});
      } else {
        decide_all(S, pol, sg);
      }
      launch(c, k_lm_apply, dim3(fixed_grid(4)), dim3(APPLY_THREADS), 0, L.d, sg, labels, S.size, S.sig, S.target,
             S.counters);
      // moves to empty communities (kernels return at once when there are none)
      const int32_t* n_empty = S.counters + 2;
      launch(c, k_free_flags, dim3(fixed_grid(4)), dim3(256), 0, (const int32_t*)S.size, N, S.tmp32a, n_empty);
      scan_excl(c, S.tmp32a, S.tmp32a, N, (int32_t*)nullptr, n_empty);
      launch(c, k_free_scatter, dim3(fixed_grid(4)), dim3(256), 0, (const int32_t*)S.size, (const int32_t*)S.tmp32a, N,
             S.freelist, n_empty);
      launch(c, k_empty_flags, dim3(fixed_grid(4)), dim3(256), 0, (const int32_t*)S.target, N, S.tmp32b, n_empty);
      scan_excl(c, S.tmp32b, S.tmp32b, N, (int32_t*)nullptr, n_empty);
      launch(c, k_empty_assign, dim3(fixed_grid(4)), dim3(256), 0, L.d, (const int32_t*)S.target,
             (const int32_t*)S.tmp32b, (const int32_t*)S.freelist, labels, S.size, S.sig, S.counters);
      launch(c, k_reset_targets, dim3(fixed_grid(4)), dim3(256), 0, sg, S.target, S.counters);
      launch(c, k_zero_empty, dim3(1), dim3(1), 0, S.counters);
    }
    const int64_t moved = *static_cast<const int64_t*>(readback(c, S.counters, sizeof(int64_t)));
    check_status(c, "local moving");
    out.rounds++;
    out.moves += moved;
    if (moved == 0) break;
  }
  S.lm_moves += out.moves;
  return out;
}

}  // namespace mslice
