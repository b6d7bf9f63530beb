// Refinement (the Leiden refinement phase named in Sec. 3.2; Traag et al.
// 2019) in its greedy form.  Inside every local-moving community C each node
// starts as its own sub-community; one pass of K sub-rounds (class tag 1,
// round 0).  A node still alone in its sub-community and well connected to C,
//   2^64 W(v,C\v) >= od sum_s Lambda_s k_{v,s} (K_{C,s} - k_{v,s}),
// joins the well-connected sub-community R of C (reached by one of its edges
// inside C) with the largest positive key
//   2^64 W(v,R) - od sum_s Lambda_s k_{v,s} K_{R,s}
// (ties to the smallest label).  Well connected:
//   2^64 W(R,C\R) >= od sum_s Lambda_s K_{R,s} (K_{C,s} - K_{R,s}).
// A singleton sub-community whose node is active in the same sub-round is
// not a target, so a joined node never leaves and every sub-community stays
// connected.  A non-empty sub-community label L always contains node L, so a
// singleton's label is its node.
//
// W(R,C\R) is maintained incrementally: when the set M of nodes joins R,
//   W(R u M, C\(R u M)) = W(R,C\R) + sum_{v in M} [W(v,C\v) - 2 W(v,R)]
//                         - sum_{v in M} W(v, M\v).
#include "decide.cuh"
#include "solver.h"

namespace mslice {

namespace {

__device__ __forceinline__ u128 lam_k_x(const u128* lam, int32_t s, long long k, long long x) {
  return lam[s] * (u128)(ull)k * (u128)(ull)x;
}

// Per node: W(v,C\v), eligibility, initial sub-community state.
__global__ void k_ref_init(LevelDev g, const int32_t* P, SigStore sig, const u128* lam, int32_t* R, int32_t* sizeR,
                           long long* Wc, long long* Wout, uint8_t* elig, SigStore kr, long long* PR) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = (((int64_t)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5); v < g.N; v += warps) {
    const int32_t C = P[v];
    const Omega om = node_omega(g, (int32_t)v);
    long long w = 0;
    for (int64_t e = g.rowptr[v] + lane; e < g.rowptr[v + 1]; e += 32) {
      int32_t u;
      long long W;
      if (edge_at(g, e, u, W, om) && P[u] == C) w += W;
    }
    w = warp_sum(w);
    // a long (snapshot, strength) list is shared by the lanes; a short one
    // (every level-0 node's) is walked by lane 0 alone
    int64_t b, e;
    slice_range(g, (int32_t)v, b, e);
    const bool wide = e - b > 32;
    u128 rhs = 0;
    if (wide || lane == 0)
      for (int64_t j = b + (wide ? lane : 0); j < e; j += (wide ? 32 : 1)) {
        int32_t s;
        long long k;
        slice_entry(g, (int32_t)v, j, s, k);
        rhs += lam_k_x(lam, s, k, ss_get(sig, C, s) - k);
        ss_add(kr, (int32_t)v, s, k);
      }
    if (wide) rhs = warp_sum_u128(rhs);
    if (lane == 0) {
      R[v] = (int32_t)v;
      PR[v] = (long long)(((unsigned long long)(uint32_t)C << 32) | (uint32_t)v);
      sizeR[v] = 1;
      Wc[v] = w;
      Wout[v] = w;
      elig[v] = ((((i128)w) << P_BITS) - (i128)((u128)(ull)null_scale(g, om) * rhs)) >= 0 ? 1 : 0;
    }
  }
}

__global__ void k_classes(LevelDev g, uint64_t seed, uint64_t it, uint64_t lvl, int K, uint8_t* cls) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.N; v += (int64_t)gridDim.x * blockDim.x)
    cls[v] = (uint8_t)vertex_class(seed, 1, it, lvl, 0, local_id(g, (int32_t)v), K);
}

__global__ void k_zero_rhs(ull* rhs, int64_t n2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x)
    rhs[i] = 0;
}

// sum_s Lambda_s K_{R,s} (K_{C,s} - K_{R,s}) for every sub-community with
// more than one node (singletons reuse their eligibility).
__global__ void k_rhs_accum(SigStore kr, const int32_t* sizeR, const int32_t* P, SigStore sig, const u128* lam,
                            ull* rhs) {
  const uint64_t span = ss_span(kr);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < span; i += (uint64_t)gridDim.x * blockDim.x) {
    int32_t Rl, s;
    long long K;
    if (!ss_entry(kr, i, Rl, s, K)) continue;
    if (sizeR[Rl] <= 1) continue;
    const long long KC = ss_get(sig, P[Rl], s);
    atomic_add_u128(&rhs[2 * (int64_t)Rl], lam_k_x(lam, s, K, KC - K));
  }
}

// (A sub-community label L is a node of the level, so its omega is that
// node's instance's.)
// Also packs what a candidate probe reads of sub-community L, as of the
// sub-round start, into one word: size | class << 32 | well-connected << 40.
__global__ void k_wc(LevelDev g, const int32_t* sizeR, const long long* Wout, const ull* rhs, const uint8_t* elig,
                     const uint8_t* cls, uint8_t* wc, unsigned long long* desc) {
  for (int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; L < g.N; L += (int64_t)gridDim.x * blockDim.x) {
    const int32_t sz = sizeR[L];
    uint8_t f = 0;
    if (sz == 1) {
      f = elig[L];
    } else if (sz > 1) {
      const u128 x = ((u128)rhs[2 * L + 1] << 64) | rhs[2 * L];
      const long long nd = null_scale(g, node_omega(g, (int32_t)L));
      f = ((((i128)Wout[L]) << P_BITS) - (i128)((u128)(ull)nd * x)) >= 0 ? 1 : 0;
    }
    wc[L] = f;
    desc[L] = (unsigned long long)(uint32_t)sz | ((unsigned long long)cls[L] << 32) | ((unsigned long long)f << 40);
  }
}

template <bool DENSE>
struct RefPolicy {
  static constexpr int MIN_BLOCKS = DENSE ? MSLICE_DENSE_MIN_BLOCKS : MSLICE_GROUP_MIN_BLOCKS;
  LevelDev g;
  const int32_t* P;
  const int32_t* R;
  const unsigned long long* desc;  // size, class, well-connectedness (k_wc)
  const long long* PR;  // (P << 32) | R of every node, kept with R
  const int32_t* sizeR;
  const uint8_t* elig;
  const uint8_t* wc;
  const uint8_t* cls;
  SigStore kr;
  const u128* lam;
  int32_t* target;
  long long* Wsel;
  int q;

  struct Probe {
    Slot first;
    int32_t size;
    uint8_t cls, wc;
  };
  // Per node: at level 0 the snapshot s and A = nd * Lambda_s * k.
  struct VCtx {
    int32_t s, Pv;
    bool single;
    long long k;
    Omega om;
    u128 A;
  };

  __device__ bool begin(int32_t v) const { return sizeR[R[v]] == 1 && elig[v]; }
  __device__ VCtx vctx(int32_t v) const {
    VCtx c;
    c.single = g.is0 != 0;
    c.s = 0;
    c.k = 0;
    c.A = 0;
    c.Pv = P[v];
    c.om = node_omega(g, v);
    if (c.single) {
      c.k = g.k0[v];
      c.s = node_slice0(g, v);
      if (c.k > 0) c.A = (u128)(ull)null_scale(g, c.om) * lam[c.s] * (u128)(ull)c.k;
    }
    return c;
  }
  __device__ void skip(int32_t v) const { target[v] = NO_MOVE; }
  __device__ bool edge(int32_t v, const VCtx& vc, int64_t e, int32_t& key, long long& w) const {
    int32_t u;
    if (!edge_at(g, e, u, w, vc.om)) return false;
    const unsigned long long pr = (unsigned long long)PR[u];  // (P[u], R[u]) in one load
    if ((int32_t)(pr >> 32) != vc.Pv) return false;
    key = (int32_t)(uint32_t)pr;
    return true;
  }
  __device__ int32_t own_key(int32_t) const { return -1; }
  __device__ i128 own(int32_t, const VCtx&, long long) const { return 0; }
  __device__ Probe probe(int32_t, const VCtx& vc, int32_t X) const {
    Probe p;
    const unsigned long long d = desc[X];
    p.size = (int32_t)(uint32_t)d;
    p.cls = (uint8_t)(d >> 32);
    p.wc = (uint8_t)(d >> 40);
    p.first = (vc.single && vc.k > 0) ? sst_first<DENSE>(kr, X, vc.s) : Slot{EMPTY_KEY, 0};
    return p;
  }
  // A singleton sub-community's label is its node, so cls[X] is the class of
  // that node.
  __device__ Cand cand(int32_t v, const VCtx& vc, int32_t X, long long W, const Probe& p) const {
    if (p.size == 1 && p.cls == q) return Cand{0, INT32_MAX};
    if (!p.wc) return Cand{0, INT32_MAX};
    i128 G;
    if (vc.single) {
      const long long x = vc.k > 0 ? sst_resolve<DENSE>(kr, X, vc.s, p.first) : 0;
      G = (((i128)W) << P_BITS) - (i128)(vc.A * (u128)(ull)x);
    } else {
      int64_t b, e;
      slice_range(g, v, b, e);
      u128 ns = 0;
      for (int64_t j = b; j < e; ++j) {
        int32_t s;
        long long k;
        slice_entry(g, v, j, s, k);
        ns += lam_k_x(lam, s, k, sst_get<DENSE>(kr, X, s));
      }
      G = (((i128)W) << P_BITS) - (i128)((u128)(ull)null_scale(g, vc.om) * ns);
    }
    if (G <= 0) return Cand{0, INT32_MAX};
    return Cand{G, X};
  }
  // slice-parallel scoring (block tiers, aggregated levels); own() is 0
  __device__ int64_t slice_count(int32_t v) const { return g.is0 ? 0 : g.sptr[v + 1] - g.sptr[v]; }
  __device__ bool own_walks_slices() const { return false; }
  __device__ u128 null_part(int32_t v, const VCtx&, int32_t X, bool, int t, int nt) const {
    int64_t b, e;
    slice_range(g, v, b, e);
    u128 acc = 0;
    for (int64_t j = b + t; j < e; j += nt) {
      int32_t s;
      long long k;
      slice_entry(g, v, j, s, k);
      acc += lam_k_x(lam, s, k, sst_get<DENSE>(kr, X, s));
    }
    return acc;
  }
  __device__ Cand cand_ns(int32_t, const VCtx& vc, int32_t X, long long W, const u128& ns) const {
    const unsigned long long d = desc[X];
    if ((int32_t)(uint32_t)d == 1 && (uint8_t)(d >> 32) == q) return Cand{0, INT32_MAX};
    if (!(uint8_t)(d >> 40)) return Cand{0, INT32_MAX};
    const i128 G = (((i128)W) << P_BITS) - (i128)((u128)(ull)null_scale(g, vc.om) * ns);
    if (G <= 0) return Cand{0, INT32_MAX};
    return Cand{G, X};
  }
  __device__ i128 own_ns(int32_t, const VCtx&, long long, const u128&) const { return 0; }
  __device__ void finish(int32_t v, const Cand& best, long long Wb, const i128&, const VCtx&) const {
    if (best.label != INT32_MAX) {
      target[v] = best.label;
      Wsel[v] = Wb;
    } else {
      target[v] = NO_MOVE;
    }
  }
};

typedef TierSegs Segs3;

__device__ __forceinline__ int seg3_total(const Segs3& sg) {
  int t = 0;
#pragma unroll
  for (int i = 0; i < NTIERS; ++i) t += *sg.count[i];
  return t;
}
__device__ __forceinline__ bool seg3_item(const Segs3& sg, int64_t idx, int32_t& v) {
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

// One warp per active node: movers compute W(v, M_t \ v) over their edges to
// other movers with the same target, then update sizes, K_{R,s} and W(R,C\R).
__global__ void k_ref_apply(LevelDev g, Segs3 sg, const int32_t* P, const int32_t* target, const long long* Wc,
                            const long long* Wsel, int32_t* R, int32_t* sizeR, long long* Wout, SigStore kr,
                            long long* PR) {
  const int lane = threadIdx.x & 31;
  const int total = seg3_total(sg);
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t idx = (((int64_t)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5); idx < total; idx += warps) {
    int32_t v;
    if (!seg3_item(sg, idx, v)) break;
    const int32_t t = target[v];
    if (t < 0) continue;
    long long wp = 0;
    const Omega om = node_omega(g, v);
    for (int64_t e = g.rowptr[v] + lane; e < g.rowptr[v + 1]; e += 32) {
      int32_t u;
      long long W;
      // a target lies in the mover's own community, so target[u] == t
      // implies P[u] == P[v]
      if (edge_at(g, e, u, W, om) && target[u] == t) wp += W;
    }
    wp = warp_sum(wp);
    if (lane == 0) {
      R[v] = t;
      PR[v] = (long long)(((unsigned long long)(uint32_t)P[v] << 32) | (uint32_t)t);
      atomicSub(&sizeR[v], 1);
      atomicAdd(&sizeR[t], 1);
      atomicAdd((ull*)&Wout[t], (ull)(Wc[v] - 2 * Wsel[v] - wp));
      Wout[v] = 0;
    }
    // the sub-community rows take the node's list: by the warp when long
    int64_t b, e;
    slice_range(g, v, b, e);
    const bool wide = e - b > 32;
    if (wide || lane == 0)
      for (int64_t j = b + (wide ? lane : 0); j < e; j += (wide ? 32 : 1)) {
        int32_t s;
        long long k;
        slice_entry(g, v, j, s, k);
        ss_add(kr, v, s, -k);
        ss_add(kr, t, s, k);
      }
  }
}

__global__ void k_ref_reset(Segs3 sg, int32_t* target) {
  const int total = seg3_total(sg);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int32_t v;
    if (seg3_item(sg, idx, v)) target[v] = NO_MOVE;
  }
}

unsigned fixed_grid(int per_sm) { return 152u * (unsigned)per_sm; }

}  // namespace

void bucket(Solver& S, const Level& L, uint64_t tag, int it, int lvl, int r, const int32_t* active,
            const int32_t* r_dev = nullptr);
TierSegs bucket_segments(Solver& S, int q);

template <bool DENSE>
static void refine_impl(Solver& S, const Level& L, const int32_t* P, int it, int lvl) {
  Ctx& c = *S.c;
  const int32_t N = L.d.N;
  if (N == 0) return;
  clear_store(S, S.kr);
  long long* PR = c.ws->get<long long>("ref_PR", N);
  launch(c, k_ref_init, dim3(fixed_grid(8)), dim3(256), 0, L.d, P, S.sig, (const u128*)S.lam, S.R, S.sizeR, S.Wc,
         S.Wout, S.elig, S.kr, PR);
  bucket(S, L, 1, it, lvl, 0, S.inst_active);
  RefPolicy<DENSE> pol;
  pol.g = L.d;
  pol.P = P;
  pol.R = S.R;
  pol.PR = PR;
  unsigned long long* desc = c.ws->get<unsigned long long>("ref_desc", N);
  pol.desc = desc;
  pol.sizeR = S.sizeR;
  pol.elig = S.elig;
  pol.wc = S.wc;
  pol.kr = S.kr;
  pol.lam = S.lam;
  pol.target = S.target;
  pol.Wsel = S.Wsel;
  pol.cls = S.cls;
  launch(c, k_classes, dim3(fixed_grid(8)), dim3(256), 0, L.d, S.p.seed, (uint64_t)it, (uint64_t)lvl, S.p.K, S.cls);
  for (int q = 0; q < S.p.K; ++q) {
    // well-connectedness of every sub-community at the sub-round start
    if (q > 0) {
      launch(c, k_zero_rhs, dim3(fixed_grid(8)), dim3(256), 0, S.rhs, 2 * (int64_t)N);
      launch(c, k_rhs_accum, dim3(fixed_grid(8)), dim3(256), 0, S.kr, (const int32_t*)S.sizeR, P, S.sig,
             (const u128*)S.lam, S.rhs);
    }
    launch(c, k_wc, dim3(fixed_grid(8)), dim3(256), 0, L.d, (const int32_t*)S.sizeR, (const long long*)S.Wout,
           (const ull*)S.rhs, (const uint8_t*)S.elig, (const uint8_t*)S.cls, S.wc, desc);
    pol.q = q;
    const Segs3 sg = bucket_segments(S, q);
    decide_all(c, pol, sg, S.tier_cnt, S.gkeys, S.gvals, S.goff);
    launch(c, k_ref_apply, dim3(fixed_grid(8)), dim3(256), 0, L.d, sg, P, (const int32_t*)S.target,
           (const long long*)S.Wc, (const long long*)S.Wsel, S.R, S.sizeR, S.Wout, S.kr, PR);
    launch(c, k_ref_reset, dim3(fixed_grid(4)), dim3(256), 0, sg, S.target);
  }
}

void refine(Solver& S, const Level& L, const int32_t* P, int it, int lvl) {
  if (S.kr.d)
    refine_impl<true>(S, L, P, it, lvl);
  else
    refine_impl<false>(S, L, P, it, lvl);
}

}  // namespace mslice
