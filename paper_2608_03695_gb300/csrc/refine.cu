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

// Per node: W(v,C\v), eligibility, initial sub-community state.  G lanes per
// node (G = 32 at aggregated levels, whose long (snapshot, strength) lists
// the lanes share; fewer at level 0, whose rows are short and whose nodes
// hold one snapshot each, so a warp takes several nodes at once).
template <int G>
__global__ void k_ref_init(LevelDev g, const int32_t* P, SigStore sig, const u128* lam, int32_t* R, int32_t* sizeR,
                           long long* Wc, long long* Wout, uint8_t* elig, SigStore kr, long long* PR) {
  const int lane = threadIdx.x & 31, gl = lane % G;
  const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane - gl));
  const int64_t groups = ((int64_t)gridDim.x * blockDim.x) / G;
  // every lane of a warp runs the same number of iterations (shuffles below)
  const int64_t first = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t warp_first = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) / G;
  for (int64_t v0 = warp_first; v0 < g.N; v0 += groups) {
    const int64_t v = v0 + (first - warp_first);
    const bool ok = v < g.N;
    const int32_t C = ok ? P[v] : 0;
    const Omega om = ok ? node_omega(g, (int32_t)v) : Omega{1, 1};
    long long w = 0;
    if (ok)
      for (int64_t e = g.rowptr[v] + gl; e < g.rowptr[v + 1]; e += G) {
        int32_t u;
        long long W;
        if (edge_at(g, e, u, W, om) && P[u] == C) w += W;
      }
#pragma unroll
    for (int m = G / 2; m >= 1; m >>= 1) w += __shfl_xor_sync(gmask, w, m);
    // a long (snapshot, strength) list is shared by the lanes of the group;
    // a short one (every level-0 node's) is walked by its first lane
    int64_t b = 0, e = 0;
    if (ok) slice_range(g, (int32_t)v, b, e);
    const bool wide = G == 32 && e - b > 32;
    u128 rhs = 0;
    if (ok && (wide || gl == 0))
      for (int64_t j = b + (wide ? gl : 0); j < e; j += (wide ? G : 1)) {
        int32_t s;
        long long k;
        slice_entry(g, (int32_t)v, j, s, k);
        rhs += lam_k_x(lam, s, k, ss_get(sig, C, s) - k);
        ss_add(kr, (int32_t)v, s, k);
      }
    if (G == 32 && __any_sync(0xffffffffu, wide)) rhs = warp_sum_u128(rhs);
    if (ok && gl == 0) {
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
  // randomised refinement: the key of target X when X is allowed and the
  // key is >= 0 (cand() without its strict-gain filter)
  __device__ bool rand_key(int32_t v, const VCtx& vc, int32_t X, long long W, i128& G) const {
    const Probe p = probe(v, vc, X);
    if (p.size == 1 && p.cls == q) return false;
    if (!p.wc) return false;
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
    return G >= 0;
  }
};

// ---------------------------------------------------------------------------
// Randomised refinement (Traag et al.: an eligible singleton joins a target X
// with probability proportional to exp(dQ_X / theta) among the targets with
// dQ_X >= 0, staying weighing exp(0)).  With dQ = G / (2^63 2M) (G the exact
// key, 2M = od*2mu) the weight of a candidate is 2^40 exp(-(Gmax - G) /
// (2^63 2M theta)), evaluated by an integer recipe that every implementation
// follows bit for bit:
//   Y  = floor(d / (2M theta_num))   (0 weight when Y >= 2^96)
//   yF = floor(Y theta_den / 2^31)   (y in Q32; 0 weight when y >= 64)
//   u  = yF * LOG2E                  (y log2 e in Q64; LOG2E = round(log2(e) 2^32))
//   I  = floor(u / 2^64)             (0 weight when I >= 40), f = u mod 2^64
//   g  = floor(f LN2 / 2^64)         (f ln 2 in Q62; LN2 = round(ln(2) 2^62))
//   e^-g = its Taylor series in Q62 (term_k = floor(floor(term_{k-1} g / 2^62) / k),
//          alternating signs, ending at the first zero term)
//   weight = floor(e^-g / 2^(22 + I))   (Q40).
// The draw R = class_hash(seed, 2, it, level, 0, node) / 2^32 sets the
// threshold floor(R * total / 2^32); the first candidate, in the order
// staying, then ascending label, whose cumulative weight exceeds it wins.
constexpr ull LOG2E_Q32 = 6196328019ull;
constexpr ull LN2_Q62 = 3196577161300663915ull;

__device__ __forceinline__ int bitlen128(u128 x) {
  const ull hi = (ull)(x >> 64);
  return hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)(ull)x);
}

// floor(d / div) for d >= div, in integers: the top 64 bits of d times the
// reciprocal R give an estimate q_est <= the quotient (both factors are
// truncated) and, below 2^59, within 2 of it (relative errors 2^-63 and
// 2^-62), corrected by subtracting div from the remainder.  A larger
// estimate returns false with q_est in q (the caller then needs only to know
// whether the quotient reaches 2^69, or divides exactly).
__device__ __forceinline__ bool udiv_recip(u128 d, const RandDiv& rd, u128& q) {
  const int ld = bitlen128(d);
  const int sd = ld > 64 ? ld - 64 : 0;
  const ull dt = (ull)(d >> sd);
  q = ((u128)dt * (u128)rd.R) >> (rd.k - sd);  // k - sd <= 126 since d >= div
  if (q >> 59) return false;
  u128 r = d - q * rd.div;
  while (r >= rd.div) {
    r -= rd.div;
    ++q;
  }
  return true;
}

// floor((2^64 - 1) / k) for k = 2..40, computed by the compiler: floor(x / k)
// is then the high product with it, corrected upward (by at most 2).
struct SmallRecips {
  ull r[41];
  constexpr SmallRecips() : r() {
    for (int k = 2; k <= 40; ++k) r[k] = ~0ull / (ull)k;
  }
};
__device__ constexpr SmallRecips SMALL_RECIPS{};

__device__ __forceinline__ ull div_small(ull x, int k) {
  if (k == 1) return x;
  ull q = __umul64hi(x, SMALL_RECIPS.r[k]);
  while ((q + 1) * (ull)k <= x) ++q;
  return q;
}

// The weight of a key difference d.  (Every intermediate of the series fits
// 64 bits: g < 2^62 and each term is at most 2^62, so the products are
// 64x64 -> 128 and the divisions 64-bit; the values are those of the 128-bit
// statement above.)  Kept out of line: one copy of the series instead of one
// per call site left the warp-per-node kernel 20 registers lighter and
// refinement 7% faster (fewer instruction-cache misses).
__device__ __noinline__ ull rand_weight(u128 d, const RandDiv& rd, ull td) {
  u128 Y = 0;
  if (d >= rd.div && !udiv_recip(d, rd, Y)) {
    // Y >= q_est >= 2^69 makes Y * theta_den / 2^31 >= 64 * 2^32: weight 0
    if (Y >> 69) return 0;
    Y = d / rd.div;
  }
  if (Y >> 96) return 0;
  const u128 yF = (Y * (u128)td) >> 31;
  if (yF >= ((u128)64 << 32)) return 0;
  const u128 u = yF * (u128)LOG2E_Q32;
  const ull I = (ull)(u >> 64);
  if (I >= 40) return 0;
  const ull g = (ull)(((u128)(ull)u * (u128)LN2_Q62) >> 64);
  ull term = 1ull << 62;
  long long sum = (long long)term;
  for (int k = 1; k <= 40; ++k) {
    term = div_small((ull)(((u128)term * (u128)g) >> 62), k);
    if (term == 0) break;
    sum += (k & 1) ? -(long long)term : (long long)term;
  }
  return (ull)sum >> (22 + I);
}

struct RandParams {
  uint64_t seed, it, lvl;
  const RandDiv* div;  // 2M theta_num of every instance
  ull td;              // theta_den
};

__device__ __forceinline__ i128 shfl_xor_i128(i128 x, int m, unsigned mask) {
  ull lo = (ull)(u128)x, hi = (ull)((u128)x >> 64);
  lo = __shfl_xor_sync(mask, lo, m);
  hi = __shfl_xor_sync(mask, hi, m);
  return (i128)(((u128)hi << 64) | lo);
}

// Maximum / sum over a team of NT threads: a group of NT <= 32 aligned lanes
// (mask: its lanes), or a block of NT threads through sm (one word per warp;
// every thread gets the result; two barriers).
template <int NT>
__device__ __forceinline__ i128 team_max_i128(i128 x, unsigned mask, u128* sm) {
#pragma unroll
  for (int m = (NT < 32 ? NT : 32) / 2; m >= 1; m >>= 1) {
    const i128 o = shfl_xor_i128(x, m, mask);
    if (o > x) x = o;
  }
  if constexpr (NT > 32) {
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = (u128)x;
    __syncthreads();
    x = 0;
    for (int w = 0; w < NT / 32; ++w)
      if ((i128)sm[w] > x) x = (i128)sm[w];
    __syncthreads();
  }
  return x;
}

template <int NT>
__device__ __forceinline__ u128 team_sum_u128(u128 x, unsigned mask, u128* sm) {
  ull lo = (ull)x, hi = (ull)(x >> 64);
#pragma unroll
  for (int m = (NT < 32 ? NT : 32) / 2; m >= 1; m >>= 1) {
    const ull l2 = __shfl_xor_sync(mask, lo, m), h2 = __shfl_xor_sync(mask, hi, m);
    const ull nl = lo + l2;
    hi += h2 + (nl < lo ? 1ull : 0ull);
    lo = nl;
  }
  x = ((u128)hi << 64) | lo;
  if constexpr (NT > 32) {
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = x;
    __syncthreads();
    x = 0;
    for (int w = 0; w < NT / 32; ++w) x += sm[w];
    __syncthreads();
  }
  return x;
}

// One node's randomised choice over the candidate keys listed in its table
// (slots cand[0..n), or every slot when cand is null), by a team of NT
// threads: t is the thread's rank in the team, base the team's first lane
// (groups), mask its lanes; a block (NT > 32) uses sm (NT/32 + 1 words).
// Returns the chosen label (INT32_MAX: stay) and its weight W through Wb,
// on every thread of the team.
template <class Pol, int NT>
__device__ int32_t rand_choose(const Pol& pol, int32_t v, const typename Pol::VCtx& vc, const RandParams& rp,
                               const int32_t* K, const long long* V, ull* WT, const uint16_t* cand, int64_t n,
                               int bits, int t, int base, unsigned mask, u128* sm128, long long& Wb) {
  constexpr bool BLOCK = NT > 32;
  const RandDiv rd = rp.div[node_inst(pol.g, v)];
  // pass 1: largest allowed key (staying: 0); with at most one candidate per
  // thread its key is kept for pass 2
  const bool one_each = n <= NT;
  i128 G1 = 0;
  bool ok1 = false;
  i128 gmax = 0;
  for (int64_t j = t; j < n; j += NT) {
    const int slot = cand ? cand[j] : (int)j;
    const int32_t X = K[slot];
    i128 G = 0;
    const bool ok = X >= 0 && pol.rand_key(v, vc, X, V[slot], G);
    if (ok && G > gmax) gmax = G;
    G1 = G;
    ok1 = ok;
  }
  gmax = team_max_i128<NT>(gmax, mask, sm128);
  // pass 2: weights (0 for a slot that is not a candidate) and their total.
  // With fewer candidates than threads, thread n weighs staying in the same
  // pass (one weight evaluation per thread instead of two in a row).
  u128 part = 0;
  ull wstay = 0;
  const bool stay_lane = n < NT;
  if (stay_lane) {
    const int slot = t < n ? (cand ? cand[t] : t) : 0;
    const bool has = t < n ? ok1 : t == n;
    const u128 d = t < n ? (u128)(gmax - G1) : (u128)gmax;
    const ull w = has ? rand_weight(d, rd, rp.td) : 0;
    if (t < n) {
      WT[slot] = w;
      part = w;
    }
    if (BLOCK) {
      if (t == n) sm128[NT / 32] = w;  // read after the first barrier of the sum below
    } else {
      wstay = __shfl_sync(mask, w, base + (int)n);
    }
  } else {
    for (int64_t j = t; j < n; j += NT) {
      const int slot = cand ? cand[j] : (int)j;
      const int32_t X = K[slot];
      i128 G = G1;
      ull w = 0;
      if (one_each ? ok1 : (X >= 0 && pol.rand_key(v, vc, X, V[slot], G)))
        w = rand_weight((u128)(gmax - G), rd, rp.td);
      WT[slot] = w;
      part += w;
    }
  }
  if (BLOCK && stay_lane) {
    // team_sum_u128's barriers order the write above before this read
    part = team_sum_u128<NT>(part, mask, sm128);
    wstay = (ull)sm128[NT / 32];
    __syncthreads();  // before a later node's write of the word
  } else {
    part = team_sum_u128<NT>(part, mask, sm128);
    if (!BLOCK) __syncwarp(mask);  // WT written by the team
  }
  if (!stay_lane) wstay = rand_weight((u128)gmax, rd, rp.td);
  const u128 total = part + wstay;
  const ull R = class_hash(rp.seed, 2, rp.it, rp.lvl, 0, local_id(pol.g, v)) >> 32;
  const u128 thr = ((u128)R * total) >> 32;
  if (BLOCK) {
    if (threadIdx.x == 0) sm128[0] = ~(u128)0;  // "no candidate chosen"
    __syncthreads();
  }
  // pass 3: the candidate whose interval [cum, cum + w) holds thr, in
  // ascending label order after staying.  Few candidates: each thread sums
  // the weights of the smaller labels for its own candidates.  Many: a
  // binary search for the smallest label L with wstay + sum_{label <= L} w
  // > thr (about 31 team sums instead of n^2 work).
  int32_t chosen = INT32_MAX;
  long long wchosen = 0;
  if (!(thr < wstay) && n <= 64) {
    for (int64_t j = t; j < n; j += NT) {
      const int slot = cand ? cand[j] : (int)j;
      const ull wj = WT[slot];
      if (wj == 0) continue;
      const int32_t X = K[slot];
      u128 cb = wstay;
      for (int64_t i = 0; i < n; ++i) {
        const int s2 = cand ? cand[i] : (int)i;
        const ull wi = WT[s2];
        if (wi && K[s2] < X) cb += wi;
      }
      if (cb <= thr && thr < cb + wj) {
        chosen = X;
        wchosen = V[slot];
      }
    }
  } else if (!(thr < wstay)) {
    int64_t lo = -1, hi = INT32_MAX;  // wstay + C(lo) <= thr < wstay + C(hi)
    while (hi - lo > 1) {
      const int64_t mid = lo + (hi - lo) / 2;
      u128 c = 0;
      for (int64_t j = t; j < n; j += NT) {
        const int slot = cand ? cand[j] : (int)j;
        const ull wj = WT[slot];
        if (wj && K[slot] <= mid) c += wj;
      }
      c = team_sum_u128<NT>(c, mask, sm128);
      if (wstay + c > thr)
        hi = mid;
      else
        lo = mid;
    }
    // hi is a candidate's label; the team's first thread reports it
    if (t == 0) {
      chosen = (int32_t)hi;
      wchosen = table_get(K, V, bits, (int32_t)hi);
    }
  }
  // at most one thread holds the choice: hand it to every thread
  if (BLOCK) {
    if (chosen != INT32_MAX) sm128[0] = ((u128)(uint32_t)chosen << 64) | (u128)(ull)wchosen;
    __syncthreads();
    const u128 r = sm128[0];
    __syncthreads();
    if (r == ~(u128)0) {
      chosen = INT32_MAX;
      wchosen = 0;
    } else {
      chosen = (int32_t)(uint32_t)(r >> 64);
      wchosen = (long long)(ull)r;
    }
  } else {
    const unsigned hit = __ballot_sync(mask, chosen != INT32_MAX) & mask;
    if (hit) {
      const int src = __ffs(hit) - 1;
      chosen = __shfl_sync(mask, chosen, src);
      wchosen = __shfl_sync(mask, wchosen, src);
    }
  }
  Wb = wchosen;
  return chosen;
}

// Randomised decisions, degree tiers 0-2: G lanes per node, 2^BITS-slot
// tables per group in shared memory, with the weights beside them; the
// distinct target labels are listed as their slots are claimed, and only
// those slots are reset.  THREADS keeps the static tables within 48 KB per
// block.  All three tiers use a warp per node: most of a node's work is per
// candidate (a probe and an integer exponential), which a warp spreads over
// its lanes, and 4- or 8-lane groups were measured slower (refinement 74
// against 57 ms per solve of the power-law workload at theta = 1/100).
template <bool DENSE, int G, int BITS, int THREADS>
__global__ void __launch_bounds__(THREADS, 512 / THREADS)
    k_ref_random_groups(RefPolicy<DENSE> pol, const int32_t* list, const int32_t* count_ptr, RandParams rp) {
  constexpr int GPW = 32 / G, NG = (THREADS / 32) * GPW, SLOTS = 1 << BITS, MAXC = SLOTS / 2;
  __shared__ int32_t hk[NG][SLOTS];
  __shared__ long long hv[NG][SLOTS];
  __shared__ ull hw[NG][SLOTS];
  __shared__ uint16_t cl[NG][MAXC];
  __shared__ int32_t ncand[NG];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int gl = lane % G, gi = lane / G, gx = w * GPW + gi;
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (gi * G));
  int32_t* K = hk[gx];
  long long* V = hv[gx];
  ull* WT = hw[gx];
  uint16_t* CL = cl[gx];
  for (int i = gl; i < SLOTS; i += G) {
    K[i] = -1;
    V[i] = 0;
  }
  if (gl == 0) ncand[gx] = 0;
  __syncwarp(gmask);
  const int count = *count_ptr;
  for (int idx = blockIdx.x * NG + gx; idx < count; idx += gridDim.x * NG) {
    const int32_t v = list[idx];
    if (!pol.begin(v)) {
      if (gl == 0) pol.skip(v);
      continue;
    }
    const typename RefPolicy<DENSE>::VCtx vc = pol.vctx(v);
    for (int64_t e = pol.g.rowptr[v] + gl; e < pol.g.rowptr[v + 1]; e += G) {
      int32_t key;
      long long wgt;
      if (pol.edge(v, vc, e, key, wgt)) {
        bool fresh;
        const int slot = table_add_slot(K, V, BITS, key, wgt, fresh);
#if MSLICE_CHECKED
        if (slot < 0) atomicOr(pol.g.chk, ERR_BOUNDS);
#endif
        if (fresh) CL[atomicAdd(&ncand[gx], 1)] = (uint16_t)slot;
      }
    }
    __syncwarp(gmask);
    const int n = ncand[gx];
    long long Wb;
    const int32_t X =
        rand_choose<RefPolicy<DENSE>, G>(pol, v, vc, rp, K, V, WT, CL, n, BITS, gl, gi * G, gmask, nullptr, Wb);
    if (gl == 0) pol.finish(v, Cand{0, X}, Wb, 0, vc);
    __syncwarp(gmask);
    for (int j = gl; j < n; j += G) {
      const int slot = CL[j];
      K[slot] = -1;
      V[slot] = 0;
    }
    if (gl == 0) ncand[gx] = 0;
    __syncwarp(gmask);
  }
}

// Randomised decisions, tiers 3 and 4: one block per node, the table in
// shared memory (degree <= 1024) or in global scratch at goff[v].
template <bool DENSE>
__global__ void __launch_bounds__(256) k_ref_random_block(RefPolicy<DENSE> pol, const int32_t* list,
                                                          const int32_t* count_ptr, RandParams rp, int32_t* gkeys,
                                                          long long* gvals, ull* gwts, const int64_t* goff,
                                                          unsigned* status, int in_global) {
  constexpr int BITS = 11, SLOTS = 1 << BITS;
  __shared__ int32_t hk[SLOTS];
  __shared__ long long hv[SLOTS];
  __shared__ ull hw[SLOTS];
  __shared__ uint16_t cl[SLOTS / 2];
  __shared__ int32_t ncand;
  __shared__ u128 sm128[9];  // 8 warp partials, then staying's weight
  if (!in_global) {
    for (int i = threadIdx.x; i < SLOTS; i += 256) {
      hk[i] = -1;
      hv[i] = 0;
    }
    if (threadIdx.x == 0) ncand = 0;
    __syncthreads();
  }
  const int count = *count_ptr;
  for (int idx = blockIdx.x; idx < count; idx += gridDim.x) {
    const int32_t v = list[idx];
    if (!pol.begin(v)) {
      if (threadIdx.x == 0) pol.skip(v);
      continue;
    }
    const typename RefPolicy<DENSE>::VCtx vc = pol.vctx(v);
    const int64_t beg = pol.g.rowptr[v], end = pol.g.rowptr[v + 1];
    long long Wb;
    int32_t X;
    if (!in_global) {
      const int bits = table_bits_for_degree(end - beg);
      for (int64_t e = beg + threadIdx.x; e < end; e += 256) {
        int32_t key;
        long long wgt;
        if (pol.edge(v, vc, e, key, wgt)) {
          bool fresh;
          const int slot = table_add_slot(hk, hv, bits, key, wgt, fresh);
#if MSLICE_CHECKED
          if (slot < 0) atomicOr(pol.g.chk, ERR_BOUNDS);
#endif
          if (fresh) cl[atomicAdd(&ncand, 1)] = (uint16_t)slot;
        }
      }
      __syncthreads();
      const int n = ncand;
      X = rand_choose<RefPolicy<DENSE>, 256>(pol, v, vc, rp, hk, hv, hw, cl, n, bits, threadIdx.x, 0, 0xffffffffu,
                                             sm128, Wb);
      if (threadIdx.x == 0) pol.finish(v, Cand{0, X}, Wb, 0, vc);
      __syncthreads();
      for (int j = threadIdx.x; j < n; j += 256) {
        const int slot = cl[j];
        hk[slot] = -1;
        hv[slot] = 0;
      }
      if (threadIdx.x == 0) ncand = 0;
      __syncthreads();
    } else {
      const int bits = table_bits_for_degree(end - beg);
      const int64_t S = 1ll << bits;
      int32_t* K = gkeys + goff[v];
      long long* V = gvals + goff[v];
      ull* WT = gwts + goff[v];
      for (int64_t i = threadIdx.x; i < S; i += 256) {
        K[i] = -1;
        V[i] = 0;
      }
      __syncthreads();
      for (int64_t e = beg + threadIdx.x; e < end; e += 256) {
        int32_t key;
        long long wgt;
        if (pol.edge(v, vc, e, key, wgt)) gtable_add(K, V, bits, key, wgt, status);
      }
      __syncthreads();
      X = rand_choose<RefPolicy<DENSE>, 256>(pol, v, vc, rp, K, V, WT, nullptr, S, bits, threadIdx.x, 0, 0xffffffffu,
                                             sm128, Wb);
      if (threadIdx.x == 0) pol.finish(v, Cand{0, X}, Wb, 0, vc);
      __syncthreads();
    }
  }
}

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
// Nodes of tiers [T0, T1) of a sub-round's segments.
template <int T0, int T1>
__device__ __forceinline__ int seg3_total_in(const Segs3& sg) {
  int t = 0;
#pragma unroll
  for (int i = T0; i < T1; ++i) t += *sg.count[i];
  return t;
}
template <int T0, int T1>
__device__ __forceinline__ bool seg3_item_in(const Segs3& sg, int64_t idx, int32_t& v) {
#pragma unroll
  for (int t = T0; t < T1; ++t) {
    const int cnt = *sg.count[t];
    if (idx < cnt) {
      v = sg.list[t][idx];
      return true;
    }
    idx -= cnt;
  }
  return false;
}

// Applies the sub-round's refinement moves of tiers [T0, T1): G lanes per
// node (8 for the short rows of the low tiers, a warp otherwise).
template <int G, int T0, int T1>
__global__ void k_ref_apply(LevelDev g, Segs3 sg, const int32_t* P, const int32_t* target, const long long* Wc,
                            const long long* Wsel, int32_t* R, int32_t* sizeR, long long* Wout, SigStore kr,
                            long long* PR) {
  const int lane = threadIdx.x & 31, gl = lane % G;
  const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane - gl));
  const int total = seg3_total_in<T0, T1>(sg);
  const int64_t groups = ((int64_t)gridDim.x * blockDim.x) / G;
  // every lane of a warp runs the same number of iterations (shuffles below)
  const int64_t first = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t warp_first = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) / G;
  for (int64_t i0 = warp_first; i0 < total; i0 += groups) {
    const int64_t idx = i0 + (first - warp_first);
    int32_t v = 0, t = NO_MOVE;
    if (idx < total && seg3_item_in<T0, T1>(sg, idx, v)) t = target[v];
    long long wp = 0;
    if (t >= 0) {
      const Omega om = node_omega(g, v);
      for (int64_t e = g.rowptr[v] + gl; e < g.rowptr[v + 1]; e += G) {
        int32_t u;
        long long W;
        // a target lies in the mover's own community, so target[u] == t
        // implies P[u] == P[v]
        if (edge_at(g, e, u, W, om) && target[u] == t) wp += W;
      }
    }
#pragma unroll
    for (int m = G / 2; m >= 1; m >>= 1) wp += __shfl_xor_sync(gmask, wp, m);
    if (t < 0) continue;
    if (gl == 0) {
      R[v] = t;
      PR[v] = (long long)(((unsigned long long)(uint32_t)P[v] << 32) | (uint32_t)t);
      atomicSub(&sizeR[v], 1);
      atomicAdd(&sizeR[t], 1);
      atomicAdd((ull*)&Wout[t], (ull)(Wc[v] - 2 * Wsel[v] - wp));
      Wout[v] = 0;
    }
    // the sub-community rows take the node's list: by the group when long
    int64_t b, e;
    slice_range(g, v, b, e);
    const bool wide = e - b > G;
    if (wide || gl == 0)
      for (int64_t j = b + (wide ? gl : 0); j < e; j += (wide ? G : 1)) {
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

// Launches the randomised decisions of one sub-round: the tiers decide
// disjoint nodes with separate scratch, so they run concurrently, heaviest
// first, each on its own side stream (as the greedy tiers do).
template <bool DENSE>
static void random_all(Solver& S, const RefPolicy<DENSE>& pol, const TierSegs& sg, const RandParams& rp) {
  Ctx& c = *S.c;
  const int32_t* cnt = S.tier_cnt;
  StreamFan* f = c.fan;
  cudaStream_t st[NTIERS] = {c.stream, c.stream, c.stream, c.stream, c.stream};
  bool used[StreamFan::kSide] = {false, false, false, false};
  if (f) {
    int busy = 0;
    for (int t = 0; t < NTIERS; ++t) busy += cnt[t] > 0;
    if (busy > 1) {
      check_cuda(cudaEventRecord(f->fork, c.stream), "event");
      for (int t = NTIERS - 1; t >= 1; --t)
        if (cnt[t] > 0) {
          const int k = NTIERS - 1 - t;
          check_cuda(cudaStreamWaitEvent(f->side[k], f->fork, 0), "event");
          st[t] = f->side[k];
          used[k] = true;
        }
    }
  }
  for (int t = NTIERS - 1; t >= 3; --t)
    if (cnt[t] > 0)
      launch_on(c, st[t], k_ref_random_block<DENSE>, dim3(152 * 4), dim3(256), 0, pol, sg.list[t], sg.count[t], rp,
                S.gkeys, S.gvals, S.gwts, (const int64_t*)S.goff, c.d_status, (int)(t == NTIERS - 1));
  if (cnt[2] > 0)
    launch_on(c, st[2], k_ref_random_groups<DENSE, 32, 9, 128>, dim3(152 * 8), dim3(128), 0, pol, sg.list[2],
              sg.count[2], rp);
  if (cnt[1] > 0)
    launch_on(c, st[1], k_ref_random_groups<DENSE, 32, 9, 128>, dim3(152 * 8), dim3(128), 0, pol, sg.list[1],
              sg.count[1], rp);
  if (cnt[0] > 0)
    launch_on(c, st[0], k_ref_random_groups<DENSE, 32, 9, 128>, dim3(152 * 8), dim3(128), 0, pol, sg.list[0],
              sg.count[0], rp);
  for (int k = 0; k < StreamFan::kSide; ++k)
    if (used[k]) {
      check_cuda(cudaEventRecord(f->join[k], f->side[k]), "event");
      check_cuda(cudaStreamWaitEvent(c.stream, f->join[k], 0), "event");
    }
}

template <bool DENSE>
static void refine_impl(Solver& S, const Level& L, const int32_t* P, int it, int lvl) {
  Ctx& c = *S.c;
  const int32_t N = L.d.N;
  if (N == 0) return;
  clear_store(S, S.kr);
  long long* PR = c.ws->get<long long>("ref_PR", N);
  if (L.d.is0)
    launch(c, k_ref_init<8>, dim3(fixed_grid(8)), dim3(256), 0, L.d, P, S.sig, (const u128*)S.lam, S.R, S.sizeR,
           S.Wc, S.Wout, S.elig, S.kr, PR);
  else
    launch(c, k_ref_init<32>, dim3(fixed_grid(8)), dim3(256), 0, L.d, P, S.sig, (const u128*)S.lam, S.R, S.sizeR,
           S.Wc, S.Wout, S.elig, S.kr, PR);
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
    if (S.p.theta_num > 0) {
      random_all<DENSE>(S, pol, sg, RandParams{S.p.seed, (uint64_t)it, (uint64_t)lvl, S.rdiv, (ull)S.p.theta_den});
    } else {
      decide_all(c, pol, sg, S.tier_cnt, S.gkeys, S.gvals, S.goff);
    }
    launch(c, k_ref_apply<8, 0, 2>, dim3(fixed_grid(8)), dim3(256), 0, L.d, sg, P, (const int32_t*)S.target,
           (const long long*)S.Wc, (const long long*)S.Wsel, S.R, S.sizeR, S.Wout, S.kr, PR);
    launch(c, k_ref_apply<32, 2, NTIERS>, dim3(fixed_grid(8)), dim3(256), 0, L.d, sg, P, (const int32_t*)S.target,
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
