// Multislice-Leiden ORACLE -- test infrastructure only (see oracle.h).
//
// Plain single-threaded C++: std::map / std::vector containers, no blocking,
// no fusion, no parallelism.  Each function names the passage of the paper
// ("Accelerating Dynamic Graph Clustering on GPU Architectures with cuGraph")
// that it follows; where the paper is silent, the comment states the reading
// this implementation takes.
//
// Units.  Integer edge weights w >= 1 and rationals gamma = gn/gd,
// omega = on/od.  An adjacency weight W is kept in units of 1/od: an
// intra-slice edge of weight w counts od*w, a coupling edge counts on.
// Node strengths k, community sums Sigma and 2m_s are raw (unscaled) sums of
// intra-slice weights, as in the null term of Eq. multislice-modularity.
#include "oracle.h"

#include <algorithm>
#include <cstring>
#include <map>
#include <vector>

typedef __int128 i128;
typedef unsigned __int128 u128;

namespace {

const int P_BITS = 64;  // quantisation exponent P of the null coefficient

// ---------------------------------------------------------------------------
// Counter-based hash: the SplitMix64 output finaliser (Steele, Lea & Flood,
// "Fast splittable pseudorandom number generators", OOPSLA 2014), written
// from its published definition.
uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

// Vertex class of node v for (seed, tag, iteration, level, round) (reading:
// the synchronous schedule draws one class in [0, K) per node and round from
// a counter-based hash; tag 0 = local moving, 1 = refinement).
int vertex_class(uint64_t seed, uint64_t tag, uint64_t it, uint64_t lvl, uint64_t r, uint64_t v, int K) {
  uint64_t h = mix64(seed ^ mix64(tag ^ mix64(it ^ mix64(lvl ^ mix64(r ^ mix64(v))))));
  return (int)(h % (uint64_t)K);
}

// ---------------------------------------------------------------------------
// A level of the optimisation: nodes, symmetric weighted adjacency (no
// self-loops) and per-node slice-strength vectors k_{v,s} (only k > 0 kept).
struct Level {
  int64_t N = 0;
  std::vector<std::vector<std::pair<int32_t, int64_t>>> adj;   // (u, W) sorted by u
  std::vector<std::vector<std::pair<int32_t, int64_t>>> kvec;  // (s, k) sorted by s
  int64_t nnz() const {
    int64_t t = 0;
    for (const auto& a : adj) t += (int64_t)a.size();
    return t;
  }
};

// Null models.  ORC_NULL_MULTISLICE: the per-slice null term of Eq.
// multislice-modularity.  ORC_NULL_GLOBAL: plain modularity (Eq. modularity)
// on the supra-adjacency of Eq. supra-adjacency, the proxy Sec. 3.2 runs with
// cuGraph's Leiden: coupling edges count in the degrees and one null term
// covers the whole supra-graph.  For the global model the strengths and sums
// below are kept in units of 1/od (k' = od*k + on*c, c = the node's coupling
// edges), the null "slice" is single (index 0) and the key's null scale is 1
// instead of od.
// ORC_NULL_CPM: the temporal Constant Potts Model Sec. 3.2 names as an
// alternative quality function on the supra-graph (Traag et al.): the null
// term of snapshot s is gamma_s per ordered pair of its nodes, i.e. Eq.
// multislice-modularity with every node's null strength 1 and 2m_s replaced
// by 1.  So every node has the entry (s, 1), the null slices are the
// snapshots with mass 1, Lambda_s = floor(gamma_s 2^P), and the key's null
// scale stays od.
//
// General coupling (the omega^(sr) and gamma^(s) of Eq. multislice-modularity):
// omega^(sr) = cw[pair]/od, with pair = min(s,r) for ORDINAL coupling (only
// |s-r| = 1 coupled) and pair = s*T + r for CATEGORICAL coupling (every pair
// s != r).  Without a table every coupled pair has numerator on.  gamma^(s)
// = gsn[s]/gsd[s], or gn/gd for every slice without a table.  cstr[s] is the
// coupling strength of one node of slice s, sum_r omega_num^(sr).
struct Problem {
  int32_t T = 0;
  int64_t n = 0;
  int64_t gn = 1, gd = 1, on = 1, od = 1;
  int32_t coupling = ORC_ORDINAL;
  bool omega_table = false;
  std::vector<int64_t> cw;
  bool gamma_table = false;
  std::vector<int64_t> gsn, gsd;
  std::vector<int64_t> cstr;
  int64_t twoM_all = 0;  // od * 2mu: od*sum(2m_s) + n*sum_s cstr[s]
  int32_t null_model = ORC_NULL_MULTISLICE;
  int64_t ns = 1;              // null scale of the key: od (multislice) or 1 (global)
  std::vector<int64_t> two_m;  // 2m_s of every snapshot
  std::vector<int64_t> two_m_null;  // masses of the null slices: 2m_s, or {2M'} (global)
  std::vector<u128> lambda;    // Lambda of every null slice
};

bool valid_rational(int64_t num, int64_t den, bool allow_zero) {
  const int64_t lim = (int64_t)1 << 31;
  if (den < 1 || den > lim) return false;
  if (num < (allow_zero ? 0 : 1) || num > lim) return false;
  return true;
}

// Numerator of omega^(sr) over od (0 when s and r are not coupled).
int64_t coupling_num(const Problem& p, int32_t s, int32_t r) {
  if (s == r) return 0;
  if (p.coupling == ORC_ORDINAL) return (s - r == 1 || r - s == 1) ? p.cw[std::min(s, r)] : 0;
  return p.cw[(int64_t)s * p.T + r];
}

// The coupling table and the per-slice resolutions from the optional
// general specification (EINVAL for a bad one).
int setup_general(const orc_general* g, Problem& p) {
  const int32_t T = p.T;
  p.coupling = g ? g->coupling : ORC_ORDINAL;
  if (p.coupling != ORC_ORDINAL && p.coupling != ORC_CATEGORICAL) return ORC_EINVAL;
  const int64_t npairs = p.coupling == ORC_ORDINAL ? (T > 1 ? T - 1 : 0) : (int64_t)T * T;
  p.omega_table = g && g->omega_num;
  p.cw.assign(npairs, p.on);
  if (p.coupling == ORC_CATEGORICAL)
    for (int32_t s = 0; s < T; ++s) p.cw[(int64_t)s * T + s] = 0;
  if (p.omega_table) {
    for (int64_t q = 0; q < npairs; ++q) {
      if (!valid_rational(g->omega_num[q], p.od, true)) return ORC_EINVAL;
      p.cw[q] = g->omega_num[q];
    }
    if (p.coupling == ORC_CATEGORICAL)
      for (int32_t s = 0; s < T; ++s) {
        if (p.cw[(int64_t)s * T + s] != 0) return ORC_EINVAL;
        for (int32_t r = 0; r < s; ++r)
          if (p.cw[(int64_t)s * T + r] != p.cw[(int64_t)r * T + s]) return ORC_EINVAL;
      }
  }
  p.gamma_table = g && (g->gamma_num || g->gamma_den);
  p.gsn.assign(T, p.gn);
  p.gsd.assign(T, p.gd);
  if (p.gamma_table) {
    if (!g->gamma_num || !g->gamma_den) return ORC_EINVAL;
    if (p.null_model == ORC_NULL_GLOBAL) return ORC_EINVAL;  // one null term: one resolution
    for (int32_t s = 0; s < T; ++s) {
      if (!valid_rational(g->gamma_num[s], g->gamma_den[s], false)) return ORC_EINVAL;
      p.gsn[s] = g->gamma_num[s];
      p.gsd[s] = g->gamma_den[s];
    }
  }
  p.cstr.assign(T, 0);
  for (int32_t s = 0; s < T; ++s)
    for (int32_t r = 0; r < T; ++r) p.cstr[s] += coupling_num(p, s, r);
  return ORC_OK;
}

// Input validation (reading: the paper takes simple undirected snapshots; this
// implementation rejects self-loops, duplicates, asymmetric entries and
// weights < 1, and requires every snapshot to have the same n).
int validate(const orc_csr* slices, int32_t T) {
  if (T < 1 || slices == nullptr) return ORC_EINVAL;
  int64_t n = slices[0].n;
  if (n < 0 || n > ((int64_t)1 << 31) - 1) return ORC_EINVAL;
  if (n * (int64_t)T > ((int64_t)1 << 31) - 1) return ORC_EINVAL;
  for (int32_t s = 0; s < T; ++s) {
    const orc_csr& A = slices[s];
    if (A.n != n) return ORC_EINVAL;
    if (n > 0 && A.indptr == nullptr) return ORC_EINVAL;
    if (n == 0) continue;
    if (A.indptr[0] != 0) return ORC_EINVAL;
    for (int64_t i = 0; i < n; ++i)
      if (A.indptr[i + 1] < A.indptr[i]) return ORC_EINVAL;
    for (int64_t i = 0; i < n; ++i) {
      for (int64_t e = A.indptr[i]; e < A.indptr[i + 1]; ++e) {
        int32_t j = A.indices[e];
        if (j < 0 || j >= n || j == i) return ORC_EINVAL;
        if (e > A.indptr[i] && A.indices[e - 1] >= j) return ORC_EINVAL;
        if (A.weights[e] < 1) return ORC_EINVAL;
        // symmetric: entry (j, i) with the same weight
        const int32_t* b = A.indices + A.indptr[j];
        const int32_t* en = A.indices + A.indptr[j + 1];
        const int32_t* f = std::lower_bound(b, en, (int32_t)i);
        if (f == en || *f != i) return ORC_EINVAL;
        if (A.weights[A.indptr[j] + (f - b)] != A.weights[e]) return ORC_EINVAL;
      }
    }
  }
  return ORC_OK;
}

// 2m_s and the quantised null coefficients
//   Lambda_s = floor(gn * 2^P / (gd * 2m_s))   (0 for an edgeless slice).
// Reading: with per-slice denominators 2m_s, an exact comparison of gains of
// multi-slice nodes would need lcm(2m_s); both implementations instead
// compare keys built from Lambda_s, i.e. they optimise Q_MS with
// gamma'_s = Lambda_s*2m_s/2^P, within 2m_s/2^64 of gamma (relative).
// Global model: one null slice of mass 2M' = od*sum(2m_s) + n*sum_s cstr[s]
// (the supra-graph's total weight in units of 1/od) and
//   Lambda' = floor(gn * 2^P / (gd * 2M')).
// Per-slice resolutions: Lambda_s = floor(gsn[s] * 2^P / (gsd[s] * 2m_s)).
void slice_masses(const orc_csr* slices, Problem& p) {
  p.two_m.assign(p.T, 0);
  for (int32_t s = 0; s < p.T; ++s) {
    int64_t t = 0;
    for (int64_t e = 0; e < (p.n > 0 ? slices[s].indptr[p.n] : 0); ++e) t += slices[s].weights[e];
    p.two_m[s] = t;
  }
  {
    int64_t sum2m = 0, csum = 0;
    for (int64_t t : p.two_m) sum2m += t;
    for (int64_t c : p.cstr) csum += c;
    p.twoM_all = p.od * sum2m + p.n * csum;
  }
  if (p.null_model == ORC_NULL_GLOBAL) {
    int64_t sum2m = 0;
    for (int64_t t : p.two_m) sum2m += t;
    int64_t csum = 0;
    for (int64_t c : p.cstr) csum += c;
    p.two_m_null.assign(1, p.od * sum2m + p.n * csum);
    p.ns = 1;
  } else if (p.null_model == ORC_NULL_CPM) {
    p.two_m_null.assign(p.T, 1);
    p.ns = p.od;
  } else {
    p.two_m_null = p.two_m;
    p.ns = p.od;
  }
  p.lambda.assign(p.two_m_null.size(), 0);
  const bool global = p.null_model == ORC_NULL_GLOBAL;
  for (size_t s = 0; s < p.two_m_null.size(); ++s) {
    const int64_t t = p.two_m_null[s];
    const int64_t num = global ? p.gn : p.gsn[s], den = global ? p.gd : p.gsd[s];
    if (t > 0) p.lambda[s] = (((u128)(uint64_t)num) << P_BITS) / ((u128)(uint64_t)den * (u128)(uint64_t)t);
  }
}

// Overflow guard: every key below stays inside a signed 128-bit integer when
//   2M' = od*sum(2m_s) + n*sum_s cstr[s] < 2^61   and   gamma_s*od*sum(2m_s) < 2^61
// for every s (gamma*2M' < 2^61 for the global model, whose strengths include
// the coupling; gamma_s*od*n*N < 2^61 for CPM, whose null sums count nodes:
// sum_s k_{v,s} Sigma_{c,s} <= N*n).
int check_bounds(const Problem& p) {
  u128 sum2m = 0;
  for (int64_t t : p.two_m) sum2m += (u128)(uint64_t)t;
  u128 csum = 0;
  for (int64_t c : p.cstr) csum += (u128)(uint64_t)c;
  u128 lim = (u128)1 << 61;
  const u128 twoM = (u128)(uint64_t)p.od * sum2m + (u128)(uint64_t)p.n * csum;
  if (twoM >= lim) return ORC_EOVERFLOW;
  if (p.null_model == ORC_NULL_GLOBAL) {
    if ((u128)(uint64_t)p.gn * twoM >= lim * (u128)(uint64_t)p.gd) return ORC_EOVERFLOW;
    return ORC_OK;
  }
  const u128 mass = p.null_model == ORC_NULL_CPM ? (u128)(uint64_t)p.n * (u128)(uint64_t)(p.n * p.T) : sum2m;
  for (int32_t s = 0; s < p.T; ++s)
    if ((u128)(uint64_t)p.gsn[s] * (u128)(uint64_t)p.od * mass >= lim * (u128)(uint64_t)p.gsd[s])
      return ORC_EOVERFLOW;
  return ORC_OK;
}

// Level 0: the supra-graph of Eq. supra-adjacency.  Supra-node v = s*n + i.
// Intra-slice edge (i,j) of snapshot s -> (s*n+i, s*n+j) with W = od*w.
// Coupling (i,s)-(i,r) with W = omega_num^(sr), omitted when that is 0:
// ordinal r = s-1 and s+1 with W = on unless a table is given; categorical
// every r != s.
Level build_level0(const orc_csr* slices, const Problem& p) {
  Level L;
  L.N = p.n * p.T;
  L.adj.assign(L.N, {});
  L.kvec.assign(L.N, {});
  for (int32_t s = 0; s < p.T; ++s) {
    for (int64_t i = 0; i < p.n; ++i) {
      int64_t v = (int64_t)s * p.n + i;
      auto& a = L.adj[v];
      for (int32_t r = 0; r < s; ++r)
        if (coupling_num(p, s, r) > 0) a.push_back({(int32_t)((int64_t)r * p.n + i), coupling_num(p, s, r)});
      int64_t k = 0;
      for (int64_t e = slices[s].indptr[i]; e < slices[s].indptr[i + 1]; ++e) {
        a.push_back({(int32_t)((int64_t)s * p.n + slices[s].indices[e]), p.od * (int64_t)slices[s].weights[e]});
        k += slices[s].weights[e];
      }
      for (int32_t r = s + 1; r < p.T; ++r)
        if (coupling_num(p, s, r) > 0) a.push_back({(int32_t)((int64_t)r * p.n + i), coupling_num(p, s, r)});
      if (p.null_model == ORC_NULL_GLOBAL) {
        // k' = od*k + (coupling strength of v), one null slice
        const int64_t kp = p.od * k + p.cstr[s];
        if (kp > 0) L.kvec[v].push_back({0, kp});
      } else if (p.null_model == ORC_NULL_CPM) {
        L.kvec[v].push_back({s, 1});  // every node weighs 1 in its snapshot's null term
      } else if (k > 0) {
        L.kvec[v].push_back({s, k});
      }
    }
  }
  return L;
}

// Sum_s Lambda_s * k_{v,s} * X_s over the slices of v, where X_s is supplied by
// `get` (a community or sub-community slice sum).
template <class F>
u128 null_sum(const Problem& p, const std::vector<std::pair<int32_t, int64_t>>& kv, F get) {
  u128 t = 0;
  for (const auto& sk : kv) {
    int64_t x = get(sk.first);
    t += p.lambda[sk.first] * (u128)(uint64_t)sk.second * (u128)(uint64_t)x;
  }
  return t;
}

// Exact move key (Eq. multislice-modularity; the change of Q_MS when v joins
// community c is 2/(2mu) * [g(v,c) - g(v,a)] with
//   g(v,c) = W(v,c\v)/od - sum_s gamma k_{v,s} Sigma_{c\v,s} / 2m_s).
// Scaled by od*2^P and with gamma/2m_s quantised to Lambda_s/2^P:
//   G(v,c) = 2^P W(v,c\v) - od * sum_s Lambda_s k_{v,s} Sigma_{c\v,s}.
// Global model (Eq. modularity on the supra-graph, all in units of 1/od):
// g(v,c) = W(v,c\v) - gamma k'_v Sigma'_{c\v} / 2M', so
//   G(v,c) = 2^P W(v,c\v) - Lambda' k'_v Sigma'_{c\v}   (null scale 1).
i128 key(const Problem& p, int64_t W, u128 nullsum) {
  return (((i128)W) << P_BITS) - (i128)((u128)(uint64_t)p.ns * nullsum);
}

typedef std::map<int32_t, int64_t> SliceMap;  // slice -> sum

// ---------------------------------------------------------------------------
// Local moving (Louvain/Leiden move phase, Sec. 3.2) under the synchronous
// schedule.  Reading (the paper gives none): in round r, sub-round q, every
// node whose class is q decides against the state at the start of the
// sub-round; then all decisions are applied at once.
struct MoveResult {
  int64_t rounds = 0, moves = 0, first_round_moves = 0;
};

const int32_t NO_MOVE = -1;
const int32_t TO_EMPTY = -2;

MoveResult local_move(const Level& G, const Problem& p, const orc_opts& o, std::vector<int32_t>& c, int it, int lvl,
                      int max_rounds, orc_stats* st) {
  MoveResult res;
  const int64_t N = G.N;
  std::vector<int64_t> size(N, 0);
  for (int64_t v = 0; v < N; ++v) size[c[v]]++;
  std::vector<SliceMap> Sigma(N);  // Sigma[c][s]
  for (int64_t v = 0; v < N; ++v)
    for (const auto& sk : G.kvec[v]) Sigma[c[v]][sk.first] += sk.second;
  auto sig = [&](int32_t comm, int32_t s) -> int64_t {
    auto it2 = Sigma[comm].find(s);
    return it2 == Sigma[comm].end() ? 0 : it2->second;
  };
  const int64_t nnz = G.nnz();
  for (int r = 0; r < max_rounds; ++r) {
    int64_t moved = 0;
    res.rounds++;
    if (st) {
      st->lm_rounds++;
      st->lm_edges += nnz;
    }
    for (int q = 0; q < o.K; ++q) {
      std::vector<int32_t> target(N, NO_MOVE);
      // ---- decide (reads the sub-round snapshot only) ----
      for (int64_t v = 0; v < N; ++v) {
        if (vertex_class(o.seed, 0, it, lvl, r, v, o.K) != q) continue;
        const int32_t a = c[v];
        std::map<int32_t, int64_t> Wmap;  // neighbour community -> W(v, c)
        for (const auto& uw : G.adj[v]) Wmap[c[uw.first]] += uw.second;
        const int64_t Wa = Wmap.count(a) ? Wmap[a] : 0;
        const i128 Ga = key(p, Wa, null_sum(p, G.kvec[v], [&](int32_t s) {
                              int64_t kvs = 0;
                              for (const auto& sk : G.kvec[v])
                                if (sk.first == s) kvs = sk.second;
                              return sig(a, s) - kvs;  // Sigma_{a\v,s}
                            }));
        int32_t best = a;
        i128 Gbest = Ga;
        for (const auto& cw : Wmap) {  // ascending community label
          if (cw.first == a) continue;
          const i128 Gc = key(p, cw.second, null_sum(p, G.kvec[v], [&](int32_t s) { return sig(cw.first, s); }));
          if (Gc > Gbest || (Gc == Gbest && cw.first < best)) {
            best = cw.first;
            Gbest = Gc;
          }
        }
        // An empty community (key 0) is a candidate when v is not alone; it
        // ranks after every label on ties.
        if (size[a] > 1 && Gbest < 0) {
          best = TO_EMPTY;
          Gbest = 0;
        }
        if (!(Gbest > Ga)) continue;  // strict improvement only
        // Singleton-swap guard: a node alone in its community moves into
        // another singleton community only if that label is smaller.
        if (size[a] == 1 && best != TO_EMPTY && size[best] == 1 && best > a) continue;
        target[v] = best;
      }
      // ---- apply ----
      int64_t n_moves = 0;
      for (int64_t v = 0; v < N; ++v) {
        if (target[v] < 0) continue;
        const int32_t a = c[v], b = target[v];
        size[a]--;
        size[b]++;
        for (const auto& sk : G.kvec[v]) {
          Sigma[a][sk.first] -= sk.second;
          Sigma[b][sk.first] += sk.second;
        }
        c[v] = b;
        n_moves++;
      }
      // Moves to an empty community: in ascending node order, the ascending
      // labels that are unused once every other move is applied and the
      // movers themselves have left (reading; the paper is silent).
      std::vector<int64_t> empties;
      for (int64_t v = 0; v < N; ++v) {
        if (target[v] != TO_EMPTY) continue;
        const int32_t a = c[v];
        size[a]--;
        for (const auto& sk : G.kvec[v]) Sigma[a][sk.first] -= sk.second;
        empties.push_back(v);
      }
      if (!empties.empty()) {
        int32_t L = 0;
        for (int64_t v : empties) {
          while (size[L] != 0) ++L;
          c[v] = L;
          size[L] = 1;
          for (const auto& sk : G.kvec[v]) Sigma[L][sk.first] += sk.second;
          ++L;
          n_moves++;
        }
      }
      moved += n_moves;
    }
    res.moves += moved;
    if (r == 0) res.first_round_moves = moved;
    if (st) st->lm_moves += moved;
    if (moved == 0) break;
  }
  return res;
}

// ---------------------------------------------------------------------------
// Randomised refinement (Traag et al. 2019: a node joins a target X with
// probability proportional to exp(dH_X / theta) among the targets with
// dH_X >= 0, staying alone included).  Reading: with the exact keys G (the
// gain dQ = 2G / (2^P od 2mu)), the weight of a candidate c is
//   E(Gmax - G_c) ~= 2^40 exp(-(Gmax - G_c) / (2^(P-1) od 2mu theta)),
// evaluated by one fixed-point integer recipe (so every implementation gets
// the same bits):
//   Y  = floor(d / (2M * theta_num))            (2M = od*2mu, an integer)
//   yF = floor(Y * theta_den / 2^31)            (y = d/(2^63 2M theta), Q32)
//   u  = yF * LOG2E                             (y log2 e, Q64; LOG2E = round(log2(e) 2^32))
//   I  = floor(u / 2^64), f = u mod 2^64        (2^-y log2e = 2^-I 2^-(f/2^64))
//   g  = floor(f * LN2 / 2^64)                  (f ln 2, Q62; LN2 = round(ln 2 * 2^62))
//   e^-g by its Taylor series in Q62 (term_k = floor(term_{k-1} g / 2^62) / k,
//   alternating signs, stopping when a term is 0)
//   E  = floor(e^-g / 2^(22 + I))               (Q40); 0 when Y >= 2^96, yF >= 64*2^32 or I >= 40.
// The draw: R = the class hash's 64-bit value for (seed, tag 2, it, level,
// round 0, node) shifted right by 32; the threshold floor(R * total / 2^32)
// picks the first candidate, in the order stay, then ascending label, whose
// cumulative weight exceeds it.
const uint64_t LOG2E_Q32 = 6196328019ull;
const uint64_t LN2_Q62 = 3196577161300663915ull;

uint64_t exp_weight(u128 d, u128 div, uint64_t td) {
  const u128 Y = d / div;
  if (Y >> 96) return 0;
  const u128 yF = (Y * (u128)td) >> 31;
  if (yF >= ((u128)64 << 32)) return 0;
  const u128 u = yF * (u128)LOG2E_Q32;
  const uint64_t I = (uint64_t)(u >> 64);
  if (I >= 40) return 0;
  const uint64_t f = (uint64_t)u;
  const u128 g = ((u128)f * (u128)LN2_Q62) >> 64;
  u128 term = (u128)1 << 62;
  i128 sum = (i128)term;
  for (int k = 1; k <= 40; ++k) {
    term = ((term * g) >> 62) / (u128)k;
    if (term == 0) break;
    sum += (k & 1) ? -(i128)term : (i128)term;
  }
  return (uint64_t)((u128)sum >> (22 + I));
}

uint64_t class_hash(uint64_t seed, uint64_t tag, uint64_t it, uint64_t lvl, uint64_t r, uint64_t v) {
  return mix64(seed ^ mix64(tag ^ mix64(it ^ mix64(lvl ^ mix64(r ^ mix64(v))))));
}

// ---------------------------------------------------------------------------
// Refinement (Leiden, Sec. 3.2; Traag et al. 2019, refinement phase) in the
// greedy limit (theta = 0; theta > 0: randomised, above).  Inside each local-moving community C every node starts as
// its own sub-community; one pass of K sub-rounds (class tag 1, round 0).
// A node still alone in its sub-community and well connected to C joins the
// well-connected sub-community R of C with the largest positive key
//   2^P W(v,R) - od * sum_s Lambda_s k_{v,s} K_{R,s}
// (ties -> smallest label).  A singleton sub-community whose node is active
// in the same sub-round is not a target.  Well-connectedness of a set X in C:
//   2^P W(X, C\X) >= od * sum_s Lambda_s K_{X,s} (K_{C,s} - K_{X,s}).
std::vector<int32_t> refine(const Level& G, const Problem& p, const orc_opts& o, const std::vector<int32_t>& P, int it,
                            int lvl) {
  const int64_t N = G.N;
  std::vector<int32_t> R(N);
  for (int64_t v = 0; v < N; ++v) R[v] = (int32_t)v;
  std::vector<SliceMap> KC(N);  // K_{C,s} of local-moving communities
  for (int64_t v = 0; v < N; ++v)
    for (const auto& sk : G.kvec[v]) KC[P[v]][sk.first] += sk.second;
  auto kc = [&](int32_t C, int32_t s) -> int64_t {
    auto f = KC[C].find(s);
    return f == KC[C].end() ? 0 : f->second;
  };
  std::vector<int64_t> Wc(N, 0);  // W(v, C\v)
  for (int64_t v = 0; v < N; ++v)
    for (const auto& uw : G.adj[v])
      if (P[uw.first] == P[v]) Wc[v] += uw.second;

  for (int q = 0; q < o.K; ++q) {
    // snapshot statistics, recomputed from scratch
    std::vector<int64_t> sizeR(N, 0), Wout(N, 0), member(N, -1);
    std::vector<SliceMap> KR(N);
    std::vector<int32_t> PofR(N, -1);
    for (int64_t v = 0; v < N; ++v) {
      sizeR[R[v]]++;
      member[R[v]] = v;
      PofR[R[v]] = P[v];
      for (const auto& sk : G.kvec[v]) KR[R[v]][sk.first] += sk.second;
      for (const auto& uw : G.adj[v])
        if (P[uw.first] == P[v] && R[uw.first] != R[v]) Wout[R[v]] += uw.second;
    }
    auto kr = [&](int32_t X, int32_t s) -> int64_t {
      auto f = KR[X].find(s);
      return f == KR[X].end() ? 0 : f->second;
    };
    std::vector<char> wc(N, 0);
    for (int64_t X = 0; X < N; ++X) {
      if (sizeR[X] == 0) continue;
      u128 rhs = 0;
      for (const auto& sk : KR[X])
        rhs += p.lambda[sk.first] * (u128)(uint64_t)sk.second * (u128)(uint64_t)(kc(PofR[X], sk.first) - sk.second);
      wc[X] = key(p, Wout[X], rhs) >= 0;
    }
    std::vector<int32_t> target(N, NO_MOVE);
    for (int64_t v = 0; v < N; ++v) {
      if (vertex_class(o.seed, 1, it, lvl, 0, v, o.K) != q) continue;
      if (sizeR[R[v]] != 1) continue;
      const int32_t C = P[v];
      // v alone: well connected iff 2^P W(v,C\v) >= od sum Lambda k (K_C - k)
      u128 rhs = 0;
      for (const auto& sk : G.kvec[v])
        rhs += p.lambda[sk.first] * (u128)(uint64_t)sk.second * (u128)(uint64_t)(kc(C, sk.first) - sk.second);
      if (key(p, Wc[v], rhs) < 0) continue;
      std::map<int32_t, int64_t> Wmap;
      for (const auto& uw : G.adj[v])
        if (P[uw.first] == C) Wmap[R[uw.first]] += uw.second;
      int32_t best = NO_MOVE;
      i128 Gbest = 0;  // key of staying alone
      std::vector<std::pair<int32_t, i128>> cands;  // randomised: targets with G >= 0, ascending X
      for (const auto& xw : Wmap) {
        const int32_t X = xw.first;
        if (X == R[v]) continue;
        if (sizeR[X] == 1 && vertex_class(o.seed, 1, it, lvl, 0, member[X], o.K) == q) continue;
        if (!wc[X]) continue;
        const i128 Gx = key(p, xw.second, null_sum(p, G.kvec[v], [&](int32_t s) { return kr(X, s); }));
        if (Gx >= 0) cands.push_back({X, Gx});
        if (Gx > Gbest) {  // ascending X: the first maximum is the smallest label
          best = X;
          Gbest = Gx;
        }
      }
      if (o.theta_num > 0) {
        u128 div = (u128)(uint64_t)p.twoM_all * (u128)(uint64_t)o.theta_num;
        if (div == 0) div = 1;  // no edges and no coupling: every key is 0
        const uint64_t td = (uint64_t)o.theta_den;
        u128 total = exp_weight((u128)Gbest, div, td);  // staying: key 0
        for (const auto& xc : cands) total += exp_weight((u128)(Gbest - xc.second), div, td);
        const uint64_t Rd = class_hash(o.seed, 2, it, lvl, 0, v) >> 32;
        const u128 thr = ((u128)Rd * total) >> 32;
        u128 cum = exp_weight((u128)Gbest, div, td);
        best = NO_MOVE;
        if (!(thr < cum))
          for (const auto& xc : cands) {
            cum += exp_weight((u128)(Gbest - xc.second), div, td);
            if (thr < cum) {
              best = xc.first;
              break;
            }
          }
      }
      target[v] = best;
    }
    for (int64_t v = 0; v < N; ++v)
      if (target[v] >= 0) R[v] = target[v];
  }
  return R;
}

int64_t count_distinct(const std::vector<int32_t>& x, int64_t N) {
  std::vector<char> seen(N, 0);
  int64_t d = 0;
  for (int32_t v : x)
    if (!seen[v]) {
      seen[v] = 1;
      ++d;
    }
  return d;
}

uint64_t level_checksum(const Level& L) {
  uint64_t h = 0;
  for (int64_t x = 0; x < L.N; ++x) {
    for (const auto& yw : L.adj[x]) h += mix64(mix64(mix64((uint64_t)yw.second) ^ (uint64_t)yw.first) ^ (uint64_t)x);
    for (const auto& sk : L.kvec[x])
      h += mix64(mix64(mix64((uint64_t)sk.second) ^ (uint64_t)sk.first) ^ ((uint64_t)x + 0x9E3779B97F4A7C15ULL));
  }
  return h;
}

// Aggregation (Louvain/Leiden, Sec. 3.2): one node per refined community,
// numbered by ascending refined label; edge weights summed between distinct
// new nodes (self-loops dropped: no key or check below reads them and Q is
// always evaluated on level 0); slice vectors summed; the initial label of a
// new node is the smallest new id inside its local-moving community.
Level aggregate(const Level& G, const std::vector<int32_t>& P, const std::vector<int32_t>& R,
                std::vector<int32_t>& next_labels, std::vector<int32_t>& map) {
  const int64_t N = G.N;
  std::vector<int32_t> newid(N, -1);
  std::vector<char> used(N, 0);
  for (int64_t v = 0; v < N; ++v) used[R[v]] = 1;
  int32_t Np = 0;
  for (int64_t L = 0; L < N; ++L)
    if (used[L]) newid[L] = Np++;
  std::vector<std::map<int32_t, int64_t>> adjm(Np), km(Np);
  map.assign(N, 0);
  for (int64_t v = 0; v < N; ++v) {
    const int32_t x = newid[R[v]];
    map[v] = x;
    for (const auto& uw : G.adj[v]) {
      const int32_t y = newid[R[uw.first]];
      if (y != x) adjm[x][y] += uw.second;
    }
    for (const auto& sk : G.kvec[v]) km[x][sk.first] += sk.second;
  }
  Level H;
  H.N = Np;
  H.adj.resize(Np);
  H.kvec.resize(Np);
  for (int32_t x = 0; x < Np; ++x) {
    for (const auto& e : adjm[x]) H.adj[x].push_back(e);
    for (const auto& e : km[x])
      if (e.second > 0) H.kvec[x].push_back(e);
  }
  std::vector<int32_t> minid(N, INT32_MAX);
  for (int64_t v = 0; v < N; ++v) minid[P[v]] = std::min(minid[P[v]], map[v]);
  next_labels.assign(Np, 0);
  for (int64_t v = 0; v < N; ++v) next_labels[map[v]] = minid[P[v]];
  return H;
}

// Canonical labels: renumbered by first occurrence over supra-node order.
void canonicalise(std::vector<int32_t>& x) {
  std::map<int32_t, int32_t> ren;
  for (auto& l : x) {
    auto f = ren.find(l);
    if (f == ren.end()) f = ren.emplace(l, (int32_t)ren.size()).first;
    l = f->second;
  }
}

// u128 -> double, round to nearest (the compiler's conversion).
double u128_to_double(u128 x) { return (double)x; }

// Q_MS in FP64 (Eq. multislice-modularity):
//   2mu Q = I + omega*J - sum_s gamma_s (sum_c Sigma_{c,s}^2) / 2m_s,
//   I = sum of intra-slice weights over ordered pairs in one community,
//   omega*J = sum of omega^(sr) over ordered coupling pairs in one community
//             (J counts them when every coupled pair has the same omega),
//   2mu = sum_s 2m_s + n * sum_s sum_r omega^(sr).
// Fixed evaluation order (reading, shared by both implementations): slice
// terms as (double)S_s/(double)2m_s summed in ascending s, then omega*J as
// ((double)on*(double)J)/(double)od (uniform omega) or (double)Jw/(double)od
// (Jw = the integer sum of the pairs' numerators), then the numerator
// (I + omega*J) - gamma*sum, then the division.  With per-slice resolutions
// each slice term is first multiplied by (double)gsn/(double)gsd and the
// products are summed ascending instead.
// Global model, Eq. modularity on the supra-graph with total weight 2mu:
//   Q = (I + omega*J) / 2mu - gamma * S' / (2mu)^2,
//   S' = sum_c (sum_{v in c} k'_v)^2 in units of 1/od^2, so the second term is
//   evaluated as S' / (2M')^2 with 2M' = od*2mu.
// Fixed order: I + omega*J as above, divided by 2mu; S' (double) divided by
// ((double)2M' * (double)2M'); times gamma; subtracted.
struct PairSums {
  int64_t I = 0, J = 0, Jw = 0;
};

// I, J and Jw of a level-0 labelling; calls per_node(v, s, k) for every node.
template <class F>
PairSums pair_sums(const orc_csr* slices, const Problem& p, const std::vector<int32_t>& labels, F per_node) {
  PairSums ps;
  const int64_t n = p.n;
  for (int32_t s = 0; s < p.T; ++s) {
    for (int64_t i = 0; i < n; ++i) {
      const int64_t v = (int64_t)s * n + i;
      int64_t k = 0;
      for (int64_t e = slices[s].indptr[i]; e < slices[s].indptr[i + 1]; ++e) {
        const int64_t u = (int64_t)s * n + slices[s].indices[e];
        if (labels[u] == labels[v]) ps.I += slices[s].weights[e];
        k += slices[s].weights[e];
      }
      for (int32_t r = 0; r < p.T; ++r) {
        const bool coupled = p.coupling == ORC_ORDINAL ? (r == s - 1 || r == s + 1) : r != s;
        if (!coupled || labels[(int64_t)r * n + i] != labels[v]) continue;
        ps.J++;
        ps.Jw += coupling_num(p, s, r);
      }
      per_node(v, s, k);
    }
  }
  return ps;
}

double omega_J(const Problem& p, const PairSums& ps) {
  if (p.omega_table) return (double)ps.Jw / (double)p.od;
  return ((double)p.on * (double)ps.J) / (double)p.od;
}

double modularity_global(const orc_csr* slices, const Problem& p, const std::vector<int32_t>& labels) {
  std::map<int32_t, u128> sig;  // Sigma'_c
  const PairSums ps = pair_sums(slices, p, labels, [&](int64_t v, int32_t s, int64_t k) {
    sig[labels[v]] += (u128)(uint64_t)(p.od * k + p.cstr[s]);
  });
  u128 S = 0;
  for (const auto& cs : sig) S += cs.second * cs.second;
  const int64_t twoM = p.two_m_null[0];
  if (twoM == 0) return 0.0;  // reading: no edges and no coupling -> Q = 0
  const double wJ = omega_J(p, ps);
  const double gam = (double)p.gn / (double)p.gd;
  const double twomu = (double)twoM / (double)p.od;
  const double first = ((double)ps.I + wJ) / twomu;
  const double null = u128_to_double(S) / ((double)twoM * (double)twoM);
  return first - gam * null;
}

double modularity_of(const orc_csr* slices, const Problem& p, const std::vector<int32_t>& labels) {
  if (p.null_model == ORC_NULL_GLOBAL) return modularity_global(slices, p, labels);
  const int64_t n = p.n;
  std::map<int32_t, SliceMap> sig;
  const bool cpm = p.null_model == ORC_NULL_CPM;  // node counts over masses 1
  const PairSums ps = pair_sums(slices, p, labels,
                                [&](int64_t v, int32_t s, int64_t k) { sig[labels[v]][s] += cpm ? 1 : k; });
  std::vector<u128> S(p.T, 0);
  for (const auto& cs : sig)
    for (const auto& sk : cs.second) S[sk.first] += (u128)(uint64_t)sk.second * (u128)(uint64_t)sk.second;
  double nullsum = 0.0;
  for (int32_t s = 0; s < p.T; ++s) {
    if (p.two_m_null[s] == 0) continue;
    const double term = u128_to_double(S[s]) / (double)p.two_m_null[s];
    nullsum += p.gamma_table ? ((double)p.gsn[s] / (double)p.gsd[s]) * term : term;
  }
  const double wJ = omega_J(p, ps);
  const double gam = (double)p.gn / (double)p.gd;
  int64_t sum2m = 0, csum = 0;
  for (int64_t t : p.two_m) sum2m += t;
  for (int64_t c : p.cstr) csum += c;
  const int64_t twomu_num = p.od * sum2m + n * csum;
  if (twomu_num == 0) return 0.0;  // reading: no edges and no coupling -> Q = 0
  const double twomu = (double)twomu_num / (double)p.od;
  const double num = ((double)ps.I + wJ) - (p.gamma_table ? nullsum : gam * nullsum);
  return num / twomu;
}

// Key G(v, c) of node v of a level for community c under `labels` (c = -1:
// an empty community, key 0): the key of Eq. multislice-modularity's gain
// as stated above `key`, with W(v, c\v) summed over v's entries (a level has
// no self-loops) and Sigma_{c\v,s} over the other members of c.
i128 level_key(const Level& G, const Problem& p, const int32_t* labels, int64_t v, int64_t c) {
  if (c < 0) return 0;
  int64_t W = 0;
  for (const auto& uw : G.adj[v])
    if (labels[uw.first] == c) W += uw.second;
  SliceMap sig;
  for (int64_t u = 0; u < G.N; ++u)
    if (labels[u] == c && u != v)
      for (const auto& sk : G.kvec[u]) sig[sk.first] += sk.second;
  return key(p, W, null_sum(p, G.kvec[v], [&](int32_t s) { return sig.count(s) ? sig[s] : 0; }));
}

// A local-moving partition P and a refinement R of it (labels in [0, N),
// every R-community inside one P-community), as aggregation takes them.
int check_partitions(int64_t N, const int32_t* P, const int32_t* R) {
  std::vector<int32_t> parent(N, -1);
  for (int64_t v = 0; v < N; ++v) {
    if (P[v] < 0 || P[v] >= N || R[v] < 0 || R[v] >= N) return ORC_EINVAL;
    if (parent[R[v]] >= 0 && parent[R[v]] != P[v]) return ORC_EINVAL;
    parent[R[v]] = P[v];
  }
  return ORC_OK;
}

int setup(const orc_csr* slices, int32_t T, int64_t gn, int64_t gd, int64_t on, int64_t od, Problem& p,
          int32_t null_model, const orc_general* gen) {
  int rc = validate(slices, T);
  if (rc) return rc;
  if (!valid_rational(gn, gd, false) || !valid_rational(on, od, true)) return ORC_EINVAL;
  if (null_model != ORC_NULL_MULTISLICE && null_model != ORC_NULL_GLOBAL && null_model != ORC_NULL_CPM)
    return ORC_EINVAL;
  p.null_model = null_model;
  p.T = T;
  p.n = slices[0].n;
  p.gn = gn;
  p.gd = gd;
  p.on = on;
  p.od = od;
  rc = setup_general(gen, p);
  if (rc) return rc;
  slice_masses(slices, p);
  return check_bounds(p);
}

}  // namespace

extern "C" {

uint64_t orc_mix64(uint64_t x) { return mix64(x); }

uint64_t orc_exp_weight(uint64_t d_lo, uint64_t d_hi, uint64_t div_lo, uint64_t div_hi, uint64_t theta_den) {
  const u128 d = ((u128)d_hi << 64) | d_lo, div = ((u128)div_hi << 64) | div_lo;
  if (div == 0) return 0;
  return exp_weight(d, div, theta_den);
}

void orc_default_opts(orc_opts* o) {
  o->n_iterations = 2;  // two optimisation passes (paper Sec. 4)
  o->K = 4;
  o->max_rounds = 100;
  o->max_levels = 32;
  o->seed = 0;
  o->stop_level = -1;
  o->stop_stage = 0;
  o->stop_rounds = 0;
  o->null_model = ORC_NULL_MULTISLICE;
  o->theta_num = 0;
  o->theta_den = 1;
}

int orc_lambda(const orc_csr* slices, int32_t T, int64_t gn, int64_t gd, uint64_t* lam, int64_t* two_m) {
  Problem p;
  int rc = setup(slices, T, gn, gd, 1, 1, p, ORC_NULL_MULTISLICE, nullptr);
  if (rc) return rc;
  for (int32_t s = 0; s < T; ++s) {
    lam[2 * s] = (uint64_t)p.lambda[s];
    lam[2 * s + 1] = (uint64_t)(p.lambda[s] >> 64);
    two_m[s] = p.two_m[s];
  }
  return ORC_OK;
}

int orc_modularity(const orc_csr* slices, int32_t T, const int32_t* labels, int64_t gn, int64_t gd, int64_t on,
                   int64_t od, int32_t null_model, const orc_general* gen, double* Q_out) {
  Problem p;
  int rc = setup(slices, T, gn, gd, on, od, p, null_model, gen);
  if (rc) return rc;
  const int64_t N = p.n * T;
  std::vector<int32_t> lab(labels, labels + N);
  for (int32_t l : lab)
    if (l < 0 || l >= N) return ORC_EINVAL;
  *Q_out = modularity_of(slices, p, lab);
  return ORC_OK;
}

int orc_move_key(const orc_csr* slices, int32_t T, const int32_t* labels, int64_t gn, int64_t gd, int64_t on,
                 int64_t od, int32_t null_model, const orc_general* gen, int64_t v, int64_t c, uint64_t out[2]) {
  Problem p;
  int rc = setup(slices, T, gn, gd, on, od, p, null_model, gen);
  if (rc) return rc;
  Level G = build_level0(slices, p);
  if (v < 0 || v >= G.N) return ORC_EINVAL;
  const i128 Gk = level_key(G, p, labels, v, c);
  out[0] = (uint64_t)(u128)Gk;
  out[1] = (uint64_t)((u128)Gk >> 64);
  return ORC_OK;
}

int orc_aggregate(const orc_csr* slices, int32_t T, int64_t on, int64_t od, int32_t null_model,
                  const orc_general* gen, const int32_t* P, const int32_t* R, orc_level_out* out) {
  Problem p;
  int rc = setup(slices, T, 1, 1, on, od, p, null_model, gen);
  if (rc) return rc;
  const Level G = build_level0(slices, p);
  rc = check_partitions(G.N, P, R);
  if (rc) return rc;
  std::vector<int32_t> Pv(P, P + G.N), Rv(R, R + G.N), nl, mp;
  const Level H = aggregate(G, Pv, Rv, nl, mp);
  int64_t ns = 0;
  for (const auto& kv : H.kvec) ns += (int64_t)kv.size();
  out->N = H.N;
  out->nnz = H.nnz();
  out->ns = ns;
  if (!out->rowptr) return ORC_OK;  // sizes only
  if (out->cap_N < H.N || out->cap_nnz < out->nnz || out->cap_ns < ns) return ORC_EINVAL;
  int64_t e = 0, j = 0;
  for (int64_t x = 0; x < H.N; ++x) {
    out->rowptr[x] = e;
    out->sptr[x] = j;
    for (const auto& yw : H.adj[x]) {
      out->col[e] = yw.first;
      out->W[e++] = yw.second;
    }
    for (const auto& sk : H.kvec[x]) {
      out->sidx[j] = sk.first;
      out->sval[j++] = sk.second;
    }
    out->init_labels[x] = nl[x];
  }
  out->rowptr[H.N] = e;
  out->sptr[H.N] = j;
  std::copy(mp.begin(), mp.end(), out->node_map);
  return ORC_OK;
}

int orc_level_key(const orc_csr* slices, int32_t T, int64_t gn, int64_t gd, int64_t on, int64_t od,
                  int32_t null_model, const orc_general* gen, const int32_t* P, const int32_t* R,
                  const int32_t* labels1, int64_t x, int64_t c, uint64_t out[2]) {
  Problem p;
  int rc = setup(slices, T, gn, gd, on, od, p, null_model, gen);
  if (rc) return rc;
  const Level G = build_level0(slices, p);
  rc = check_partitions(G.N, P, R);
  if (rc) return rc;
  std::vector<int32_t> Pv(P, P + G.N), Rv(R, R + G.N), nl, mp;
  const Level H = aggregate(G, Pv, Rv, nl, mp);
  if (x < 0 || x >= H.N || c >= H.N) return ORC_EINVAL;
  for (int64_t y = 0; y < H.N; ++y)
    if (labels1[y] < 0 || labels1[y] >= H.N) return ORC_EINVAL;
  const i128 Gk = level_key(H, p, labels1, x, c);
  out[0] = (uint64_t)(u128)Gk;
  out[1] = (uint64_t)((u128)Gk >> 64);
  return ORC_OK;
}

int orc_count_improving(const orc_csr* slices, int32_t T, const int32_t* labels, int64_t gn, int64_t gd, int64_t on,
                        int64_t od, int32_t null_model, const orc_general* gen, int64_t* count) {
  Problem p;
  int rc = setup(slices, T, gn, gd, on, od, p, null_model, gen);
  if (rc) return rc;
  Level G = build_level0(slices, p);
  std::vector<int64_t> size(G.N, 0);
  std::vector<SliceMap> Sigma(G.N);
  for (int64_t v = 0; v < G.N; ++v) {
    if (labels[v] < 0 || labels[v] >= G.N) return ORC_EINVAL;
    size[labels[v]]++;
    for (const auto& sk : G.kvec[v]) Sigma[labels[v]][sk.first] += sk.second;
  }
  int64_t cnt = 0;
  for (int64_t v = 0; v < G.N; ++v) {
    const int32_t a = labels[v];
    std::map<int32_t, int64_t> Wmap;
    for (const auto& uw : G.adj[v]) Wmap[labels[uw.first]] += uw.second;
    auto ga = key(p, Wmap.count(a) ? Wmap[a] : 0, null_sum(p, G.kvec[v], [&](int32_t s) {
                    int64_t kvs = 0;
                    for (const auto& sk : G.kvec[v])
                      if (sk.first == s) kvs = sk.second;
                    return (Sigma[a].count(s) ? Sigma[a][s] : 0) - kvs;  // Sigma_{a\v,s}
                  }));
    bool imp = (size[a] > 1 && ga < 0);
    for (const auto& cw : Wmap) {
      if (cw.first == a) continue;
      auto gc = key(p, cw.second, null_sum(p, G.kvec[v], [&](int32_t s) {
                      return Sigma[cw.first].count(s) ? Sigma[cw.first][s] : 0;
                    }));
      if (gc > ga) imp = true;
    }
    cnt += imp;
  }
  *count = cnt;
  return ORC_OK;
}

int orc_leiden(const orc_csr* slices, int32_t T, int64_t gn, int64_t gd, int64_t on, int64_t od, const orc_opts* o,
               const orc_general* gen, const int32_t* init_labels, int32_t* labels_out, int64_t labels_cap,
               double* Q_out, orc_stats* st) {
  orc_opts opt;
  orc_default_opts(&opt);
  if (o) opt = *o;
  if (opt.theta_num < 0 || opt.theta_den < 1 || opt.theta_num > ((int64_t)1 << 31) || opt.theta_den > ((int64_t)1 << 31))
    return ORC_EINVAL;
  Problem p;
  int rc = setup(slices, T, gn, gd, on, od, p, opt.null_model, gen);
  if (rc) return rc;
  if (opt.n_iterations < 1 || opt.K < 1 || opt.max_rounds < 1 || opt.max_levels < 1) return ORC_EINVAL;
  orc_stats local{};
  if (!st) st = &local;
  std::memset(st, 0, sizeof(*st));

  const Level L0 = build_level0(slices, p);
  const int64_t N0 = L0.N;
  std::vector<int32_t> labels(N0);
  for (int64_t v = 0; v < N0; ++v) {
    labels[v] = init_labels ? init_labels[v] : (int32_t)v;
    if (labels[v] < 0 || labels[v] >= N0) return ORC_EINVAL;
  }
  std::vector<int32_t> prev;
  for (int it = 0; it < opt.n_iterations; ++it) {
    st->iterations = it + 1;
    Level cur_store;
    const Level* cur = &L0;
    std::vector<int32_t> c = labels;
    std::vector<std::vector<int32_t>> maps;
    int lvl = 0;
    for (;; ++lvl) {
      const bool stop_here = (it == 0 && opt.stop_level == lvl);
      int rounds = opt.max_rounds;
      if (stop_here && opt.stop_rounds > 0) rounds = opt.stop_rounds;
      if (stop_here && opt.stop_rounds < 0) rounds = 0;  // keep the level's initial labels
      MoveResult mr = local_move(*cur, p, opt, c, it, lvl, rounds, st);
      if (lvl == 0) st->last_level0_moves = mr.moves;
      if (stop_here && opt.stop_stage == 1) {
        if ((int64_t)c.size() > labels_cap) return ORC_EINVAL;
        std::copy(c.begin(), c.end(), labels_out);
        st->out_n = (int64_t)c.size();
        st->levels = lvl + 1;
        return ORC_OK;
      }
      if (count_distinct(c, cur->N) == cur->N) {  // every community is a single node
        st->stop_reason = 1;
        break;
      }
      if (lvl + 1 >= opt.max_levels) {
        st->stop_reason = 2;
        break;
      }
      std::vector<int32_t> R = refine(*cur, p, opt, c, it, lvl);
      if (stop_here && opt.stop_stage == 2) {
        if ((int64_t)R.size() > labels_cap) return ORC_EINVAL;
        std::copy(R.begin(), R.end(), labels_out);
        st->out_n = (int64_t)R.size();
        st->levels = lvl + 1;
        return ORC_OK;
      }
      if (count_distinct(R, cur->N) == cur->N) {  // aggregation would not shrink the graph
        st->stop_reason = 3;
        break;
      }
      std::vector<int32_t> nl, mp;
      Level nxt = aggregate(*cur, c, R, nl, mp);
      if (stop_here && opt.stop_stage == 3) {
        if ((int64_t)nl.size() > labels_cap) return ORC_EINVAL;
        std::copy(nl.begin(), nl.end(), labels_out);
        st->out_n = (int64_t)nl.size();
        st->next_n = nxt.N;
        st->next_nnz = nxt.nnz();
        st->next_checksum = level_checksum(nxt);
        st->levels = lvl + 1;
        return ORC_OK;
      }
      maps.push_back(std::move(mp));
      cur_store = std::move(nxt);
      cur = &cur_store;
      c = std::move(nl);
    }
    st->levels = lvl + 1;
    // flatten the level maps down to supra-nodes
    std::vector<int32_t> out(N0);
    for (int64_t v = 0; v < N0; ++v) {
      int64_t x = v;
      for (const auto& m : maps) x = m[x];
      out[v] = c[x];
    }
    canonicalise(out);
    const bool same = (it > 0 && out == prev);
    prev = out;
    labels = out;
    if (same) break;
  }
  if (labels_cap < N0) return ORC_EINVAL;
  std::copy(prev.begin(), prev.end(), labels_out);
  st->out_n = N0;
  if (Q_out) *Q_out = modularity_of(slices, p, prev);
  return ORC_OK;
}

}  // extern "C"
