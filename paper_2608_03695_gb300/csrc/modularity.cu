// Multislice modularity (Eq. multislice-modularity) of a level-0 labelling,
// from exact integer sums:
//   2mu Q = I + omega*J - gamma * sum_s S_s / 2m_s
//   I   = intra-snapshot weight over ordered pairs inside one community,
//   J   = ordered coupling pairs inside one community (general coupling:
//         omega*J = Jw/od, Jw the sum of the pairs' numerators),
//   S_s = sum_c Sigma_{c,s}^2 (128-bit),
//   2mu = sum_s 2m_s + n * sum_{s,r} omega^(sr)  (2*omega*n*(T-1) ordinal).
// Per-snapshot gamma: each slice term is multiplied by its gamma before the
// ascending sum, and the sum is subtracted as it is.
// Temporal CPM: S_s counts nodes (Sigma = node counts) and its slice term is
// S_s itself (a mass of 1) for every snapshot.
// The FP64 combination follows one fixed order (slice terms in ascending s,
// then omega*J, the numerator, the division), with explicitly rounded
// operations so no contraction changes the result.
//
// Global null model (plain modularity of the supra-graph, Eq. modularity):
//   Q = (I + omega*J) / 2mu - gamma * S' / (2M')^2,
//   S' = sum_c Sigma'_c^2 with Sigma' in units of 1/od, 2M' = od*2mu;
// FP64 order: I + omega*J, divided by 2mu; S' divided by the product
// 2M'*2M' (each converted first); times gamma; subtracted.
//
// Also: canonical relabelling (first occurrence order), distinct counting
// and the order-free level checksum used by the step-level tests.
#include <cstring>
#include <vector>

#include "solver.h"

namespace mslice {

namespace {

// I and J of every instance (IJ: 2 words per instance).  A single instance
// accumulates per warp before one atomic; batches add per row.
__global__ void k_IJ(LevelDev g, const int32_t* labels, ull* IJ, int32_t B) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  ull I = 0, J = 0;
  for (int64_t v = (((int64_t)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5); v < g.N; v += warps) {
    const int32_t c = labels[v];
    ull Iv = 0, Jv = 0;
    for (int64_t e = g.rowptr[v] + lane; e < g.rowptr[v + 1]; e += 32) {
      const int2 x = g.adj0[e];
      if (labels[x.x] == c) {
        if (x.y > 0)
          Iv += (ull)x.y;
        else
          Jv += g.cw ? (ull)g.cw[-x.y - 1] : 1ull;  // weighted by the pair's numerator with a table
      }
    }
    if (B == 1) {
      I += Iv;
      J += Jv;
    } else {
      Iv = warp_sum(Iv);
      Jv = warp_sum(Jv);
      if (lane == 0) {
        const int32_t i = node_inst(g, (int32_t)v);
        if (Iv) atomicAdd(&IJ[2 * i], Iv);
        if (Jv) atomicAdd(&IJ[2 * i + 1], Jv);
      }
    }
  }
  if (B == 1) {
    I = warp_sum(I);
    J = warp_sum(J);
    if (lane == 0) {
      if (I) atomicAdd(&IJ[0], I);
      if (J) atomicAdd(&IJ[1], J);
    }
  }
}

// S_s += Sigma_{c,s}^2 over the table; per-block partial sums in shared
// memory when T is small enough, global 128-bit atomics otherwise.
__global__ void k_S(SigStore h, int32_t T, ull* S) {
  extern __shared__ ull sm[];  // 2*T words when used
  const bool use_sm = T <= 1024;
  if (use_sm) {
    for (int i = threadIdx.x; i < 2 * T; i += blockDim.x) sm[i] = 0;
    __syncthreads();
  }
  const uint64_t span = ss_span(h);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < span; i += (uint64_t)gridDim.x * blockDim.x) {
    int32_t cc, s;
    long long val;
    if (!ss_entry(h, i, cc, s, val)) continue;
    const u128 sq = (u128)(ull)val * (u128)(ull)val;
    if (use_sm)
      atomic_add_u128(&sm[2 * s], sq);
    else
      atomic_add_u128(&S[2 * s], sq);
  }
  if (use_sm) {
    __syncthreads();
    for (int s = threadIdx.x; s < T; s += blockDim.x) {
      const u128 x = ((u128)sm[2 * s + 1] << 64) | sm[2 * s];
      if (x) atomic_add_u128(&S[2 * s], x);
    }
  }
}

struct QInst {
  int64_t n;
  int32_t T, soff;
  long long gn, gd, on, od;
  long long csum;      // n * sum_{s,r} omega_num^(sr): the coupling part of 2mu, in units of 1/od
  int32_t table, gtab;  // the instance has its own omega^(sr) table / per-snapshot gamma
};

// omega*J of an instance: with its own table, (double)Jw/od; otherwise
// (on*J)/od.  IJ's second word holds Jw when the solve has a coupling table
// (weighted) -- an instance without one then had every pair weigh on, so
// J = Jw/on.
__device__ __forceinline__ double omega_J(const QInst& p, ull Jword, int32_t weighted) {
  if (p.table) return __ddiv_rn(__ull2double_rn(Jword), __ll2double_rn(p.od));
  const ull J = weighted ? (p.on > 0 ? Jword / (ull)p.on : 0ull) : Jword;
  return __ddiv_rn(__dmul_rn(__ll2double_rn(p.on), __ull2double_rn(J)), __ll2double_rn(p.od));
}

// Q of every instance (one thread each), in the fixed FP64 order.  S holds
// one 128-bit sum per null slice: per snapshot (Q_MS) or per instance
// (global model).  gs: per-snapshot gamma (num, den) pairs, when any
// instance has them.
// The slice terms of Q_MS, one thread per snapshot: S_s / 2m_s (CPM: S_s,
// a mass of 1), times gamma_s when the instance has per-snapshot gamma.
// k_Q adds them in ascending s, so the result is that of one sequential
// evaluation.
__global__ void k_slice_terms(const ull* S, const int64_t* two_m, int32_t T, const int32_t* slice_inst,
                              const QInst* qi, int32_t cpm, const long long* gs, double* terms) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < T; s += gridDim.x * blockDim.x) {
    const long long t = two_m[s];
    double term = 0.0;
    if (t > 0 || cpm) {
      const u128 x = ((u128)S[2 * s + 1] << 64) | S[2 * s];
      term = cpm ? u128_to_double(x) : __ddiv_rn(u128_to_double(x), __ll2double_rn(t));
      if (qi[slice_inst ? slice_inst[s] : 0].gtab)
        term = __dmul_rn(__ddiv_rn(__ll2double_rn(gs[2 * s]), __ll2double_rn(gs[2 * s + 1])), term);
    }
    terms[s] = term;
  }
}

__global__ void k_Q(const ull* IJ, const ull* S, const int64_t* two_m, const QInst* qi, int32_t B, int32_t global,
                    int32_t cpm, int32_t weighted, const double* terms, double* Q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  const QInst p = qi[i];
  if (global) {
    long long sum2m = 0;
    for (int s = p.soff; s < p.soff + p.T; ++s) sum2m += two_m[s];
    const long long twoM = p.od * sum2m + p.csum;
    if (twoM == 0) {
      Q[i] = 0.0;
      return;
    }
    const u128 x = ((u128)S[2 * i + 1] << 64) | S[2 * i];
    const double wJ = omega_J(p, IJ[2 * i + 1], weighted);
    const double gam = __ddiv_rn(__ll2double_rn(p.gn), __ll2double_rn(p.gd));
    const double twomu = __ddiv_rn(__ll2double_rn(twoM), __ll2double_rn(p.od));
    const double first = __ddiv_rn(__dadd_rn(__ull2double_rn(IJ[2 * i]), wJ), twomu);
    const double tM = __ll2double_rn(twoM);
    const double null = __ddiv_rn(u128_to_double(x), __dmul_rn(tM, tM));
    Q[i] = __dsub_rn(first, __dmul_rn(gam, null));
    return;
  }
  double nullsum = 0.0;
  long long sum2m = 0;
  for (int s = p.soff; s < p.soff + p.T; ++s) {
    const long long t = two_m[s];
    sum2m += t;
    if (t > 0 || cpm) nullsum = __dadd_rn(nullsum, terms[s]);  // ascending s
  }
  const double wJ = omega_J(p, IJ[2 * i + 1], weighted);
  const double gam = __ddiv_rn(__ll2double_rn(p.gn), __ll2double_rn(p.gd));
  const long long twomu_num = p.od * sum2m + p.csum;
  if (twomu_num == 0) {
    Q[i] = 0.0;
    return;
  }
  const double twomu = __ddiv_rn(__ll2double_rn(twomu_num), __ll2double_rn(p.od));
  const double num = __dsub_rn(__dadd_rn(__ull2double_rn(IJ[2 * i]), wJ), p.gtab ? nullsum : __dmul_rn(gam, nullsum));
  Q[i] = __ddiv_rn(num, twomu);
}

__global__ void k_first(const int32_t* x, int64_t N, int32_t* first) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
    atomicMin(&first[x[v]], (int32_t)v);
}

__global__ void k_first_flag(const int32_t* x, const int32_t* first, int64_t N, int32_t* flag) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
    flag[v] = first[x[v]] == (int32_t)v ? 1 : 0;
}

// Renumbered labels, counted from the instance's first community.
__global__ void k_canon(const int32_t* x, const int32_t* first, const int32_t* rank, int64_t N, const int32_t* inst,
                        const int32_t* inst_off, int32_t* out) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
    out[v] = rank[first[x[v]]] - (inst ? rank[inst_off[inst[v]]] : 0);
}

__global__ void k_mark(const int32_t* x, int64_t N, int32_t* flag) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
    flag[x[v]] = 1;
}

__global__ void k_checksum(LevelDev g, ull* out) {
  ull h = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.N; v += (int64_t)gridDim.x * blockDim.x) {
    for (int64_t e = g.rowptr[v]; e < g.rowptr[v + 1]; ++e)
      h += mix64(mix64(mix64((ull)g.W[e]) ^ (ull)g.col[e]) ^ (ull)v);
    for (int64_t j = g.sptr[v]; j < g.sptr[v + 1]; ++j)
      h += mix64(mix64(mix64((ull)g.sval[j]) ^ (ull)g.sidx[j]) ^ ((ull)v + 0x9E3779B97F4A7C15ULL));
  }
  h = warp_sum(h);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, h);
}

unsigned gsz(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

void modularity(Solver& S, const int32_t* labels0, double* Q) {
  Ctx& c = *S.c;
  const SupraGraph& G = *S.G0;
  const int32_t B = G.B;
  LevelDev g = level0_view(G, S);  // (S.Tn / S.kn set up by setup_null_model)
  configure_stores(S, G.N);
  sigma_rebuild(S, Level{g}, labels0);
  const int32_t Tn = S.Tn;
  ull* acc = c.ws->get<ull>("q_acc", 2 * (size_t)B + 2 * (size_t)Tn);
  double* dQ = c.ws->get<double>("q_out", B);
  QInst* dqi = c.ws->get<QInst>("q_inst", B);
  std::vector<QInst> qi(B);
  for (int32_t i = 0; i < B; ++i) {
    const InstInfo& in = G.inst[i];
    qi[i] = QInst{in.n, in.T, in.soff, S.gn_h[i], S.gd_h[i], S.on_h[i], S.od_h[i], S.csum_h[i],
                  (int32_t)S.has_cw_h[i], (int32_t)S.has_gs_h[i]};
  }
  check_cuda(cudaMemcpyAsync(dqi, qi.data(), B * sizeof(QInst), cudaMemcpyHostToDevice, c.stream), "copy");
  check_cuda(cudaMemsetAsync(acc, 0, (2 * (size_t)B + 2 * (size_t)Tn) * sizeof(ull), c.stream), "memset");
  if (G.N > 0) launch(c, k_IJ, dim3(gsz(G.N * 32)), dim3(256), 0, g, labels0, acc, B);
  const size_t smem = Tn <= 1024 ? 2 * (size_t)Tn * sizeof(ull) : 0;
  const int64_t span = S.sig.d ? S.sig.rows * S.sig.T : (int64_t)S.sig.h.cap;
  launch(c, k_S, dim3(gsz(span)), dim3(256), smem, S.sig, Tn, acc + 2 * B);
  double* terms = c.ws->get<double>("q_terms", G.T > 0 ? G.T : 1);
  if (!S.p.global_null && G.T > 0)
    launch(c, k_slice_terms, dim3(grid_for(G.T, 256)), dim3(256), 0, (const ull*)(acc + 2 * B),
           (const int64_t*)G.two_m, G.T, (const int32_t*)(G.B > 1 ? G.slice_inst : nullptr), (const QInst*)dqi,
           (int32_t)(S.p.cpm ? 1 : 0), (const long long*)S.gs_d, terms);
  launch(c, k_Q, dim3(grid_for(B, 128)), dim3(128), 0, (const ull*)acc, (const ull*)(acc + 2 * B),
         (const int64_t*)G.two_m, (const QInst*)dqi, B, (int32_t)(S.p.global_null ? 1 : 0), (int32_t)(S.p.cpm ? 1 : 0),
         (int32_t)(S.cw_d ? 1 : 0), (const double*)terms, dQ);
  // B values go straight to the caller's (pageable) array
  check_cuda(cudaMemcpyAsync(Q, dQ, B * sizeof(double), cudaMemcpyDeviceToHost, c.stream), "copy");
  sync(c);
}

void canonicalise(Solver& S, const int32_t* x, int32_t* out, int64_t N) {
  Ctx& c = *S.c;
  if (N == 0) return;
  int32_t* first = S.tmp32a;
  int32_t* rank = S.tmp32b;
  fill_i32(c, first, INT32_MAX, N);
  launch(c, k_first, dim3(gsz(N)), dim3(256), 0, x, N, first);
  int32_t* flag = S.freelist;
  launch(c, k_first_flag, dim3(gsz(N)), dim3(256), 0, x, (const int32_t*)first, N, flag);
  // rank has N + 1 entries: rank[N] counts every community
  check_cuda(cudaMemsetAsync(flag + N, 0, sizeof(int32_t), c.stream), "memset");
  scan_excl(c, flag, rank, N + 1, (int32_t*)nullptr);
  const SupraGraph& G = *S.G0;
  launch(c, k_canon, dim3(gsz(N)), dim3(256), 0, x, (const int32_t*)first, (const int32_t*)rank, N,
         (const int32_t*)G.inst0, (const int32_t*)G.inst_off0, out);
}

int64_t count_distinct(Solver& S, const int32_t* x, int64_t N) {
  Ctx& c = *S.c;
  if (N == 0) return 0;
  int32_t* flag = S.freelist;
  check_cuda(cudaMemsetAsync(flag, 0, N * sizeof(int32_t), c.stream), "memset");
  launch(c, k_mark, dim3(gsz(N)), dim3(256), 0, x, N, flag);
  int32_t* d_tot = c.ws->get<int32_t>("cd_tot", 1);
  scan_excl(c, flag, S.tmp32a, N, d_tot);
  return *static_cast<const int32_t*>(readback(c, d_tot, sizeof(int32_t)));
}

uint64_t level_checksum(Solver& S, const Level& L) {
  Ctx& c = *S.c;
  ull* d = c.ws->get<ull>("ck_out", 1);
  check_cuda(cudaMemsetAsync(d, 0, sizeof(ull), c.stream), "memset");
  if (L.d.N > 0) launch(c, k_checksum, dim3(gsz(L.d.N)), dim3(256), 0, L.d, d);
  return *static_cast<const ull*>(readback(c, d, sizeof(ull)));
}

}  // namespace mslice
