// The Leiden driver (Sec. 3.2: Leiden = local moving, refinement,
// aggregation) over one or more independent instances laid out in one
// supra-graph:
//   for it in 0..n_iterations-1 (the paper caps runs at two passes, Sec. 4):
//     level 0 starts from the warm-start / previous labels (singletons first)
//     per level: local moving; an instance stops if every community is one
//     node; all stop at max_levels; refinement; an instance stops if it
//     merged nothing; aggregation
//     flatten the last level's labels to supra-nodes, canonicalise within
//     each instance; an instance whose iteration returned the labels it
//     started from takes no part in later iterations
//   Q of every instance (its own gamma and omega).
// A stopped instance is frozen: its nodes are never bucketed for a decision,
// so they neither move nor merge, refinement leaves them singletons and
// aggregation maps them one to one with their communities kept.  The level
// loop runs while some instance is unfrozen, and every instance's labels are
// those of a solve of that instance alone.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "../../include/mslice.h"
#include "solver.h"

namespace mslice {

namespace {

__global__ void k_gather(const int32_t* labels, const int32_t* node_of0, int64_t N0, int32_t* out) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N0; v += (int64_t)gridDim.x * blockDim.x)
    out[v] = labels[node_of0[v]];
}

// diff[i] = 1 when instance i's labels changed.
__global__ void k_differs(const int32_t* a, const int32_t* b, int64_t N, const int32_t* inst, int32_t* diff) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
    if (a[v] != b[v]) diff[inst ? inst[v] : 0] = 1;
}

// Freezes the instances whose labels did not change; counts the rest.
__global__ void k_freeze(const int32_t* diff, int32_t* active, int32_t B, int32_t* n_active) {
  __shared__ int tot;
  if (threadIdx.x == 0) tot = 0;
  __syncthreads();
  int n = 0;
  for (int32_t i = threadIdx.x; i < B; i += blockDim.x) {
    if (!diff[i]) active[i] = 0;
    n += active[i];
  }
  atomicAdd(&tot, n);
  __syncthreads();
  if (threadIdx.x == 0) *n_active = tot;
}

// cnt[i] = number of distinct values of x within instance i (flag marks the
// values present).
__global__ void k_mark(const int32_t* x, int64_t N, int32_t* flag) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
    flag[x[v]] = 1;
}

__global__ void k_inst_count(const int32_t* flag, int64_t N, const int32_t* inst, int32_t* cnt) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
    if (flag[v]) atomicAdd(&cnt[inst[v]], 1);
}

// Freezes every instance whose values are all distinct (each node its own
// community); counts the instances still active.
__global__ void k_freeze_settled(const int32_t* cnt, const int32_t* inst_off, int32_t* active, int32_t B,
                                 int32_t* n_active) {
  __shared__ int tot;
  if (threadIdx.x == 0) tot = 0;
  __syncthreads();
  int n = 0;
  for (int32_t i = threadIdx.x; i < B; i += blockDim.x) {
    if (cnt[i] == inst_off[i + 1] - inst_off[i]) active[i] = 0;
    n += active[i];
  }
  atomicAdd(&tot, n);
  __syncthreads();
  if (threadIdx.x == 0) *n_active = tot;
}

__global__ void k_add_offsets(int32_t* x, int64_t N, const int32_t* inst, const int32_t* inst_off) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
    x[v] += inst_off[inst[v]];
}

__global__ void k_check_labels(const int32_t* x, int64_t N, const int32_t* inst, const int32_t* inst_off,
                               unsigned* status) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t hi = inst ? inst_off[inst[i] + 1] - inst_off[inst[i]] : N;
    if (x[i] < 0 || x[i] >= hi) atomicOr(status, ERR_BAD_INPUT);
  }
}

unsigned gsz(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

// Batch: freezes the instances of level L whose values x are all distinct;
// returns the number of instances still active.
int32_t freeze_settled(Solver& S, const Level& L, const int32_t* x) {
  Ctx& c = *S.c;
  const int64_t N = L.d.N;
  const int32_t B = S.B;
  int32_t* flag = S.freelist;
  int32_t* cnt = S.inst_cnt;  // B + 1 entries: counts, then the active total
  check_cuda(cudaMemsetAsync(flag, 0, N * sizeof(int32_t), c.stream), "memset");
  check_cuda(cudaMemsetAsync(cnt, 0, (B + 1) * sizeof(int32_t), c.stream), "memset");
  if (N > 0) {
    launch(c, k_mark, dim3(gsz(N)), dim3(256), 0, x, N, flag);
    launch(c, k_inst_count, dim3(gsz(N)), dim3(256), 0, (const int32_t*)flag, N, L.d.inst, cnt);
  }
  launch(c, k_freeze_settled, dim3(1), dim3(256), 0, (const int32_t*)cnt, L.d.inst_off, S.inst_active, B, cnt + B);
  const int32_t act = *static_cast<const int32_t*>(readback(c, cnt + B, sizeof(int32_t)));
  // the empty-community pass expects its per-instance counters zeroed
  check_cuda(cudaMemsetAsync(cnt, 0, (B + 1) * sizeof(int32_t), c.stream), "memset");
  return act;
}

}  // namespace

PhaseClock::~PhaseClock() {
  for (auto& s : spans) {
    cudaEventDestroy(s.second.first);
    cudaEventDestroy(s.second.second);
  }
}

cudaEvent_t PhaseClock::begin() {
  cudaEvent_t e;
  check_cuda(cudaEventCreate(&e), "event");
  check_cuda(cudaEventRecord(e, c.stream), "event");
  return e;
}

void PhaseClock::end(int phase, cudaEvent_t b) {
  cudaEvent_t e;
  check_cuda(cudaEventCreate(&e), "event");
  check_cuda(cudaEventRecord(e, c.stream), "event");
  spans.push_back({phase, {b, e}});
}

void PhaseClock::totals(double out[5]) {
  sync(c);
  for (int i = 0; i < 5; ++i) out[i] = 0;
  for (auto& s : spans) {
    float ms = 0;
    check_cuda(cudaEventElapsedTime(&ms, s.second.first, s.second.second), "event time");
    out[s.first] += ms;
  }
}

void check_label_ranges(Ctx& c, const SupraGraph& G, const int32_t* d) {
  if (G.N == 0) return;
  check_cuda(cudaMemsetAsync(c.d_status, 0, sizeof(unsigned), c.stream), "memset");
  launch(c, k_check_labels, dim3(gsz(G.N)), dim3(256), 0, d, G.N, (const int32_t*)(G.B > 1 ? G.inst0 : nullptr),
         (const int32_t*)G.inst_off0, c.d_status);
  check_status(c, "labels");
}

// The snapshots coupled to s: [lo, s) and (s, hi) (ordinal: s-1 and s+1;
// categorical: all), so loops over an instance's pairs cost T times the
// partners, not T^2.
static inline void partners(int32_t coupling, int32_t T, int32_t s, int32_t& lo, int32_t& hi) {
  lo = coupling == 0 ? std::max(s - 1, 0) : 0;
  hi = coupling == 0 ? std::min(s + 2, T) : T;
}

long long pair_num(const InstParams& j, int32_t coupling, int32_t T, int32_t s, int32_t r) {
  if (s == r) return 0;
  if (coupling == 0 && s - r != 1 && r - s != 1) return 0;
  if (j.cw.empty()) return j.on;
  return j.cw[coupling == 0 ? std::min(s, r) : (int64_t)s * T + r];
}

void check_bounds(int64_t n, int32_t T, int32_t coupling, const int64_t* two_m, const InstParams& j, int nm) {
  u128 sum2m = 0, csum = 0;
  for (int32_t s = 0; s < T; ++s) {
    sum2m += (u128)(ull)two_m[s];
    int32_t lo, hi;
    partners(coupling, T, s, lo, hi);
    for (int32_t r = lo; r < hi; ++r) csum += (u128)(ull)pair_num(j, coupling, T, s, r);
  }
  const u128 lim = (u128)1 << 61;
  const u128 twoM = (u128)(ull)j.od * sum2m + (u128)(ull)n * csum;
  if (twoM >= lim) fail(MSLICE_EOVERFLOW, "omega_den*sum(2m_s) + n*sum(omega_num^(sr)) must stay below 2^61");
  if (nm == NULL_SUPRA_GLOBAL) {
    if ((u128)(ull)j.gn * twoM >= lim * (u128)(ull)j.gd)
      fail(MSLICE_EOVERFLOW, "global null model: gamma*(omega_den*sum(2m_s) + n*sum(omega_num^(sr))) must stay below 2^61");
    return;
  }
  const u128 mass = nm == NULL_CPM ? (u128)(ull)n * (u128)(ull)(n * T) : sum2m;
  for (int32_t s = 0; s < (j.gsn.empty() ? 1 : T); ++s) {
    const long long gn = j.gsn.empty() ? j.gn : j.gsn[s], gd = j.gsn.empty() ? j.gd : j.gsd[s];
    if ((u128)(ull)gn * (u128)(ull)j.od * mass >= lim * (u128)(ull)gd)
      fail(MSLICE_EOVERFLOW, nm == NULL_CPM ? "CPM: gamma*omega_den*n*N must stay below 2^61"
                                            : "gamma*omega_den*sum(2m_s) must stay below 2^61");
  }
}

namespace {

// Every level-0 node weighs 1 in CPM's null term.
__global__ void k_ones(int64_t* x, int64_t N) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
    x[v] = 1;
}

// k'_v = od*k_v + cstr[s], s the snapshot of v (batches: slice0 gives it;
// cstr is indexed by global snapshot).
__global__ void k_null_strength(const int64_t* k, int64_t N, int64_t n, const int32_t* slice0, const int32_t* inst0,
                                const long long* cstr, const long long* od, int64_t* kn) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = inst0 ? inst0[v] : 0;
    const int64_t s = slice0 ? (int64_t)slice0[v] : v / n;
    kn[v] = od[i] * k[v] + cstr[s];
  }
}

}  // namespace

void setup_null_model(Solver& S) {
  Ctx& c = *S.c;
  const SupraGraph& G = *S.G0;
  bool any_gs = false;
  for (uint8_t x : S.has_gs_h) any_gs = any_gs || x;
  if (S.p.cpm) {
    // node counts as strengths, masses 1: Lambda_s = floor(gamma_s 2^64)
    S.Tn = G.T > 0 ? G.T : 1;
    S.lam = c.ws->get<u128>("lam", S.Tn);
    std::vector<u128> lam(G.T);
    for (int32_t i = 0; i < G.B; ++i) {
      const InstInfo& in = G.inst[i];
      for (int32_t s = in.soff; s < in.soff + in.T; ++s) {
        const long long gn = any_gs ? S.gs_h[2 * s] : S.gn_h[i], gd = any_gs ? S.gs_h[2 * s + 1] : S.gd_h[i];
        lam[s] = (((u128)(ull)gn) << P_BITS) / (u128)(ull)gd;
      }
    }
    if (G.T > 0)
      check_cuda(cudaMemcpyAsync(S.lam, lam.data(), G.T * sizeof(u128), cudaMemcpyHostToDevice, c.stream), "copy");
    S.kn = c.ws->get<int64_t>("k_null", S.N0 > 0 ? S.N0 : 1);
    if (G.N > 0) launch(c, k_ones, dim3(grid_for(G.N, 256) < 4096 ? grid_for(G.N, 256) : 4096), dim3(256), 0, S.kn, G.N);
    sync(c);  // lam is pageable host memory
    return;
  }
  if (!S.p.global_null) {
    S.Tn = G.T > 0 ? G.T : 1;
    S.lam = c.ws->get<u128>("lam", S.Tn);
    if (G.T > 0 && !any_gs) {
      compute_lambda(c, G, S.gn_d, S.gd_d, S.lam);
    } else if (G.T > 0) {
      // per-snapshot gamma: Lambda_s = floor(gsn 2^64 / (gsd 2m_s)), from the host table
      std::vector<u128> lam(G.T);
      const std::vector<long long>& gs = S.gs_h;
      for (int32_t s = 0; s < G.T; ++s) {
        const long long t = G.two_m_host[s];
        lam[s] = t > 0 ? (((u128)(ull)gs[2 * s]) << P_BITS) / ((u128)(ull)gs[2 * s + 1] * (u128)(ull)t) : (u128)0;
      }
      check_cuda(cudaMemcpyAsync(S.lam, lam.data(), G.T * sizeof(u128), cudaMemcpyHostToDevice, c.stream), "copy");
      sync(c);  // lam is pageable host memory
    }
    return;
  }
  // one null slice per instance, 2M' = od*sum 2m_s + n*sum cstr in units of 1/od
  S.Tn = G.B;
  std::vector<u128> lam(G.B);
  for (int32_t i = 0; i < G.B; ++i) {
    const InstInfo& in = G.inst[i];
    long long sum2m = 0;
    for (int32_t s = in.soff; s < in.soff + in.T; ++s) sum2m += G.two_m_host[s];
    const long long twoM = S.od_h[i] * sum2m + S.csum_h[i];
    lam[i] = twoM > 0 ? (((u128)(ull)S.gn_h[i]) << P_BITS) / ((u128)(ull)S.gd_h[i] * (u128)(ull)twoM) : (u128)0;
  }
  S.lam = c.ws->get<u128>("lam", S.Tn);
  check_cuda(cudaMemcpyAsync(S.lam, lam.data(), G.B * sizeof(u128), cudaMemcpyHostToDevice, c.stream), "copy");
  long long* cstr = c.ws->get<long long>("cstr", G.T > 0 ? G.T : 1);
  if (G.T > 0)
    check_cuda(cudaMemcpyAsync(cstr, S.cstr_h.data(), G.T * sizeof(long long), cudaMemcpyHostToDevice, c.stream),
               "copy");
  S.kn = c.ws->get<int64_t>("k_null", S.N0 > 0 ? S.N0 : 1);
  if (G.N > 0) {
    const bool batch = G.B > 1;
    launch(c, k_null_strength, dim3(grid_for(G.N, 256) < 4096 ? grid_for(G.N, 256) : 4096), dim3(256), 0,
           (const int64_t*)G.k, G.N, G.n > 0 ? G.n : 1, (const int32_t*)(batch ? G.slice0 : nullptr),
           (const int32_t*)(batch ? G.inst0 : nullptr), (const long long*)cstr, (const long long*)S.od_d, S.kn);
  }
  sync(c);  // lam and cstr are pageable host memory
}

void set_instances(Ctx& c, Solver& S, const std::vector<InstParams>& jobs) {
  const int32_t B = (int32_t)jobs.size();
  S.B = B;
  S.p.gn = jobs[0].gn;
  S.p.gd = jobs[0].gd;
  S.p.on = jobs[0].on;
  S.p.od = jobs[0].od;
  S.gn_h.resize(B);
  S.gd_h.resize(B);
  S.on_h.resize(B);
  S.od_h.resize(B);
  std::vector<long long> hp(4 * (size_t)B);
  for (int32_t i = 0; i < B; ++i) {
    hp[i] = S.gn_h[i] = jobs[i].gn;
    hp[B + i] = S.gd_h[i] = jobs[i].gd;
    hp[2 * B + i] = S.on_h[i] = jobs[i].on;
    hp[3 * B + i] = S.od_h[i] = jobs[i].od;
  }
  long long* par = c.ws->get<long long>("s_params", 4 * (size_t)B);
  S.gn_d = par;
  S.gd_d = par + B;
  S.on_d = par + 2 * B;
  S.od_d = par + 3 * B;
  check_cuda(cudaMemcpyAsync(par, hp.data(), hp.size() * sizeof(long long), cudaMemcpyHostToDevice, c.stream), "copy");
  // coupling sums of every snapshot and instance; the tables when any
  // instance has one (the others' slots then hold their uniform omega)
  const SupraGraph& G = *S.G0;
  S.cstr_h.assign(G.T, 0);
  S.csum_h.assign(B, 0);
  S.has_cw_h.assign(B, 0);
  S.has_gs_h.assign(B, 0);
  S.cpl_edges = 0;
  bool any_cw = false, any_gs = false;
  for (int32_t i = 0; i < B; ++i) {
    const InstInfo& in = G.inst[i];
    S.has_cw_h[i] = !jobs[i].cw.empty();
    S.has_gs_h[i] = !jobs[i].gsn.empty();
    any_cw = any_cw || S.has_cw_h[i];
    any_gs = any_gs || S.has_gs_h[i];
    long long sum = 0;
    for (int32_t s = 0; s < in.T; ++s) {
      int32_t lo, hi;
      partners(in.coupling, in.T, s, lo, hi);
      for (int32_t r = lo; r < hi; ++r) {
        const long long x = pair_num(jobs[i], in.coupling, in.T, s, r);
        S.cstr_h[in.soff + s] += x;
        sum += x;
        if (x > 0) S.cpl_edges += in.n;
      }
    }
    S.csum_h[i] = in.n * sum;
  }
  std::vector<long long> cw;
  std::vector<long long>& gs = S.gs_h;
  gs.clear();
  S.cw_d = nullptr;
  S.gs_d = nullptr;
  if (any_cw && G.ncw > 0) {
    cw.assign(G.ncw, 0);
    for (int32_t i = 0; i < B; ++i) {
      const InstInfo& in = G.inst[i];
      for (int32_t s = 0; s < in.T; ++s) {
        int32_t lo, hi;
        partners(in.coupling, in.T, s, lo, hi);
        for (int32_t r = std::max(lo, in.coupling == 0 ? s + 1 : lo); r < hi; ++r)  // ordinal: slot s is (s, s+1)
          cw[in.cwoff + (in.coupling == 0 ? s : (int64_t)s * in.T + r)] = pair_num(jobs[i], in.coupling, in.T, s, r);
      }
    }
    S.cw_d = c.ws->get<long long>("s_cw", G.ncw);
    check_cuda(cudaMemcpyAsync(S.cw_d, cw.data(), G.ncw * sizeof(long long), cudaMemcpyHostToDevice, c.stream),
               "copy");
  }
  if (any_gs && G.T > 0) {
    gs.assign(2 * (size_t)G.T, 0);
    for (int32_t i = 0; i < B; ++i) {
      const InstInfo& in = G.inst[i];
      for (int32_t s = 0; s < in.T; ++s) {
        gs[2 * (in.soff + s)] = S.has_gs_h[i] ? jobs[i].gsn[s] : jobs[i].gn;
        gs[2 * (in.soff + s) + 1] = S.has_gs_h[i] ? jobs[i].gsd[s] : jobs[i].gd;
      }
    }
    S.gs_d = c.ws->get<long long>("s_gs", 2 * (size_t)G.T);
    check_cuda(cudaMemcpyAsync(S.gs_d, gs.data(), gs.size() * sizeof(long long), cudaMemcpyHostToDevice, c.stream),
               "copy");
  }
  // randomised refinement: 2M theta_num of every instance
  S.rdiv = nullptr;
  if (S.p.theta_num > 0) {
    std::vector<RandDiv> rd(B);
    for (int32_t i = 0; i < B; ++i) {
      const InstInfo& in = G.inst[i];
      long long sum2m = 0;
      for (int32_t s = in.soff; s < in.soff + in.T; ++s) sum2m += G.two_m_host[s];
      u128 d = (u128)(ull)(S.od_h[i] * sum2m + S.csum_h[i]) * (u128)(ull)S.p.theta_num;
      if (d == 0) d = 1;  // an edgeless instance: every key is 0
      int L = 0;
      while (L < 128 && (d >> L) != 0) ++L;
      // R = floor(2^k / div) by binary long division (the remainder stays
      // below 2 div < 2^93; the quotient below 2^64)
      const int k = 62 + L;
      u128 r = 0;
      ull R = 0;
      for (int b = k; b >= 0; --b) {
        r = (r << 1) | (u128)(b == k ? 1 : 0);
        R <<= 1;
        if (r >= d) {
          r -= d;
          R |= 1;
        }
      }
      rd[i].div = d;
      rd[i].R = R;
      rd[i].k = k;
      rd[i].pad_ = 0;
    }
    S.rdiv = c.ws->get<RandDiv>("s_rdiv", B);
    check_cuda(cudaMemcpyAsync(S.rdiv, rd.data(), B * sizeof(RandDiv), cudaMemcpyHostToDevice, c.stream), "copy");
  }
  sync(c);  // hp, cw, gs and rd are pageable host memory
}

void run_leiden(Ctx& c, const SupraGraph& G, const std::vector<InstParams>& jobs, const SolveParams& p,
                int stop_level, int stop_stage, int stop_rounds, const int32_t* init, int32_t* out, Solver& S,
                RunOut& ro) {
  PhaseClock clock(c);
  cudaEvent_t t_all = clock.begin();
  const int32_t B = G.B;
  S.c = &c;
  S.G0 = &G;
  S.p = p;
  S.N0 = G.N;
  set_instances(c, S, jobs);
  const int64_t N0 = G.N;
  solver_alloc(S);
  S.inst_active = c.ws->get<int32_t>("s_active", B);
  int32_t* iter_active = c.ws->get<int32_t>("s_iter_active", B);
  fill_i32(c, iter_active, 1, B);
  setup_null_model(S);

  int32_t* labA = c.ws->get<int32_t>("lab_A", N0);
  int32_t* labB = c.ws->get<int32_t>("lab_B", N0);
  int32_t* lab0 = c.ws->get<int32_t>("lab_0", N0);
  int32_t* prev = c.ws->get<int32_t>("lab_prev", N0);
  int32_t* outc = c.ws->get<int32_t>("lab_out", N0);
  int32_t* node_of0 = c.ws->get<int32_t>("node_of0", N0);
  int32_t* diff = c.ws->get<int32_t>("diff_flag", B + 1);
  if (init) {
    check_cuda(cudaMemcpyAsync(lab0, init, N0 * sizeof(int32_t), cudaMemcpyDeviceToDevice, c.stream), "copy");
    check_label_ranges(c, G, lab0);
    if (B > 1 && N0 > 0)
      launch(c, k_add_offsets, dim3(gsz(N0)), dim3(256), 0, lab0, N0, (const int32_t*)G.inst0,
             (const int32_t*)G.inst_off0);
  } else {
    iota_i32(c, lab0, N0);
  }

  Level L0;
  L0.d = level0_view(G, S);
  if (MSLICE_CHECKED) L0.d.chk = c.d_status;
  L0.nnz = G.nnz;
  L0.nnz_eff = G.nnz_intra + S.cpl_edges;
  L0.ns = N0;

  bool debug_done = false;
  bool have_prev = false;
  for (int it = 0; it < p.n_iterations && !debug_done; ++it) {
    ro.iterations = it + 1;
    Level cur = L0;
    int32_t* lab = labA;
    int32_t* lab_next = labB;
    check_cuda(cudaMemcpyAsync(lab, lab0, N0 * sizeof(int32_t), cudaMemcpyDeviceToDevice, c.stream), "copy");
    check_cuda(cudaMemcpyAsync(S.inst_active, iter_active, B * sizeof(int32_t), cudaMemcpyDeviceToDevice, c.stream),
               "copy");
    iota_i32(c, node_of0, N0);
    int lvl = 0;
    for (;; ++lvl) {
      const bool stop_here = (it == 0 && stop_level == lvl);
      int rounds = p.max_rounds;
      if (stop_here && stop_rounds > 0) rounds = stop_rounds;
      if (stop_here && stop_rounds < 0) rounds = 0;
      // MSLICE_TRACE: host wall time of each step of the level (synchronised)
      auto wall = [&]() -> double {
        if (!c.trace) return 0.0;
        sync(c);
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
      };
      double tw[6] = {wall(), 0, 0, 0, 0, 0};
      prepare_level(S, cur);
      tw[1] = wall();
      cudaEvent_t t0 = clock.begin();
      const MoveOut mo = local_move(S, cur, lab, it, lvl, rounds);
      clock.end(1, t0);
      if (mo.capped) {
        // a level that ran out of rounds still moving: the cost of cycling
        sync(c);
        float ms = 0;
        check_cuda(cudaEventElapsedTime(&ms, t0, clock.spans.back().second.second), "event time");
        ro.ms_capped += ms;
        ro.capped_levels++;
        ro.capped_rounds += mo.rounds;
      }
      if (c.trace) {
        sync(c);
        float ms = 0;
        cudaEventElapsedTime(&ms, t0, clock.spans.back().second.second);
        fprintf(stderr, "[mslice level] it=%d lvl=%d N=%d nnz=%lld ns=%lld rounds=%lld moves=%lld lm_ms=%.3f\n", it,
                lvl, cur.d.N, (long long)cur.nnz, (long long)cur.ns, (long long)mo.rounds, (long long)mo.moves, ms);
      }
      if (lvl == 0) ro.last_level0_moves = mo.moves;
      if (stop_here && stop_stage == 1) {
        check_cuda(cudaMemcpyAsync(out, lab, cur.d.N * sizeof(int32_t), cudaMemcpyDeviceToDevice, c.stream), "copy");
        ro.out_n = cur.d.N;
        ro.levels = lvl + 1;
        debug_done = true;
        break;
      }
      tw[2] = wall();
      const bool settled = B > 1 ? freeze_settled(S, cur, lab) == 0 : count_distinct(S, lab, cur.d.N) == cur.d.N;
      tw[3] = wall();
      if (c.trace)
        fprintf(stderr, "[mslice steps] it=%d lvl=%d prepare_ms=%.3f local_move_ms=%.3f count_ms=%.3f\n", it, lvl,
                tw[1] - tw[0], tw[2] - tw[1], tw[3] - tw[2]);
      if (settled) {
        ro.stop_reason = 1;
        break;
      }
      if (lvl + 1 >= p.max_levels) {
        ro.stop_reason = 2;
        break;
      }
      tw[4] = wall();
      cudaEvent_t t1 = clock.begin();
      refine(S, cur, lab, it, lvl);
      clock.end(2, t1);
      tw[5] = wall();
      if (c.trace) fprintf(stderr, "[mslice steps] it=%d lvl=%d refine_ms=%.3f\n", it, lvl, tw[5] - tw[4]);
      if (stop_here && stop_stage == 2) {
        check_cuda(cudaMemcpyAsync(out, S.R, cur.d.N * sizeof(int32_t), cudaMemcpyDeviceToDevice, c.stream), "copy");
        ro.out_n = cur.d.N;
        ro.levels = lvl + 1;
        debug_done = true;
        break;
      }
      if (B > 1 && freeze_settled(S, cur, S.R) == 0) {
        ro.stop_reason = 3;
        break;
      }
      Level nxt;
      int64_t ck = 0;
      cudaEvent_t t2 = clock.begin();
      const bool shrunk = aggregate(S, cur, lab, nxt, (lvl % 2 == 0) ? "LA" : "LB", lab_next, node_of0,
                                    (stop_here && stop_stage == 3) ? &ck : nullptr);
      clock.end(3, t2);
      if (c.trace) fprintf(stderr, "[mslice steps] it=%d lvl=%d aggregate_ms=%.3f\n", it, lvl, wall() - tw[5]);
      if (!shrunk) {
        ro.stop_reason = 3;
        break;
      }
      if (stop_here && stop_stage == 3) {
        check_cuda(cudaMemcpyAsync(out, lab_next, nxt.d.N * sizeof(int32_t), cudaMemcpyDeviceToDevice, c.stream),
                   "copy");
        ro.out_n = nxt.d.N;
        ro.next_n = nxt.d.N;
        ro.next_nnz = nxt.nnz;
        ro.next_checksum = (uint64_t)ck;
        ro.levels = lvl + 1;
        debug_done = true;
        break;
      }
      cur = nxt;
      std::swap(lab, lab_next);
    }
    if (debug_done) break;
    ro.levels = lvl + 1;
    // flatten to supra-nodes and canonicalise within each instance
    int32_t* flat = lab_next;  // free buffer of N0 entries
    if (N0 > 0) launch(c, k_gather, dim3(gsz(N0)), dim3(256), 0, (const int32_t*)lab, (const int32_t*)node_of0, N0, flat);
    canonicalise(S, flat, outc, N0);
    bool all_frozen = false;
    if (have_prev) {
      check_cuda(cudaMemsetAsync(diff, 0, (B + 1) * sizeof(int32_t), c.stream), "memset");
      if (N0 > 0)
        launch(c, k_differs, dim3(gsz(N0)), dim3(256), 0, (const int32_t*)outc, (const int32_t*)prev, N0,
               (const int32_t*)(B > 1 ? G.inst0 : nullptr), diff);
      launch(c, k_freeze, dim3(1), dim3(256), 0, (const int32_t*)diff, iter_active, B, diff + B);
      all_frozen = *static_cast<const int32_t*>(readback(c, diff + B, sizeof(int32_t))) == 0;
    }
    std::swap(prev, outc);
    have_prev = true;
    // the next iteration starts from these labels; canonical labels count
    // from 0 within each instance, so shift them back into its id range
    check_cuda(cudaMemcpyAsync(lab0, prev, N0 * sizeof(int32_t), cudaMemcpyDeviceToDevice, c.stream), "copy");
    if (B > 1 && N0 > 0)
      launch(c, k_add_offsets, dim3(gsz(N0)), dim3(256), 0, lab0, N0, (const int32_t*)G.inst0,
             (const int32_t*)G.inst_off0);
    if (all_frozen) break;
  }
  if (!debug_done) {
    ro.Q.assign(B, 0.0);
    cudaEvent_t t3 = clock.begin();
    modularity(S, lab0, ro.Q.data());
    clock.end(4, t3);
    if (N0 > 0) check_cuda(cudaMemcpyAsync(out, prev, N0 * sizeof(int32_t), cudaMemcpyDeviceToDevice, c.stream), "copy");
    ro.out_n = N0;
  }
  clock.end(0, t_all);
  clock.totals(ro.ms);
  check_status(c, "leiden");
}

}  // namespace mslice
