// C ABI of the mslice library (include/mslice.h) and the Leiden driver.
//
// Driver (Sec. 3.2: Leiden = local moving, refinement, aggregation):
//   for it in 0..n_iterations-1 (the paper caps runs at two passes, Sec. 4):
//     level 0 starts from the warm-start / previous labels (singletons first)
//     per level: local moving; stop if every community is one node or at
//     max_levels; refinement; stop if it merged nothing; aggregation
//     flatten the last level's labels to supra-nodes, canonicalise,
//     stop early when an iteration returns the labels it started from
//   Q of the final labels (exact gamma).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <functional>
#include <new>
#include <string>
#include <vector>

#include "../../include/mslice.h"
#include "solver.h"

namespace mslice {

static thread_local std::string g_last_error;

void fail(int code, const std::string& msg) { throw Error{code, msg}; }

void set_last_error(const std::string& msg) { g_last_error = msg; }

void check_cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return;
  const int code = (e == cudaErrorMemoryAllocation) ? MSLICE_ENOMEM : MSLICE_ECUDA;
  fail(code, std::string(what) + ": " + cudaGetErrorString(e));
}

Workspace::~Workspace() { release_all(); }

void* Workspace::get_bytes(const std::string& name, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  auto it = bufs_.find(name);
  if (it != bufs_.end()) {
    if (it->second.second >= bytes) return it->second.first;
    cudaFreeAsync(it->second.first, stream);
    bufs_.erase(it);
  }
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, bytes, stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(MSLICE_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes for " + name + " failed");
  }
  bufs_[name] = {p, bytes};
  return p;
}

void Workspace::release(const std::string& name) {
  auto it = bufs_.find(name);
  if (it == bufs_.end()) return;
  cudaFreeAsync(it->second.first, stream);
  bufs_.erase(it);
}

void Workspace::release_all() {
  for (auto& kv : bufs_) cudaFreeAsync(kv.second.first, stream);
  if (!bufs_.empty()) cudaStreamSynchronize(stream);
  bufs_.clear();
}

size_t Workspace::bytes_held() const {
  size_t t = 0;
  for (const auto& kv : bufs_) t += kv.second.second;
  return t;
}

void sync(Ctx& c) { check_cuda(cudaStreamSynchronize(c.stream), "stream synchronize"); }

void trace_begin(Ctx& c, const void*, cudaEvent_t* e0) {
  check_cuda(cudaEventCreate(e0), "event");
  check_cuda(cudaEventRecord(*e0, c.stream), "event");
}

void trace_end(Ctx& c, const void* k, cudaEvent_t e0) {
  cudaEvent_t e1;
  check_cuda(cudaEventCreate(&e1), "event");
  check_cuda(cudaEventRecord(e1, c.stream), "event");
  c.trace->push_back({k, {e0, e1}});
}

// Per-kernel totals of a traced call, printed to stderr.
static void trace_report(Ctx& c) {
  sync(c);
  std::map<std::string, std::pair<int64_t, double>> agg;
  double tot = 0;
  for (auto& t : *c.trace) {
    float ms = 0;
    cudaEventElapsedTime(&ms, t.second.first, t.second.second);
    cudaEventDestroy(t.second.first);
    cudaEventDestroy(t.second.second);
    const char* name = nullptr;
    if (cudaFuncGetName(&name, t.first) != cudaSuccess || !name) name = "?";
    auto& a = agg[name];
    a.first++;
    a.second += ms;
    tot += ms;
  }
  cudaGetLastError();
  c.trace->clear();
  std::vector<std::pair<double, std::string>> order;
  for (auto& kv : agg) order.push_back({kv.second.second, kv.first});
  std::sort(order.rbegin(), order.rend());
  fprintf(stderr, "[mslice trace] %.3f ms in %zu kernel kinds\n", tot, order.size());
  for (auto& o : order) {
    const auto& a = agg[o.second];
    fprintf(stderr, "[mslice trace] %9.3f ms %5.1f%% %7lld launches %8.1f us/launch  %.110s\n", a.second,
            100.0 * a.second / (tot > 0 ? tot : 1), (long long)a.first, 1e3 * a.second / a.first, o.second.c_str());
  }
}

void* readback(Ctx& c, const void* dptr, size_t bytes) {
  check_cuda(cudaMemcpyAsync(c.pinned, dptr, bytes, cudaMemcpyDeviceToHost, c.stream), "readback");
  sync(c);
  return c.pinned;
}

void check_status(Ctx& c, const char* where) {
  const unsigned st = *static_cast<const unsigned*>(readback(c, c.d_status, sizeof(unsigned)));
  if (st == 0) return;
  check_cuda(cudaMemsetAsync(c.d_status, 0, sizeof(unsigned), c.stream), "memset");
  if (st & ERR_BAD_INPUT) fail(MSLICE_EINVAL, std::string(where) + ": malformed input");
  if (st & ERR_HASH_FULL) fail(MSLICE_ECUDA, std::string(where) + ": internal hash table overflow");
  fail(MSLICE_ECUDA, std::string(where) + ": internal error");
}

namespace {

__global__ void k_check_labels(const int32_t* x, int64_t N, int64_t hi, unsigned* status) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    if (x[i] < 0 || x[i] >= hi) atomicOr(status, ERR_BAD_INPUT);
}

__global__ void k_gather(const int32_t* labels, const int32_t* node_of0, int64_t N0, int32_t* out) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N0; v += (int64_t)gridDim.x * blockDim.x)
    out[v] = labels[node_of0[v]];
}

__global__ void k_differs(const int32_t* a, const int32_t* b, int64_t N, int32_t* flag) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
    if (a[v] != b[v]) *flag = 1;
}

unsigned gsz(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

// CUDA-event phase timing: events recorded on the handle's stream.
struct PhaseClock {
  Ctx& c;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> spans;
  explicit PhaseClock(Ctx& cc) : c(cc) {}
  ~PhaseClock() {
    for (auto& s : spans) {
      cudaEventDestroy(s.second.first);
      cudaEventDestroy(s.second.second);
    }
  }
  cudaEvent_t begin() {
    cudaEvent_t e;
    check_cuda(cudaEventCreate(&e), "event");
    check_cuda(cudaEventRecord(e, c.stream), "event");
    return e;
  }
  void end(int phase, cudaEvent_t b) {
    cudaEvent_t e;
    check_cuda(cudaEventCreate(&e), "event");
    check_cuda(cudaEventRecord(e, c.stream), "event");
    spans.push_back({phase, {b, e}});
  }
  void totals(double out[5]) {
    sync(c);
    for (int i = 0; i < 5; ++i) out[i] = 0;
    for (auto& s : spans) {
      float ms = 0;
      check_cuda(cudaEventElapsedTime(&ms, s.second.first, s.second.second), "event time");
      out[s.first] += ms;
    }
  }
};

}  // namespace
}  // namespace mslice

using namespace mslice;

struct mslice_graph {
  SupraGraph G;
  Workspace ws;
  cudaStream_t stream = nullptr;
  unsigned* d_status = nullptr;
  void* pinned = nullptr;
  long long on = 1, od = 1;
  int64_t launches = 0;
  Ctx ctx() {
    Ctx c;
    c.stream = stream;
    c.ws = &ws;
    c.d_status = d_status;
    c.pinned = pinned;
    return c;
  }
  ~mslice_graph() {
    ws.release_all();
    G.mem.release_all();
    if (pinned) cudaFreeHost(pinned);
  }
};

namespace {

int guard(const std::function<void()>& f) {
  try {
    f();
    g_last_error.clear();
    return MSLICE_OK;
  } catch (const Error& e) {
    g_last_error = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return MSLICE_ENOMEM;
  }
}

// Freed stream-ordered allocations stay in the device's default pool, so
// handles created and released in a loop do not pay for fresh allocations.
void keep_pool_memory() {
  static bool done = false;
  if (done) return;
  int dev = 0;
  cudaMemPool_t pool;
  if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  done = true;
}

bool rational_ok(int64_t num, int64_t den, bool allow_zero) {
  const int64_t lim = (int64_t)1 << 31;
  return den >= 1 && den <= lim && num >= (allow_zero ? 0 : 1) && num <= lim;
}

void check_bounds(const SupraGraph& G, long long gn, long long gd, long long on, long long od) {
  u128 sum2m = 0;
  for (int64_t t : G.two_m_host) sum2m += (u128)(ull)t;
  const u128 ncpl = (u128)(ull)G.n * (u128)(ull)(G.T - 1);
  const u128 lim = (u128)1 << 61;
  if ((u128)(ull)od * sum2m + 2 * (u128)(ull)on * ncpl >= lim)
    fail(MSLICE_EOVERFLOW, "omega_den*sum(2m_s) + 2*omega_num*n*(T-1) must stay below 2^61");
  if ((u128)(ull)gn * (u128)(ull)od * sum2m >= lim * (u128)(ull)gd)
    fail(MSLICE_EOVERFLOW, "gamma*omega_den*sum(2m_s) must stay below 2^61");
}

void check_labels(Ctx& c, const int32_t* d, int64_t N) {
  if (N == 0) return;
  check_cuda(cudaMemsetAsync(c.d_status, 0, sizeof(unsigned), c.stream), "memset");
  launch(c, k_check_labels, dim3(gsz(N)), dim3(256), 0, d, N, N, c.d_status);
  check_status(c, "labels");
}

}  // namespace

extern "C" {

void mslice_default_opts(mslice_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->n_iterations = 2;
  o->K = 4;
  o->max_rounds = 100;
  o->max_levels = 32;
  o->seed = 0;
  o->gamma_num = 1;
  o->gamma_den = 1;
  o->omega_num = 1;
  o->omega_den = 1;
  o->flags = 0;
  o->stop_level = -1;
  o->stop_stage = 0;
  o->stop_rounds = 0;
}

const char* mslice_last_error(void) { return g_last_error.c_str(); }

int mslice_build_ex(const mslice_csr* slices, int32_t T, mslice_coupling cpl, int64_t omega_num, int64_t omega_den,
                    int32_t flags, void* stream, mslice_handle* out) {
  mslice_graph* h = nullptr;
  const int rc = guard([&] {
    if (!out) fail(MSLICE_EINVAL, "null output handle");
    *out = nullptr;
    if (!slices || T < 1) fail(MSLICE_EINVAL, "need T >= 1 snapshots");
    if (cpl != MSLICE_ORDINAL) fail(MSLICE_EINVAL, "unsupported coupling");
    if (!rational_ok(omega_num, omega_den, true)) fail(MSLICE_EINVAL, "omega must be a rational >= 0");
    const int64_t n = slices[0].n;
    if (n < 0 || n > INT32_MAX || n * (int64_t)T > INT32_MAX) fail(MSLICE_EINVAL, "n*T must fit in int32");
    for (int32_t s = 0; s < T; ++s)
      if (slices[s].n != n) fail(MSLICE_EINVAL, "snapshots must have the same n");
    h = new mslice_graph();
    h->stream = static_cast<cudaStream_t>(stream);
    h->ws.stream = h->stream;
    h->G.mem.stream = h->stream;
    keep_pool_memory();
    h->on = omega_num;
    h->od = omega_den;
    check_cuda(cudaMallocHost(&h->pinned, 4096), "pinned buffer");
    h->d_status = h->ws.get<unsigned>("status", 4);
    Ctx c = h->ctx();
    check_cuda(cudaMemsetAsync(h->d_status, 0, 16, c.stream), "memset");
    const bool dev = (flags & MSLICE_DEVICE_PTRS) != 0;
    std::vector<const int64_t*> ip(T);
    std::vector<const int32_t*> ix(T), wt(T);
    std::vector<int64_t> nnz(T);
    for (int32_t s = 0; s < T; ++s) {
      if (n > 0 && !slices[s].indptr) fail(MSLICE_EINVAL, "null indptr");
      int64_t z = 0;
      if (n > 0) {
        if (dev)
          check_cuda(cudaMemcpy(&z, slices[s].indptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost), "copy");
        else
          z = slices[s].indptr[n];
      }
      if (z < 0) fail(MSLICE_EINVAL, "negative nnz");
      if (z > 0 && (!slices[s].indices || !slices[s].weights)) fail(MSLICE_EINVAL, "null indices/weights");
      nnz[s] = z;
      if (dev) {
        ip[s] = slices[s].indptr;
        ix[s] = slices[s].indices;
        wt[s] = slices[s].weights;
      } else {
        const std::string tag = std::to_string(s);
        int64_t* dip = h->ws.get<int64_t>("in_ip" + tag, n + 1);
        int32_t* dix = h->ws.get<int32_t>("in_ix" + tag, z);
        int32_t* dwt = h->ws.get<int32_t>("in_wt" + tag, z);
        if (n > 0) {
          check_cuda(cudaMemcpyAsync(dip, slices[s].indptr, (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                                     c.stream), "copy");
        } else {
          check_cuda(cudaMemsetAsync(dip, 0, sizeof(int64_t), c.stream), "memset");
        }
        if (z > 0) {
          check_cuda(cudaMemcpyAsync(dix, slices[s].indices, z * sizeof(int32_t), cudaMemcpyHostToDevice, c.stream),
                     "copy");
          check_cuda(cudaMemcpyAsync(dwt, slices[s].weights, z * sizeof(int32_t), cudaMemcpyHostToDevice, c.stream),
                     "copy");
        }
        ip[s] = dip;
        ix[s] = dix;
        wt[s] = dwt;
      }
    }
    build_supra(c, ip, ix, wt, nnz, n, h->G);
    h->launches += c.launches;
    // staged host copies are not needed after the build
    if (!dev)
      for (int32_t s = 0; s < T; ++s) {
        const std::string tag = std::to_string(s);
        h->ws.release("in_ip" + tag);
        h->ws.release("in_ix" + tag);
        h->ws.release("in_wt" + tag);
      }
    *out = h;
  });
  if (rc != MSLICE_OK && h) delete h;
  return rc;
}

int mslice_build(const mslice_csr* slices, int32_t T, mslice_coupling cpl, int64_t omega_num, int64_t omega_den,
                 mslice_handle* out) {
  return mslice_build_ex(slices, T, cpl, omega_num, omega_den, 0, nullptr, out);
}

int mslice_info(mslice_handle h, int64_t* N, int32_t* T, int64_t* n, int64_t* nnz) {
  if (!h) {
    g_last_error = "null handle";
    return MSLICE_EINVAL;
  }
  if (N) *N = h->G.N;
  if (T) *T = h->G.T;
  if (n) *n = h->G.n;
  if (nnz) *nnz = h->G.nnz;
  return MSLICE_OK;
}

void mslice_free(mslice_handle h) { delete h; }

int64_t mslice_kernel_launches(mslice_handle h) { return h ? h->launches : -1; }

int mslice_leiden_ex(mslice_handle h, const mslice_opts* o, const int32_t* init_labels, int32_t* labels_out,
                     double* Q_out, mslice_stats* st) {
  return guard([&] {
    if (!h) fail(MSLICE_EINVAL, "null handle");
    mslice_opts opt;
    mslice_default_opts(&opt);
    if (o) opt = *o;
    if (opt.n_iterations < 1 || opt.K < 1 || opt.max_rounds < 1 || opt.max_levels < 1)
      fail(MSLICE_EINVAL, "n_iterations, K, max_rounds and max_levels must be >= 1");
    if (opt.K > 64) fail(MSLICE_EINVAL, "K must be at most 64");
    if (!rational_ok(opt.gamma_num, opt.gamma_den, false)) fail(MSLICE_EINVAL, "gamma must be a rational > 0");
    if (!rational_ok(opt.omega_num, opt.omega_den, true)) fail(MSLICE_EINVAL, "omega must be a rational >= 0");
    if (!labels_out && h->G.N > 0) fail(MSLICE_EINVAL, "null labels_out");
    const bool dev = (opt.flags & MSLICE_DEVICE_PTRS) != 0;
    const SupraGraph& G = h->G;
    check_bounds(G, opt.gamma_num, opt.gamma_den, opt.omega_num, opt.omega_den);
    Ctx c = h->ctx();
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_spans;
    c.profile = (opt.flags & MSLICE_PROFILE) != 0;
    c.prof_spans = &prof_spans;
    std::vector<std::pair<const void*, std::pair<cudaEvent_t, cudaEvent_t>>> trace;
    if (std::getenv("MSLICE_TRACE")) c.trace = &trace;
    PhaseClock clock(c);
    cudaEvent_t t_all = clock.begin();

    Solver S;
    S.c = &c;
    S.G0 = &G;
    S.p.gn = opt.gamma_num;
    S.p.gd = opt.gamma_den;
    S.p.on = opt.omega_num;
    S.p.od = opt.omega_den;
    S.p.K = opt.K;
    S.p.max_rounds = opt.max_rounds;
    S.p.max_levels = opt.max_levels;
    S.p.n_iterations = opt.n_iterations;
    S.p.seed = opt.seed;
    S.N0 = G.N;
    const int64_t N0 = G.N;
    solver_alloc(S);
    S.lam = h->ws.get<u128>("lam", G.T);
    compute_lambda(c, G, S.p.gn, S.p.gd, S.lam);

    int32_t* labA = h->ws.get<int32_t>("lab_A", N0);
    int32_t* labB = h->ws.get<int32_t>("lab_B", N0);
    int32_t* lab0 = h->ws.get<int32_t>("lab_0", N0);
    int32_t* prev = h->ws.get<int32_t>("lab_prev", N0);
    int32_t* outc = h->ws.get<int32_t>("lab_out", N0);
    int32_t* node_of0 = h->ws.get<int32_t>("node_of0", N0);
    int32_t* dflag = h->ws.get<int32_t>("diff_flag", 1);
    if (init_labels) {
      if (dev)
        check_cuda(cudaMemcpyAsync(lab0, init_labels, N0 * sizeof(int32_t), cudaMemcpyDeviceToDevice, c.stream), "copy");
      else
        check_cuda(cudaMemcpyAsync(lab0, init_labels, N0 * sizeof(int32_t), cudaMemcpyHostToDevice, c.stream), "copy");
      check_labels(c, lab0, N0);
    } else {
      iota_i32(c, lab0, N0);
    }

    mslice_stats stats;
    std::memset(&stats, 0, sizeof(stats));
    const LevelDev d0 = level0_view(G, S.p.on, S.p.od);
    Level L0;
    L0.d = d0;
    L0.nnz = G.nnz;
    L0.nnz_eff = S.p.on > 0 ? G.nnz : G.nnz_intra;
    L0.ns = N0;

    bool debug_done = false;
    bool have_prev = false;
    for (int it = 0; it < opt.n_iterations && !debug_done; ++it) {
      stats.iterations = it + 1;
      Level cur = L0;
      int32_t* lab = labA;
      int32_t* lab_next = labB;
      check_cuda(cudaMemcpyAsync(lab, lab0, N0 * sizeof(int32_t), cudaMemcpyDeviceToDevice, c.stream), "copy");
      iota_i32(c, node_of0, N0);
      int lvl = 0;
      for (;; ++lvl) {
        const bool stop_here = (it == 0 && opt.stop_level == lvl);
        int rounds = opt.max_rounds;
        if (stop_here && opt.stop_rounds > 0) rounds = opt.stop_rounds;
        if (stop_here && opt.stop_rounds < 0) rounds = 0;
        prepare_level(S, cur);
        cudaEvent_t t0 = clock.begin();
        const MoveOut mo = local_move(S, cur, lab, it, lvl, rounds);
        clock.end(1, t0);
        if (c.trace) {
          sync(c);
          float ms = 0;
          cudaEventElapsedTime(&ms, t0, clock.spans.back().second.second);
          fprintf(stderr, "[mslice level] it=%d lvl=%d N=%d nnz=%lld rounds=%lld moves=%lld lm_ms=%.3f tiers=%d/%d/%d/%d/%d\n",
                  it, lvl, cur.d.N, (long long)cur.nnz, (long long)mo.rounds, (long long)mo.moves, ms, S.tier_cnt[0],
                  S.tier_cnt[1], S.tier_cnt[2], S.tier_cnt[3], S.tier_cnt[4]);
        }
        if (lvl == 0) stats.last_level0_moves = mo.moves;
        if (stop_here && opt.stop_stage == 1) {
          check_cuda(cudaMemcpyAsync(labels_out, lab, cur.d.N * sizeof(int32_t),
                                     dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c.stream), "copy");
          stats.out_n = cur.d.N;
          stats.levels = lvl + 1;
          debug_done = true;
          break;
        }
        if (count_distinct(S, lab, cur.d.N) == cur.d.N) {
          stats.stop_reason = 1;
          break;
        }
        if (lvl + 1 >= opt.max_levels) {
          stats.stop_reason = 2;
          break;
        }
        cudaEvent_t t1 = clock.begin();
        refine(S, cur, lab, it, lvl);
        clock.end(2, t1);
        if (stop_here && opt.stop_stage == 2) {
          check_cuda(cudaMemcpyAsync(labels_out, S.R, cur.d.N * sizeof(int32_t),
                                     dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c.stream), "copy");
          stats.out_n = cur.d.N;
          stats.levels = lvl + 1;
          debug_done = true;
          break;
        }
        Level nxt;
        int64_t ck = 0;
        cudaEvent_t t2 = clock.begin();
        const bool shrunk = aggregate(S, cur, lab, nxt, (lvl % 2 == 0) ? "LA" : "LB", lab_next, node_of0,
                                      (stop_here && opt.stop_stage == 3) ? &ck : nullptr);
        clock.end(3, t2);
        if (!shrunk) {
          stats.stop_reason = 3;
          break;
        }
        if (stop_here && opt.stop_stage == 3) {
          check_cuda(cudaMemcpyAsync(labels_out, lab_next, nxt.d.N * sizeof(int32_t),
                                     dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c.stream), "copy");
          stats.out_n = nxt.d.N;
          stats.next_n = nxt.d.N;
          stats.next_nnz = nxt.nnz;
          stats.next_checksum = (uint64_t)ck;
          stats.levels = lvl + 1;
          debug_done = true;
          break;
        }
        cur = nxt;
        std::swap(lab, lab_next);
      }
      if (debug_done) break;
      stats.levels = lvl + 1;
      // flatten to supra-nodes and canonicalise
      int32_t* flat = lab_next;  // free buffer of size N0
      if (N0 > 0) launch(c, k_gather, dim3(gsz(N0)), dim3(256), 0, (const int32_t*)lab, (const int32_t*)node_of0, N0, flat);
      canonicalise(S, flat, outc, N0);
      bool same = false;
      if (have_prev && N0 > 0) {
        check_cuda(cudaMemsetAsync(dflag, 0, sizeof(int32_t), c.stream), "memset");
        launch(c, k_differs, dim3(gsz(N0)), dim3(256), 0, (const int32_t*)outc, (const int32_t*)prev, N0, dflag);
        same = *static_cast<const int32_t*>(readback(c, dflag, sizeof(int32_t))) == 0;
      } else if (have_prev) {
        same = true;
      }
      std::swap(prev, outc);
      have_prev = true;
      check_cuda(cudaMemcpyAsync(lab0, prev, N0 * sizeof(int32_t), cudaMemcpyDeviceToDevice, c.stream), "copy");
      if (same) break;
    }
    if (!debug_done) {
      double Q = 0.0;
      cudaEvent_t t3 = clock.begin();
      modularity(S, prev, &Q);
      clock.end(4, t3);
      if (N0 > 0)
        check_cuda(cudaMemcpyAsync(labels_out, prev, N0 * sizeof(int32_t),
                                   dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c.stream), "copy");
      stats.out_n = N0;
      if (Q_out) *Q_out = Q;
    }
    clock.end(0, t_all);
    double ms[5];
    clock.totals(ms);
    check_status(c, "leiden");
    stats.ms_total = ms[0];
    stats.ms_local_move = ms[1];
    stats.ms_refine = ms[2];
    stats.ms_aggregate = ms[3];
    stats.ms_modularity = ms[4];
    stats.lm_rounds = S.lm_rounds;
    stats.lm_edges = S.lm_edges;
    stats.lm_moves = S.lm_moves;
    stats.kernel_launches = c.launches;
    h->launches += c.launches;
    if (c.trace) trace_report(c);
    if (c.profile) {
      double dms = 0;
      for (auto& sp : prof_spans) {
        float ms = 0;
        check_cuda(cudaEventElapsedTime(&ms, sp.first, sp.second), "event time");
        dms += ms;
        cudaEventDestroy(sp.first);
        cudaEventDestroy(sp.second);
      }
      stats.ms_decide = dms;
      stats.decide_launches = (int64_t)prof_spans.size();
      stats.decide_bytes = c.prof_bytes;
    }
    if (st) *st = stats;
  });
}

int mslice_leiden(mslice_handle h, int64_t gamma_num, int64_t gamma_den, int64_t omega_num, int64_t omega_den,
                  int32_t max_levels, uint64_t seed, int32_t* labels_out, double* Q_out) {
  mslice_opts o;
  mslice_default_opts(&o);
  o.gamma_num = gamma_num;
  o.gamma_den = gamma_den;
  o.omega_num = omega_num;
  o.omega_den = omega_den;
  o.max_levels = max_levels;
  o.seed = seed;
  return mslice_leiden_ex(h, &o, nullptr, labels_out, Q_out, nullptr);
}

int mslice_modularity_ex(mslice_handle h, const int32_t* labels, int64_t gamma_num, int64_t gamma_den,
                         int64_t omega_num, int64_t omega_den, int32_t flags, double* Q_out) {
  return guard([&] {
    if (!h) fail(MSLICE_EINVAL, "null handle");
    if (!rational_ok(gamma_num, gamma_den, false)) fail(MSLICE_EINVAL, "gamma must be a rational > 0");
    if (!rational_ok(omega_num, omega_den, true)) fail(MSLICE_EINVAL, "omega must be a rational >= 0");
    const SupraGraph& G = h->G;
    if (!labels && G.N > 0) fail(MSLICE_EINVAL, "null labels");
    check_bounds(G, gamma_num, gamma_den, omega_num, omega_den);
    Ctx c = h->ctx();
    Solver S;
    S.c = &c;
    S.G0 = &G;
    S.p.gn = gamma_num;
    S.p.gd = gamma_den;
    S.p.on = omega_num;
    S.p.od = omega_den;
    S.N0 = G.N;
    const int64_t N = G.N > 0 ? G.N : 1;
    S.sig_used = h->ws.get<ull>("m_used", 1);
    int32_t* lab = h->ws.get<int32_t>("m_lab", N);
    if (G.N > 0) {
      const bool dev = (flags & MSLICE_DEVICE_PTRS) != 0;
      check_cuda(cudaMemcpyAsync(lab, labels, G.N * sizeof(int32_t),
                                 dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c.stream), "copy");
      check_labels(c, lab, G.N);
    }
    double Q = 0.0;
    modularity(S, lab, &Q);
    check_status(c, "modularity");
    h->launches += c.launches;
    if (Q_out) *Q_out = Q;
  });
}

int mslice_modularity(mslice_handle h, const int32_t* labels, int64_t gamma_num, int64_t gamma_den,
                      int64_t omega_num, int64_t omega_den, double* Q_out) {
  return mslice_modularity_ex(h, labels, gamma_num, gamma_den, omega_num, omega_den, 0, Q_out);
}

}  // extern "C"
