// C ABI of the mslice library (include/mslice.h): argument checks, host and
// device buffers, handles and batches around the driver (driver.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <functional>
#include <new>
#include <string>
#include <unordered_set>
#include <vector>

#include "../../include/mslice.h"
#include "solver.h"

namespace mslice {

static thread_local std::string g_last_error;

void fail(int code, const std::string& msg) { throw Error{code, msg}; }

void set_last_error(const std::string& msg) { g_last_error = msg; }

// Freed stream-ordered allocations stay in the device's default pool, so
// handles created and released in a loop do not pay for fresh allocations.
void keep_pool_memory() {
  static std::once_flag once;
  std::call_once(once, [] {
  int dev = 0;
  cudaMemPool_t pool;
  if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  });
}


void check_cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return;
  const int code = (e == cudaErrorMemoryAllocation) ? MSLICE_ENOMEM : MSLICE_ECUDA;
  fail(code, std::string(what) + ": " + cudaGetErrorString(e));
}

Workspace::~Workspace() { release_all(); }

// Host-side fault injection for the tests: with MSLICE_FAIL_ALLOC_AFTER=k in
// the environment, every device allocation after the first k (counted since
// the variable last changed) fails as if the device were out of memory.
static bool injected_alloc_failure() {
  static std::mutex mu;
  static std::string last;
  static long long count = 0;
  const char* e = std::getenv("MSLICE_FAIL_ALLOC_AFTER");
  std::lock_guard<std::mutex> lk(mu);
  const std::string cur = e ? e : "";
  if (cur != last) {
    last = cur;
    count = 0;
  }
  if (cur.empty()) return false;
  return count++ >= std::atoll(cur.c_str());
}

void* Workspace::get_bytes(const std::string& name, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  auto it = bufs_.find(name);
  if (it != bufs_.end()) {
    if (it->second.second >= bytes) return it->second.first;
    cudaFreeAsync(it->second.first, stream);
    bufs_.erase(it);
  }
  if (injected_alloc_failure())
    fail(MSLICE_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes for " + name + " failed (injected)");
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, bytes, stream);
  if (e == cudaErrorMemoryAllocation) {
    // The device pool keeps freed memory for reuse (keep_pool_memory); when
    // that leaves too little for this request, wait for pending frees,
    // return the pool's unused memory and try once more.
    cudaGetLastError();
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaDeviceSynchronize() == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess && cudaMemPoolTrimTo(pool, 0) == cudaSuccess)
      e = cudaMallocAsync(&p, bytes, stream);
  }
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

namespace {
std::mutex g_coop_mu;
cudaEvent_t g_coop_ev[64] = {};
}  // namespace

CoopOrder::CoopOrder(cudaStream_t s) : s_(s) {
  g_coop_mu.lock();
  if (cudaGetDevice(&dev_) != cudaSuccess || dev_ < 0 || dev_ >= 64) dev_ = 0;
  if (!g_coop_ev[dev_]) {
    if (cudaEventCreateWithFlags(&g_coop_ev[dev_], cudaEventDisableTiming) != cudaSuccess) g_coop_ev[dev_] = nullptr;
  } else {
    cudaStreamWaitEvent(s_, g_coop_ev[dev_], 0);
  }
}

CoopOrder::~CoopOrder() {
  if (g_coop_ev[dev_]) cudaEventRecord(g_coop_ev[dev_], s_);
  g_coop_mu.unlock();
}

void StreamFan::create() {
  int lo = 0, hi = 0;
  check_cuda(cudaDeviceGetStreamPriorityRange(&lo, &hi), "stream priorities");
  for (int k = 0; k < kSide; ++k) {
    // side 0 and 1 carry the block-per-node tiers: highest priority, so their
    // blocks are placed before the group tiers' queued blocks
    check_cuda(cudaStreamCreateWithPriority(&side[k], cudaStreamNonBlocking, k < 2 ? hi : lo), "stream");
    check_cuda(cudaEventCreateWithFlags(&join[k], cudaEventDisableTiming), "event");
  }
  check_cuda(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming), "event");
}

void StreamFan::destroy() {
  for (int k = 0; k < kSide; ++k) {
    if (side[k]) cudaStreamSynchronize(side[k]);
    if (side[k]) cudaStreamDestroy(side[k]);
    if (join[k]) cudaEventDestroy(join[k]);
    side[k] = nullptr;
    join[k] = nullptr;
  }
  if (fork) cudaEventDestroy(fork);
  fork = nullptr;
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
  if (bytes > PINNED_BYTES) fail(MSLICE_ECUDA, "readback larger than the pinned staging buffer");
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
  if (st & ERR_BOUNDS) fail(MSLICE_ECUDA, std::string(where) + ": bound check failed (checked build)");
  fail(MSLICE_ECUDA, std::string(where) + ": internal error");
}

}  // namespace mslice

using namespace mslice;

struct mslice_graph {
  SupraGraph G;
  uint64_t serial = 0;  // unique per built graph (batches cache their concatenation by it)
  Workspace ws;
  cudaStream_t stream = nullptr;
  unsigned* d_status = nullptr;
  void* pinned = nullptr;
  long long on = 1, od = 1;
  int64_t launches = 0;
  StreamFan fan;
  bool own_stream = false;
  Ctx ctx() {
    Ctx c;
    c.stream = stream;
    c.fan = fan.fork ? &fan : nullptr;
    c.ws = &ws;
    c.d_status = d_status;
    c.pinned = pinned;
    return c;
  }
  ~mslice_graph() {
    ws.release_all();
    G.mem.release_all();
    fan.destroy();
    if (pinned) cudaFreeHost(pinned);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }
};


struct mslice_batch_s {
  cudaStream_t stream = nullptr;
  Workspace ws;
  unsigned* d_status = nullptr;
  void* pinned = nullptr;
  int32_t flags = 0;
  // instances, in add order
  std::vector<mslice_graph*> graphs;
  std::vector<InstParams> jobs;
  std::vector<int64_t> off{0};     // first supra-node of every instance (B+1)
  std::vector<int32_t> init;       // warm starts (local ids), filled with singletons where none was given
  bool any_init = false;
  // concatenated supra-graph and the graph serials it was built from
  SupraGraph G;
  std::vector<uint64_t> G_serials;
  bool solved = false;
  std::vector<double> Q;
  int64_t launches = 0;
  StreamFan fan;
  bool own_stream = false;
  Ctx ctx() {
    Ctx c;
    c.stream = stream;
    c.fan = fan.fork ? &fan : nullptr;
    c.ws = &ws;
    c.d_status = d_status;
    c.pinned = pinned;
    return c;
  }
  ~mslice_batch_s() {
    ws.release_all();
    G.mem.release_all();
    fan.destroy();
    if (pinned) cudaFreeHost(pinned);
    if (own_stream && stream) cudaStreamDestroy(stream);
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

bool rational_ok(int64_t num, int64_t den, bool allow_zero) {
  const int64_t lim = (int64_t)1 << 31;
  return den >= 1 && den <= lim && num >= (allow_zero ? 0 : 1) && num <= lim;
}

void sync_stream(cudaStream_t s) { check_cuda(cudaStreamSynchronize(s), "stream synchronize"); }

void check_opts(const mslice_opts& opt) {
  if (opt.n_iterations < 1 || opt.K < 1 || opt.max_rounds < 1 || opt.max_levels < 1)
    fail(MSLICE_EINVAL, "n_iterations, K, max_rounds and max_levels must be >= 1");
  if (opt.K > 64) fail(MSLICE_EINVAL, "K must be at most 64");
  if (!rational_ok(opt.theta_num, opt.theta_den, true)) fail(MSLICE_EINVAL, "theta must be a rational >= 0");
  const int32_t* t = opt.tier_cuts;
  if (t[0] || t[1] || t[2] || t[3]) {
    int32_t lo = 0;
    for (int k = 0; k < 4; ++k) {
      if (t[k] < lo || t[k] > TIER_MAX[k])
        fail(MSLICE_EINVAL, "tier cuts must be ascending and within the tiers' capacities (16, 32, " +
                                std::to_string(TIER_MAX[2]) + ", 1024)");
      lo = t[k];
    }
  }
}

// The null model the flags select (EINVAL for two at once).
int null_model_of(int32_t flags) {
  const bool g = (flags & MSLICE_NULL_GLOBAL) != 0, cpm = (flags & MSLICE_NULL_CPM) != 0;
  if (g && cpm) fail(MSLICE_EINVAL, "MSLICE_NULL_GLOBAL and MSLICE_NULL_CPM exclude each other");
  return g ? NULL_SUPRA_GLOBAL : cpm ? NULL_CPM : NULL_MULTISLICE;
}

// The instance parameters of a solve on graph G: the uniform rationals and,
// when gen gives them, the validated tables (EINVAL for bad ones).
InstParams inst_params(const SupraGraph& G, int64_t gn, int64_t gd, int64_t on, int64_t od, const mslice_general* gen,
                       bool global_null) {
  if (!rational_ok(gn, gd, false)) fail(MSLICE_EINVAL, "gamma must be a rational > 0");
  if (!rational_ok(on, od, true)) fail(MSLICE_EINVAL, "omega must be a rational >= 0");
  InstParams j{gn, gd, on, od};
  if (!gen) return j;
  const int32_t T = G.T;
  if (gen->omega_num) {
    const int64_t slots = coupling_slots(G.coupling, T);
    j.cw.assign(gen->omega_num, gen->omega_num + slots);
    for (long long x : j.cw)
      if (!rational_ok(x, od, true)) fail(MSLICE_EINVAL, "omega^(sr) numerators must lie in [0, 2^31]");
    if (G.coupling != 0)
      for (int32_t s = 0; s < T; ++s) {
        if (j.cw[(int64_t)s * T + s] != 0) fail(MSLICE_EINVAL, "categorical omega^(ss) must be 0");
        for (int32_t r = 0; r < s; ++r)
          if (j.cw[(int64_t)s * T + r] != j.cw[(int64_t)r * T + s])
            fail(MSLICE_EINVAL, "categorical omega^(sr) must be symmetric");
      }
  }
  if (gen->gamma_num || gen->gamma_den) {
    if (!gen->gamma_num || !gen->gamma_den) fail(MSLICE_EINVAL, "gamma_num and gamma_den go together");
    if (global_null) fail(MSLICE_EINVAL, "per-snapshot gamma does not apply to the global null model");
    j.gsn.assign(gen->gamma_num, gen->gamma_num + T);
    j.gsd.assign(gen->gamma_den, gen->gamma_den + T);
    for (int32_t s = 0; s < T; ++s)
      if (!rational_ok(j.gsn[s], j.gsd[s], false)) fail(MSLICE_EINVAL, "gamma^(s) must be rationals > 0");
  }
  return j;
}

TierCuts cuts_of(const mslice_opts& opt) {
  TierCuts c;
  const int32_t* t = opt.tier_cuts;
  if (t[0] || t[1] || t[2] || t[3])
    for (int k = 0; k < 4; ++k) c.t[k] = t[k];
  return c;
}

// One solve (a single instance or a batch) with the options' schedule;
// fills the stats, prints the MSLICE_TRACE kernel table when set.
void run_solve(Ctx& c, const SupraGraph& G, const std::vector<InstParams>& jobs, const mslice_opts& opt,
               const int32_t* init, int32_t* out, Solver& S, RunOut& ro, mslice_stats& stats) {
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_spans;
  c.profile = (opt.flags & MSLICE_PROFILE) != 0;
  c.prof_spans = &prof_spans;
  std::vector<std::pair<const void*, std::pair<cudaEvent_t, cudaEvent_t>>> trace;
  if (std::getenv("MSLICE_TRACE")) c.trace = &trace;
  SolveParams p;
  p.K = opt.K;
  p.max_rounds = opt.max_rounds;
  p.max_levels = opt.max_levels;
  p.n_iterations = opt.n_iterations;
  p.seed = opt.seed;
  p.cuts = cuts_of(opt);
  p.autotune = (opt.flags & MSLICE_AUTOTUNE) != 0;
  p.global_null = null_model_of(opt.flags) == NULL_SUPRA_GLOBAL;
  p.theta_num = opt.theta_num;
  p.theta_den = opt.theta_den;
  p.cpm = null_model_of(opt.flags) == NULL_CPM;
  run_leiden(c, G, jobs, p, opt.stop_level, opt.stop_stage, opt.stop_rounds, init, out, S, ro);
  std::memset(&stats, 0, sizeof(stats));
  stats.iterations = (int32_t)ro.iterations;
  stats.levels = (int32_t)ro.levels;
  stats.out_n = ro.out_n;
  stats.next_n = ro.next_n;
  stats.next_nnz = ro.next_nnz;
  stats.next_checksum = ro.next_checksum;
  stats.stop_reason = (int32_t)ro.stop_reason;
  stats.last_level0_moves = ro.last_level0_moves;
  stats.ms_total = ro.ms[0];
  stats.ms_local_move = ro.ms[1];
  stats.ms_refine = ro.ms[2];
  stats.ms_aggregate = ro.ms[3];
  stats.ms_modularity = ro.ms[4];
  stats.ms_capped = ro.ms_capped;
  stats.capped_levels = ro.capped_levels;
  stats.capped_rounds = ro.capped_rounds;
  stats.lm_rounds = S.lm_rounds;
  stats.lm_edges = S.lm_edges;
  stats.lm_moves = S.lm_moves;
  stats.kernel_launches = c.launches;
  stats.host_launches = c.host_launches;
  for (int k = 0; k < 4; ++k) stats.tier_cuts[k] = S.p.cuts.t[k];
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
  o->theta_num = 0;
  o->theta_den = 1;
}

const char* mslice_last_error(void) { return g_last_error.c_str(); }

int mslice_build_ex(const mslice_csr* slices, int32_t T, mslice_coupling cpl, int64_t omega_num, int64_t omega_den,
                    int32_t flags, void* stream, mslice_handle* out) {
  mslice_graph* h = nullptr;
  const int rc = guard([&] {
    if (!out) fail(MSLICE_EINVAL, "null output handle");
    *out = nullptr;
    if (!slices || T < 1) fail(MSLICE_EINVAL, "need T >= 1 snapshots");
    if (cpl != MSLICE_ORDINAL && cpl != MSLICE_CATEGORICAL) fail(MSLICE_EINVAL, "unsupported coupling");
    if (!rational_ok(omega_num, omega_den, true)) fail(MSLICE_EINVAL, "omega must be a rational >= 0");
    const int64_t n = slices[0].n;
    if (n < 0 || n > INT32_MAX || n * (int64_t)T > INT32_MAX) fail(MSLICE_EINVAL, "n*T must fit in int32");
    for (int32_t s = 0; s < T; ++s)
      if (slices[s].n != n) fail(MSLICE_EINVAL, "snapshots must have the same n");
    h = new mslice_graph();
    static std::atomic<uint64_t> next_serial{1};
    h->serial = next_serial++;
    h->stream = static_cast<cudaStream_t>(stream);
    if (!h->stream) {
      // a stream of the handle's own that, like the legacy default stream it
      // stands for, waits for the legacy stream's work (and can be captured)
      check_cuda(cudaStreamCreate(&h->stream), "stream");
      h->own_stream = true;
    }
    h->ws.stream = h->stream;
    h->G.mem.stream = h->stream;
    keep_pool_memory();
    h->on = omega_num;
    h->od = omega_den;
    check_cuda(cudaMallocHost(&h->pinned, PINNED_BYTES), "pinned buffer");
    if (!std::getenv("MSLICE_SERIAL_TIERS")) h->fan.create();
    h->d_status = h->ws.get<unsigned>("status", 4);
    Ctx c = h->ctx();
    check_cuda(cudaMemsetAsync(h->d_status, 0, 16, c.stream), "memset");
    const bool dev = (flags & MSLICE_DEVICE_PTRS) != 0;
    std::vector<const int64_t*> ip(T);
    std::vector<const int32_t*> ix(T), wt(T);
    std::vector<int64_t> nnz(T), eoff(T + 1, 0);
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
      eoff[s + 1] = eoff[s] + z;
      if (dev) {
        ip[s] = slices[s].indptr;
        ix[s] = slices[s].indices;
        wt[s] = slices[s].weights;
      }
    }
    if (!dev) {
      // host snapshots: one staging buffer per array kind.  Up to 64
      // snapshots are copied one by one (pinned inputs stream straight in);
      // longer sequences are packed on the host first, so many small
      // snapshots cost three copies instead of 3T.
      const size_t nip = (size_t)T * (n + 1);
      int64_t* dip = h->ws.get<int64_t>("in_ip", nip);
      int32_t* dix = h->ws.get<int32_t>("in_ix", eoff[T]);
      int32_t* dwt = h->ws.get<int32_t>("in_wt", eoff[T]);
      if (n == 0) {
        check_cuda(cudaMemsetAsync(dip, 0, nip * sizeof(int64_t), c.stream), "memset");
      } else if (T <= 64) {
        for (int32_t s = 0; s < T; ++s) {
          check_cuda(cudaMemcpyAsync(dip + (size_t)s * (n + 1), slices[s].indptr, (n + 1) * sizeof(int64_t),
                                     cudaMemcpyHostToDevice, c.stream), "copy");
          if (nnz[s] > 0) {
            check_cuda(cudaMemcpyAsync(dix + eoff[s], slices[s].indices, nnz[s] * sizeof(int32_t),
                                       cudaMemcpyHostToDevice, c.stream), "copy");
            check_cuda(cudaMemcpyAsync(dwt + eoff[s], slices[s].weights, nnz[s] * sizeof(int32_t),
                                       cudaMemcpyHostToDevice, c.stream), "copy");
          }
        }
      } else {
        std::vector<int64_t> hip(nip);
        std::vector<int32_t> hix(eoff[T]), hwt(eoff[T]);
        for (int32_t s = 0; s < T; ++s) {
          std::memcpy(&hip[(size_t)s * (n + 1)], slices[s].indptr, (n + 1) * sizeof(int64_t));
          if (nnz[s] > 0) {
            std::memcpy(&hix[eoff[s]], slices[s].indices, nnz[s] * sizeof(int32_t));
            std::memcpy(&hwt[eoff[s]], slices[s].weights, nnz[s] * sizeof(int32_t));
          }
        }
        check_cuda(cudaMemcpyAsync(dip, hip.data(), nip * sizeof(int64_t), cudaMemcpyHostToDevice, c.stream), "copy");
        if (eoff[T] > 0) {
          check_cuda(cudaMemcpyAsync(dix, hix.data(), eoff[T] * sizeof(int32_t), cudaMemcpyHostToDevice, c.stream),
                     "copy");
          check_cuda(cudaMemcpyAsync(dwt, hwt.data(), eoff[T] * sizeof(int32_t), cudaMemcpyHostToDevice, c.stream),
                     "copy");
        }
        sync(c);  // the host staging vectors go out of scope
      }
      for (int32_t s = 0; s < T; ++s) {
        ip[s] = dip + (size_t)s * (n + 1);
        ix[s] = dix + eoff[s];
        wt[s] = dwt + eoff[s];
      }
    }
    build_supra(c, ip, ix, wt, nnz, n, h->G, (int32_t)cpl);
    h->launches += c.launches;
    // staged host copies are not needed after the build
    if (!dev) {
      h->ws.release("in_ip");
      h->ws.release("in_ix");
      h->ws.release("in_wt");
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
  return mslice_leiden_general(h, o, nullptr, init_labels, labels_out, Q_out, st);
}

int mslice_leiden_general(mslice_handle h, const mslice_opts* o, const mslice_general* gen, const int32_t* init_labels,
                          int32_t* labels_out, double* Q_out, mslice_stats* st) {
  return guard([&] {
    if (!h) fail(MSLICE_EINVAL, "null handle");
    mslice_opts opt;
    mslice_default_opts(&opt);
    if (o) opt = *o;
    check_opts(opt);
    const int nm = null_model_of(opt.flags);
    const SupraGraph& G = h->G;
    const InstParams job =
        inst_params(G, opt.gamma_num, opt.gamma_den, opt.omega_num, opt.omega_den, gen, nm == NULL_SUPRA_GLOBAL);
    if (!labels_out && h->G.N > 0) fail(MSLICE_EINVAL, "null labels_out");
    const bool dev = (opt.flags & MSLICE_DEVICE_PTRS) != 0;
    check_bounds(G.n, G.T, G.coupling, G.two_m_host.data(), job, nm);
    const int64_t N0 = G.N;
    Ctx c = h->ctx();
    const int32_t* init = nullptr;
    if (init_labels && N0 > 0) {
      if (dev) {
        init = init_labels;
      } else {
        int32_t* d = h->ws.get<int32_t>("in_init", N0);
        check_cuda(cudaMemcpyAsync(d, init_labels, N0 * sizeof(int32_t), cudaMemcpyHostToDevice, c.stream), "copy");
        init = d;
      }
    }
    int32_t* out = dev ? labels_out : h->ws.get<int32_t>("out_lab", N0 > 0 ? N0 : 1);
    mslice_stats stats;
    RunOut ro;
    Solver S;
    run_solve(c, G, {job}, opt, init, out, S, ro, stats);
    if (!dev && ro.out_n > 0) {
      check_cuda(cudaMemcpyAsync(labels_out, out, ro.out_n * sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream),
                 "copy");
      sync(c);
    }
    h->launches += c.launches;
    if (Q_out && !ro.Q.empty()) *Q_out = ro.Q[0];
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
  mslice_opts o;
  mslice_default_opts(&o);
  o.gamma_num = gamma_num;
  o.gamma_den = gamma_den;
  o.omega_num = omega_num;
  o.omega_den = omega_den;
  o.flags = flags;
  return mslice_modularity_general(h, labels, &o, nullptr, Q_out);
}

int mslice_modularity_general(mslice_handle h, const int32_t* labels, const mslice_opts* o, const mslice_general* gen,
                              double* Q_out) {
  return guard([&] {
    if (!h) fail(MSLICE_EINVAL, "null handle");
    mslice_opts opt;
    mslice_default_opts(&opt);
    if (o) opt = *o;
    const int32_t flags = opt.flags;
    const SupraGraph& G = h->G;
    const int nm = null_model_of(flags);
    const InstParams job =
        inst_params(G, opt.gamma_num, opt.gamma_den, opt.omega_num, opt.omega_den, gen, nm == NULL_SUPRA_GLOBAL);
    if (!labels && G.N > 0) fail(MSLICE_EINVAL, "null labels");
    check_bounds(G.n, G.T, G.coupling, G.two_m_host.data(), job, nm);
    Ctx c = h->ctx();
    Solver S;
    S.c = &c;
    S.G0 = &G;
    S.N0 = G.N;
    S.p.global_null = nm == NULL_SUPRA_GLOBAL;
    S.p.cpm = nm == NULL_CPM;
    set_instances(c, S, {job});
    setup_null_model(S);
    const int64_t N = G.N > 0 ? G.N : 1;
    S.sig_used = h->ws.get<ull>("m_used", 1);
    int32_t* lab = h->ws.get<int32_t>("m_lab", N);
    if (G.N > 0) {
      const bool dev = (flags & MSLICE_DEVICE_PTRS) != 0;
      check_cuda(cudaMemcpyAsync(lab, labels, G.N * sizeof(int32_t),
                                 dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c.stream), "copy");
      check_label_ranges(c, G, lab);
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

int mslice_batch_create(int32_t flags, void* stream, mslice_batch* out) {
  mslice_batch b = nullptr;
  const int rc = guard([&] {
    if (!out) fail(MSLICE_EINVAL, "null output batch");
    *out = nullptr;
    b = new mslice_batch_s();
    b->flags = flags;
    b->stream = static_cast<cudaStream_t>(stream);
    if (!b->stream) {
      check_cuda(cudaStreamCreate(&b->stream), "stream");
      b->own_stream = true;
    }
    b->ws.stream = b->stream;
    b->G.mem.stream = b->stream;
    keep_pool_memory();
    check_cuda(cudaMallocHost(&b->pinned, PINNED_BYTES), "pinned buffer");
    if (!std::getenv("MSLICE_SERIAL_TIERS")) b->fan.create();
    b->d_status = b->ws.get<unsigned>("status", 4);
    check_cuda(cudaMemsetAsync(b->d_status, 0, 16, b->stream), "memset");
    sync_stream(b->stream);
    *out = b;
  });
  if (rc != MSLICE_OK && b) delete b;
  return rc;
}

int mslice_batch_add(mslice_batch b, mslice_handle g, int64_t gamma_num, int64_t gamma_den, int64_t omega_num,
                     int64_t omega_den, const int32_t* init_labels, int32_t* index_out) {
  return mslice_batch_add_general(b, g, gamma_num, gamma_den, omega_num, omega_den, nullptr, init_labels, index_out);
}

int mslice_batch_add_general(mslice_batch b, mslice_handle g, int64_t gamma_num, int64_t gamma_den,
                             int64_t omega_num, int64_t omega_den, const mslice_general* gen,
                             const int32_t* init_labels, int32_t* index_out) {
  return guard([&] {
    if (!b || !g) fail(MSLICE_EINVAL, "null batch or graph");
    const SupraGraph& G = g->G;
    const InstParams job = inst_params(G, gamma_num, gamma_den, omega_num, omega_den, gen, false);
    check_bounds(G.n, G.T, G.coupling, G.two_m_host.data(), job, NULL_MULTISLICE);
    const int64_t N = G.N;
    if (b->off.back() + N > INT32_MAX) fail(MSLICE_EINVAL, "the batch must hold fewer than 2^31 supra-nodes");
    if ((int64_t)b->graphs.size() >= INT32_MAX) fail(MSLICE_EINVAL, "too many instances");
    std::vector<int32_t> lab(N);
    if (init_labels && N > 0) {
      if (b->flags & MSLICE_DEVICE_PTRS)
        check_cuda(cudaMemcpy(lab.data(), init_labels, N * sizeof(int32_t), cudaMemcpyDeviceToHost), "copy");
      else
        std::memcpy(lab.data(), init_labels, N * sizeof(int32_t));
      for (int64_t v = 0; v < N; ++v)
        if (lab[v] < 0 || lab[v] >= N) fail(MSLICE_EINVAL, "init labels must lie in [0, N)");
    } else {
      for (int64_t v = 0; v < N; ++v) lab[v] = (int32_t)v;
    }
    b->init.insert(b->init.end(), lab.begin(), lab.end());
    b->any_init = b->any_init || init_labels != nullptr;
    b->graphs.push_back(g);
    b->jobs.push_back(job);
    b->off.push_back(b->off.back() + N);
    b->solved = false;
    if (index_out) *index_out = (int32_t)b->graphs.size() - 1;
  });
}

int mslice_batch_run(mslice_batch b, const mslice_opts* o, mslice_stats* st) {
  return guard([&] {
    if (!b) fail(MSLICE_EINVAL, "null batch");
    if (b->graphs.empty()) fail(MSLICE_EINVAL, "empty batch");
    mslice_opts opt;
    mslice_default_opts(&opt);
    if (o) opt = *o;
    check_opts(opt);
    if (opt.stop_level >= 0) fail(MSLICE_EINVAL, "debug stops apply to single solves only");
    const int nm = null_model_of(opt.flags);
    if (nm != NULL_MULTISLICE)
      for (size_t i = 0; i < b->graphs.size(); ++i) {
        const SupraGraph& Gi = b->graphs[i]->G;
        const InstParams& j = b->jobs[i];
        if (nm == NULL_SUPRA_GLOBAL && !j.gsn.empty())
          fail(MSLICE_EINVAL, "per-snapshot gamma does not apply to the global null model");
        check_bounds(Gi.n, Gi.T, Gi.coupling, Gi.two_m_host.data(), j, nm);
      }
    Ctx c = b->ctx();
    std::vector<uint64_t> serials;
    for (mslice_graph* g : b->graphs) serials.push_back(g->serial);
    // one instance: solved on its handle's graph, no copy
    const bool single = b->graphs.size() == 1;
    if (!single && serials != b->G_serials) {
      std::vector<const SupraGraph*> parts;
      for (mslice_graph* g : b->graphs) parts.push_back(&g->G);
      b->G_serials.clear();
      concat_instances(c, parts, b->G);
      b->G_serials = serials;
    }
    const SupraGraph& G = single ? b->graphs[0]->G : b->G;
    const int64_t N = G.N;
    int32_t* init = nullptr;
    if (b->any_init && N > 0) {
      init = b->ws.get<int32_t>("b_init", N);
      check_cuda(cudaMemcpyAsync(init, b->init.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice, c.stream), "copy");
    }
    int32_t* out = b->ws.get<int32_t>("b_out", N > 0 ? N : 1);
    opt.flags &= MSLICE_PROFILE | MSLICE_AUTOTUNE | MSLICE_NULL_GLOBAL | MSLICE_NULL_CPM;
    mslice_stats stats;
    RunOut ro;
    Solver S;
    b->solved = false;
    run_solve(c, G, b->jobs, opt, init, out, S, ro, stats);
    b->Q = ro.Q;
    b->solved = true;
    b->launches += c.launches;
    if (st) *st = stats;
  });
}

int mslice_batch_results(mslice_batch b, int32_t i, int32_t* labels_out, double* Q_out) {
  return guard([&] {
    if (!b) fail(MSLICE_EINVAL, "null batch");
    if (!b->solved) fail(MSLICE_EINVAL, "the batch has not been run since its last change");
    const int32_t B = (int32_t)b->graphs.size();
    if (i < -1 || i >= B) fail(MSLICE_EINVAL, "instance index out of range");
    const int64_t lo = i < 0 ? 0 : b->off[i], hi = i < 0 ? b->off[B] : b->off[i + 1];
    if (hi > lo) {
      if (!labels_out) fail(MSLICE_EINVAL, "null labels_out");
      const int32_t* out = b->ws.get<int32_t>("b_out", b->off.back() > 0 ? b->off.back() : 1);
      const bool dev = (b->flags & MSLICE_DEVICE_PTRS) != 0;
      check_cuda(cudaMemcpyAsync(labels_out, out + lo, (hi - lo) * sizeof(int32_t),
                                 dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream), "copy");
      sync_stream(b->stream);
    }
    if (Q_out) {
      if (i < 0)
        std::memcpy(Q_out, b->Q.data(), B * sizeof(double));
      else
        *Q_out = b->Q[i];
    }
  });
}

int mslice_batch_info(mslice_batch b, int32_t* B, int64_t* N, int64_t* offsets) {
  if (!b) {
    g_last_error = "null batch";
    return MSLICE_EINVAL;
  }
  if (B) *B = (int32_t)b->graphs.size();
  if (N) *N = b->off.back();
  if (offsets) std::memcpy(offsets, b->off.data(), b->off.size() * sizeof(int64_t));
  return MSLICE_OK;
}

int mslice_batch_clear(mslice_batch b) {
  if (!b) {
    g_last_error = "null batch";
    return MSLICE_EINVAL;
  }
  b->graphs.clear();
  b->jobs.clear();
  b->off.assign(1, 0);
  b->init.clear();
  b->any_init = false;
  b->solved = false;
  return MSLICE_OK;
}

int64_t mslice_batch_kernel_launches(mslice_batch b) { return b ? b->launches : -1; }

void mslice_batch_free(mslice_batch b) { delete b; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Windowed optimisation of a long snapshot sequence.  Sec. 4 names windowed
// optimisation for its 7,375-snapshot case and gives no procedure; the
// reading:
//   * windows of W snapshots start at 0, stride, 2*stride, ..., the last start
//     clamped to T - W so every window holds W snapshots and the last ends at
//     T (one window [0, T) when T <= W);
//   * window 0 starts from singletons; window k is warm-started by the
//     serving rule with the actual shift e = start_k - start_{k-1}: local
//     snapshot j takes the previous window's labels of local snapshot
//     min(j + e, W - 1);
//   * stitching: window k's communities in order of first occurrence; one
//     whose first supra-node lies in the overlap (the first W - e snapshots)
//     continues the stitched label of that supra-node unless an earlier
//     community of the window took it; any other gets the next fresh label;
//     window k's labels then overwrite its snapshots' stitched labels;
//   * the stitched labels are renumbered by first occurrence at the end.
// Each window is a complete solve (build + Leiden + Q) on the caller's
// stream; stitching runs on the host over the window's labels.

namespace mslice {
namespace windowed {

__global__ void k_window_init(const int32_t* prev, int64_t n, int32_t w, int32_t shift, int32_t* init) {
  const int64_t N = n * w;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = v / n, i = v - j * n;
    init[v] = prev[min(j + shift, (int64_t)w - 1) * n + i];
  }
}

std::vector<int32_t> window_starts(int32_t T, int32_t W, int32_t stride) {
  std::vector<int32_t> st{0};
  if (T <= W) return st;
  while (st.back() + W < T) st.push_back(std::min(st.back() + stride, T - W));
  return st;
}

}  // namespace windowed
}  // namespace mslice

extern "C" int mslice_leiden_windowed(const mslice_csr* slices, int32_t T, int32_t W, int32_t stride,
                                      const mslice_opts* o, void* stream, int32_t* labels_out, double* Q_windows,
                                      int32_t q_cap, int32_t* n_windows, mslice_stats* st) {
  cudaStream_t own = nullptr;
  Workspace ws;
  SupraGraph G;
  StreamFan fan;
  void* pinned = nullptr;
  const int rc = guard([&] {
    if (!slices || T < 1) fail(MSLICE_EINVAL, "need T >= 1 snapshots");
    if (W < 1) fail(MSLICE_EINVAL, "W must be >= 1");
    if (T > W && (stride < 1 || stride >= W)) fail(MSLICE_EINVAL, "stride must lie in [1, W) so windows overlap");
    mslice_opts opt;
    mslice_default_opts(&opt);
    if (o) opt = *o;
    check_opts(opt);
    if (opt.stop_level >= 0) fail(MSLICE_EINVAL, "debug stops apply to single solves only");
    if (!rational_ok(opt.gamma_num, opt.gamma_den, false)) fail(MSLICE_EINVAL, "gamma must be a rational > 0");
    if (!rational_ok(opt.omega_num, opt.omega_den, true)) fail(MSLICE_EINVAL, "omega must be a rational >= 0");
    const int nm = null_model_of(opt.flags);
    const int64_t n = slices[0].n;
    const int32_t Wn = std::min(W, T);
    if (n < 0 || n > INT32_MAX || n * (int64_t)Wn > INT32_MAX) fail(MSLICE_EINVAL, "n*W must fit in int32");
    for (int32_t s = 0; s < T; ++s)
      if (slices[s].n != n) fail(MSLICE_EINVAL, "snapshots must have the same n");
    if (!labels_out && n > 0) fail(MSLICE_EINVAL, "null labels_out");
    const bool dev = (opt.flags & MSLICE_DEVICE_PTRS) != 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!s) {
      check_cuda(cudaStreamCreate(&own), "stream");
      s = own;
    }
    ws.stream = s;
    G.mem.stream = s;
    keep_pool_memory();
    check_cuda(cudaMallocHost(&pinned, PINNED_BYTES), "pinned buffer");
    if (!std::getenv("MSLICE_SERIAL_TIERS")) fan.create();
    Ctx c;
    c.stream = s;
    c.fan = fan.fork ? &fan : nullptr;
    c.ws = &ws;
    c.d_status = ws.get<unsigned>("status", 4);
    c.pinned = pinned;
    check_cuda(cudaMemsetAsync(c.d_status, 0, 16, s), "memset");
    // snapshot arrays on the device: one staging copy per array kind
    std::vector<int64_t> nnz(T), eoff(T + 1, 0);
    for (int32_t t = 0; t < T; ++t) {
      if (n > 0 && !slices[t].indptr) fail(MSLICE_EINVAL, "null indptr");
      int64_t z = 0;
      if (n > 0) {
        if (dev)
          check_cuda(cudaMemcpy(&z, slices[t].indptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost), "copy");
        else
          z = slices[t].indptr[n];
      }
      if (z < 0) fail(MSLICE_EINVAL, "negative nnz");
      if (z > 0 && (!slices[t].indices || !slices[t].weights)) fail(MSLICE_EINVAL, "null indices/weights");
      nnz[t] = z;
      eoff[t + 1] = eoff[t] + z;
    }
    std::vector<const int64_t*> ip(T);
    std::vector<const int32_t*> ix(T), wt(T);
    if (dev) {
      for (int32_t t = 0; t < T; ++t) {
        ip[t] = slices[t].indptr;
        ix[t] = slices[t].indices;
        wt[t] = slices[t].weights;
      }
    } else {
      std::vector<int64_t> hip((size_t)T * (n + 1));
      std::vector<int32_t> hix(eoff[T]), hwt(eoff[T]);
      for (int32_t t = 0; t < T; ++t) {
        if (n > 0) std::memcpy(&hip[(size_t)t * (n + 1)], slices[t].indptr, (n + 1) * sizeof(int64_t));
        if (nnz[t] > 0) {
          std::memcpy(&hix[eoff[t]], slices[t].indices, nnz[t] * sizeof(int32_t));
          std::memcpy(&hwt[eoff[t]], slices[t].weights, nnz[t] * sizeof(int32_t));
        }
      }
      int64_t* dip = ws.get<int64_t>("w_ip", hip.size());
      int32_t* dix = ws.get<int32_t>("w_ix", eoff[T]);
      int32_t* dwt = ws.get<int32_t>("w_wt", eoff[T]);
      if (!hip.empty())
        check_cuda(cudaMemcpyAsync(dip, hip.data(), hip.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s), "copy");
      if (eoff[T] > 0) {
        check_cuda(cudaMemcpyAsync(dix, hix.data(), eoff[T] * sizeof(int32_t), cudaMemcpyHostToDevice, s), "copy");
        check_cuda(cudaMemcpyAsync(dwt, hwt.data(), eoff[T] * sizeof(int32_t), cudaMemcpyHostToDevice, s), "copy");
      }
      sync(c);  // the host staging arrays go out of scope
      for (int32_t t = 0; t < T; ++t) {
        ip[t] = dip + (size_t)t * (n + 1);
        ix[t] = dix + eoff[t];
        wt[t] = dwt + eoff[t];
      }
    }
    const std::vector<int32_t> starts = windowed::window_starts(T, W, stride);
    if (n_windows) *n_windows = (int32_t)starts.size();
    const InstParams job{opt.gamma_num, opt.gamma_den, opt.omega_num, opt.omega_den};
    SolveParams sp;
    sp.K = opt.K;
    sp.max_rounds = opt.max_rounds;
    sp.max_levels = opt.max_levels;
    sp.n_iterations = opt.n_iterations;
    sp.seed = opt.seed;
    sp.cuts = cuts_of(opt);
    sp.global_null = nm == NULL_SUPRA_GLOBAL;
    sp.cpm = nm == NULL_CPM;
    sp.theta_num = opt.theta_num;
    sp.theta_den = opt.theta_den;
    const int64_t Nw = n * Wn;
    int32_t* prev = ws.get<int32_t>("w_prev", Nw);
    int32_t* init = ws.get<int32_t>("w_init", Nw);
    int32_t* out = ws.get<int32_t>("w_out", Nw);
    std::vector<int64_t> stitched((size_t)n * T, -1);
    std::vector<int32_t> lab(Nw);
    std::vector<int64_t> first;
    int64_t fresh = 0;
    mslice_stats acc;
    std::memset(&acc, 0, sizeof(acc));
    for (size_t k = 0; k < starts.size(); ++k) {
      const int32_t a = starts[k], b = std::min(a + W, T), w = b - a;
      const int32_t e = k == 0 ? 0 : a - starts[k - 1];
      build_supra(c, std::vector<const int64_t*>(ip.begin() + a, ip.begin() + b),
                  std::vector<const int32_t*>(ix.begin() + a, ix.begin() + b),
                  std::vector<const int32_t*>(wt.begin() + a, wt.begin() + b),
                  std::vector<int64_t>(nnz.begin() + a, nnz.begin() + b), n, G);
      check_bounds(n, w, 0, G.two_m_host.data(), job, nm);
      const int64_t N = n * w;
      if (k > 0 && N > 0)
        launch(c, windowed::k_window_init, dim3(grid_for(N, 256) < 4096 ? grid_for(N, 256) : 4096), dim3(256), 0,
               (const int32_t*)prev, n, w, e, init);
      Solver S;
      RunOut ro;
      run_leiden(c, G, {job}, sp, -1, 0, 0, k > 0 ? init : nullptr, out, S, ro);
      if (N > 0) {
        check_cuda(cudaMemcpyAsync(lab.data(), out, N * sizeof(int32_t), cudaMemcpyDeviceToHost, s), "copy");
        check_cuda(cudaMemcpyAsync(prev, out, N * sizeof(int32_t), cudaMemcpyDeviceToDevice, s), "copy");
      }
      sync(c);
      if (Q_windows && (int32_t)k < q_cap && !ro.Q.empty()) Q_windows[k] = ro.Q[0];
      acc.lm_rounds += S.lm_rounds;
      acc.lm_edges += S.lm_edges;
      acc.lm_moves += S.lm_moves;
      acc.ms_total += ro.ms[0];
      acc.ms_local_move += ro.ms[1];
      acc.ms_refine += ro.ms[2];
      acc.ms_aggregate += ro.ms[3];
      acc.ms_modularity += ro.ms[4];
      acc.ms_capped += ro.ms_capped;
      acc.capped_levels += ro.capped_levels;
      acc.capped_rounds += ro.capped_rounds;
      acc.iterations = std::max<int32_t>(acc.iterations, (int32_t)ro.iterations);
      acc.levels = std::max<int32_t>(acc.levels, (int32_t)ro.levels);
      // stitching (canonical labels: first occurrence order is label order)
      int32_t ncomm = 0;
      for (int64_t v = 0; v < N; ++v) ncomm = std::max(ncomm, lab[v] + 1);
      first.assign(ncomm, N);
      for (int64_t v = N - 1; v >= 0; --v) first[lab[v]] = v;
      const int64_t overlap = k == 0 ? 0 : (int64_t)(w - e) * n;
      std::vector<int64_t> map(ncomm);
      std::unordered_set<int64_t> used;
      for (int32_t cc = 0; cc < ncomm; ++cc) {
        bool cont = false;
        if (first[cc] < overlap) {
          const int64_t L = stitched[(size_t)a * n + first[cc]];
          if (used.insert(L).second) {
            map[cc] = L;
            cont = true;
          }
        }
        if (!cont) map[cc] = fresh++;
      }
      for (int64_t v = 0; v < N; ++v) stitched[(size_t)a * n + v] = map[lab[v]];
    }
    // renumber by first occurrence
    std::map<int64_t, int32_t> seen;
    for (size_t v = 0; v < stitched.size(); ++v) {
      auto it = seen.find(stitched[v]);
      if (it == seen.end()) it = seen.emplace(stitched[v], (int32_t)seen.size()).first;
      labels_out[v] = it->second;
    }
    acc.out_n = (int64_t)stitched.size();
    acc.kernel_launches = c.launches;
    acc.host_launches = c.host_launches;
    for (int kk = 0; kk < 4; ++kk) acc.tier_cuts[kk] = sp.cuts.t[kk];
    if (st) *st = acc;
  });
  ws.release_all();
  G.mem.release_all();
  fan.destroy();
  if (pinned) cudaFreeHost(pinned);
  if (own) cudaStreamDestroy(own);
  return rc;
}
