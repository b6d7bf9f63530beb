// Serving runtime (mslice_server_*): sliding windows of live temporal graphs
// solved warm-started, with admission by device-memory footprint and
// continuous batching over several worker streams.
//
// Windowing bounds the supra-graph of a long snapshot stream (Sec. 4 names
// windowed optimisation for the case where the coupling grows with the
// snapshot count).  Per live graph the device holds a ring of W + 1 slice
// buffers (the W slices of the window and one staging buffer for the next
// snapshot) and the labels of the current window.  A request:
//   1. copies its snapshot into the staging buffer,
//   2. builds the supra-graph of the advanced window (device to device),
//   3. derives the initial labels from the previous result (k_shift_init),
//   4. is solved, batched with the other requests its worker admitted,
//   5. on success the staging buffer joins the window, the oldest slice
//      buffer (if the window was full) becomes the next staging buffer, and
//      the result becomes the window's labels.
// A failed request leaves the window as it was.
//
// Scheduling: every worker owns a CUDA stream and its own scratch; a free
// worker takes, in arrival order, the requests of graphs with nothing in
// flight whose estimated footprint fits the remaining budget.  Later requests
// of a graph wait for its earlier ones (each warm-starts from the previous
// result), and the scan stops at the first eligible request that does not fit
// (no overtaking, so a large request is not starved).
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/mslice.h"
#include "solver.h"

namespace mslice {

namespace {

// init[v] for supra-node v = j*n + i of the new window (j < w_new): the
// label of (min(j + shift, w_prev - 1), i) in the previous window's labels
// (instance-local ids, as the batched solve expects).
__global__ void k_shift_init(const int32_t* prev, int64_t n, int32_t w_prev, int32_t w_new, int32_t shift,
                             int32_t* init) {
  const int64_t N = n * w_new;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = v / n, i = v - j * n;
    const int64_t src = min(j + shift, (int64_t)w_prev - 1);
    init[v] = prev[src * n + i];
  }
}

__global__ void k_iota_seg(int32_t* x, int64_t N) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
    x[v] = (int32_t)v;
}

unsigned gsz(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

}  // namespace mslice

using namespace mslice;

namespace {

using Clock = std::chrono::steady_clock;

struct SrvGraph {
  int64_t n = 0;
  Workspace mem;                 // slice buffers and window labels
  std::vector<int64_t*> ip;      // W + 1 ring buffers
  std::vector<int32_t*> ix, wt;
  std::vector<int64_t> cap_ix;   // capacity (entries) of ix/wt of every buffer
  std::vector<int64_t> nnz;      // entries of the slice in every buffer
  std::vector<int> window;       // buffer indices of the window, oldest first
  int32_t* labels = nullptr;     // canonical labels of the current window (n * window.size())
  bool busy = false;             // a request of this graph is in flight
};

struct SrvRequest {
  int64_t id = 0;
  int32_t graph = 0;
  std::vector<int64_t> indptr;
  std::vector<int32_t> indices, weights;
  int64_t nnz = 0;
  bool done = false;
  mslice_request_info info{};
  std::string msg;
  std::vector<int32_t> labels;
};

struct Worker {
  int id = 0;
  cudaStream_t stream = nullptr;
  StreamFan fan;
  Workspace ws;
  SupraGraph batch;
  unsigned* d_status = nullptr;
  void* pinned = nullptr;
};

}  // namespace

struct mslice_server_s {
  mslice_server_opts opt{};
  int device = 0;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<int64_t> queue;
  std::map<int64_t, std::unique_ptr<SrvRequest>> reqs;
  std::vector<std::unique_ptr<SrvGraph>> graphs;
  int64_t used = 0;
  int inflight_batches = 0;
  int64_t next_id = 1;
  bool stop = false;
  std::vector<std::unique_ptr<Worker>> slots;
  std::vector<std::thread> workers;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

  // Device bytes a request holds while solved: the window's supra-graph
  // (24 B per supra-node, 8 B per entry), the solver's per-node scratch and
  // hash tables (~250 B per supra-node) and the aggregation's row buffers and
  // large-row tables (~44 B per entry).
  // Supra-nodes of the window a request will solve.
  int64_t window_nodes(const SrvRequest& r) const {
    const SrvGraph& g = *graphs[r.graph];
    return g.n * std::min<int64_t>((int64_t)g.window.size() + 1, opt.window);
  }

  int null_model() const {
    return (opt.solve.flags & MSLICE_NULL_GLOBAL) ? NULL_SUPRA_GLOBAL
           : (opt.solve.flags & MSLICE_NULL_CPM) ? NULL_CPM
                                                  : NULL_MULTISLICE;
  }

  int64_t footprint(const SrvRequest& r) const {
    const SrvGraph& g = *graphs[r.graph];
    const int W = opt.window;
    const int keep = std::min<int>((int)g.window.size(), W - 1);
    int64_t nnz = r.nnz;
    for (int k = (int)g.window.size() - keep; k < (int)g.window.size(); ++k) nnz += g.nnz[g.window[k]];
    const int64_t w = keep + 1;
    const int64_t N = g.n * w;
    nnz += 2 * g.n * (w - 1);
    const int64_t strengths = null_model() != NULL_MULTISLICE ? 8 : 0;  // k' or CPM's node weights
    return (274 + strengths) * N + 52 * nnz + (1 << 20);
  }
};

namespace {

// Stages a request's snapshot in its graph's spare buffer; returns the
// buffer index.
int stage_slice(Ctx& c, SrvGraph& g, const SrvRequest& r, int W) {
  std::vector<bool> in_window(W + 1, false);
  for (int b : g.window) in_window[b] = true;
  int p = 0;
  while (in_window[p]) ++p;
  const std::string tag = std::to_string(p);
  g.ip[p] = g.mem.get<int64_t>("ip" + tag, g.n + 1);
  if (r.nnz > g.cap_ix[p] || !g.ix[p]) {
    g.ix[p] = g.mem.get<int32_t>("ix" + tag, r.nnz);
    g.wt[p] = g.mem.get<int32_t>("wt" + tag, r.nnz);
    g.cap_ix[p] = std::max<int64_t>(r.nnz, 1);
  }
  check_cuda(cudaMemcpyAsync(g.ip[p], r.indptr.data(), (g.n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c.stream),
             "copy");
  if (r.nnz > 0) {
    check_cuda(cudaMemcpyAsync(g.ix[p], r.indices.data(), r.nnz * sizeof(int32_t), cudaMemcpyHostToDevice, c.stream),
               "copy");
    check_cuda(cudaMemcpyAsync(g.wt[p], r.weights.data(), r.nnz * sizeof(int32_t), cudaMemcpyHostToDevice, c.stream),
               "copy");
  }
  g.nnz[p] = r.nnz;
  return p;
}

void finish(mslice_server_s* s, SrvRequest* r, int code, const std::string& msg) {
  r->info.status = code;
  r->msg = msg;
  r->info.t_done = s->now();
}

// Solves one admitted batch on a worker.
void run_batch(mslice_server_s* s, Worker& slot, std::vector<SrvRequest*>& batch) {
  const int W = s->opt.window;
  Ctx c;
  c.stream = slot.stream;
  c.fan = slot.fan.fork ? &slot.fan : nullptr;
  c.ws = &slot.ws;
  c.d_status = slot.d_status;
  c.pinned = slot.pinned;
  struct Part {
    SrvRequest* r;
    SrvGraph* g;
    int buf;
    std::vector<int> window;
    std::unique_ptr<SupraGraph> G;
  };
  std::vector<Part> parts;
  // 1-2: stage the snapshot, build the advanced window's supra-graph
  for (SrvRequest* r : batch) {
    SrvGraph& g = *s->graphs[r->graph];
    g.mem.stream = slot.stream;
    Part p{r, &g, -1, {}, std::make_unique<SupraGraph>()};
    p.G->mem.stream = slot.stream;
    try {
      p.buf = stage_slice(c, g, *r, W);
      p.window = g.window;
      if ((int)p.window.size() == W) p.window.erase(p.window.begin());
      p.window.push_back(p.buf);
      std::vector<const int64_t*> ip;
      std::vector<const int32_t*> ix, wt;
      std::vector<int64_t> nnz;
      for (int b : p.window) {
        ip.push_back(g.ip[b]);
        ix.push_back(g.ix[b]);
        wt.push_back(g.wt[b]);
        nnz.push_back(g.nnz[b]);
      }
      build_supra(c, ip, ix, wt, nnz, g.n, *p.G);
      check_bounds(g.n, p.G->T, 0, p.G->two_m_host.data(),
                   InstParams{s->opt.gamma_num, s->opt.gamma_den, s->opt.omega_num, s->opt.omega_den}, s->null_model());
      parts.push_back(std::move(p));
    } catch (const Error& e) {
      finish(s, r, e.code, e.msg);
    }
  }
  if (parts.empty()) return;
  try {
    // 3: initial labels, instance after instance
    int64_t N = 0;
    for (Part& p : parts) N += p.G->N;
    int32_t* init = slot.ws.get<int32_t>("srv_init", N);
    int32_t* out = slot.ws.get<int32_t>("srv_out", N);
    int64_t off = 0;
    for (Part& p : parts) {
      const int32_t w_prev = (int32_t)p.g->window.size();
      const int32_t w_new = (int32_t)p.window.size();
      if (p.G->N > 0) {
        if (w_prev == 0)
          launch(c, k_iota_seg, dim3(gsz(p.G->N)), dim3(256), 0, init + off, p.G->N);
        else
          launch(c, k_shift_init, dim3(gsz(p.G->N)), dim3(256), 0, (const int32_t*)p.g->labels, p.g->n, w_prev, w_new,
                 (int32_t)(w_prev == W ? 1 : 0), init + off);
      }
      off += p.G->N;
    }
    // 4: one solve over the batch
    const SupraGraph* G = parts[0].G.get();
    if (parts.size() > 1) {
      std::vector<const SupraGraph*> gs;
      for (Part& p : parts) gs.push_back(p.G.get());
      slot.batch.mem.stream = slot.stream;
      concat_instances(c, gs, slot.batch);
      G = &slot.batch;
    }
    std::vector<InstParams> jobs(parts.size(), InstParams{s->opt.gamma_num, s->opt.gamma_den, s->opt.omega_num,
                                                          s->opt.omega_den});
    SolveParams sp;
    sp.K = s->opt.solve.K;
    sp.max_rounds = s->opt.solve.max_rounds;
    sp.max_levels = s->opt.solve.max_levels;
    sp.n_iterations = s->opt.solve.n_iterations;
    sp.seed = s->opt.solve.seed;
    sp.global_null = s->null_model() == NULL_SUPRA_GLOBAL;
    sp.theta_num = s->opt.solve.theta_num;
    sp.theta_den = s->opt.solve.theta_den;
    sp.cpm = s->null_model() == NULL_CPM;
    for (int k = 0; k < 4; ++k)
      if (s->opt.solve.tier_cuts[0] || s->opt.solve.tier_cuts[1] || s->opt.solve.tier_cuts[2] ||
          s->opt.solve.tier_cuts[3])
        sp.cuts.t[k] = s->opt.solve.tier_cuts[k];
    Solver S;
    RunOut ro;
    const double tb = s->now();
    run_leiden(c, *G, jobs, sp, -1, 0, 0, init, out, S, ro);
    const double te = s->now();
    // 5: results become the windows' labels
    off = 0;
    for (size_t k = 0; k < parts.size(); ++k) {
      Part& p = parts[k];
      const int64_t Ni = p.G->N;
      p.g->labels = p.g->mem.get<int32_t>("labels", Ni);
      if (Ni > 0)
        check_cuda(cudaMemcpyAsync(p.g->labels, out + off, Ni * sizeof(int32_t), cudaMemcpyDeviceToDevice, c.stream),
                   "copy");
      p.r->labels.resize(Ni);
      if (Ni > 0)
        check_cuda(cudaMemcpyAsync(p.r->labels.data(), out + off, Ni * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                   c.stream), "copy");
      p.g->window = p.window;
      p.r->info.Q = ro.Q[k];
      p.r->info.slices = (int32_t)p.window.size();
      p.r->info.N = Ni;
      p.r->info.batch_size = (int32_t)parts.size();
      p.r->info.t_batch_start = tb;
      p.r->info.t_batch_end = te;
      off += Ni;
    }
    sync(c);
    for (Part& p : parts) finish(s, p.r, MSLICE_OK, "");
  } catch (const Error& e) {
    for (Part& p : parts) finish(s, p.r, e.code, e.msg);
  }
}

void worker_loop(mslice_server_s* s, Worker* slot) {
  cudaSetDevice(s->device);
  for (;;) {
    std::vector<SrvRequest*> batch;
    int64_t fp_total = 0, nodes_total = 0;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        // admission scan in arrival order
        std::vector<bool> seen(s->graphs.size(), false);
        for (int64_t id : s->queue) {
          SrvRequest* r = s->reqs[id].get();
          if (seen[r->graph]) continue;  // an earlier request of this graph is still queued
          seen[r->graph] = true;
          SrvGraph& g = *s->graphs[r->graph];
          if (g.busy) continue;
          const int64_t fp = s->footprint(*r);
          const bool alone = s->used == 0 && fp_total == 0;
          if (!alone && s->used + fp_total + fp > s->opt.hbm_budget) break;
          const int64_t nodes = s->window_nodes(*r);
          if (!batch.empty() && nodes_total + nodes > s->opt.max_batch_nodes) break;
          nodes_total += nodes;
          r->info.footprint = fp;
          fp_total += fp;
          batch.push_back(r);
          g.busy = true;
          if ((int)batch.size() >= s->opt.max_batch) break;
        }
        if (!batch.empty()) break;
        if (s->stop && s->queue.empty()) return;
        s->cv_work.wait(lk);
      }
      for (SrvRequest* r : batch) {
        for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
          if (*it == r->id) {
            s->queue.erase(it);
            break;
          }
        r->info.t_admit = s->now();
        r->info.slot = slot->id;
      }
      s->used += fp_total;
      s->inflight_batches++;
    }
    run_batch(s, *slot, batch);
    slot->ws.release_all();  // the memory goes back to the device pool for the other workers
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->used -= fp_total;
      s->inflight_batches--;
      for (SrvRequest* r : batch) {
        s->graphs[r->graph]->busy = false;
        r->done = true;
      }
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

int guard_srv(const std::function<void()>& f) {
  try {
    f();
    set_last_error("");
    return MSLICE_OK;
  } catch (const Error& e) {
    set_last_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    return MSLICE_ENOMEM;
  }
}

}  // namespace

extern "C" {

void mslice_server_default_opts(mslice_server_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->window = 8;
  o->n_slots = 2;
  o->max_batch = 64;
  o->max_batch_nodes = (int64_t)1 << 21;
  o->hbm_budget = 0;
  o->gamma_num = o->gamma_den = o->omega_num = o->omega_den = 1;
  mslice_default_opts(&o->solve);
}

int mslice_server_create(const mslice_server_opts* o, mslice_server* out) {
  mslice_server s = nullptr;
  const int rc = guard_srv([&] {
    if (!out) fail(MSLICE_EINVAL, "null output server");
    *out = nullptr;
    mslice_server_opts opt;
    mslice_server_default_opts(&opt);
    if (o) opt = *o;
    if (opt.window < 1 || opt.n_slots < 1 || opt.n_slots > 64 || opt.max_batch < 1 || opt.hbm_budget < 0 ||
        opt.max_batch_nodes < 1)
      fail(MSLICE_EINVAL, "window, n_slots (<= 64), max_batch and max_batch_nodes must be >= 1, hbm_budget >= 0");
    const mslice_opts& so = opt.solve;
    if (so.n_iterations < 1 || so.K < 1 || so.K > 64 || so.max_rounds < 1 || so.max_levels < 1)
      fail(MSLICE_EINVAL, "bad schedule options");
    if (so.theta_num < 0 || so.theta_num > ((int64_t)1 << 31) || so.theta_den < 1 || so.theta_den > ((int64_t)1 << 31))
      fail(MSLICE_EINVAL, "theta must be a rational >= 0");
    if ((so.flags & MSLICE_NULL_GLOBAL) && (so.flags & MSLICE_NULL_CPM))
      fail(MSLICE_EINVAL, "MSLICE_NULL_GLOBAL and MSLICE_NULL_CPM exclude each other");
    if (so.tier_cuts[0] || so.tier_cuts[1] || so.tier_cuts[2] || so.tier_cuts[3]) {
      int32_t lo = 0;
      for (int k = 0; k < 4; ++k) {
        if (so.tier_cuts[k] < lo || so.tier_cuts[k] > TIER_MAX[k]) fail(MSLICE_EINVAL, "bad tier cuts");
        lo = so.tier_cuts[k];
      }
    }
    const int64_t lim = (int64_t)1 << 31;
    if (opt.gamma_num < 1 || opt.gamma_num > lim || opt.gamma_den < 1 || opt.gamma_den > lim || opt.omega_num < 0 ||
        opt.omega_num > lim || opt.omega_den < 1 || opt.omega_den > lim)
      fail(MSLICE_EINVAL, "gamma must be a rational > 0 and omega >= 0");
    s = new mslice_server_s();
    s->opt = opt;
    s->t0 = Clock::now();
    check_cuda(cudaGetDevice(&s->device), "device");
    keep_pool_memory();
    if (s->opt.hbm_budget == 0) {
      size_t fr = 0, tot = 0;
      check_cuda(cudaMemGetInfo(&fr, &tot), "memory info");
      s->opt.hbm_budget = (int64_t)(0.8 * (double)fr);
    }
    for (int k = 0; k < opt.n_slots; ++k) {
      auto slot = std::make_unique<Worker>();
      slot->id = k;
      check_cuda(cudaStreamCreateWithFlags(&slot->stream, cudaStreamNonBlocking), "stream");
      if (!std::getenv("MSLICE_SERIAL_TIERS")) slot->fan.create();
      slot->ws.stream = slot->stream;
      slot->batch.mem.stream = slot->stream;
      check_cuda(cudaMallocHost(&slot->pinned, PINNED_BYTES), "pinned buffer");
      check_cuda(cudaMalloc(&slot->d_status, 16), "status word");
      check_cuda(cudaMemset(slot->d_status, 0, 16), "memset");
      s->slots.push_back(std::move(slot));
    }
    for (auto& slot : s->slots) s->workers.emplace_back(worker_loop, s, slot.get());
    *out = s;
  });
  if (rc != MSLICE_OK && s) mslice_server_free(s);
  return rc;
}

int mslice_server_add_graph(mslice_server s, int64_t n, int32_t* graph_id) {
  return guard_srv([&] {
    if (!s) fail(MSLICE_EINVAL, "null server");
    if (n < 1 || n * (int64_t)s->opt.window > INT32_MAX) fail(MSLICE_EINVAL, "n*window must fit in int32");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->graphs.size() >= (size_t)INT32_MAX) fail(MSLICE_EINVAL, "too many graphs");
    auto g = std::make_unique<SrvGraph>();
    g->n = n;
    const int R = s->opt.window + 1;
    g->ip.assign(R, nullptr);
    g->ix.assign(R, nullptr);
    g->wt.assign(R, nullptr);
    g->cap_ix.assign(R, 0);
    g->nnz.assign(R, 0);
    s->graphs.push_back(std::move(g));
    if (graph_id) *graph_id = (int32_t)s->graphs.size() - 1;
  });
}

int mslice_server_submit(mslice_server s, int32_t graph_id, const mslice_csr* slice, int64_t* request_id) {
  return guard_srv([&] {
    if (!s || !slice) fail(MSLICE_EINVAL, "null server or slice");
    int64_t n = 0;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (graph_id < 0 || graph_id >= (int32_t)s->graphs.size()) fail(MSLICE_EINVAL, "unknown graph");
      n = s->graphs[graph_id]->n;
      if (s->stop) fail(MSLICE_EINVAL, "server is stopping");
    }
    if (slice->n != n) fail(MSLICE_EINVAL, "slice n differs from the graph's");
    if (!slice->indptr) fail(MSLICE_EINVAL, "null indptr");
    auto r = std::make_unique<SrvRequest>();
    r->graph = graph_id;
    r->nnz = slice->indptr[n];
    if (slice->indptr[0] != 0 || r->nnz < 0) fail(MSLICE_EINVAL, "malformed row pointers");
    if (r->nnz > 0 && (!slice->indices || !slice->weights)) fail(MSLICE_EINVAL, "null indices/weights");
    r->indptr.assign(slice->indptr, slice->indptr + n + 1);
    if (r->nnz > 0) {
      r->indices.assign(slice->indices, slice->indices + r->nnz);
      r->weights.assign(slice->weights, slice->weights + r->nnz);
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      r->id = s->next_id++;
      r->info.t_submit = s->now();
      r->info.slot = -1;
      if (request_id) *request_id = r->id;
      s->queue.push_back(r->id);
      s->reqs[r->id] = std::move(r);
    }
    s->cv_work.notify_one();
  });
}

int mslice_server_wait(mslice_server s, int64_t request_id, int32_t* labels_out, mslice_request_info* info) {
  std::unique_ptr<SrvRequest> r;
  {
    if (!s) {
      set_last_error("null server");
      return MSLICE_EINVAL;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) {
      set_last_error("unknown request");
      return MSLICE_EINVAL;
    }
    SrvRequest* p = it->second.get();
    s->cv_done.wait(lk, [&] { return p->done; });
    r = std::move(it->second);
    s->reqs.erase(it);
  }
  if (info) *info = r->info;
  if (r->info.status != MSLICE_OK) {
    set_last_error(r->msg);
    return r->info.status;
  }
  if (labels_out && !r->labels.empty()) std::memcpy(labels_out, r->labels.data(), r->labels.size() * sizeof(int32_t));
  set_last_error("");
  return MSLICE_OK;
}

}  // extern "C"

namespace {

// Marks an idle graph busy for a checkpoint or restore (no request of it may
// be queued or in flight); released by the destructor.
struct IdleGraph {
  mslice_server_s* s;
  SrvGraph* g = nullptr;
  IdleGraph(mslice_server_s* srv, int32_t graph_id) : s(srv) {
    std::lock_guard<std::mutex> lk(s->mu);
    if (graph_id < 0 || graph_id >= (int32_t)s->graphs.size()) fail(MSLICE_EINVAL, "unknown graph");
    SrvGraph* gg = s->graphs[graph_id].get();
    if (gg->busy) fail(MSLICE_EINVAL, "the graph has a request in flight");
    for (int64_t id : s->queue)
      if (s->reqs[id]->graph == graph_id) fail(MSLICE_EINVAL, "the graph has queued requests");
    gg->busy = true;
    g = gg;
  }
  ~IdleGraph() {
    if (!g) return;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      g->busy = false;
    }
    s->cv_work.notify_all();
  }
};

// A private stream, scratch and status word for work done on the caller's
// thread.
struct CallerCtx {
  cudaStream_t stream = nullptr;
  Workspace ws;
  unsigned* d_status = nullptr;
  void* pinned = nullptr;
  Ctx c;
  CallerCtx() {
    check_cuda(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking), "stream");
    ws.stream = stream;
    check_cuda(cudaMallocHost(&pinned, PINNED_BYTES), "pinned buffer");
    d_status = ws.get<unsigned>("status", 4);
    check_cuda(cudaMemsetAsync(d_status, 0, 16, stream), "memset");
    c.stream = stream;
    c.ws = &ws;
    c.d_status = d_status;
    c.pinned = pinned;
  }
  ~CallerCtx() {
    ws.release_all();
    if (pinned) cudaFreeHost(pinned);
    if (stream) cudaStreamDestroy(stream);
  }
};

}  // namespace

extern "C" {

int mslice_server_window_info(mslice_server s, int32_t graph_id, int32_t* slices, int64_t* nnz) {
  return guard_srv([&] {
    if (!s) fail(MSLICE_EINVAL, "null server");
    IdleGraph ig(s, graph_id);
    if (slices) *slices = (int32_t)ig.g->window.size();
    if (nnz)
      for (size_t k = 0; k < ig.g->window.size(); ++k) nnz[k] = ig.g->nnz[ig.g->window[k]];
  });
}

int mslice_server_window_read(mslice_server s, int32_t graph_id, int32_t k, int64_t* indptr, int32_t* indices,
                              int32_t* weights, int32_t* labels) {
  return guard_srv([&] {
    if (!s) fail(MSLICE_EINVAL, "null server");
    IdleGraph ig(s, graph_id);
    SrvGraph& g = *ig.g;
    const int32_t w = (int32_t)g.window.size();
    check_cuda(cudaSetDevice(s->device), "device");
    if (k == -1) {
      if (w > 0) {
        if (!labels) fail(MSLICE_EINVAL, "null labels");
        check_cuda(cudaMemcpy(labels, g.labels, g.n * w * sizeof(int32_t), cudaMemcpyDeviceToHost), "copy");
      }
      return;
    }
    if (k < 0 || k >= w) fail(MSLICE_EINVAL, "no such snapshot in the window");
    const int b = g.window[k];
    if (!indptr || (g.nnz[b] > 0 && (!indices || !weights))) fail(MSLICE_EINVAL, "null output arrays");
    check_cuda(cudaMemcpy(indptr, g.ip[b], (g.n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost), "copy");
    if (g.nnz[b] > 0) {
      check_cuda(cudaMemcpy(indices, g.ix[b], g.nnz[b] * sizeof(int32_t), cudaMemcpyDeviceToHost), "copy");
      check_cuda(cudaMemcpy(weights, g.wt[b], g.nnz[b] * sizeof(int32_t), cudaMemcpyDeviceToHost), "copy");
    }
  });
}

int mslice_server_window_restore(mslice_server s, int32_t graph_id, const mslice_csr* slices, int32_t nslices,
                                 const int32_t* labels) {
  return guard_srv([&] {
    if (!s) fail(MSLICE_EINVAL, "null server");
    if (!slices || !labels || nslices < 1 || nslices > s->opt.window)
      fail(MSLICE_EINVAL, "need 1..window snapshots and their labels");
    IdleGraph ig(s, graph_id);
    SrvGraph& g = *ig.g;
    const int64_t n = g.n, N = n * nslices;
    for (int32_t k = 0; k < nslices; ++k) {
      if (slices[k].n != n || !slices[k].indptr) fail(MSLICE_EINVAL, "snapshot n differs from the graph's");
      const int64_t z = slices[k].indptr[n];
      if (slices[k].indptr[0] != 0 || z < 0) fail(MSLICE_EINVAL, "malformed row pointers");
      if (z > 0 && (!slices[k].indices || !slices[k].weights)) fail(MSLICE_EINVAL, "null indices/weights");
    }
    for (int64_t v = 0; v < N; ++v)
      if (labels[v] < 0 || labels[v] >= N) fail(MSLICE_EINVAL, "labels must lie in [0, n * nslices)");
    check_cuda(cudaSetDevice(s->device), "device");
    CallerCtx cc;
    Ctx& c = cc.c;
    // upload to scratch and validate as a build would, before touching the ring
    std::vector<const int64_t*> ip(nslices);
    std::vector<const int32_t*> ix(nslices), wt(nslices);
    std::vector<int64_t> nnz(nslices);
    for (int32_t k = 0; k < nslices; ++k) {
      const std::string tag = std::to_string(k);
      nnz[k] = slices[k].indptr[n];
      int64_t* dip = cc.ws.get<int64_t>("r_ip" + tag, n + 1);
      int32_t* dix = cc.ws.get<int32_t>("r_ix" + tag, nnz[k]);
      int32_t* dwt = cc.ws.get<int32_t>("r_wt" + tag, nnz[k]);
      check_cuda(cudaMemcpyAsync(dip, slices[k].indptr, (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c.stream),
                 "copy");
      if (nnz[k] > 0) {
        check_cuda(cudaMemcpyAsync(dix, slices[k].indices, nnz[k] * sizeof(int32_t), cudaMemcpyHostToDevice,
                                   c.stream), "copy");
        check_cuda(cudaMemcpyAsync(dwt, slices[k].weights, nnz[k] * sizeof(int32_t), cudaMemcpyHostToDevice,
                                   c.stream), "copy");
      }
      ip[k] = dip;
      ix[k] = dix;
      wt[k] = dwt;
    }
    {
      SupraGraph check;
      check.mem.stream = c.stream;
      build_supra(c, ip, ix, wt, nnz, n, check);
      check_bounds(n, check.T, 0, check.two_m_host.data(),
                   InstParams{s->opt.gamma_num, s->opt.gamma_den, s->opt.omega_num, s->opt.omega_den}, s->null_model());
    }
    // valid: the ring's buffers 0..nslices-1 take the snapshots
    g.mem.stream = c.stream;
    for (int32_t k = 0; k < nslices; ++k) {
      const std::string tag = std::to_string(k);
      g.ip[k] = g.mem.get<int64_t>("ip" + tag, n + 1);
      if (nnz[k] > g.cap_ix[k] || !g.ix[k]) {
        g.ix[k] = g.mem.get<int32_t>("ix" + tag, nnz[k]);
        g.wt[k] = g.mem.get<int32_t>("wt" + tag, nnz[k]);
        g.cap_ix[k] = std::max<int64_t>(nnz[k], 1);
      }
      check_cuda(cudaMemcpyAsync(g.ip[k], ip[k], (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, c.stream), "copy");
      if (nnz[k] > 0) {
        check_cuda(cudaMemcpyAsync(g.ix[k], ix[k], nnz[k] * sizeof(int32_t), cudaMemcpyDeviceToDevice, c.stream),
                   "copy");
        check_cuda(cudaMemcpyAsync(g.wt[k], wt[k], nnz[k] * sizeof(int32_t), cudaMemcpyDeviceToDevice, c.stream),
                   "copy");
      }
      g.nnz[k] = nnz[k];
    }
    g.labels = g.mem.get<int32_t>("labels", N);
    check_cuda(cudaMemcpyAsync(g.labels, labels, N * sizeof(int32_t), cudaMemcpyHostToDevice, c.stream), "copy");
    check_cuda(cudaStreamSynchronize(c.stream), "stream synchronize");
    g.mem.stream = nullptr;  // the private stream ends with this call
    g.window.clear();
    for (int32_t k = 0; k < nslices; ++k) g.window.push_back(k);
  });
}

void mslice_server_free(mslice_server s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& slot : s->slots) {
    slot->ws.release_all();
    slot->batch.mem.release_all();
    if (slot->stream) cudaStreamSynchronize(slot->stream);
    if (slot->d_status) cudaFree(slot->d_status);
    if (slot->pinned) cudaFreeHost(slot->pinned);
  }
  for (auto& g : s->graphs) g->mem.release_all();
  for (auto& slot : s->slots) {
    slot->fan.destroy();
    if (slot->stream) cudaStreamDestroy(slot->stream);
  }
  delete s;
}

}  // extern "C"
