// Aggregation (Louvain/Leiden, Sec. 3.2): one node per refined
// sub-community, numbered by ascending sub-community label.  Edges between
// different new nodes are keyed (x*N' + y), radix-sorted and reduced by key
// (weights summed); self-loops are dropped because no key or check reads
// them and Q is always evaluated on level 0.  Snapshot strengths k_{x,s} are
// the refinement's K_{R,s} table, sorted by (x, s).  The initial label of a
// new node is the smallest new id inside its local-moving community.
#include "solver.h"

namespace mslice {

namespace {

__global__ void k_present(const int32_t* sizeR, int32_t N, int32_t* flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = sizeR[i] > 0 ? 1 : 0;
}

// One warp per row; surviving entries are compacted with one atomic per warp
// step (their order is fixed afterwards by the sort).
__global__ void k_emit_edges(LevelDev g, const int32_t* R, const int32_t* newid, uint64_t Np, uint64_t* keys,
                             long long* vals, ull* cursor) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = (((int64_t)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5); v < g.N; v += warps) {
    const uint64_t x = (uint64_t)newid[R[v]];
    const int64_t b = g.rowptr[v], e = g.rowptr[v + 1];
    const Omega om = node_omega(g, (int32_t)v);
    for (int64_t base = b; base < e; base += 32) {
      const int64_t i = base + lane;
      bool keep = false;
      uint64_t key = 0;
      long long W = 0;
      if (i < e) {
        int32_t u;
        if (edge_at(g, i, u, W, om)) {
          const uint64_t y = (uint64_t)newid[R[u]];
          if (y != x) {
            keep = true;
            key = x * Np + y;
          }
        }
      }
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (m == 0) continue;
      ull pos = 0;
      if (lane == 0) pos = atomicAdd(cursor, (ull)__popc(m));
      pos = __shfl_sync(0xffffffffu, pos, 0);
      if (keep) {
        const ull o = pos + __popc(m & ((1u << lane) - 1u));
        keys[o] = key;
        vals[o] = W;
      }
    }
  }
}

// Hashed K_{R,s}: entries in table order, sorted afterwards.
__global__ void k_emit_slices(SigStore kr, const int32_t* newid, uint64_t T, uint64_t* keys, long long* vals,
                              ull* cursor) {
  const int lane = threadIdx.x & 31;
  const uint64_t span = ss_span(kr);
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < span; base += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = base + threadIdx.x;
    bool keep = false;
    uint64_t key = 0;
    long long val = 0;
    if (i < span) {
      int32_t Rl, s;
      if (ss_entry(kr, i, Rl, s, val)) {
        keep = true;
        key = (uint64_t)newid[Rl] * T + (uint64_t)s;
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (m == 0) continue;
    ull pos = 0;
    if (lane == 0) pos = atomicAdd(cursor, (ull)__popc(m));
    pos = __shfl_sync(0xffffffffu, pos, 0);
    if (keep) {
      const ull o = pos + __popc(m & ((1u << lane) - 1u));
      keys[o] = key;
      vals[o] = val;
    }
  }
}

// Dense K_{R,s}: rows are already in (new id, snapshot) order, since new ids
// rank the present labels; count and copy the non-zero entries row by row.
__global__ void k_dense_slice_counts(const long long* d, int32_t T, const int32_t* sizeR, const int32_t* newid,
                                     int32_t N, int32_t* cnt) {
  for (int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; L < N; L += (int64_t)gridDim.x * blockDim.x) {
    if (sizeR[L] <= 0) continue;
    int32_t c = 0;
    for (int32_t s = 0; s < T; ++s) c += d[L * T + s] != 0;
    cnt[newid[L]] = c;
  }
}

__global__ void k_dense_slice_fill(const long long* d, int32_t T, const int32_t* sizeR, const int32_t* newid,
                                   int32_t N, const int64_t* sptr, int32_t* sidx, long long* sval) {
  for (int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; L < N; L += (int64_t)gridDim.x * blockDim.x) {
    if (sizeR[L] <= 0) continue;
    int64_t o = sptr[newid[L]];
    for (int32_t s = 0; s < T; ++s) {
      const long long x = d[L * T + s];
      if (x != 0) {
        sidx[o] = s;
        sval[o] = x;
        ++o;
      }
    }
  }
}

__global__ void k_seg_flags(const uint64_t* keys, int64_t m, int32_t* flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void k_zero_ll(long long* p, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = 0;
}

__global__ void k_seg_reduce(const uint64_t* keys, const long long* vals, const int32_t* flag, const int64_t* pos,
                             int64_t m, uint64_t* ukeys, long long* usum) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t id = pos[i] + flag[i] - 1;
    if (flag[i]) ukeys[id] = keys[i];
    atomicAdd((ull*)&usum[id], (ull)vals[i]);
  }
}

// Unique (row, col) keys -> per-row counts and the column array.
__global__ void k_rows_of(const uint64_t* ukeys, int64_t mu, uint64_t div, int32_t* cnt, int32_t* col) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < mu; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = ukeys[i];
    atomicAdd(&cnt[k / div], 1);
    col[i] = (int32_t)(k % div);
  }
}

__global__ void k_slices_of(const uint64_t* keys, const long long* vals, int64_t ms, uint64_t T, int32_t* cnt,
                            int32_t* sidx, long long* sval) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ms; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    atomicAdd(&cnt[k / T], 1);
    sidx[i] = (int32_t)(k % T);
    sval[i] = vals[i];
  }
}

__global__ void k_min_init(const int32_t* P, const int32_t* R, const int32_t* newid, int32_t N, int32_t* minid) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
    atomicMin(&minid[P[v]], newid[R[v]]);
}

__global__ void k_next_labels(const int32_t* P, const int32_t* R, const int32_t* newid, const int32_t* minid,
                              int32_t N, int32_t* next) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
    next[newid[R[v]]] = minid[P[v]];
}

// Batches: instance of every new node and the first new id of every instance.
__global__ void k_next_inst(LevelDev g, const int32_t* R, const int32_t* newid, int32_t* inst_next, int32_t* off_next) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.N; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = newid[R[v]];
    const int32_t i = g.inst[v];
    inst_next[x] = i;
    atomicMin(&off_next[i], x);
  }
}

__global__ void k_compose(const int32_t* R, const int32_t* newid, int64_t N0, int32_t* node_of0) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N0; v += (int64_t)gridDim.x * blockDim.x)
    node_of0[v] = newid[R[node_of0[v]]];
}

__global__ void k_max_deg(const int64_t* rowptr, int32_t N, int32_t* mx) {
  int32_t m = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (int32_t)(rowptr[v + 1] - rowptr[v]));
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(mx, m);
}

unsigned gsz(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

int bits_for(uint64_t maxval) {
  int b = 0;
  while (b < 64 && (maxval >> b) != 0) ++b;
  return b < 1 ? 1 : b;
}

}  // namespace

bool aggregate(Solver& S, const Level& L, const int32_t* P, Level& next, const std::string& slot,
               int32_t* next_labels, int32_t* node_of0, int64_t* checksum) {
  Ctx& c = *S.c;
  const int32_t N = L.d.N;
  // new ids = ranks of the present sub-community labels
  int32_t* flag = S.tmp32a;
  int32_t* newid = S.tmp32b;
  launch(c, k_present, dim3(gsz(N)), dim3(256), 0, (const int32_t*)S.sizeR, N, flag);
  int32_t* d_np = c.ws->get<int32_t>("ag_np", 1);
  scan_excl(c, flag, newid, N, d_np);
  const int32_t Np = *static_cast<const int32_t*>(readback(c, d_np, sizeof(int32_t)));
  if (Np == N) return false;

  // ---- edges ----
  const int64_t cap = L.nnz > 0 ? L.nnz : 1;
  uint64_t* k0 = c.ws->get<uint64_t>("ag_k0", cap);
  long long* v0 = c.ws->get<long long>("ag_v0", cap);
  uint64_t* k1 = c.ws->get<uint64_t>("ag_k1", cap);
  long long* v1 = c.ws->get<long long>("ag_v1", cap);
  ull* cursor = c.ws->get<ull>("ag_cursor", 2);
  check_cuda(cudaMemsetAsync(cursor, 0, 2 * sizeof(ull), c.stream), "memset");
  launch(c, k_emit_edges, dim3(gsz((int64_t)N * 32)), dim3(256), 0, L.d, (const int32_t*)S.R, (const int32_t*)newid,
         (uint64_t)Np, k0, v0, cursor);
  const int64_t m = (int64_t) * static_cast<const ull*>(readback(c, cursor, sizeof(ull)));
  const SortBufs sorted = radix_sort_pairs(c, k0, v0, k1, v1, m, bits_for((uint64_t)Np * (uint64_t)Np - 1));
  int32_t* sflag = c.ws->get<int32_t>("ag_flag", m + 1);
  int64_t* spos = c.ws->get<int64_t>("ag_pos", m + 1);
  int64_t* d_mu = c.ws->get<int64_t>("ag_mu", 1);
  launch(c, k_seg_flags, dim3(gsz(m)), dim3(256), 0, (const uint64_t*)sorted.keys, m, sflag);
  scan_excl(c, sflag, spos, m, d_mu);
  const int64_t mu = m > 0 ? *static_cast<const int64_t*>(readback(c, d_mu, sizeof(int64_t))) : 0;
  // unique keys/sums go to the buffers the sort did not leave its result in
  uint64_t* ukeys = sorted.keys == k0 ? k1 : k0;
  long long* usum = sorted.vals == v0 ? v1 : v0;
  launch(c, k_zero_ll, dim3(gsz(mu)), dim3(256), 0, usum, mu);
  launch(c, k_seg_reduce, dim3(gsz(m)), dim3(256), 0, (const uint64_t*)sorted.keys, (const long long*)sorted.vals,
         (const int32_t*)sflag, (const int64_t*)spos, m, ukeys, usum);

  next.d = LevelDev{};
  next.d.N = Np;
  next.d.is0 = 0;
  next.d.on = L.d.on;
  next.d.od = L.d.od;
  next.d.on_i = L.d.on_i;
  next.d.od_i = L.d.od_i;
  if (L.d.inst) {
    int32_t* inst_next = c.ws->get<int32_t>(slot + "_inst", (size_t)Np);
    int32_t* off_next = c.ws->get<int32_t>(slot + "_ioff", (size_t)S.B + 1);
    fill_i32(c, off_next, Np, (int64_t)S.B + 1);
    launch(c, k_next_inst, dim3(gsz(N)), dim3(256), 0, L.d, (const int32_t*)S.R, (const int32_t*)newid, inst_next,
           off_next);
    next.d.inst = inst_next;
    next.d.inst_off = off_next;
  }
  int64_t* rowptr = c.ws->get<int64_t>(slot + "_rowptr", (size_t)Np + 1);
  int32_t* col = c.ws->get<int32_t>(slot + "_col", mu);
  long long* W = c.ws->get<long long>(slot + "_W", mu);
  int32_t* cnt = c.ws->get<int32_t>("ag_cnt", (size_t)Np + 1);
  check_cuda(cudaMemsetAsync(cnt, 0, ((size_t)Np + 1) * sizeof(int32_t), c.stream), "memset");
  launch(c, k_rows_of, dim3(gsz(mu)), dim3(256), 0, (const uint64_t*)ukeys, mu, (uint64_t)Np, cnt, col);
  scan_excl(c, cnt, rowptr, (int64_t)Np + 1, (int64_t*)nullptr);
  check_cuda(cudaMemcpyAsync(W, usum, mu * sizeof(long long), cudaMemcpyDeviceToDevice, c.stream), "copy");
  next.d.rowptr = rowptr;
  next.d.col = col;
  next.d.W = W;
  next.nnz = mu;
  next.nnz_eff = mu;

  // ---- snapshot strengths ----
  const uint64_t T = (uint64_t)S.G0->T;
  int64_t* sptr = c.ws->get<int64_t>(slot + "_sptr", (size_t)Np + 1);
  int64_t ms = 0;
  int32_t* sidx = nullptr;
  long long* sval = nullptr;
  check_cuda(cudaMemsetAsync(cnt, 0, ((size_t)Np + 1) * sizeof(int32_t), c.stream), "memset");
  if (S.kr.d) {
    launch(c, k_dense_slice_counts, dim3(gsz(N)), dim3(256), 0, (const long long*)S.kr.d, (int32_t)T,
           (const int32_t*)S.sizeR, (const int32_t*)newid, N, cnt);
    int64_t* d_ms = c.ws->get<int64_t>("ag_ms", 1);
    scan_excl(c, cnt, sptr, (int64_t)Np + 1, d_ms);
    ms = *static_cast<const int64_t*>(readback(c, d_ms, sizeof(int64_t)));
    sidx = c.ws->get<int32_t>(slot + "_sidx", ms);
    sval = c.ws->get<long long>(slot + "_sval", ms);
    launch(c, k_dense_slice_fill, dim3(gsz(N)), dim3(256), 0, (const long long*)S.kr.d, (int32_t)T,
           (const int32_t*)S.sizeR, (const int32_t*)newid, N, (const int64_t*)sptr, sidx, sval);
  } else {
    const int64_t scap = (int64_t)S.kr.h.cap;
    uint64_t* sk0 = c.ws->get<uint64_t>("ag_sk0", scap);
    long long* sv0 = c.ws->get<long long>("ag_sv0", scap);
    uint64_t* sk1 = c.ws->get<uint64_t>("ag_sk1", scap);
    long long* sv1 = c.ws->get<long long>("ag_sv1", scap);
    launch(c, k_emit_slices, dim3(gsz(scap)), dim3(256), 0, S.kr, (const int32_t*)newid, T, sk0, sv0, cursor + 1);
    ms = (int64_t) * static_cast<const ull*>(readback(c, cursor + 1, sizeof(ull)));
    const SortBufs ss = radix_sort_pairs(c, sk0, sv0, sk1, sv1, ms, bits_for((uint64_t)Np * T - 1));
    sidx = c.ws->get<int32_t>(slot + "_sidx", ms);
    sval = c.ws->get<long long>(slot + "_sval", ms);
    launch(c, k_slices_of, dim3(gsz(ms)), dim3(256), 0, (const uint64_t*)ss.keys, (const long long*)ss.vals, ms, T,
           cnt, sidx, sval);
    scan_excl(c, cnt, sptr, (int64_t)Np + 1, (int64_t*)nullptr);
  }
  next.d.sptr = sptr;
  next.d.sidx = sidx;
  next.d.sval = sval;
  next.ns = ms;

  // ---- initial labels, level map ----
  int32_t* minid = flag;  // reuse
  fill_i32(c, minid, INT32_MAX, N);
  launch(c, k_min_init, dim3(gsz(N)), dim3(256), 0, P, (const int32_t*)S.R, (const int32_t*)newid, N, minid);
  launch(c, k_next_labels, dim3(gsz(N)), dim3(256), 0, P, (const int32_t*)S.R, (const int32_t*)newid,
         (const int32_t*)minid, N, next_labels);
  if (node_of0)
    launch(c, k_compose, dim3(gsz(S.N0)), dim3(256), 0, (const int32_t*)S.R, (const int32_t*)newid, S.N0, node_of0);
  int32_t* d_mx = c.ws->get<int32_t>("ag_mx", 1);
  check_cuda(cudaMemsetAsync(d_mx, 0, sizeof(int32_t), c.stream), "memset");
  launch(c, k_max_deg, dim3(gsz(Np)), dim3(256), 0, (const int64_t*)rowptr, Np, d_mx);
  next.max_deg = *static_cast<const int32_t*>(readback(c, d_mx, sizeof(int32_t)));
  if (checksum) *checksum = (int64_t)level_checksum(S, next);
  return true;
}

}  // namespace mslice
