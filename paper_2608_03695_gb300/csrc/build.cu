// Supra-graph builder (Eq. supra-adjacency): the level-0 CSR over N = n*T
// supra-nodes.  Row v = s*n + i holds, in ascending column order, the
// coupling entries to the copies of i in earlier snapshots, the snapshot-s row
// of i shifted by s*n, and the coupling entries to later copies.  Ordinal
// coupling (Eq. supra-adjacency) couples s with s-1 and s+1; categorical
// coupling (the all-pairs omega^(sr) of Eq. multislice-modularity) with every
// other snapshot.  Entries are 8-byte {col, w} pairs; w <= 0 flags a coupling
// entry and names its pair's slot (-w-1) in a table of omega numerators, so
// omega (uniform or per pair) is applied at solve time and a sweep needs no
// rebuild.
#include "build.h"

#include "../../include/mslice.h"

#include <algorithm>

namespace mslice {

namespace {

struct SliceTable {
  const int64_t* const* indptr;
  const int32_t* const* indices;
  const int32_t* const* weights;
};

// indptr of every snapshot: starts at 0, non-decreasing, ends at nnz_s.
__global__ void k_check_indptr(SliceTable st, const int64_t* nnz, int32_t T, int64_t n, unsigned* status) {
  const int64_t total = n * (int64_t)T;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < total; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = (int32_t)(v / n);
    const int64_t i = v - (int64_t)s * n;
    const int64_t a = st.indptr[s][i], b = st.indptr[s][i + 1];
    bool bad = (b < a) || (a < 0) || (b > nnz[s]);
    if (i == 0 && a != 0) bad = true;
    if (i == n - 1 && b != nnz[s]) bad = true;
    if (bad) atomicOr(status, ERR_BAD_INPUT);
  }
}

// Row contents: sorted strictly ascending, in range, no self-loop, w >= 1,
// and the mirrored entry (j, i) present with the same weight.  One warp per
// supra-row.
__global__ void k_check_rows(SliceTable st, int32_t T, int64_t n, unsigned* status) {
  const int64_t total = n * (int64_t)T;
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = (((int64_t)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5); v < total; v += warps) {
    const int32_t s = (int32_t)(v / n);
    const int64_t i = v - (int64_t)s * n;
    const int64_t* ip = st.indptr[s];
    const int32_t* ix = st.indices[s];
    const int32_t* wt = st.weights[s];
    const int64_t a = ip[i], b = ip[i + 1];
    bool bad = false;
    for (int64_t e = a + lane; e < b; e += 32) {
      const int32_t j = ix[e];
      const int32_t w = wt[e];
      if (j < 0 || j >= n || j == i || w < 1) {
        bad = true;
        continue;
      }
      if (e > a && ix[e - 1] >= j) bad = true;
      // binary search for i in row j
      int64_t lo = ip[j], hi = ip[j + 1];
      while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (ix[mid] < i)
          lo = mid + 1;
        else
          hi = mid;
      }
      if (lo >= ip[j + 1] || ix[lo] != i || wt[lo] != w) bad = true;
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, ERR_BAD_INPUT);
  }
}

// Coupled snapshots of snapshot s: [lo, s) below and (s, hi) above.
__device__ __forceinline__ void coupled_range(int32_t coupling, int32_t T, int32_t s, int32_t& lo, int32_t& hi) {
  lo = coupling == 0 ? (s > 0 ? s - 1 : 0) : 0;
  hi = coupling == 0 ? (s + 2 < T ? s + 2 : T) : T;
}

// The flag of the coupling entry from snapshot s to r: -(slot + 1).
__device__ __forceinline__ int32_t coupling_flag(int32_t coupling, int32_t T, int32_t s, int32_t r) {
  return coupling == 0 ? -((s < r ? s : r) + 1) : -(s * T + r + 1);
}

__global__ void k_row_len(SliceTable st, int32_t T, int64_t n, int32_t coupling, int64_t* len) {
  const int64_t total = n * (int64_t)T;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < total; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = (int32_t)(v / n);
    const int64_t i = v - (int64_t)s * n;
    int32_t lo, hi;
    coupled_range(coupling, T, s, lo, hi);
    len[v] = (st.indptr[s][i + 1] - st.indptr[s][i]) + (s - lo) + (hi - s - 1);
  }
}

// One warp per supra-row: copies the shifted snapshot row, adds the coupling
// flags, and writes k_v = sum of the row's intra weights.
__global__ void k_fill_rows(SliceTable st, int32_t T, int64_t n, int32_t coupling, const int64_t* rowptr, int2* adj,
                            int64_t* k) {
  const int64_t total = n * (int64_t)T;
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = (((int64_t)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5); v < total; v += warps) {
    const int32_t s = (int32_t)(v / n);
    const int64_t i = v - (int64_t)s * n;
    const int64_t a = st.indptr[s][i], b = st.indptr[s][i + 1];
    int32_t lo, hi;
    coupled_range(coupling, T, s, lo, hi);
    int64_t out = rowptr[v];
    for (int32_t r = lo + lane; r < s; r += 32)
      adj[out + (r - lo)] = make_int2((int32_t)((int64_t)r * n + i), coupling_flag(coupling, T, s, r));
    out += s - lo;
    const int32_t off = (int32_t)((int64_t)s * n);
    long long ksum = 0;
    for (int64_t e = a + lane; e < b; e += 32) {
      const int32_t w = st.weights[s][e];
      adj[out + (e - a)] = make_int2(st.indices[s][e] + off, w);
      ksum += w;
    }
    ksum = warp_sum(ksum);
    for (int32_t r = s + 1 + lane; r < hi; r += 32)
      adj[out + (b - a) + (r - s - 1)] = make_int2((int32_t)((int64_t)r * n + i), coupling_flag(coupling, T, s, r));
    if (lane == 0) k[v] = ksum;
  }
}

// 2m_s = sum of k_v over the rows of snapshot s: blockIdx.y is the snapshot,
// blocks stride over its rows, one atomic per block.
__global__ void k_slice_mass(const int64_t* k, int64_t n, ull* two_m) {
  __shared__ ull sm[32];
  const int32_t s = blockIdx.y;
  ull t = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    t += (ull)k[(int64_t)s * n + i];
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x < 32) {
    ull x = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0ull;
    x = warp_sum(x);
    if (threadIdx.x == 0 && x) atomicAdd(&two_m[s], x);
  }
}

__global__ void k_lambda(const int64_t* two_m, int32_t T, const int32_t* slice_inst, const long long* gn,
                         const long long* gd, u128* lam) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= T) return;
  const int32_t i = slice_inst ? slice_inst[s] : 0;
  const long long t = two_m[s];
  lam[s] = t > 0 ? (((u128)(ull)gn[i]) << P_BITS) / ((u128)(ull)gd[i] * (u128)(ull)t) : (u128)0;
}

// Copies one instance into the concatenated arrays (coupling flags move to
// the instance's slots of the batch's table).
__global__ void k_append(int64_t Ni, const int64_t* rowptr, const int2* adj, const int64_t* k, int64_t n, int32_t inst,
                         int64_t noff, int64_t eoff, int32_t soff, int32_t cwoff, int64_t* rowptr_o, int2* adj_o,
                         int64_t* k_o, int32_t* slice0, int32_t* inst0) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < Ni; v += (int64_t)gridDim.x * blockDim.x) {
    rowptr_o[noff + v] = rowptr[v] + eoff;
    k_o[noff + v] = k[v];
    slice0[noff + v] = soff + (int32_t)(v / n);
    inst0[noff + v] = inst;
  }
  const int64_t nnz = rowptr[Ni];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const int2 x = adj[e];
    adj_o[eoff + e] = make_int2(x.x + (int32_t)noff, x.y <= 0 ? x.y - cwoff : x.y);
  }
}

__global__ void k_slice_inst(int32_t* slice_inst, int32_t soff, int32_t T, int32_t inst) {
  for (int s = threadIdx.x; s < T; s += blockDim.x) slice_inst[soff + s] = inst;
}

unsigned gs(int64_t n, int per) {
  int64_t g = (n + per - 1) / per;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

void build_supra(Ctx& c, const std::vector<const int64_t*>& indptr, const std::vector<const int32_t*>& indices,
                 const std::vector<const int32_t*>& weights, const std::vector<int64_t>& nnz, int64_t n,
                 SupraGraph& g, int32_t coupling) {
  const int32_t T = (int32_t)indptr.size();
  if (coupling != 0 && (int64_t)T * T >= INT32_MAX) fail(MSLICE_EINVAL, "categorical coupling needs T*T < 2^31");
  g.T = T;
  g.coupling = coupling;
  g.ncw = coupling_slots(coupling, T);
  g.n = n;
  g.N = n * T;
  // device table of snapshot pointers
  const int64_t** d_ip = c.ws->get<const int64_t*>("b_ip", T);
  const int32_t** d_ix = c.ws->get<const int32_t*>("b_ix", T);
  const int32_t** d_wt = c.ws->get<const int32_t*>("b_wt", T);
  int64_t* d_nnz = c.ws->get<int64_t>("b_nnz", T);
  check_cuda(cudaMemcpyAsync(d_ip, indptr.data(), T * sizeof(void*), cudaMemcpyHostToDevice, c.stream), "copy");
  check_cuda(cudaMemcpyAsync(d_ix, indices.data(), T * sizeof(void*), cudaMemcpyHostToDevice, c.stream), "copy");
  check_cuda(cudaMemcpyAsync(d_wt, weights.data(), T * sizeof(void*), cudaMemcpyHostToDevice, c.stream), "copy");
  check_cuda(cudaMemcpyAsync(d_nnz, nnz.data(), T * sizeof(int64_t), cudaMemcpyHostToDevice, c.stream), "copy");
  SliceTable st{d_ip, d_ix, d_wt};
  check_cuda(cudaMemsetAsync(c.d_status, 0, sizeof(unsigned), c.stream), "memset");
  if (g.N > 0) {
    launch(c, k_check_indptr, dim3(gs(g.N, 256)), dim3(256), 0, st, (const int64_t*)d_nnz, T, n, c.d_status);
    check_status(c, "snapshot row pointers");
    launch(c, k_check_rows, dim3(gs(g.N * 32, 256)), dim3(256), 0, st, T, n, c.d_status);
    check_status(c, "snapshot rows");
  }
  int64_t* len = c.ws->get<int64_t>("b_len", g.N + 1);
  g.rowptr = static_cast<int64_t*>(g.mem.get_bytes("rowptr0", (g.N + 1) * sizeof(int64_t)));
  if (g.N > 0) launch(c, k_row_len, dim3(gs(g.N, 256)), dim3(256), 0, st, T, n, coupling, len);
  int64_t* d_total = c.ws->get<int64_t>("b_total", 1);
  scan_excl(c, len, g.rowptr, g.N, d_total);
  check_cuda(cudaMemcpyAsync(g.rowptr + g.N, d_total, sizeof(int64_t), cudaMemcpyDeviceToDevice, c.stream), "copy");
  g.nnz = *static_cast<int64_t*>(readback(c, d_total, sizeof(int64_t)));
  g.adj = static_cast<int2*>(g.mem.get_bytes("adj0", (g.nnz ? g.nnz : 1) * sizeof(int2)));
  g.k = static_cast<int64_t*>(g.mem.get_bytes("k0", (g.N ? g.N : 1) * sizeof(int64_t)));
  g.two_m = static_cast<int64_t*>(g.mem.get_bytes("two_m", T * sizeof(int64_t)));
  check_cuda(cudaMemsetAsync(g.two_m, 0, T * sizeof(int64_t), c.stream), "memset");
  if (g.N > 0) {
    launch(c, k_fill_rows, dim3(gs(g.N * 32, 256)), dim3(256), 0, st, T, n, coupling, (const int64_t*)g.rowptr,
           g.adj, g.k);
    unsigned gx = (unsigned)std::min<int64_t>((n + 255) / 256, 64);
    launch(c, k_slice_mass, dim3(gx, T), dim3(256), 0, (const int64_t*)g.k, n, (ull*)g.two_m);
  }
  g.two_m_host.resize(T);
  check_cuda(cudaMemcpyAsync(g.two_m_host.data(), g.two_m, T * sizeof(int64_t), cudaMemcpyDeviceToHost, c.stream),
             "copy");
  sync(c);
  g.nnz_intra = g.nnz - coupling_entries(coupling, n, T);
  g.B = 1;
  g.inst.assign(1, InstInfo{n, 0, T, 0, coupling, 0});
}

void compute_lambda(Ctx& c, const SupraGraph& g, const long long* gn, const long long* gd, u128* lam) {
  launch(c, k_lambda, dim3(grid_for(g.T, 128)), dim3(128), 0, (const int64_t*)g.two_m, g.T,
         (const int32_t*)g.slice_inst, gn, gd, lam);
}

void concat_instances(Ctx& c, const std::vector<const SupraGraph*>& parts, SupraGraph& out) {
  const int32_t B = (int32_t)parts.size();
  out.B = B;
  out.inst.assign(B, InstInfo{});
  int64_t N = 0, nnz = 0, nnz_intra = 0, ncw = 0;
  int32_t T = 0;
  for (int32_t i = 0; i < B; ++i) {
    out.inst[i] = InstInfo{parts[i]->n, N, parts[i]->T, T, parts[i]->coupling, ncw};
    N += parts[i]->N;
    nnz += parts[i]->nnz;
    nnz_intra += parts[i]->nnz_intra;
    T += parts[i]->T;
    ncw += parts[i]->ncw;
  }
  if (ncw >= INT32_MAX) fail(MSLICE_EINVAL, "the batch's coupling tables need fewer than 2^31 slots");
  out.ncw = ncw;
  out.coupling = -1;  // per instance
  out.N = N;
  out.T = T;
  out.n = parts.empty() ? 0 : parts[0]->n;
  out.nnz = nnz;
  out.nnz_intra = nnz_intra;
  out.rowptr = static_cast<int64_t*>(out.mem.get_bytes("rowptr0", (N + 1) * sizeof(int64_t)));
  out.adj = static_cast<int2*>(out.mem.get_bytes("adj0", (nnz ? nnz : 1) * sizeof(int2)));
  out.k = static_cast<int64_t*>(out.mem.get_bytes("k0", (N ? N : 1) * sizeof(int64_t)));
  out.two_m = static_cast<int64_t*>(out.mem.get_bytes("two_m", (T ? T : 1) * sizeof(int64_t)));
  out.slice0 = static_cast<int32_t*>(out.mem.get_bytes("slice0", (N ? N : 1) * sizeof(int32_t)));
  out.inst0 = static_cast<int32_t*>(out.mem.get_bytes("inst0", (N ? N : 1) * sizeof(int32_t)));
  out.inst_off0 = static_cast<int32_t*>(out.mem.get_bytes("inst_off0", (B + 1) * sizeof(int32_t)));
  out.slice_inst = static_cast<int32_t*>(out.mem.get_bytes("slice_inst", (T ? T : 1) * sizeof(int32_t)));
  std::vector<int32_t> offs(B + 1);
  int64_t eoff = 0;
  out.two_m_host.clear();
  for (int32_t i = 0; i < B; ++i) {
    const SupraGraph& p = *parts[i];
    offs[i] = (int32_t)out.inst[i].noff;
    if (p.N > 0)
      launch(c, k_append, dim3(gs(std::max<int64_t>(p.N, p.nnz), 256)), dim3(256), 0, p.N, (const int64_t*)p.rowptr,
             (const int2*)p.adj, (const int64_t*)p.k, p.n, i, out.inst[i].noff, eoff, out.inst[i].soff,
             (int32_t)out.inst[i].cwoff, out.rowptr, out.adj, out.k, out.slice0, out.inst0);
    if (p.T > 0) {
      check_cuda(cudaMemcpyAsync(out.two_m + out.inst[i].soff, p.two_m, p.T * sizeof(int64_t),
                                 cudaMemcpyDeviceToDevice, c.stream), "copy");
      launch(c, k_slice_inst, dim3(1), dim3(256), 0, out.slice_inst, out.inst[i].soff, p.T, i);
    }
    for (int64_t t : p.two_m_host) out.two_m_host.push_back(t);
    eoff += p.nnz;
  }
  offs[B] = (int32_t)N;
  check_cuda(cudaMemcpyAsync(out.rowptr + N, &nnz, sizeof(int64_t), cudaMemcpyHostToDevice, c.stream), "copy");
  check_cuda(cudaMemcpyAsync(out.inst_off0, offs.data(), (B + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, c.stream),
             "copy");
  sync(c);
}

}  // namespace mslice
