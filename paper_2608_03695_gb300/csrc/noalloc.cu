// mslice_modularity_noalloc: Q_MS of a labelling, computed without allocating
// any device memory.
//
// Some callers cannot call cudaMalloc (or any routine that allocates device
// memory): plug-ins that must stay inside a memory budget fixed by their host
// application, and services that pre-reserve all device memory at start-up
// and hand out slices of it.  For them this entry point keeps all of its
// scratch in one fixed array that is part of the library image (below).
// Every GPU that loads the library holds that array until the process exits.
// The call copies a small pointer table from host memory and synchronises its
// stream before it returns, so it must not be issued on a stream that is
// being captured into a CUDA graph.
//
// The computation is the same as mslice_modularity (same integer sums, same
// FP64 evaluation order), read straight from the caller's snapshot arrays.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mslice.h"
#include "common.cuh"

namespace mslice {
void set_last_error(const std::string& msg);
}

namespace {

using namespace mslice;

// Scratch of the allocation-free entry point: 32 MiB in 8-byte words.
constexpr size_t NOALLOC_WORDS = (size_t)4 << 20;
static __device__ __align__(256) ull g_noalloc_scratch[NOALLOC_WORDS];

// Word layout inside the scratch (T snapshots, N = n*T supra-nodes):
//   [0]            status bits
//   [1]            Q (double)
//   [2, 4)         I, J
//   [4, 4+3T)      pointer table: indptr, indices, weights of each snapshot
//   [.., +2T)      S_s as 128-bit (lo, hi)
//   [.., +T)       2m_s
//   [.., +N*T)     Sigma_{c,s}, dense rows of T words
constexpr uint64_t W_STATUS = 0, W_Q = 1, W_IJ = 2, W_PTRS = 4;

size_t words_needed(int64_t N, int64_t T) { return (size_t)(W_PTRS + 3 * T + 2 * T + T + N * T); }

struct Layout {
  int64_t n, N;
  int32_t T;
  ull* base;
  const int64_t* const* ip;
  const int32_t* const* ix;
  const int32_t* const* wt;
  ull* S;
  long long* two_m;
  long long* sig;
};

__global__ void k_na_clear(ull* p, size_t words) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (size_t)gridDim.x * blockDim.x) p[i] = 0;
}

// The snapshot conventions of mslice_build, except symmetry: row pointers
// monotone within [0, nnz_s]; index and weight arrays present when a
// snapshot has entries; columns in [0, n), strictly ascending within a row
// (no duplicates) and never the row itself (no self-loops); weights >= 1;
// labels in [0, N).  A violation sets a status bit, and nothing is read out
// of bounds (a row is walked only after its bounds and arrays checked out).
__global__ void k_na_check(Layout L, const int32_t* labels) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < L.N; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = (int32_t)(v / L.n);
    const int64_t i = v - (int64_t)s * L.n;
    const int64_t* ip = L.ip[s];
    const int32_t* ix = L.ix[s];
    const int32_t* wt = L.wt[s];
    const int64_t a = ip[i], b = ip[i + 1], nnz = ip[L.n];
    bool bad = a < 0 || b < a || b > nnz || (i == 0 && a != 0) || (nnz > 0 && (!ix || !wt));
    if (!bad)
      for (int64_t e = a; e < b; ++e) {
        const int32_t j = ix[e];
        if (j < 0 || j >= L.n || j == i || wt[e] < 1 || (e > a && ix[e - 1] >= j)) {
          bad = true;
          break;
        }
      }
    if (labels[v] < 0 || labels[v] >= L.N) bad = true;
    if (bad) atomicOr((unsigned*)&L.base[W_STATUS], 1u);
  }
}

// Per supra-node: strength into Sigma and 2m_s, same-community intra weight
// into I and same-community coupling neighbours into J.
__global__ void k_na_sums(Layout L, const int32_t* labels) {
  if (L.base[W_STATUS]) return;
  ull I = 0, J = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < L.N; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = (int32_t)(v / L.n);
    const int64_t i = v - (int64_t)s * L.n;
    const int32_t c = labels[v];
    const int64_t off = (int64_t)s * L.n;
    long long k = 0;
    for (int64_t e = L.ip[s][i]; e < L.ip[s][i + 1]; ++e) {
      const int32_t w = L.wt[s][e];
      k += w;
      if (labels[off + L.ix[s][e]] == c) I += (ull)w;
    }
    if (s > 0 && labels[v - L.n] == c) J++;
    if (s < L.T - 1 && labels[v + L.n] == c) J++;
    if (k) {
      atomicAdd((ull*)&L.sig[(int64_t)c * L.T + s], (ull)k);
      atomicAdd((ull*)&L.two_m[s], (ull)k);
    }
  }
  I = warp_sum(I);
  J = warp_sum(J);
  if ((threadIdx.x & 31) == 0) {
    if (I) atomicAdd(&L.base[W_IJ], I);
    if (J) atomicAdd(&L.base[W_IJ + 1], J);
  }
}

__global__ void k_na_squares(Layout L) {
  if (L.base[W_STATUS]) return;
  const int64_t span = L.N * L.T;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < span; i += (int64_t)gridDim.x * blockDim.x) {
    const long long x = L.sig[i];
    if (x) atomic_add_u128(&L.S[2 * (i % L.T)], (u128)(ull)x * (u128)(ull)x);
  }
}

// Q in the fixed FP64 order shared with mslice_modularity, after the overflow
// guard of the library's conventions.
__global__ void k_na_q(Layout L, long long gn, long long gd, long long on, long long od) {
  if (L.base[W_STATUS]) return;
  u128 sum2m = 0;
  for (int s = 0; s < L.T; ++s) sum2m += (u128)(ull)L.two_m[s];
  const u128 lim = (u128)1 << 61;
  const u128 ncpl = (u128)(ull)L.n * (u128)(ull)(L.T - 1);
  if ((u128)(ull)od * sum2m + 2 * (u128)(ull)on * ncpl >= lim || (u128)(ull)gn * (u128)(ull)od * sum2m >= lim * (u128)(ull)gd) {
    L.base[W_STATUS] |= 2u;
    return;
  }
  double nullsum = 0.0;
  for (int s = 0; s < L.T; ++s) {
    const long long t = L.two_m[s];
    if (t > 0) {
      const u128 x = ((u128)L.S[2 * s + 1] << 64) | L.S[2 * s];
      nullsum = __dadd_rn(nullsum, __ddiv_rn(u128_to_double(x), __ll2double_rn(t)));
    }
  }
  const double wJ = __ddiv_rn(__dmul_rn(__ll2double_rn(on), __ull2double_rn(L.base[W_IJ + 1])), __ll2double_rn(od));
  const double gam = __ddiv_rn(__ll2double_rn(gn), __ll2double_rn(gd));
  const long long twomu_num = od * (long long)sum2m + 2 * on * L.n * (long long)(L.T - 1);
  double Q = 0.0;
  if (twomu_num != 0) {
    const double twomu = __ddiv_rn(__ll2double_rn(twomu_num), __ll2double_rn(od));
    const double num = __dsub_rn(__dadd_rn(__ull2double_rn(L.base[W_IJ]), wJ), __dmul_rn(gam, nullsum));
    Q = __ddiv_rn(num, twomu);
  }
  L.base[W_Q] = (ull)__double_as_longlong(Q);
}

// Device address of the scratch array, looked up once per device (with that
// device current) and cached.  The cached address belongs to the device's
// primary context; after cudaDeviceReset on that device it is stale, and
// this entry point must not be called there again in the same process.
ull* scratch_address(int dev, std::string& err) {
  static std::mutex mu;
  static std::vector<ull*> cache;
  std::lock_guard<std::mutex> lock(mu);
  if ((size_t)dev >= cache.size()) cache.resize(dev + 1, nullptr);
  if (!cache[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return nullptr;
    }
    cache[dev] = static_cast<ull*>(p);
  }
  return cache[dev];
}

unsigned grid_of(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 8) g = 152 * 8;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

extern "C" int mslice_modularity_noalloc(const mslice_csr* slices, int32_t T, const int32_t* labels,
                                         int64_t gamma_num, int64_t gamma_den, int64_t omega_num, int64_t omega_den,
                                         void* stream, double* Q_out) {
  auto fail = [](int code, const std::string& m) {
    mslice::set_last_error(m);
    return code;
  };
  const int64_t lim = (int64_t)1 << 31;
  if (!slices || T < 1 || !Q_out) return fail(MSLICE_EINVAL, "need T >= 1 snapshots and an output");
  if (gamma_den < 1 || gamma_den > lim || gamma_num < 1 || gamma_num > lim || omega_den < 1 || omega_den > lim ||
      omega_num < 0 || omega_num > lim)
    return fail(MSLICE_EINVAL, "gamma must be a rational > 0 and omega a rational >= 0");
  const int64_t n = slices[0].n;
  if (n < 0 || n > INT32_MAX || n * (int64_t)T > INT32_MAX) return fail(MSLICE_EINVAL, "n*T must fit in int32");
  for (int32_t s = 0; s < T; ++s)
    if (slices[s].n != n || (n > 0 && !slices[s].indptr)) return fail(MSLICE_EINVAL, "snapshots must share n");
  const int64_t N = n * (int64_t)T;
  const size_t words = words_needed(N, T);
  if (words > NOALLOC_WORDS)
    return fail(MSLICE_EINVAL, "n*T*T = " + std::to_string(N * (int64_t)T) +
                                   " exceeds the allocation-free scratch (at most about 4.1M (node, snapshot) x T "
                                   "words, 32 MiB)");
  if (N > 0 && !labels) return fail(MSLICE_EINVAL, "null labels");
  // A CUDA error left pending by the caller's earlier work is reported, not
  // consumed: the launch checks below would otherwise clear it and blame this
  // call for it.
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess)
    return fail(MSLICE_ECUDA, std::string("a CUDA error from earlier work is pending: ") + cudaGetErrorString(e));
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(MSLICE_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  std::string err;
  ull* base = scratch_address(dev, err);
  if (!base) return fail(MSLICE_ECUDA, err);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Layout L;
  L.n = n;
  L.N = N;
  L.T = T;
  L.base = base;
  L.ip = reinterpret_cast<const int64_t* const*>(base + W_PTRS);
  L.ix = reinterpret_cast<const int32_t* const*>(base + W_PTRS + T);
  L.wt = reinterpret_cast<const int32_t* const*>(base + W_PTRS + 2 * T);
  L.S = base + W_PTRS + 3 * T;
  L.two_m = reinterpret_cast<long long*>(base + W_PTRS + 5 * T);
  L.sig = reinterpret_cast<long long*>(base + W_PTRS + 6 * T);
  // everything that accumulates starts from zero on every call
  k_na_clear<<<grid_of((int64_t)words), 256, 0, st>>>(base, words);
  std::vector<const void*> ptrs(3 * (size_t)T);
  for (int32_t s = 0; s < T; ++s) {
    ptrs[s] = slices[s].indptr;
    ptrs[T + s] = slices[s].indices;
    ptrs[2 * T + s] = slices[s].weights;
  }
  e = cudaMemcpyAsync(base + W_PTRS, ptrs.data(), ptrs.size() * sizeof(void*), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail(MSLICE_ECUDA, std::string("copy: ") + cudaGetErrorString(e));
  if (N > 0) {
    k_na_check<<<grid_of(N), 256, 0, st>>>(L, labels);
    k_na_sums<<<grid_of(N), 256, 0, st>>>(L, labels);
    k_na_squares<<<grid_of(N * T), 256, 0, st>>>(L);
  }
  k_na_q<<<1, 1, 0, st>>>(L, gamma_num, gamma_den, omega_num, omega_den);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(MSLICE_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  ull out[2];
  e = cudaMemcpyAsync(out, base, 2 * sizeof(ull), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(MSLICE_ECUDA, std::string("readback: ") + cudaGetErrorString(e));
  if (out[0] & 1u)
    return fail(MSLICE_EINVAL,
                "malformed snapshot (row pointers, missing arrays, unsorted or repeated columns, self-loop, weight "
                "< 1) or label out of [0, N)");
  if (out[0] & 2u) return fail(MSLICE_EOVERFLOW, "the 2^61 bounds of the library conventions do not hold");
  double Q;
  std::memcpy(&Q, &out[1], sizeof(double));
  *Q_out = Q;
  mslice::set_last_error("");
  return MSLICE_OK;
}
