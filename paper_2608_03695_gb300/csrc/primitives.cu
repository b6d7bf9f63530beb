// Device-wide primitives: exclusive scan (reduce-then-scan over 4096-element
// tiles), fills.
#include "internal.h"

namespace mslice {

namespace {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <class T>
__device__ __forceinline__ T block_excl_scan(T x, T* sm, T& total) {
  // sm: at least 32 entries
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T incl = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) sm[w] = incl;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    T v = lane < nw ? sm[lane] : T(0);
    T vi = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, vi, d);
      if (lane >= d) vi += y;
    }
    if (lane < nw) sm[lane] = vi - v;
    if (lane == nw - 1) sm[32] = vi;
  }
  __syncthreads();
  T r = incl - x + sm[w];
  total = sm[32];
  __syncthreads();
  return r;
}

template <class In, class Acc>
__global__ void k_tile_reduce(const In* in, int64_t n, Acc* bsum, const int32_t* cond) {
  if (cond && *cond == 0) return;
  __shared__ Acc sm[33];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  Acc t = 0;
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    int64_t i = base + (int64_t)j * SCAN_THREADS + threadIdx.x;
    if (i < n) t += (Acc)in[i];
  }
  Acc tot;
  block_excl_scan<Acc>(t, sm, tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

template <class In, class Out, class Acc>
__global__ void k_tile_scan(const In* in, Out* out, int64_t n, const Acc* boff, Out* d_total, const int32_t* cond) {
  if (cond && *cond == 0) return;
  __shared__ Acc sm[33];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  Acc v[SCAN_ITEMS];
  Acc t = 0;
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    int64_t i = base + j;
    v[j] = (i < n) ? (Acc)in[i] : Acc(0);
    t += v[j];
  }
  Acc tot;
  Acc p = block_excl_scan<Acc>(t, sm, tot) + (boff ? boff[blockIdx.x] : Acc(0));
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    int64_t i = base + j;
    if (i < n) out[i] = (Out)p;
    p += v[j];
  }
  if (d_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
    *d_total = (Out)((boff ? boff[blockIdx.x] : Acc(0)) + tot);
}

template <class In, class Out, class Acc>
void scan_impl(Ctx& c, const In* in, Out* out, int64_t n, Out* d_total, int depth, const int32_t* cond) {
  if (n <= 0) {
    if (d_total) check_cuda(cudaMemsetAsync(d_total, 0, sizeof(Out), c.stream), "memset");
    return;
  }
  const unsigned nb = grid_for(n, SCAN_TILE);
  if (nb == 1) {
    launch(c, k_tile_scan<In, Out, Acc>, dim3(1), dim3(SCAN_THREADS), 0, in, out, n, (const Acc*)nullptr, d_total,
           cond);
    return;
  }
  Acc* bsum = c.ws->get<Acc>("scan_bsum" + std::to_string(depth), nb);
  launch(c, k_tile_reduce<In, Acc>, dim3(nb), dim3(SCAN_THREADS), 0, in, n, bsum, cond);
  scan_impl<Acc, Acc, Acc>(c, bsum, bsum, (int64_t)nb, (Acc*)nullptr, depth + 1, cond);
  launch(c, k_tile_scan<In, Out, Acc>, dim3(nb), dim3(SCAN_THREADS), 0, in, out, n, (const Acc*)bsum, d_total, cond);
}

__global__ void k_fill_i32(int32_t* p, int32_t v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}
__global__ void k_fill_i64(int64_t* p, int64_t v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}
__global__ void k_iota_i32(int32_t* p, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = (int32_t)i;
}

unsigned grid_stride(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

void scan_excl(Ctx& c, const int32_t* in, int64_t* out, int64_t n, int64_t* d_total, const int32_t* cond) {
  scan_impl<int32_t, int64_t, long long>(c, in, out, n, d_total, 0, cond);
}
void scan_excl(Ctx& c, const int64_t* in, int64_t* out, int64_t n, int64_t* d_total, const int32_t* cond) {
  scan_impl<int64_t, int64_t, long long>(c, in, out, n, d_total, 0, cond);
}
void scan_excl(Ctx& c, const int32_t* in, int32_t* out, int64_t n, int32_t* d_total, const int32_t* cond) {
  scan_impl<int32_t, int32_t, long long>(c, in, out, n, d_total, 0, cond);
}

void fill_i32(Ctx& c, int32_t* p, int32_t v, int64_t n) {
  if (n > 0) launch(c, k_fill_i32, dim3(grid_stride(n)), dim3(256), 0, p, v, n);
}
void fill_i64(Ctx& c, int64_t* p, int64_t v, int64_t n) {
  if (n > 0) launch(c, k_fill_i64, dim3(grid_stride(n)), dim3(256), 0, p, v, n);
}
void iota_i32(Ctx& c, int32_t* p, int64_t n) {
  if (n > 0) launch(c, k_iota_i32, dim3(grid_stride(n)), dim3(256), 0, p, n);
}

}  // namespace mslice
