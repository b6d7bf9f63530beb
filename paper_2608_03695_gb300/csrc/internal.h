// Host-side internals of the mslice library: error handling, device
// workspace, launch bookkeeping and the kernel entry wrappers shared between
// translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "common.cuh"

namespace mslice {

struct Error {
  int code;
  std::string msg;
};

[[noreturn]] void fail(int code, const std::string& msg);
// Message returned by mslice_last_error() in the calling thread.
void set_last_error(const std::string& msg);
// Raises the release threshold of the device's default memory pool once per
// process, so freed stream-ordered allocations are reused, not returned.
void keep_pool_memory();
void check_cuda(cudaError_t e, const char* what);

// Growable named device buffers owned by a handle.  Contents are undefined
// after a grow; callers clear what they need.
class Workspace {
 public:
  cudaStream_t stream = nullptr;  // allocations are ordered on this stream
  ~Workspace();
  void* get_bytes(const std::string& name, size_t bytes);
  template <class T>
  T* get(const std::string& name, size_t count) {
    return static_cast<T*>(get_bytes(name, (count ? count : 1) * sizeof(T)));
  }
  void release(const std::string& name);
  void release_all();
  size_t bytes_held() const;

 private:
  std::map<std::string, std::pair<void*, size_t>> bufs_;
};

// Side streams on which the degree tiers of one decision sub-round run
// concurrently (forked from and joined back to the context's stream by
// events).  Owned by a handle, batch or server worker.
struct StreamFan {
  static constexpr int kSide = 4;
  cudaStream_t side[kSide] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kSide] = {};
  void create();   // high priority for the streams of the heaviest tiers
  void destroy();
};

struct Ctx {
  cudaStream_t stream = nullptr;
  StreamFan* fan = nullptr;      // nullptr: tiers run one after another
  bool capturing = false;        // launches are being captured into a graph
  Workspace* ws = nullptr;
  unsigned* d_status = nullptr;  // device error bits
  int64_t launches = 0;
  int64_t host_launches = 0;     // launch calls the host made (a graph launch counts once)
  bool profile = false;          // event-time the decision kernels
  // MSLICE_TRACE: every launch is bracketed by CUDA events (per-kernel table
  // printed at the end of a solve)
  std::vector<std::pair<const void*, std::pair<cudaEvent_t, cudaEvent_t>>>* trace = nullptr;
  int64_t prof_bytes = 0;        // algorithmic bytes of the timed kernels
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* prof_spans = nullptr;
  void* pinned = nullptr;        // small pinned host buffer for readbacks (>= 4 KB)
};

void trace_begin(Ctx& c, const void* k, cudaEvent_t* e0);
void trace_end(Ctx& c, const void* k, cudaEvent_t e0);

template <class... KArgs, class... Args>
inline void launch(Ctx& c, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, Args&&... args) {
  if (grid.x == 0 || grid.y == 0 || grid.z == 0) return;
  cudaEvent_t e0 = nullptr;
  if (c.trace) trace_begin(c, (const void*)k, &e0);
  k<<<grid, block, smem, c.stream>>>(std::forward<Args>(args)...);
  c.launches++;
  if (!c.capturing) c.host_launches++;
  check_cuda(cudaGetLastError(), "kernel launch");
  if (c.trace) trace_end(c, (const void*)k, e0);
}

// Orders cooperative launches device-wide: a kernel with grid-wide barriers
// starts only after the previous one (from any stream or thread of the
// process) has finished, so two such grids never hold part of the SMs each
// while waiting for the rest.  Every other kernel of the library runs to
// completion without waiting on other blocks, so a cooperative grid always
// becomes fully resident.
class CoopOrder {
 public:
  explicit CoopOrder(cudaStream_t s);  // waits for the previous cooperative kernel
  ~CoopOrder();                        // marks this stream's point as the new one
  CoopOrder(const CoopOrder&) = delete;
  CoopOrder& operator=(const CoopOrder&) = delete;

 private:
  cudaStream_t s_;
  int dev_ = 0;
};

// Cooperative launch (grid-wide barriers); the grid must be co-resident.
template <class... KArgs, class... Args>
inline void launch_coop(Ctx& c, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, Args... args) {
  void* argv[] = {(void*)&args...};
  cudaEvent_t e0 = nullptr;
  if (c.trace) trace_begin(c, (const void*)k, &e0);
  if (c.capturing) {
    // ordered as a whole by the graph's launch
    check_cuda(cudaLaunchCooperativeKernel((const void*)k, grid, block, argv, smem, c.stream), "cooperative launch");
  } else {
    CoopOrder order(c.stream);
    check_cuda(cudaLaunchCooperativeKernel((const void*)k, grid, block, argv, smem, c.stream), "cooperative launch");
    c.host_launches++;
  }
  c.launches++;
  if (c.trace) trace_end(c, (const void*)k, e0);
}

// launch() on another stream of the same context.
template <class... KArgs, class... Args>
inline void launch_on(Ctx& c, cudaStream_t s, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, Args&&... args) {
  struct Restore {
    Ctx& c;
    cudaStream_t keep;
    ~Restore() { c.stream = keep; }
  } restore{c, c.stream};
  c.stream = s;
  launch(c, k, grid, block, smem, std::forward<Args>(args)...);
}

inline unsigned grid_for(int64_t n, int per_block) {
  int64_t g = (n + per_block - 1) / per_block;
  return (unsigned)(g < 1 ? 0 : g);
}

// Size of every handle's pinned staging buffer (Ctx::pinned).
constexpr size_t PINNED_BYTES = 4096;

// Reads `bytes` (at most PINNED_BYTES) from device memory into the pinned
// buffer and synchronises.
void* readback(Ctx& c, const void* dptr, size_t bytes);
void sync(Ctx& c);
// Synchronises and throws if the device status word holds an error bit.
void check_status(Ctx& c, const char* where);

// ---- primitives (primitives.cu) ----
// out[i] = sum_{j<i} in[j] (int64 accumulation); *d_total (device, nullable)
// receives the full sum.  in and out may alias.  With `cond` (device,
// nullable) the kernels do nothing when *cond == 0, so a scan can sit in a
// stream behind work whose outcome decides whether it is needed.
void scan_excl(Ctx& c, const int32_t* in, int64_t* out, int64_t n, int64_t* d_total,
               const int32_t* cond = nullptr);
void scan_excl(Ctx& c, const int64_t* in, int64_t* out, int64_t n, int64_t* d_total,
               const int32_t* cond = nullptr);
void scan_excl(Ctx& c, const int32_t* in, int32_t* out, int64_t n, int32_t* d_total,
               const int32_t* cond = nullptr);

void fill_i32(Ctx& c, int32_t* p, int32_t v, int64_t n);
void fill_i64(Ctx& c, int64_t* p, int64_t v, int64_t n);
void iota_i32(Ctx& c, int32_t* p, int64_t n);

}  // namespace mslice
