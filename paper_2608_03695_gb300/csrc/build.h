// Level-0 supra-graph held by a handle, and its builder.
#pragma once
#include <vector>

#include "internal.h"

namespace mslice {

// One instance of a batch (a single solve is a batch of one).
struct InstInfo {
  int64_t n = 0;     // nodes per snapshot
  int64_t noff = 0;  // first supra-node
  int32_t T = 0;     // snapshots
  int32_t soff = 0;  // first global snapshot
  int32_t coupling = 0;  // MSLICE_ORDINAL or MSLICE_CATEGORICAL
  int64_t cwoff = 0;     // first slot of the instance's omega^(sr) numerators in a batch's table
};

// Slots of an instance's table of omega^(sr) numerators: ordinal, one per
// adjacent pair (slot min(s, r)); categorical, a T x T matrix (slot s*T + r).
inline int64_t coupling_slots(int32_t coupling, int32_t T) {
  return coupling == 0 ? (T > 1 ? T - 1 : 0) : (int64_t)T * T;
}

// Directed coupling entries of an instance.
inline int64_t coupling_entries(int32_t coupling, int64_t n, int32_t T) {
  if (T < 2) return 0;
  return coupling == 0 ? 2 * n * (int64_t)(T - 1) : n * (int64_t)T * (T - 1);
}

struct SupraGraph {
  int32_t T = 0;        // snapshots over all instances
  int64_t n = 0, N = 0; // n: nodes per snapshot of a single instance
  int64_t nnz = 0;        // stored entries (intra both directions + coupling flags)
  int64_t nnz_intra = 0;  // intra-snapshot entries
  int32_t coupling = 0;   // single graph: its coupling pattern (batches: per instance)
  int64_t ncw = 0;        // slots of omega^(sr) numerators over all instances
  int64_t* rowptr = nullptr;  // N+1
  // {col, w}: w >= 1 an intra-snapshot weight; w <= 0 a coupling entry whose
  // omega^(sr) numerator sits in slot -w-1 of the solve's coupling table
  int2* adj = nullptr;
  int64_t* k = nullptr;       // intra-snapshot strength of every supra-node
  int64_t* two_m = nullptr;   // T snapshot masses
  std::vector<int64_t> two_m_host;
  // batches (B > 1): instances laid out one after another
  int32_t B = 1;
  std::vector<InstInfo> inst;    // host
  int32_t* slice0 = nullptr;     // global snapshot of every supra-node
  int32_t* inst0 = nullptr;      // instance of every supra-node
  int32_t* inst_off0 = nullptr;  // first supra-node of every instance (B+1)
  int32_t* slice_inst = nullptr; // instance of every global snapshot
  Workspace mem;                 // owns the arrays above
};

// Lays the supra-graphs of several instances out one after another (node ids,
// column indices and snapshot ids shifted), with the per-node instance and
// snapshot maps the batched kernels read.  parts are only read.
void concat_instances(Ctx& c, const std::vector<const SupraGraph*>& parts, SupraGraph& out);

void build_supra(Ctx& c, const std::vector<const int64_t*>& indptr, const std::vector<const int32_t*>& indices,
                 const std::vector<const int32_t*>& weights, const std::vector<int64_t>& nnz, int64_t n,
                 SupraGraph& g, int32_t coupling = 0);

// Lambda_s = floor(gn * 2^64 / (gd * 2m_s)) (0 for an edgeless snapshot), with
// the gamma of the snapshot's instance (gn/gd: B entries each, device).
void compute_lambda(Ctx& c, const SupraGraph& g, const long long* gn, const long long* gd, u128* lam);

}  // namespace mslice
