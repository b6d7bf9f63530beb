// Level-0 supra-graph held by a handle, and its builder.
#pragma once
#include <vector>

#include "internal.h"

namespace mslice {

struct SupraGraph {
  int32_t T = 0;
  int64_t n = 0, N = 0;
  int64_t nnz = 0;        // stored entries (intra both directions + coupling flags)
  int64_t nnz_intra = 0;  // intra-snapshot entries
  int64_t* rowptr = nullptr;  // N+1
  int2* adj = nullptr;        // {col, w}; w = 0 marks a coupling entry
  int64_t* k = nullptr;       // intra-snapshot strength of every supra-node
  int64_t* two_m = nullptr;   // T snapshot masses
  std::vector<int64_t> two_m_host;
  Workspace mem;              // owns the arrays above
};

void build_supra(Ctx& c, const std::vector<const int64_t*>& indptr, const std::vector<const int32_t*>& indices,
                 const std::vector<const int32_t*>& weights, const std::vector<int64_t>& nnz, int64_t n,
                 SupraGraph& g);

// Lambda_s = floor(gn * 2^64 / (gd * 2m_s)) (0 for an edgeless snapshot).
void compute_lambda(Ctx& c, const SupraGraph& g, long long gn, long long gd, u128* lam);

}  // namespace mslice
