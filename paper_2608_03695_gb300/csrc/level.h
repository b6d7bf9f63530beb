// A level of the optimisation as the kernels see it.  Level 0 is the
// supra-graph itself ({col, w} entries, coupling flagged by w = 0, one
// snapshot per node); aggregated levels hold int64 weights already scaled to
// units of 1/omega_den and per-node lists of (snapshot, strength).
//
// A level may hold several independent instances (a batch): disjoint blocks
// of node ids, each with its own omega, gamma (through Lambda of its
// snapshots) and snapshot range.  No edge joins two instances, so no
// community ever spans two, and every per-node rule below reads only the
// node's own instance.
#pragma once
#include "internal.h"

namespace mslice {

struct LevelDev {
  int32_t N = 0;
  int32_t n = 1;  // level 0, single instance: nodes per snapshot
  int32_t is0 = 1;
  const int64_t* rowptr = nullptr;
  const int2* adj0 = nullptr;   // level 0
  const long long* cw = nullptr;  // level 0: omega^(sr) numerators by slot (nullptr: omega uniform)
  int64_t ncw = 0;
  const int64_t* k0 = nullptr;  // level 0
  const int32_t* col = nullptr; // aggregated levels
  const long long* W = nullptr;
  const int64_t* sptr = nullptr;
  const int32_t* sidx = nullptr;
  const long long* sval = nullptr;
  long long on = 1, od = 1;     // single instance
  // Null model: 0 = per-snapshot term of Q_MS; 1 = one term over the whole
  // supra-graph (plain modularity of the supra-graph).  Under 1 the
  // "snapshot" of a strength entry is the instance (one null slice each),
  // strengths are k' = od*k + on*(coupling edges) and the key's null scale is
  // 1 instead of od.
  int32_t global_null = 0;
  // batches (all nullptr for a single instance)
  const int32_t* slice0 = nullptr;    // level 0: global snapshot of every node
  const int32_t* inst = nullptr;      // instance of every node
  const int32_t* inst_off = nullptr;  // first node id of every instance at this level
  const long long* on_i = nullptr;    // omega of every instance
  const long long* od_i = nullptr;
  unsigned* chk = nullptr;            // checked builds: status word for bound violations
};

// Coupling omega = on/od of a node's instance.
struct Omega {
  long long on, od;
};

__device__ __forceinline__ int32_t node_inst(const LevelDev& g, int32_t v) { return g.inst ? g.inst[v] : 0; }

__device__ __forceinline__ Omega node_omega(const LevelDev& g, int32_t v) {
  if (g.od_i) {
    const int32_t i = node_inst(g, v);
    return Omega{g.on_i[i], g.od_i[i]};
  }
  return Omega{g.on, g.od};
}

// Scale of the key's null term: od, or 1 under the global null model (whose
// strengths are already in units of 1/od).
__device__ __forceinline__ long long null_scale(const LevelDev& g, const Omega& om) {
  return g.global_null ? 1 : om.od;
}

// Node id within its instance (the schedule's hash reads this, so a batched
// instance draws the same classes as when solved alone).
__device__ __forceinline__ uint64_t local_id(const LevelDev& g, int32_t v) {
  return g.inst_off ? (uint64_t)(v - g.inst_off[node_inst(g, v)]) : (uint64_t)v;
}

__device__ __forceinline__ int32_t node_slice0(const LevelDev& g, int32_t v) {
  return g.slice0 ? g.slice0[v] : v / g.n;
}

// Entry e of the adjacency: neighbour u and weight W in units of 1/od.
// A coupling entry weighs on (uniform omega) or its pair's numerator in the
// coupling table, and is absent when that is 0.  (om: the omega of the row's
// instance.)
__device__ __forceinline__ bool edge_at(const LevelDev& g, int64_t e, int32_t& u, long long& W, const Omega& om) {
#if MSLICE_CHECKED
  if (e < 0 || e >= g.rowptr[g.N]) {
    atomicOr(g.chk, ERR_BOUNDS);
    u = 0;
    W = 0;
    return false;
  }
  const int32_t cu = g.is0 ? g.adj0[e].x : g.col[e];
  if (cu < 0 || cu >= g.N) {
    atomicOr(g.chk, ERR_BOUNDS);
    u = 0;
    W = 0;
    return false;
  }
#endif
  if (g.is0) {
    const int2 x = __ldcs(&g.adj0[e]);
    u = x.x;
    if (x.y <= 0) {
#if MSLICE_CHECKED
      if (g.cw && (-(int64_t)x.y - 1) >= g.ncw) {
        atomicOr(g.chk, ERR_BOUNDS);
        W = 0;
        return false;
      }
#endif
      W = g.cw ? g.cw[-x.y - 1] : om.on;
      return W > 0;
    }
    W = (long long)x.y * om.od;
    return true;
  }
  u = __ldcs(&g.col[e]);
  W = __ldcs(&g.W[e]);
  return true;
}

// Snapshot-strength list of node v: entries [b, e).
__device__ __forceinline__ void slice_range(const LevelDev& g, int32_t v, int64_t& b, int64_t& e) {
  if (g.is0) {
    b = 0;
    e = g.k0[v] > 0 ? 1 : 0;
  } else {
    b = g.sptr[v];
    e = g.sptr[v + 1];
  }
}

__device__ __forceinline__ void slice_entry(const LevelDev& g, int32_t v, int64_t j, int32_t& s, long long& k) {
  if (g.is0) {
    s = node_slice0(g, v);
    k = g.k0[v];
  } else {
    s = g.sidx[j];
    k = g.sval[j];
  }
}

// Host-side level: device arrays live in the solver's workspace.
struct Level {
  LevelDev d;
  int64_t nnz = 0;       // stored entries
  int64_t nnz_eff = 0;   // entries that are edges for this omega
  int64_t ns = 0;        // snapshot-strength entries
  int32_t max_deg = 0;
};

}  // namespace mslice
