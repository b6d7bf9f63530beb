// Per-call solver state and the phases of one Leiden solve.
#pragma once
#include <vector>

#include "build.h"
#include "decide.cuh"
#include "level.h"

namespace mslice {

struct SolveParams {
  long long gn = 1, gd = 1, on = 1, od = 1;
  int32_t K = 4, max_rounds = 100, max_levels = 32, n_iterations = 2;
  uint64_t seed = 0;
  TierCuts cuts;          // degree cuts between the decision tiers
  bool autotune = false;  // choose the cuts by timing round 0 of level 0
  bool global_null = false;  // plain modularity of the supra-graph instead of Q_MS
  bool cpm = false;          // the temporal Constant Potts Model instead of Q_MS
  long long theta_num = 0, theta_den = 1;  // randomised refinement (theta_num = 0: greedy)
};

// Null models of a solve (the check_bounds argument).
enum NullModel { NULL_MULTISLICE = 0, NULL_SUPRA_GLOBAL = 1, NULL_CPM = 2 };

// CUDA-event phase timing: events recorded on the context's stream.
struct PhaseClock {
  Ctx& c;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> spans;
  explicit PhaseClock(Ctx& cc) : c(cc) {}
  ~PhaseClock();
  cudaEvent_t begin();
  void end(int phase, cudaEvent_t b);
  void totals(double out[5]);  // total ms per phase
};

// Randomised refinement's divisor of one instance, div = 2M * theta_num
// (1 <= div < 2^92), with a fixed-point reciprocal R = floor(2^k / div),
// k = 62 + bitlen(div), so 2^62 < R <= 2^63 (an estimate only: every
// quotient is corrected to the exact floor).
struct RandDiv {
  u128 div;
  unsigned long long R;
  int k;
  int pad_;
};

struct Solver {
  Ctx* c = nullptr;
  const SupraGraph* G0 = nullptr;
  SolveParams p;
  u128* lam = nullptr;  // Lambda of every null slice (Tn entries)
  int32_t Tn = 1;       // null slices: the snapshots (Q_MS) or one per instance (global model)
  int64_t* kn = nullptr;  // global model: level-0 strengths k' = od*k + (coupling strength)
  // general coupling: the omega^(sr) numerators of every instance by slot
  // (nullptr when every instance has a uniform omega), per-snapshot gamma
  // (num, den pairs; nullptr when every instance has one gamma), and host
  // sums: coupling strength of one node of every snapshot, n * the sum of
  // those per instance (the coupling part of 2mu, in units of 1/od), and the
  // level-0 coupling entries that are edges
  long long* cw_d = nullptr;
  long long* gs_d = nullptr;
  RandDiv* rdiv = nullptr;  // randomised refinement: 2M * theta_num of every instance (2M = od * 2mu)
  ull* gwts = nullptr;      // randomised refinement: weights beside gkeys/gvals
  std::vector<long long> cstr_h, csum_h, gs_h;
  std::vector<uint8_t> has_cw_h, has_gs_h;
  int64_t cpl_edges = 0;
  int64_t N0 = 0;

  // node-indexed scratch, sized for level 0 (every level is smaller)
  int32_t* target = nullptr;
  int32_t* size = nullptr;
  int32_t* tmp32a = nullptr;
  int32_t* tmp32b = nullptr;
  int32_t* freelist = nullptr;
  uint8_t* tier = nullptr;
  uint8_t* cls = nullptr;       // refinement class of every node of the level
  int32_t* lists = nullptr;     // K rows of N0 entries: nodes bucketed by class and tier
  int32_t* cursors = nullptr;   // bucket sizes per (class, tier) segment (device)
  uint16_t* bseg = nullptr;     // segment of every node in the round being bucketed
  int32_t* bcounts = nullptr;   // per segment and chunk of nodes: counts, then offsets
  int32_t* counters = nullptr;  // [0] moves in round (low), [1] moves (high), [2] moves to empty in sub-round
  ull* sig_used = nullptr;      // Sigma slots taken since its last rebuild
  int32_t empty_grid = 0;       // co-resident grid of the empty-community pass
  int32_t* empty_blk = nullptr;
  int32_t* inst_cnt = nullptr;  // per-instance counts of the empty-community pass

  // batch: B independent instances (1 for a single solve) and their
  // resolution / coupling rationals (host copies; device copies below)
  int32_t B = 1;
  std::vector<long long> gn_h, gd_h, on_h, od_h;
  long long *gn_d = nullptr, *gd_d = nullptr, *on_d = nullptr, *od_d = nullptr;
  int32_t* inst_active = nullptr;  // per instance: 1 while not converged (nullptr: all active)
  int32_t* lm_active = nullptr;    // per instance: still moving in this level's local moving
  int32_t* inst_moved = nullptr;   // per instance: moved in the current round
  int32_t* round_dev = nullptr;    // the round the device-side round loop is at
  long long* loop_acc = nullptr;   // device-side round loop: rounds run, moves, moves of the last round
  int32_t* wqueue = nullptr;       // work counters of the decision kernels, one per degree tier
  int64_t* goff = nullptr;      // global-tier table offsets
  int32_t* gkeys = nullptr;
  long long* gvals = nullptr;
  int64_t gcap = 0;

  // community slice sums Sigma_{c,s} and sub-community sums K_{R,s} of the
  // current level (dense or hashed, see configure_stores)
  SigStore sig{};
  SigStore kr{};
  HashView sig_h{}, kr_h{};
  std::vector<uint64_t> region_h;  // slot offsets of the hash regions (one per null slice, + 1)
  int64_t region_T = -1;           // null slices the regions were laid out for (-1: none yet)
  long long* sig_d = nullptr;
  long long* kr_d = nullptr;
  int64_t dense_cap = 0;
  // refinement state
  int32_t* R = nullptr;
  int32_t* sizeR = nullptr;
  long long* Wc = nullptr;
  long long* Wout = nullptr;
  long long* Wsel = nullptr;
  ull* rhs = nullptr;  // 2 words per node
  uint8_t* elig = nullptr;
  uint8_t* wc = nullptr;

  int32_t tier_off[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int32_t tier_cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};

  // statistics
  int64_t lm_rounds = 0, lm_edges = 0, lm_moves = 0;
};

void solver_alloc(Solver& S);

// Dense Sigma/K tables are used while labels x T stays within this many
// entries per table (32 MB, so the table stays resident in L2 next to the
// labels); larger levels use the hash, whose footprint follows the number of
// (node, snapshot) entries instead.  The environment variable
// MSLICE_DENSE_LIMIT overrides it; 0 forces the hashed tables.
constexpr int64_t DENSE_LIMIT = (int64_t)1 << 22;

// Points sig/kr at dense rows (allocated on demand) or the hash tables for a
// level of N nodes.  Needs the null slices (setup_null_model) first.
void configure_stores(Solver& S, int64_t N);
void clear_store(Solver& S, const SigStore& st);

// Degree tiers, global-tier scratch; once per level.
void prepare_level(Solver& S, const Level& L);

struct MoveOut {
  int64_t rounds = 0, moves = 0;
  bool capped = false;  // stopped at max_rounds while nodes were still moving
};
// Local moving of `labels` (N entries, values in [0, N)) at level lvl.
MoveOut local_move(Solver& S, const Level& L, int32_t* labels, int it, int lvl, int max_rounds);

// Refinement of the local-moving partition P; result in S.R.
void refine(Solver& S, const Level& L, const int32_t* P, int it, int lvl);

// Number of distinct values in x[0, N) (values in [0, N)).
int64_t count_distinct(Solver& S, const int32_t* x, int64_t N);

// Aggregation; returns false when the refined partition has N communities.
bool aggregate(Solver& S, const Level& L, const int32_t* P, Level& next, const std::string& slot,
               int32_t* next_labels, int32_t* node_of0, int64_t* checksum);

// Rebuilds Sigma_{c,s} of `labels` at level L.
void sigma_rebuild(Solver& S, const Level& L, const int32_t* labels);

// Canonical labels (first occurrence order within each instance) of x[0, N)
// into out.
void canonicalise(Solver& S, const int32_t* x, int32_t* out, int64_t N);

// Q_MS of level-0 labels with the true gamma, one value per instance (host
// array of B doubles).
void modularity(Solver& S, const int32_t* labels0, double* Q);

// Order-free checksum of a level (debug stage 3).
uint64_t level_checksum(Solver& S, const Level& L);

LevelDev level0_view(const SupraGraph& G, long long on, long long od);
// The level-0 view of a solve: batch maps and per-instance omega included.
LevelDev level0_view(const SupraGraph& G, const Solver& S);

// Per-instance resolution and coupling of a solve: gamma = gn/gd and omega =
// on/od, or the general form of Eq. multislice-modularity when the tables are
// given: omega^(sr) = cw[slot]/od per coupling slot (coupling_slots()) and
// gamma^(s) = gsn[s]/gsd[s] per snapshot.
struct InstParams {
  long long gn = 1, gd = 1, on = 1, od = 1;
  std::vector<long long> cw;        // empty: on for every coupled pair
  std::vector<long long> gsn, gsd;  // empty: gn/gd for every snapshot
};

// Numerator of omega^(sr) over od for an instance with this coupling pattern
// and T snapshots (0 for uncoupled pairs).
long long pair_num(const InstParams& j, int32_t coupling, int32_t T, int32_t s, int32_t r);

// Fails with MSLICE_EOVERFLOW unless the 128-bit move keys of a graph with n
// nodes per snapshot, snapshot masses two_m[0..T) and this coupling pattern
// stay in range for the instance's gamma and omega under null model nm:
// 2M' = od * sum 2m_s + n * sum_{s,r} omega_num^(sr) < 2^61, and
// gamma_s od sum 2m_s < 2^61 for every s (Q_MS); gamma 2M' < 2^61 (global
// model, whose strengths include the coupling); gamma_s od n N < 2^61 (CPM,
// whose null sums count nodes).
void check_bounds(int64_t n, int32_t T, int32_t coupling, const int64_t* two_m, const InstParams& j, int nm);

// The null model of a solve: S.Tn, the quantised coefficients S.lam (one per
// snapshot, or one per instance from 2M' for the global model) and, for the
// global model, the level-0 strengths S.kn.  Needs S.G0, S.N0, S.p and the
// instances (set_instances).
void setup_null_model(Solver& S);

// Fails with MSLICE_EINVAL unless every level-0 label d[v] (device) lies in
// [0, size of v's instance).
void check_label_ranges(Ctx& c, const SupraGraph& G, const int32_t* d);

// Output of run_leiden.
struct RunOut {
  std::vector<double> Q;  // per instance
  int64_t out_n = 0;      // labels written (N, or a debug level's size)
  int64_t levels = 0, iterations = 0, stop_reason = 0, last_level0_moves = 0;
  int64_t next_n = 0, next_nnz = 0;
  uint64_t next_checksum = 0;
  double ms[5] = {0, 0, 0, 0, 0};  // total, local moving, refinement, aggregation, Q
  double ms_capped = 0;            // local moving of the levels that stopped at max_rounds still moving
  int64_t capped_levels = 0, capped_rounds = 0;
};

// Per-instance rationals of a solve into S (host and device copies); B =
// jobs.size() must equal the instance count of the graph.
void set_instances(Ctx& c, Solver& S, const std::vector<InstParams>& jobs);

// Leiden over the instances of G (each with its InstParams).  init (device,
// nullable): level-0 labels, numbered from 0 within each instance.  out
// (device, N): canonical labels, numbered from 0 within each instance.  Debug stops
// (single instance) write a level's raw labels instead.
void run_leiden(Ctx& c, const SupraGraph& G, const std::vector<InstParams>& jobs, const SolveParams& p,
                int stop_level, int stop_stage, int stop_rounds, const int32_t* init, int32_t* out, Solver& S,
                RunOut& ro);

}  // namespace mslice
