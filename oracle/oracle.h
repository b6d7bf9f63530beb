/*
 * Multislice-Leiden ORACLE -- test infrastructure only.
 *
 * A plain, slow, single-threaded CPU statement of what the GPU library
 * computes.  Only the test-suite, the smoke check and the benchmark's CPU
 * baseline may load it; the product library never links or calls it, and the
 * two share no code.
 *
 * Method (paper: "Accelerating Dynamic Graph Clustering on GPU Architectures
 * with cuGraph", Sec. 3.2):
 *   - objective: multislice modularity Q_MS (Eq. multislice-modularity) with
 *     ordinal coupling omega between copies of a node in adjacent snapshots
 *     and the per-slice null model gamma*k_is*k_js/2m_s; or its general form
 *     (omega^(sr) per pair of slices, ordinal or categorical, and gamma^(s)
 *     per slice: orc_general); or the global null model (plain modularity of
 *     the supra-graph);
 *   - supra-graph: Eq. supra-adjacency (A^(t) blocks on the diagonal, omega*I
 *     on the first off-diagonals);
 *   - optimiser: Leiden (local moving, refinement, aggregation), as named in
 *     Sec. 3.2, run under a deterministic synchronous schedule with exact
 *     integer move keys (the paper fixes no schedule or arithmetic; the
 *     readings are listed in the design notes of the repository).
 *
 * Parity status: Q (orc_modularity) is pinned by the tests to the spectral
 * form Tr(C^T M C)/2mu (Sec. 3.2), to Newman-Girvan modularity at T=1
 * (Eq. modularity) and to the omega=0 per-slice decomposition.  The move key
 * (orc_move_key) is pinned to exact rational differences of Q_MS.  The
 * general form and the global model are pinned the same ways (exact-rational
 * dense forms, networkx on the supra-graph, exact key differences, brute
 * force, reduction to the uniform model).  The
 * partition returned by orc_leiden is "parity unpinned" by the paper (it
 * prints no partitions); it is checked against invariants only: brute-force
 * optimum bound, local optimality at convergence, connected communities,
 * clique recovery, large-omega persistence and omega=0 decoupling.
 */
#ifndef MSLICE_ORACLE_H
#define MSLICE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes (same meaning as the library's, numbered independently). */
#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_EOVERFLOW (-3)

/* Null models.  MULTISLICE: Q_MS's per-slice term gamma*k_is*k_js/2m_s.
 * GLOBAL: plain modularity (Eq. modularity) of the supra-adjacency, coupling
 * edges included in the strengths and in 2mu, one null term for the whole
 * supra-graph (the model cuGraph's Leiden optimises when it is handed the
 * supra-graph, Sec. 3.2). */
#define ORC_NULL_MULTISLICE 0
#define ORC_NULL_GLOBAL 1
/* CPM: the temporal Constant Potts Model (Sec. 3.2): snapshot s's null term
 * is gamma_s per ordered pair of its nodes; Q_CPM = (I + omega*J -
 * sum_s gamma_s sum_c n_{c,s}^2) / 2mu. */
#define ORC_NULL_CPM 2

/* Coupling patterns: ORDINAL couples (i,s) with (i,s+1); CATEGORICAL couples
 * (i,s) with (i,r) for every r != s. */
#define ORC_ORDINAL 0
#define ORC_CATEGORICAL 1

/* General form of Eq. multislice-modularity (nullable everywhere it is
 * taken; NULL = ordinal coupling with the uniform omega and gamma).
 * omega_num (nullable): numerators of omega^(sr) over the call's omega_den,
 *   each in [0, 2^31]; ORDINAL: T-1 entries, entry s for the pair (s, s+1);
 *   CATEGORICAL: a T*T row-major matrix, symmetric with a zero diagonal.
 *   NULL: every coupled pair has the call's omega_num.
 * gamma_num, gamma_den (both or neither): T per-slice resolutions gamma^(s);
 *   not with the global null model (one null term has one resolution). */
typedef struct {
  int32_t coupling;
  int32_t pad_;
  const int64_t* omega_num;
  const int64_t* gamma_num;
  const int64_t* gamma_den;
} orc_general;

/* One snapshot: symmetric CSR, sorted columns, no self-loops, weights >= 1. */
typedef struct {
  int64_t n;
  const int64_t* indptr;   /* n+1 */
  const int32_t* indices;  /* indptr[n] */
  const int32_t* weights;  /* indptr[n] */
} orc_csr;

typedef struct {
  int32_t n_iterations; /* outer Leiden passes (paper Sec. 4: two passes) */
  int32_t K;            /* sub-rounds per round */
  int32_t max_rounds;   /* local-moving rounds per level */
  int32_t max_levels;   /* aggregation levels */
  uint64_t seed;
  /* step-level debugging: when stop_level >= 0, iteration 0 stops at that
   * level after stop_stage (1 = local moving, 2 = refinement, 3 = aggregation)
   * and writes the raw level labels (not canonical) to labels_out:
   * stage 1 -> local-moving labels, stage 2 -> refined labels,
   * stage 3 -> initial labels of the next level.  stop_rounds > 0 caps the
   * local-moving rounds of that level; stop_rounds < 0 runs none there (the
   * level keeps its initial labels, so refinement can be driven directly). */
  int32_t stop_level;
  int32_t stop_stage;
  int32_t stop_rounds;
  int32_t null_model;  /* ORC_NULL_MULTISLICE (default), ORC_NULL_GLOBAL or ORC_NULL_CPM */
  int32_t pad_;
  /* refinement randomness theta = theta_num/theta_den (Traag et al.'s
   * randomised refinement); theta_num = 0 (default): the greedy limit */
  int64_t theta_num;
  int64_t theta_den;
} orc_opts;

/* The randomised refinement's fixed-point weight 2^40 exp(-d / (2^63 div /
 * theta_den)) for d (lo, hi) and div = 2M * theta_num (lo, hi): test access
 * to the integer recipe the refinement uses. */
uint64_t orc_exp_weight(uint64_t d_lo, uint64_t d_hi, uint64_t div_lo, uint64_t div_hi, uint64_t theta_den);

typedef struct {
  int32_t iterations;      /* outer iterations run */
  int32_t levels;          /* levels in the last iteration */
  int64_t lm_rounds;       /* local-moving rounds, all levels and iterations */
  int64_t lm_edges;        /* sum over those rounds of the level's directed entries */
  int64_t lm_moves;        /* node moves applied during local moving */
  int64_t last_level0_moves; /* moves in the level-0 local moving of the last iteration */
  int64_t out_n;           /* length of labels_out written */
  int64_t next_n;          /* debug stage 3: nodes of the aggregated level */
  int64_t next_nnz;        /* debug stage 3: directed entries of the aggregated level */
  uint64_t next_checksum;  /* debug stage 3: order-free checksum of the aggregated level */
  int32_t stop_reason;     /* last iteration's level loop ended because: 1 every community
                              was a single node, 2 max_levels, 3 refinement merged nothing */
  int32_t pad_;
} orc_stats;

void orc_default_opts(orc_opts* o);

/* Full multislice Leiden; labels_out holds N = n*T canonical labels
 * (renumbered by first occurrence), Q_out the FP64 Q_MS with the true gamma.
 * init_labels (nullable) must lie in [0, N). */
int orc_leiden(const orc_csr* slices, int32_t T, int64_t gamma_num, int64_t gamma_den,
               int64_t omega_num, int64_t omega_den, const orc_opts* o, const orc_general* gen,
               const int32_t* init_labels, int32_t* labels_out, int64_t labels_cap, double* Q_out,
               orc_stats* st);

/* Q of a level-0 labelling (labels in [0, N)) under null_model: Q_MS, or the
 * supra-graph's plain modularity. */
int orc_modularity(const orc_csr* slices, int32_t T, const int32_t* labels, int64_t gamma_num,
                   int64_t gamma_den, int64_t omega_num, int64_t omega_den, int32_t null_model,
                   const orc_general* gen, double* Q_out);

/* Exact integer key G(v, c) of the level-0 supra-node v for community c under
 * `labels` (c = -1 means an empty community).  Written as a signed 128-bit
 * integer in out[0] (low) / out[1] (high). */
int orc_move_key(const orc_csr* slices, int32_t T, const int32_t* labels, int64_t gamma_num,
                 int64_t gamma_den, int64_t omega_num, int64_t omega_den, int32_t null_model,
                 const orc_general* gen, int64_t v, int64_t c, uint64_t out[2]);

/* Quantised null coefficients Lambda_s, as 128-bit (lo, hi) pairs, and 2m_s. */
int orc_lambda(const orc_csr* slices, int32_t T, int64_t gamma_num, int64_t gamma_den,
               uint64_t* lambda_lohi, int64_t* two_m);

/* Number of level-0 supra-nodes that have a single move (to a neighbouring
 * community, or to an empty one when not alone) with a strictly larger key
 * than staying. */
int orc_count_improving(const orc_csr* slices, int32_t T, const int32_t* labels, int64_t gamma_num,
                        int64_t gamma_den, int64_t omega_num, int64_t omega_den, int32_t null_model,
                        const orc_general* gen, int64_t* count);

/* One aggregation step (Leiden, Sec. 3.2; the aggregation reading: new ids
 * rank the refined labels ascending, self-loops are dropped, slice strengths
 * are summed, and a new node starts in the smallest new id of its
 * local-moving community), exposed for the tests.  The caller gives the
 * level-0 local-moving partition P and a refinement R of it (labels in
 * [0, N), every R-community inside one P-community; EINVAL otherwise).
 * Written: N, nnz (directed entries) and ns (slice entries) always; the
 * arrays only when rowptr is non-null and the capacities suffice (EINVAL
 * when they do not).  Rows list columns ascending with W in units of 1/od;
 * slice lists are ascending (snapshot, strength) pairs. */
typedef struct {
  int64_t N, nnz, ns;              /* sizes of the aggregated level (out) */
  int64_t cap_N, cap_nnz, cap_ns;  /* capacities of the arrays below (in) */
  int64_t* rowptr;                 /* N + 1 */
  int32_t* col;                    /* nnz */
  int64_t* W;                      /* nnz */
  int64_t* sptr;                   /* N + 1 */
  int32_t* sidx;                   /* ns */
  int64_t* sval;                   /* ns */
  int32_t* init_labels;            /* N: initial labels of the new level */
  int32_t* node_map;               /* level-0 node count: new id of every level-0 node */
} orc_level_out;

int orc_aggregate(const orc_csr* slices, int32_t T, int64_t omega_num, int64_t omega_den, int32_t null_model,
                  const orc_general* gen, const int32_t* P, const int32_t* R, orc_level_out* out);

/* Key G(x, c) at the level that aggregating (P, R) produces, under the
 * labels labels1 of that level (c = -1: an empty community), as a signed
 * 128-bit integer in out[0] (low) / out[1] (high). */
int orc_level_key(const orc_csr* slices, int32_t T, int64_t gamma_num, int64_t gamma_den, int64_t omega_num,
                  int64_t omega_den, int32_t null_model, const orc_general* gen, const int32_t* P,
                  const int32_t* R, const int32_t* labels1, int64_t x, int64_t c, uint64_t out[2]);

/* The counter-based hash used to draw vertex classes (SplitMix64 finaliser). */
uint64_t orc_mix64(uint64_t x);

#ifdef __cplusplus
}
#endif
#endif
