/*
 * mslice -- multislice-modularity Leiden on one GPU (sm_103a), C ABI.
 *
 * The library optimises multislice modularity Q_MS (Mucha et al.), the
 * objective of Eq. multislice-modularity in "Accelerating Dynamic Graph
 * Clustering on GPU Architectures with cuGraph" (Sec. 3.2), on the
 * supra-graph of T snapshots (Eq. supra-adjacency): intra-snapshot edges with
 * the per-snapshot null model gamma*k_is*k_js/2m_s, plus ordinal coupling
 * edges of weight omega between the copies of a node in adjacent snapshots.
 * The optimiser is Leiden (local moving, refinement, aggregation; Sec. 3.2)
 * under a deterministic synchronous schedule with exact integer move keys,
 * so that repeated runs, and any other implementation of the same schedule,
 * give bit-identical partitions.
 *
 * Conventions shared by every entry point:
 *   - Status: 0 = MSLICE_OK, negative = error (below).  On error nothing is
 *     written to the outputs; mslice_last_error() describes the failure.
 *   - Snapshots: symmetric CSR over the same n nodes, int64 row pointers
 *     starting at 0, int32 column indices sorted strictly ascending in every
 *     row, no self-loops, int32 weights >= 1, entry (j,i) present with the
 *     same weight as (i,j).  Violations give MSLICE_EINVAL.
 *   - Supra-node of node i in snapshot s (0-based): v = s*n + i; N = n*T.
 *   - Rationals gamma = gamma_num/gamma_den > 0 and omega = omega_num/omega_den
 *     >= 0, each numerator and denominator in [0, 2^31] (denominators >= 1).
 *   - Overflow guard (MSLICE_EOVERFLOW): omega_den*sum_s 2m_s
 *     + 2*omega_num*n*(T-1) < 2^61 and gamma*omega_den*sum_s 2m_s < 2^61,
 *     where 2m_s is the sum of snapshot s's weights over both directions.
 *   - Ownership: inputs belong to the caller and are read only during the
 *     call.  A handle owns all device memory it allocates.  Outputs are
 *     written to caller buffers (host memory unless MSLICE_DEVICE_PTRS).
 *   - Streams: work runs on the stream given at build time (NULL: a stream of
 *     the handle's own that waits for the legacy default stream's work, as
 *     that stream would); calls return after that stream is synchronised.
 *     Calls on one handle must not overlap; different handles are
 *     independent.
 */
#ifndef MSLICE_H
#define MSLICE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MSLICE_OK 0
#define MSLICE_EINVAL (-1)    /* malformed input, bad rational, bad label */
#define MSLICE_ENOMEM (-2)    /* device allocation failed */
#define MSLICE_EOVERFLOW (-3) /* the 128-bit key bound above does not hold */
#define MSLICE_ECUDA (-4)     /* a CUDA runtime call failed */
#define MSLICE_ETIMEOUT (-5)  /* a bounded device wait gave up */

/* Input/output pointers are device pointers (build: the snapshot arrays;
 * leiden/modularity: labels). */
#define MSLICE_DEVICE_PTRS 1
/* leiden: time the local-moving decision kernels of every level-0 round with
 * CUDA events on the handle's stream, one span per sub-round (fills ms_decide
 * / decide_launches / decide_bytes; adds a little host overhead). */
#define MSLICE_PROFILE 2
/* leiden / batch run: choose the degree cuts between the decision kernels'
 * tiers by timing the candidates on round 0 of level 0 (decisions only, so
 * the result is unchanged); the cuts used are returned in mslice_stats. */
#define MSLICE_AUTOTUNE 4
/* leiden / batch run / modularity_ex / server: optimise and report the plain
 * modularity (Eq. modularity) of the supra-graph of Eq. supra-adjacency
 * instead of Q_MS -- the objective cuGraph's Leiden optimises when it is
 * handed the supra-graph (Sec. 3.2).  Coupling edges then count in the
 * strengths (k'_v = k_v + omega * coupling edges of v) and a single null term
 * gamma k'_u k'_v / 2mu covers the whole supra-graph (of one instance).  The
 * resolution is quantised once: Lambda' = floor(gamma 2^64 / 2M'), 2M' =
 * omega_den * 2mu, and the exact key's null scale is 1 instead of omega_den.
 * Bound: gamma * 2M' < 2^61 (EOVERFLOW otherwise).  Not available to
 * mslice_modularity_noalloc. */
#define MSLICE_NULL_GLOBAL 8
/* leiden / batch run / modularity / server: the temporal Constant Potts Model
 * (Sec. 3.2 names it as a quality function the supra-graph strategy takes):
 * snapshot s's null term is gamma^(s) per ordered pair of its nodes instead
 * of gamma k_is k_js / 2m_s, so resolution is a density threshold.  Reported
 * Q_CPM = (I + omega J - sum_s gamma^(s) sum_c n_{c,s}^2) / 2mu.  Keys use
 * Lambda_s = floor(gamma^(s) 2^64) with node counts as strengths; bound:
 * gamma^(s) * omega_den * n * N < 2^61 (EOVERFLOW).  Not together with
 * MSLICE_NULL_GLOBAL (EINVAL); not available to mslice_modularity_noalloc. */
#define MSLICE_NULL_CPM 16

typedef struct {
  int64_t n;              /* nodes of the snapshot (equal for all snapshots) */
  const int64_t* indptr;  /* n+1 row pointers */
  const int32_t* indices; /* indptr[n] column indices */
  const int32_t* weights; /* indptr[n] weights >= 1 */
} mslice_csr;

/* Coupling between snapshots (Eq. multislice-modularity, omega^(sr)):
 * ORDINAL links (i,s) and (i,s+1) (Eq. supra-adjacency); CATEGORICAL links
 * (i,s) and (i,r) for every r != s (needs T*T < 2^31).  The weights are
 * omega (uniform), or per pair through mslice_general. */
typedef enum { MSLICE_ORDINAL = 0, MSLICE_CATEGORICAL = 1 } mslice_coupling;

/* The general form of Eq. multislice-modularity for one solve (host arrays,
 * read during the call; every pointer nullable).
 *   omega_num: numerators of omega^(sr) over the call's omega_den, each in
 *              [0, 2^31], one per coupling slot of the handle's pattern:
 *              ORDINAL T-1 slots, slot s for the pair (s, s+1); CATEGORICAL
 *              a T*T row-major matrix, symmetric with a zero diagonal.  A
 *              pair of weight 0 is not an edge.  NULL: omega for every pair.
 *   gamma_num, gamma_den: both or neither; T per-snapshot resolutions
 *              gamma^(s), each a rational in (0, 2^31]/[1, 2^31].  NULL:
 *              gamma for every snapshot.  Not with MSLICE_NULL_GLOBAL (one
 *              null term, one resolution).
 * Keys use Lambda_s = floor(gamma^(s) 2^64 / 2m_s); the bound becomes
 * omega_den*sum 2m_s + n*sum_{s,r} omega_num^(sr) < 2^61 and
 * gamma^(s)*omega_den*sum 2m_s < 2^61 for every s (EOVERFLOW). */
typedef struct {
  const int64_t* omega_num;
  const int64_t* gamma_num;
  const int64_t* gamma_den;
} mslice_general;

typedef struct mslice_graph* mslice_handle;

typedef struct {
  int32_t n_iterations; /* outer Leiden passes; default 2 (the paper caps runs
                           at two optimisation passes, Sec. 4) */
  int32_t K;            /* synchronous sub-rounds per local-moving round, 1..64; default 4 */
  int32_t max_rounds;   /* local-moving rounds per level; default 100 */
  int32_t max_levels;   /* aggregation levels; default 32 */
  uint64_t seed;        /* seed of the counter-based class hash; default 0 */
  int64_t gamma_num, gamma_den; /* resolution; default 1/1 */
  int64_t omega_num, omega_den; /* coupling; default 1/1 (overrides the build value) */
  int32_t flags;        /* MSLICE_DEVICE_PTRS: init/labels_out are device pointers;
                           MSLICE_PROFILE, MSLICE_AUTOTUNE, MSLICE_NULL_GLOBAL: above */
  /* Step-level debugging (the library's own tests compare it stage by stage):
   * when stop_level >= 0 the first iteration stops at that level after
   * stop_stage (1 local moving, 2 refinement, 3 aggregation) and labels_out
   * receives the raw labels of that level (stage 3: the initial labels of the
   * next level); stop_rounds > 0 caps the local-moving rounds of that level,
   * stop_rounds < 0 runs none.  Set stop_level = -1 for normal use. */
  int32_t stop_level;
  int32_t stop_stage;
  int32_t stop_rounds;
  /* Degree cuts between the five decision tiers (4-lane groups, 8-lane
   * groups, a warp, a block, a block with a global table): tier t takes
   * degrees in (tier_cuts[t-1], tier_cuts[t]].  All zero (the default): 16,
   * 32, 256, 1024.  Otherwise 0 <= c0 <= 16, c0 <= c1 <= 32, c1 <= c2 <= 256,
   * c2 <= c3 <= 1024.  They change the speed only, never the result. */
  int32_t tier_cuts[4];
  /* Randomised refinement (Traag et al.): theta = theta_num/theta_den > 0
   * makes an eligible singleton join a target X with probability
   * proportional to exp(dQ_X / theta) among the targets with dQ_X >= 0,
   * staying weighing exp(0); theta_num = 0 (the default) is the greedy
   * limit (largest positive gain).  The weights are 2^40 exp(-(Gmax - G) /
   * (2^63 2M theta)) by a fixed integer recipe (2M = omega_den * 2mu) and the
   * draw comes from the schedule's hash, so results stay reproducible bit for
   * bit.  0 <= theta_num <= 2^31, 1 <= theta_den <= 2^31. */
  int64_t theta_num, theta_den;
} mslice_opts;

typedef struct {
  int32_t iterations;        /* outer iterations run */
  int32_t levels;            /* levels of the last iteration */
  int64_t lm_rounds;         /* local-moving rounds over all levels/iterations */
  int64_t lm_edges;          /* sum over those rounds of the level's directed entries */
  int64_t lm_moves;          /* node moves applied by local moving */
  int64_t last_level0_moves; /* moves of the last iteration's level-0 local moving */
  int64_t out_n;             /* labels written */
  int64_t next_n, next_nnz;  /* debug stage 3: size of the aggregated level */
  uint64_t next_checksum;    /* debug stage 3: order-free checksum of that level */
  int32_t stop_reason;       /* 1 all singletons, 2 max_levels, 3 no shrink */
  int32_t pad_;
  int64_t kernel_launches;   /* kernels this call launched */
  double ms_total;           /* device time of the call (CUDA events) */
  double ms_local_move;      /* ... of which local moving */
  double ms_refine;          /* ... refinement */
  double ms_aggregate;       /* ... aggregation */
  double ms_modularity;      /* ... Q evaluation */
  double ms_decide;          /* MSLICE_PROFILE: summed durations of the level-0 decision sub-rounds */
  int64_t decide_launches;   /* MSLICE_PROFILE: number of those sub-rounds (all degree tiers of one) */
  int64_t decide_bytes;      /* MSLICE_PROFILE: algorithmic bytes those launches move, per round
                                12 B per directed entry (column, weight, neighbour label) and 40 B
                                per node (row pointer, own label, strength, decision, the own
                                community's 16-byte table slot); probes of other candidate
                                communities are not counted, so this is a lower bound */
  int32_t tier_cuts[4];      /* degree cuts the decision tiers used (chosen by MSLICE_AUTOTUNE) */
  double ms_capped;          /* local-moving device time of the levels that stopped at max_rounds with
                                nodes still moving (the synchronous schedule cycling), part of ms_local_move */
  int64_t capped_levels;     /* number of those levels */
  int64_t capped_rounds;     /* their local-moving rounds */
  int64_t host_launches;     /* launch calls the host made for this call (kernels launched one by one, and
                                graph launches, each counting once however many kernels the graph runs) */
} mslice_stats;

/* Defaults above; stop_level = -1. */
void mslice_default_opts(mslice_opts* o);

/* Builds the level-0 supra-graph (Eq. supra-adjacency) on the device from T
 * snapshots: concatenates the snapshot rows at offset s*n, inserts the
 * ordinal coupling entries, computes k_v and 2m_s, and validates the input.
 * The coupling entries are stored as flags, so omega given here is only the
 * default for later calls.  slices[] are host arrays (copied to the device);
 * *out receives the handle.  Errors: EINVAL (T < 1, n mismatch, malformed
 * CSR, bad omega), ENOMEM, ECUDA. */
int mslice_build(const mslice_csr* slices, int32_t T, mslice_coupling cpl, int64_t omega_num,
                 int64_t omega_den, mslice_handle* out);

/* As mslice_build; flags = MSLICE_DEVICE_PTRS when the snapshot arrays are
 * device pointers; stream = cudaStream_t the handle runs on (NULL: default). */
int mslice_build_ex(const mslice_csr* slices, int32_t T, mslice_coupling cpl, int64_t omega_num,
                    int64_t omega_den, int32_t flags, void* stream, mslice_handle* out);

/* Multislice Leiden with default options and the given gamma, omega,
 * max_levels and seed.  labels_out: host int32[N], canonical labels (first
 * occurrence order over supra-nodes).  Q_out: FP64 Q_MS of those labels with
 * the exact gamma (Eq. multislice-modularity).  Errors: EINVAL, EOVERFLOW,
 * ENOMEM, ECUDA. */
int mslice_leiden(mslice_handle h, int64_t gamma_num, int64_t gamma_den, int64_t omega_num,
                  int64_t omega_den, int32_t max_levels, uint64_t seed, int32_t* labels_out,
                  double* Q_out);

/* Full-option Leiden.  init_labels (nullable) = warm start, int32[N] in
 * [0, N) (checkpoint/resume: a previous result).  labels_out has room for N
 * labels.  st (nullable) receives counters and phase times. */
int mslice_leiden_ex(mslice_handle h, const mslice_opts* o, const int32_t* init_labels,
                     int32_t* labels_out, double* Q_out, mslice_stats* st);

/* As mslice_leiden_ex with the general form gen (nullable: the uniform
 * model).  Q_out is Q_MS with the tables' omega^(sr) and gamma^(s).  Errors:
 * EINVAL (bad tables, or per-snapshot gamma with MSLICE_NULL_GLOBAL), as
 * mslice_leiden_ex otherwise. */
int mslice_leiden_general(mslice_handle h, const mslice_opts* o, const mslice_general* gen,
                          const int32_t* init_labels, int32_t* labels_out, double* Q_out, mslice_stats* st);

/* Q_MS (Eq. multislice-modularity, ordinal coupling) of int32[N] labels in
 * [0, N) (host pointer).  Errors: EINVAL, EOVERFLOW, ENOMEM, ECUDA. */
int mslice_modularity(mslice_handle h, const int32_t* labels, int64_t gamma_num, int64_t gamma_den,
                      int64_t omega_num, int64_t omega_den, double* Q_out);

/* As mslice_modularity; flags = MSLICE_DEVICE_PTRS for a device pointer,
 * MSLICE_NULL_GLOBAL for the supra-graph's plain modularity instead of Q_MS. */
int mslice_modularity_ex(mslice_handle h, const int32_t* labels, int64_t gamma_num, int64_t gamma_den,
                         int64_t omega_num, int64_t omega_den, int32_t flags, double* Q_out);

/* Q of int32[N] labels in [0, N) under the general form gen (nullable); o
 * gives gamma, omega and flags (MSLICE_DEVICE_PTRS, MSLICE_NULL_GLOBAL; o
 * nullable: the defaults).  Errors as mslice_modularity_ex. */
int mslice_modularity_general(mslice_handle h, const int32_t* labels, const mslice_opts* o,
                              const mslice_general* gen, double* Q_out);

/* Q_MS of int32[N] labels in [0, N), read straight from device snapshot
 * arrays, for callers that cannot allocate device memory: plug-ins held to a
 * memory budget by their host application, and services that reserve all
 * device memory up front and hand out slices of it.  The paper has no
 * counterpart; it is the evaluation of mslice_modularity (same integer sums
 * and FP64 order) without a handle.
 *   slices: T snapshots whose indptr/indices/weights are DEVICE pointers, with
 *           the mslice_csr conventions checked on the device (row pointers,
 *           index and weight arrays present when a snapshot has entries,
 *           columns in range, strictly ascending, no self-loops, weights
 *           >= 1), except symmetry, which is not checked;
 *   labels: device int32[N], N = n*T;  stream: cudaStream_t (NULL: default);
 *   Q_out:  host double.
 * No device memory is allocated: all scratch lives in one 32 MiB array inside
 * the library (4 + 6*T + N*T 8-byte words must fit in 4,194,304 words, else
 * MSLICE_EINVAL), which every GPU that loads the library keeps until the
 * process exits.  The first call on each device looks up that array's device
 * address (with the device current) and caches it for the process; after a
 * cudaDeviceReset of that device the cached address is stale and the call
 * must not be used there again.  Every call clears the scratch it uses, but
 * all calls share the one array, so calls that overlap on a GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * The call copies a pointer table from host memory and synchronises the
 * stream before it returns, so it must not be issued on a stream that is
 * being captured into a CUDA graph.  A CUDA error already pending from the
 * caller's earlier work makes it fail with MSLICE_ECUDA and is left pending.
 * Errors: EINVAL, EOVERFLOW, ECUDA. */
int mslice_modularity_noalloc(const mslice_csr* slices, int32_t T, const int32_t* labels, int64_t gamma_num,
                              int64_t gamma_den, int64_t omega_num, int64_t omega_den, void* stream,
                              double* Q_out);

/* ---- Windowed optimisation of long snapshot sequences ----
 *
 * Sec. 4 names windowed optimisation for sequences whose supra-graph is too
 * long to solve at once (its 7,375-snapshot case) and gives no procedure.
 * This entry point solves windows of W snapshots one after another and
 * stitches their labels:
 *   - windows start at 0, stride, 2*stride, ..., the last start clamped to
 *     T - W (every window holds W snapshots; one window [0, T) when T <= W);
 *   - window 0 starts from singletons; window k is warm-started: its local
 *     snapshot j takes the previous window's labels of local snapshot
 *     min(j + e, W - 1), e = start_k - start_{k-1} (the serving rule);
 *   - stitching: window k's communities in order of first occurrence; one
 *     whose first supra-node lies in the overlap (its first W - e snapshots)
 *     continues that supra-node's stitched label unless an earlier community
 *     of the window took it; any other gets a fresh label; window k's labels
 *     overwrite its snapshots' stitched labels;
 *   - labels_out (host int32[n*T]) gets the stitched labels renumbered by
 *     first occurrence.
 * slices: T snapshots (host arrays, or device arrays with MSLICE_DEVICE_PTRS
 * in o->flags); o: gamma, omega, schedule and null-model flags (nullable:
 * defaults; stop_level must be -1); stream: cudaStream_t (NULL: a private
 * one); Q_windows (nullable): the Q of each window's solve, at most q_cap of
 * them; *n_windows (nullable): the number of windows; st (nullable):
 * counters and phase times summed over the windows.  Every window is a full
 * solve of n*W supra-nodes; the whole sequence is never built at once.
 * Errors: EINVAL (T < 1, W < 1, stride outside [1, W) when T > W, n*W above
 * 2^31 - 1, malformed snapshots, bad options), EOVERFLOW (a window outside
 * the key bound), ENOMEM, ECUDA. */
int mslice_leiden_windowed(const mslice_csr* slices, int32_t T, int32_t W, int32_t stride, const mslice_opts* o,
                           void* stream, int32_t* labels_out, double* Q_windows, int32_t q_cap,
                           int32_t* n_windows, mslice_stats* st);

/* ---- Batches: many (graph, gamma, omega) solves in one pass ----
 *
 * Leiden's partition depends on the resolution gamma and the coupling omega
 * (Sec. 3.2), so callers sweep them, and small graphs leave the GPU bound by
 * launch overhead (Sec. 4).  A batch solves B independent instances together:
 * their supra-graphs are laid out one after another as the diagonal blocks of
 * one graph, every kernel launch of the level loop covers all instances, and
 * each instance keeps its own gamma, omega, snapshot masses and class hash
 * (computed on instance-local node ids).  No edge joins two instances and an
 * instance that has converged (all singletons, nothing merged, labels
 * unchanged over an iteration) is frozen while the others continue, so every
 * instance's labels and Q are bit-identical to those of mslice_leiden_ex on
 * that graph alone with the same options, gamma and omega.
 *
 * The batch keeps a device copy of the concatenated graphs (rebuilt by
 * mslice_batch_run only when the list of graphs changed) and solver scratch
 * for all instances: about the sum of the graphs' handle memory plus
 * ~120 bytes per supra-node.  The same graph may be added several times (a
 * gamma/omega sweep). */
typedef struct mslice_batch_s* mslice_batch;

/* Empty batch on stream (cudaStream_t; NULL = default).  flags =
 * MSLICE_DEVICE_PTRS when init_labels / labels_out of the calls below are
 * device pointers.  Errors: EINVAL, ENOMEM, ECUDA. */
int mslice_batch_create(int32_t flags, void* stream, mslice_batch* out);

/* Appends the instance (graph g, gamma, omega).  g must stay alive until the
 * next mslice_batch_run returns.  init_labels (nullable): warm start,
 * int32[N_g] in [0, N_g), copied during the call.  *index_out (nullable)
 * receives the instance index (add order, from 0).  Errors: EINVAL (bad
 * rationals or labels, more than 2^31 - 1 supra-nodes in the batch),
 * EOVERFLOW (the bound of the conventions for this graph, gamma and omega). */
int mslice_batch_add(mslice_batch b, mslice_handle g, int64_t gamma_num, int64_t gamma_den, int64_t omega_num,
                     int64_t omega_den, const int32_t* init_labels, int32_t* index_out);

/* As mslice_batch_add with the general form gen (nullable) for this
 * instance; its tables are copied during the call.  Instances of one batch
 * may mix coupling patterns, tables and uniform parameters. */
int mslice_batch_add_general(mslice_batch b, mslice_handle g, int64_t gamma_num, int64_t gamma_den,
                             int64_t omega_num, int64_t omega_den, const mslice_general* gen,
                             const int32_t* init_labels, int32_t* index_out);

/* Solves every instance.  o: schedule options shared by all instances
 * (n_iterations, K, max_rounds, max_levels, seed; MSLICE_PROFILE,
 * MSLICE_AUTOTUNE and MSLICE_NULL_GLOBAL honoured, the last for every
 * instance); its gamma/omega/init fields are not used and stop_level must be
 * -1.  st (nullable): counters summed over the batch and phase times of the
 * pass.  Errors: EINVAL (empty batch, bad options), EOVERFLOW (an instance
 * outside the global model's bound), ENOMEM, ECUDA. */
int mslice_batch_run(mslice_batch b, const mslice_opts* o, mslice_stats* st);

/* Results of the last run.  i in [0, B): labels_out gets instance i's N_i
 * canonical labels (numbered from 0 within the instance) and *Q_out its Q_MS
 * (its supra-graph modularity when run with MSLICE_NULL_GLOBAL);
 * i = -1: labels_out gets all instances' labels one after another (sum N_i
 * entries, instance i at offsets[i] of mslice_batch_info) and Q_out B values.
 * Errors: EINVAL (bad index, not run since the last add/clear). */
int mslice_batch_results(mslice_batch b, int32_t i, int32_t* labels_out, double* Q_out);

/* Instances B, total supra-nodes N, and offsets (nullable, B+1 entries):
 * first supra-node of every instance in the concatenated labels. */
int mslice_batch_info(mslice_batch b, int32_t* B, int64_t* N, int64_t* offsets);

/* Removes every instance; device memory is kept for the next runs. */
int mslice_batch_clear(mslice_batch b);

/* Kernels launched by this batch's runs; -1 for NULL. */
int64_t mslice_batch_kernel_launches(mslice_batch b);

/* Releases the batch and its device memory (NULL is ignored). */
void mslice_batch_free(mslice_batch b);

/* ---- Serving: sliding windows of live temporal graphs ----
 *
 * The supra-graph grows with the number of snapshots, and Sec. 4 names
 * windowed optimisation as the way to bound it for long streams.  A server
 * keeps, per live graph, a ring of the last W slices on the device with the
 * partition of the current window.  Each submitted snapshot is one request:
 *   - the window advances: the new slice is appended and, when W slices are
 *     held already, the oldest is evicted;
 *   - the solve is warm-started: supra-node (j, i) of the new window (slice j,
 *     node i) starts with the label that (j + e, i) had in the previous
 *     window's result, where e = 1 if a slice was evicted (else 0), capped at
 *     the previous newest slice, so the new slice's node i starts with its
 *     label in the previous newest slice; the first snapshot of a graph starts
 *     from singletons;
 *   - the result is mslice_leiden_ex on the window's slices with these initial
 *     labels and the server's gamma, omega and schedule options, bit for bit.
 * Requests are served by n_slots workers, each with its own CUDA stream.  A
 * free worker admits the queued requests, in arrival order, whose estimated
 * device footprint fits in what is left of the memory budget (at most one
 * in-flight request per graph, up to max_batch requests and max_batch_nodes
 * supra-nodes, never overtaking a request that does not fit) and solves them
 * as one batch; requests that arrive while
 * other workers' batches run are admitted as workers and memory free up, so
 * their work overlaps on the device.  A request larger than the whole budget
 * runs alone once nothing else is in flight. */
typedef struct mslice_server_s* mslice_server;

typedef struct {
  int32_t window;      /* W: slices per live graph; default 8 */
  int32_t n_slots;     /* concurrent workers (CUDA streams); default 2 */
  int32_t max_batch;   /* requests per batch; default 64 */
  int32_t pad_;
  int64_t max_batch_nodes; /* supra-nodes per batch; default 2^21, which keeps a batch's randomly
                              accessed state (~50 B per supra-node) in L2; a larger request runs
                              alone */
  int64_t hbm_budget;  /* bytes of device memory admitted work may use; 0 (default): 80% of the free
                          memory when the server is created */
  int64_t gamma_num, gamma_den, omega_num, omega_den; /* default 1/1, 1/1 */
  mslice_opts solve;   /* schedule (n_iterations, K, max_rounds, max_levels, seed, tier_cuts) and
                          the MSLICE_NULL_GLOBAL flag; defaults as mslice_default_opts;
                          gamma/omega/stop fields and the other flags are not used */
} mslice_server_opts;

/* Per-request record, times in seconds since the server was created. */
typedef struct {
  int32_t status;       /* MSLICE_OK or the request's error code */
  int32_t slices;       /* slices in the window that was solved */
  int64_t N;            /* supra-nodes of that window (labels written) */
  double Q;             /* Q_MS of the result (the supra-graph's modularity under MSLICE_NULL_GLOBAL) */
  double t_submit, t_admit, t_done;
  int32_t batch_size;   /* requests solved together with it (itself included) */
  int32_t slot;         /* worker that solved it */
  int64_t footprint;    /* estimated device bytes admitted for it */
  double t_batch_start, t_batch_end; /* the batch's solve on the device (host clock) */
} mslice_request_info;

void mslice_server_default_opts(mslice_server_opts* o);

/* Starts the workers on the current device.  Errors: EINVAL, ENOMEM, ECUDA. */
int mslice_server_create(const mslice_server_opts* o, mslice_server* out);

/* Registers a live graph of n nodes per slice; *graph_id receives its id. */
int mslice_server_add_graph(mslice_server s, int64_t n, int32_t* graph_id);

/* Queues the next snapshot of graph_id (host CSR with the mslice_csr
 * conventions, copied during the call) and returns at once; *request_id
 * receives the request's id.  A malformed snapshot fails its request
 * (EINVAL at wait) and leaves the window unchanged.  Errors: EINVAL. */
int mslice_server_submit(mslice_server s, int32_t graph_id, const mslice_csr* slice, int64_t* request_id);

/* Blocks until the request is done, then writes its N window labels
 * (canonical, host int32[N]; nullable) and its record (nullable) and forgets
 * the request.  Returns the request's status; EINVAL for an unknown id. */
int mslice_server_wait(mslice_server s, int64_t request_id, int32_t* labels_out, mslice_request_info* info);

/* Checkpoint and resume of a live graph's window: the snapshots it holds and
 * the labels of its last result, which is all the state the next request
 * reads.  The graph must be idle (no request of it queued or in flight), else
 * MSLICE_EINVAL.
 * window_info: *slices = snapshots held (0..W); nnz (nullable, one entry per
 *   snapshot held, oldest first) = their stored entries.
 * window_read: k in [0, slices): snapshot k (oldest = 0) into host indptr
 *   (n+1), indices and weights (nnz[k] each); k = -1: the window's labels into
 *   host int32[n * slices].
 * window_restore: replaces the window with nslices (1..W) host snapshots,
 *   oldest first, and their labels (host int32[n * nslices], values in
 *   [0, n * nslices)), as a previous result would have left them; the next
 *   submitted snapshot is solved from them exactly as if the server had
 *   produced them.  The snapshots are validated like a build; on any error
 *   the window is left as it was.  Errors: EINVAL, ENOMEM, ECUDA. */
int mslice_server_window_info(mslice_server s, int32_t graph_id, int32_t* slices, int64_t* nnz);
int mslice_server_window_read(mslice_server s, int32_t graph_id, int32_t k, int64_t* indptr, int32_t* indices,
                              int32_t* weights, int32_t* labels);
int mslice_server_window_restore(mslice_server s, int32_t graph_id, const mslice_csr* slices, int32_t nslices,
                                 const int32_t* labels);

/* Finishes the queued requests, stops the workers and releases the server
 * and its device memory (NULL is ignored). */
void mslice_server_free(mslice_server s);

/* Sizes of a built handle: N supra-nodes, T, n, stored level-0 entries
 * (intra + coupling, both directions). Any pointer may be NULL. */
int mslice_info(mslice_handle h, int64_t* N, int32_t* T, int64_t* n, int64_t* nnz);

/* Kernels launched on this handle since it was built (build included);
 * -1 for a NULL handle. */
int64_t mslice_kernel_launches(mslice_handle h);

/* Releases the handle and its device memory (NULL is ignored). */
void mslice_free(mslice_handle h);

/* Message of the calling thread's last error ("" if none). */
const char* mslice_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
