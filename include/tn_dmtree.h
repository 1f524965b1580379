/*
 * tn_dmtree.h -- C ABI of the GB300 density-matrix tree-approximation library.
 *
 * The library approximately contracts a closed tensor network with the
 * partitioned_contract algorithm (Sec. 3.2, Algorithm partitioned_contract):
 * partitions are absorbed one at a time along a linear path; each absorption
 * embeds the intermediate network into a low-rank MPS-shaped binary tree with
 * the density-matrix algorithm (Sec. 5, Algorithm density_matrix_alg, with the
 * memoised density matrices of Eq. dm_cache), and the last absorption closes
 * the network into the scalar Z.  All tensor arithmetic runs in the library's
 * own sm_103a CUDA kernels; there is no CPU fallback.
 *
 * Conventions (every entry point):
 *   - Dense tensors are row-major, last leg fastest.  A site tensor holds one
 *     leg per incident edge, in ascending edge-id order.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory of the ctx's device.  Pointer arrays themselves (T* const*)
 *     are always host arrays.
 *   - Inputs are owned by the caller and are not retained after a call
 *     returns, except that a batch launched by tn_contract_approx reads its
 *     plans and device inputs until tn_logz returns.
 *   - The ctx owns all device workspace; it grows on demand and is freed by
 *     tn_ctx_destroy.  One ctx must not be used by two host threads at once.
 *   - No C++ exception crosses the ABI.  Every call returns a tn_status;
 *     tn_last_error() gives a one-line reason for the last non-OK status.
 */
#ifndef TN_DMTREE_H
#define TN_DMTREE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TN_OK = 0,
  TN_ERR_INVALID = 1,      /* malformed graph, partition, path or argument      */
  TN_ERR_OOM = 2,          /* device or host allocation failed                  */
  TN_ERR_CUDA = 3,         /* a CUDA runtime call failed                        */
  TN_ERR_NONFINITE = 4,    /* NaN/Inf met in an instance (per-instance status)  */
  TN_ERR_NONPOSITIVE = 5,  /* final scalar <= 0, ln Z undefined (per instance)  */
  TN_ERR_TIMEOUT = 6,      /* a bounded device wait expired                     */
  TN_ERR_EIG_NOCONV = 7,   /* eigensolver hit its iteration cap                 */
  TN_ERR_UNSUPPORTED = 8   /* valid input outside what this build implements    */
} tn_status;

/* Arithmetic of the hot path.
 *   TN_PREC_FP64:      every contraction, eigensolver and scale in FP64.
 *   TN_PREC_TF32:      FP32 storage.  The density-matrix side (memoised
 *                      environments, K_v) on tcgen05 tensor cores as a
 *                      compensated 3-term TF32 split (hi*hi + hi*lo + lo*hi,
 *                      FP32 accumulation, ~FP32 accuracy); the value path
 *                      (local blocks M_v, projections U_v^T M_v) in FP32 FFMA,
 *                      whose rounding has no common sign (the tensor-core
 *                      accumulator's does, and a bias of one sign in the tree
 *                      tensors compounds over vertices and passes into ln Z).
 *                      The density matrix L_v = M_v R_v M_v^T is never formed:
 *                      R_v = C_v C_v^T (FP32 Cholesky with diagonal pivoting),
 *                      K_v = M_v C_v, and the leading eigenvectors of L_v are
 *                      the leading left singular vectors of K_v (FP32
 *                      bidiagonal SVD), so L_v's spectrum is resolved to
 *                      ~eps_32^2 of its largest eigenvalue, as an FP64
 *                      density matrix would be.  A pass whose shapes exceed
 *                      the factored kernels (dim A_v or a tree edge above
 *                      128, a rank above 64) runs in the TN_PREC_TF32_GRAM
 *                      form instead.  Root norm, log-scale and the closing
 *                      contraction in FP64.
 *   TN_PREC_TF32_FAST: L_v formed explicitly in plain TF32 (memoised
 *                      environments too) and an FP32 eigensolver; the value
 *                      path as in TN_PREC_TF32.  Loses eigen-directions below
 *                      ~1e-3 of the largest eigenvalue.
 *   TN_PREC_TF32_GRAM: as TN_PREC_TF32_FAST with the density side
 *                      compensated: L_v in FP32 resolves eigen-directions only
 *                      down to ~1e-7 of its largest eigenvalue.
 *   TN_PREC_BF16:      reserved; returns TN_ERR_UNSUPPORTED in this build.  */
enum {
  TN_PREC_FP64 = 0,
  TN_PREC_BF16 = 1,
  TN_PREC_TF32 = 2,
  TN_PREC_TF32_FAST = 3,
  TN_PREC_TF32_GRAM = 4
};

/* The tensor network graph G = (V, E) of Sec. 2.1.  Host memory, caller-owned.
 * edge_v[e] == -1 marks an open (uncontracted) edge; this build requires a
 * closed network (no open edges) because it returns ln Z.                  */
typedef struct {
  int32_t n_vertices;
  int32_t n_edges;
  const int32_t* edge_u;    /* [n_edges] endpoint vertex ids                 */
  const int32_t* edge_v;    /* [n_edges] other endpoint, or -1 (open)        */
  const int32_t* edge_dim;  /* [n_edges] mode size s, w(e) = ln s (Sec. 2.1) */
} tn_graph;

/* Inputs of Algorithm partitioned_contract (Sec. 3.2): the partition V_i, the
 * contraction path over it, the ansatz, the maximum bond size chi and the swap
 * batch size r.  Host memory, caller-owned.                                  */
typedef struct {
  int32_t chi_max;          /* maximum bond size chi (>= 1)                    */
  int32_t env_size;         /* vertices per partition when partition == NULL:
                               part i = vertices [i*env_size, (i+1)*env_size) */
  const int32_t* partition; /* [n_vertices] part id in 0..N-1, or NULL       */
  const int32_t* path;      /* [n_path] order in which parts are absorbed
                               (maximally unbalanced path), or NULL = 0..N-1  */
  int32_t n_path;
  int32_t ansatz;           /* 0 = MPS embedding tree (App. C); others: UNSUPPORTED */
  int32_t swap_batch;       /* swap batch size r of Algorithm approx_tensor_network
                               (<= 0: one density-matrix pass per contraction)  */
  int32_t planner;          /* 0: boundary absorption when every part fits it
                               (see tn_plan), else the general planner;
                               1: always the general planner                  */
} tn_plan_opts;

typedef struct tn_plan tn_plan_t;
typedef struct tn_ctx tn_ctx_t;

/* Summary of a plan (host).  Flop counts use the cost model of Sec. 2.2
 * (2 flops per multiply-add) over the contractions the plan will execute. */
typedef struct {
  int32_t n_steps;          /* contractions on the path (= parts - 1)          */
  int32_t n_dm_passes;      /* density_matrix_alg passes                       */
  int32_t max_legs;         /* most open legs of any intermediate              */
  int32_t max_bond;         /* largest untruncated tree-edge dimension         */
  int32_t max_eig_n;        /* largest density matrix order                    */
  int64_t site_elems;       /* doubles in one instance's packed site buffer    */
  double flops_env;         /* root-side memo density matrices (Eq. dm_cache)  */
  double flops_local;       /* local blocks M_v                                */
  double flops_density;     /* density matrices L_v = M_v L_u M_v^T            */
  double flops_project;     /* projector application U_v^T M_v and the root    */
  double flops_eig;         /* eigensolver (Householder + back-transform)      */
  int64_t n_eig;            /* eigensolves per instance                        */
  /* TN_PREC_TF32 (factored density matrices) replaces flops_density and
   * flops_eig by these three:                                                */
  double flops_factor;      /* Cholesky R_v = C_v C_v^T (D^3 / 3)              */
  double flops_kfactor;     /* K_v = M_v C_v                                   */
  double flops_svd;         /* Golub-Kahan bidiagonalisation of K_v + the
                               back-transformation of the r_v kept vectors    */
  int32_t n_exec_steps;     /* executed steps (tn_plan_step_query): the DM
                               passes, the closing contraction and, for
                               boundary plans, the exact first part          */
  int32_t general;          /* 1 if the general planner built the plan        */
} tn_plan_info;

/* One executed step of a plan (host).                                        */
typedef struct {
  int32_t kind;             /* 0 exact first part, 1 density-matrix pass,
                               2 closing contraction                           */
  int32_t n;                /* leaves of the pass's MPS tree (kind 1), chain
                               positions (kinds 0 and 2)                       */
  int32_t n_kt;             /* Kendall-Tau distance between the reference and
                               the constraint-tree ordering of the contraction
                               this pass belongs to (general plans, else 0)    */
  int32_t general;          /* 1 if the block of every position is a gather of
                               the tensors embedded there (general planner)   */
} tn_plan_step;

/* ---------------------------------------------------------------- planning
 * Build the host-side plan of Algorithm partitioned_contract for one graph:
 * partitions, the linear path, the edge ordering of every intermediate
 * (Sec. 4), the MPS embedding tree of each step (App. C) and the embedding
 * phi of its tensors (Algorithm tree_embedding), down to a flat list of
 * contraction / eigensolve / projection ops with their shapes.  Depends only
 * on the graph, never on tensor data (Sec. 3.2).  Host only; no CUDA call.
 * Supported: every part is a simple path of vertices whose i-th vertex
 * absorbs the i-th open leg of the intermediate and emits at most one new
 * open leg (boundary absorption as in the 2D lattice workloads).  Anything
 * else returns TN_ERR_UNSUPPORTED with a reason.
 * Returns TN_ERR_INVALID for malformed input.  *out is owned by the caller
 * and released with tn_plan_destroy.                                         */
tn_status tn_plan(const tn_graph* graph, const tn_plan_opts* opts, tn_plan_t** out);
tn_status tn_plan_destroy(tn_plan_t* plan);
tn_status tn_plan_query(const tn_plan_t* plan, tn_plan_info* info);
/* Shape of executed step `step` (0 .. n_exec_steps-1).  Every output array
 * is optional (NULL skips it) and host memory of the caller:
 *   leaves[n]: graph edge id of every leaf in tree order (kind 1; general
 *              plans; -1 otherwise), d[n] leaf dims, D[n] untruncated
 *              tree-edge dims (D[n-1] = 1), r[n-1] ranks after the pass
 *              (kind 1 only).                                                */
tn_status tn_plan_step_query(const tn_plan_t* plan, int32_t step, tn_plan_step* info,
                             int32_t* leaves, int32_t* d, int32_t* D, int32_t* r);
/* Offset (in doubles) of vertex v's tensor inside a packed site buffer.    */
tn_status tn_plan_site_offset(const tn_plan_t* plan, int32_t vertex, int64_t* offset);

/* ------------------------------------------------------------------- context
 * A ctx binds one CUDA device and owns the device workspace.  device is a
 * CUDA ordinal.  Fails with TN_ERR_CUDA if the device cannot be used.       */
tn_status tn_ctx_create(int32_t device, tn_ctx_t** out);
tn_status tn_ctx_destroy(tn_ctx_t* ctx);

/* --------------------------------------------------------- one DM pass
 * Algorithm density_matrix_alg (Sec. 5) on an MPS embedding tree with n leaves,
 * for n_inst independent instances of identical shape.  The intermediate
 * network is given with the tensors of each tree vertex already contracted
 * ("contract T(v) first", Sec. 5.3): blocks Y_0..Y_{n-1} of shapes
 *   Y_0: (1, d_0, D_0),  Y_k: (D_{k-1}, d_k, D_k),  Y_{n-1}: (D_{n-2}, d_{n-1}, 1)
 * packed back to back in blocks_dev[i] (device, FP64).  Tree vertex 1 joins
 * leaves x_0 and x_1 (App. C, Def. MPS tree).
 * Ranks: r_k = min(chi_k, r_{k-1} d_k, D_k, prod_{j>k} d_j) with r_0 = d_0 and
 * chi_k = chi_per_edge ? chi_per_edge[k] : chi (k = 1..n-2).
 * Output (device, FP64, caller-allocated, tree_dev[i] per instance): the tree
 * tensors packed back to back: U_1 (d_0, d_1, r_1), U_k (r_{k-1}, d_k, r_k)
 * for k = 2..n-2, then the unit-Frobenius-norm root M_r (r_{n-2}, d_{n-1}).
 * Every U_k has orthonormal columns (as a (r_{k-1} d_k) x r_k matrix); each
 * column is signed so that its largest-|.| entry is positive.
 * lognorm_dev[i] (device) receives ln ||M_r|| before scaling; status_dev[i]
 * (device) a tn_status per instance.  ranks_host (host, n-1 entries) receives
 * r_0..r_{n-2}.  Asynchronous on stream (a cudaStream_t, NULL = default).  */
tn_status tn_embed_tree(tn_ctx_t* ctx, int32_t n_inst, int32_t n_legs,
                        const int32_t* leg_dim, const int32_t* bond_dim,
                        const double* const* blocks_dev, int32_t chi,
                        const int32_t* chi_per_edge, int32_t precision,
                        double* const* tree_dev, double* lognorm_dev,
                        int32_t* status_dev, int32_t* ranks_host, void* stream);

/* ------------------------------------------------------- whole contraction
 * Algorithm partitioned_contract for a batch of n_inst instances.  Plans may
 * differ between instances (graph size, partition, path, chi): instances
 * whose plans are structurally identical form a bucket that runs as one
 * batch of launches; buckets run one after another on stream, with one
 * upload of every bucket's tables and the workspace of the largest bucket.
 * learned_chi = 1 needs a single bucket.  sites_dev[i] is a device FP64
 * buffer with every site tensor of instance i packed at tn_plan_site_offset.
 * Asynchronous on stream; results are read with tn_logz.  learned_chi = 0
 * keeps each edge's plan rank r_k; learned_chi = 1 lets the rank model of
 * ctx (tn_rank_model_load; TN_ERR_INVALID if none is loaded) choose a rank
 * chi_k <= r_k per edge under a per-pass budget (see "learned ranks");
 * learned_chi = 2 runs the batch twice, at the uniform ranks
 * min(chi_uniform, r_k) and with the learned ranks, and keeps per instance
 * the ln Z of the run whose summed discarded share sum_k sum_{j >= chi_k}
 * lam_j / sum_j lam_j is smaller (the uniform method judges the model;
 * tn_rank_judged tells which run each instance kept).  Learned ranks need
 * all instances of the batch to share one plan structure.                  */
tn_status tn_contract_approx(tn_ctx_t* ctx, const tn_plan_t* const* plans, int32_t n_inst,
                             const double* const* sites_dev, int32_t precision,
                             int32_t learned_chi, void* stream);

/* Waits for the last tn_contract_approx of ctx and copies its results (in
 * instance order, whatever the buckets) to the
 * host: logz_host[i] = ln Z of instance i (NaN if status != TN_OK) and
 * status_host[i] its tn_status.  Returns the first non-OK instance status.  */
tn_status tn_logz(tn_ctx_t* ctx, double* logz_host, int32_t* status_host, int32_t n_inst);

/* End-to-end form of tn_contract_approx + tn_logz from HOST site buffers:
 * copies sites_host[i] (host, FP64, packed as above, plans[i]'s size;
 * page-locked memory gives asynchronous copies) to ctx-owned device memory,
 * runs the batch and copies ln Z and statuses back.  Synchronous.           */
tn_status tn_contract_approx_host(tn_ctx_t* ctx, const tn_plan_t* const* plans, int32_t n_inst,
                                  const double* const* sites_host, int32_t precision,
                                  int32_t learned_chi, double* logz_host,
                                  int32_t* status_host, void* stream);

/* ------------------------------------------------------ batching support
 * The paper has no counterpart: these serve many-instance runs on one GPU.
 *
 * tn_autotune times, for every tensor-core contraction shape (M, N, K, split,
 * batch) that the given batch launches, the tile widths 64 / 128 / 256 and the
 * shared-memory budgets 70 / 104 / 200 KB of the tcgen05 kernel on the real
 * operands (every candidate computes the same values: the tile width only
 * partitions N, the K order is fixed) and keeps the fastest per shape in ctx;
 * later batches of ctx use it.  Synchronous; runs the batch once per
 * candidate of each shape (its results are discarded).  cache_path (host
 * string, may be NULL): a JSON file written for this device is loaded instead
 * of tuning; otherwise the table is written there.  No-op for TN_PREC_FP64.
 * tn_autotune_entries reports the number of tuned shapes.
 *
 * tn_batch_graph_capture records one whole batch (the arguments of
 * tn_contract_approx without learned ranks) into a CUDA graph that owns a
 * private workspace: it runs the batch once to size the workspace and place
 * the tables, then captures the same launches.  The graph reads the site
 * buffers at the given device addresses on every replay: keep them alive and
 * at the same addresses (their contents may change between replays).
 * ctx's options and autotuned tiles are copied at capture.
 * tn_batch_graph_launch replays it on stream (asynchronous);
 * tn_batch_graph_logz waits for the last replay and copies ln Z and statuses
 * to the host as tn_logz does.                                             */
typedef struct tn_batch_graph tn_batch_graph_t;
tn_status tn_autotune(tn_ctx_t* ctx, const tn_plan_t* const* plans, int32_t n_inst,
                      const double* const* sites_dev, int32_t precision, const char* cache_path);
tn_status tn_autotune_entries(const tn_ctx_t* ctx, int32_t* n_entries);
tn_status tn_batch_graph_capture(tn_ctx_t* ctx, const tn_plan_t* const* plans, int32_t n_inst,
                                 const double* const* sites_dev, int32_t precision,
                                 tn_batch_graph_t** out);
tn_status tn_batch_graph_launch(tn_batch_graph_t* graph, void* stream);
tn_status tn_batch_graph_logz(tn_batch_graph_t* graph, double* logz_host, int32_t* status_host,
                              int32_t n_inst);
tn_status tn_batch_graph_destroy(tn_batch_graph_t* graph);

/* ------------------------------------------------ allocation-free variant
 * The paper has no counterpart: this entry point exists for callers of this
 * library that cannot allocate device memory.  Examples: a host application
 * whose own allocator has already reserved nearly all device memory (a new
 * cudaMalloc would fail); a plug-in whose host forbids direct device
 * allocation; a latency-critical loop where cudaMalloc/cudaFree, which may
 * synchronise the device, are not acceptable.
 *
 * It runs the same density-matrix pass as tn_embed_tree with precision FP64
 * (same arguments, layouts, outputs and error codes, minus the ctx and the
 * precision) but allocates nothing: its workspace is one device array of
 * TN_NOALLOC_SCRATCH_BYTES (16 MiB) compiled into the library, which every
 * GPU that loads the library holds until the process exits.  A problem whose
 * workspace would exceed it returns TN_ERR_INVALID, and tn_last_error(NULL)
 * states the bytes it needs.  The caller still provides all inputs and
 * outputs (device memory it owns).  The first call on a device looks up the
 * array's device address and configures the eigensolver's shared memory;
 * make that first call before any stream capture.  All calls share the one
 * array and it keeps the previous call's contents: calls that can overlap on
 * the GPU (different streams, or host threads without ordering between them)
 * race on it and corrupt each other's results, so serialise them.  Device
 * outputs are written asynchronously on stream; ranks_host on return.      */
#define TN_NOALLOC_SCRATCH_BYTES (16u << 20)
tn_status tn_embed_tree_noalloc(int32_t n_inst, int32_t n_legs, const int32_t* leg_dim,
                                const int32_t* bond_dim, const double* const* blocks_dev,
                                int32_t chi, const int32_t* chi_per_edge,
                                double* const* tree_dev, double* lognorm_dev,
                                int32_t* status_dev, int32_t* ranks_host, void* stream);

/* ---------------------------------------------------------- learned ranks
 * The paper has no learned component: it truncates every edge to one chi.
 * These calls let a small model spend a fixed rank budget unevenly.  After
 * the eigensolve of tree vertex k of a DM pass, features of the spectrum of
 * L_k (its eigenvalues, descending, over the effective dim A_k = chi_{k-1}
 * d_k, the rows the ranks kept so far can fill) feed an MLP with BF16 weights
 * and FP32 accumulation; chi_k = rint(64 y) clamped to [1, min(r_k, dim A_k,
 * numerical rank)] (numerical rank: the last position whose eigenvalue is
 * above 1e-12 lam_1), then lowered so that every later vertex u of the pass
 * can still get rank min(2, r_u), within the pass budget sum_k min(
 * chi_uniform, r_k) (the total rank of the uniform-chi_uniform method).  Columns of U_k beyond chi_k
 * are zeroed: shapes stay those of the plan, the tree tensor network has rank
 * chi_k on that edge.
 *
 * Features (22, in order): log10(lam_k / lam_1) / 30 for k = 2, 4, 8, 12, 16,
 * 24, 32, 48, 64, 96, 128 (k clamped to dim A);
 * log10(sum_{i >= r} lam_i / sum_i lam_i) / 30 for r = 8, 16, 24, 32, 48, 64
 * (0 share when r >= dim A; negative lam count as 0); ratios and shares are
 * floored at 1e-12;
 * dim A / 128; k / (n - 1); pass index / number of DM passes; the pass
 * budget not yet spent before vertex k / (n - 1 - k) (edges left, k's
 * included) / 64; min(chi_uniform, r_k) / 64.  The last two use the
 * chi_uniform of the last tn_rank_model_load (0 before any).
 * Parameters (tn_rank_model_params() floats, in order): W1 (64 x 22,
 * row-major), b1 (64), W2 (64 x 64), b2 (64), W3 (64), b3 (1); y = W3 .
 * relu(W2 relu(W1 x + b1) + b2) + b3.                                       */

/* Number of FP32 parameters of the rank model (5697).                     */
int32_t tn_rank_model_params(void);

/* Copies n_params FP32 parameters (host) into ctx, rounded to BF16, and sets
 * the per-pass budget basis chi_uniform (>= 1).  Synchronous.  weights_host
 * NULL unloads the model.                                                   */
tn_status tn_rank_model_load(tn_ctx_t* ctx, const float* weights_host, int32_t n_params,
                             int32_t chi_uniform);

/* Spectrum records of later tn_contract_approx batches (device buffers owned
 * by the caller, each may be NULL; all NULL turns recording off).  Edge e is
 * the e-th eigensolve of a batch in launch order (pass by pass, vertex 1 to
 * n-2 within a pass); for e < cap_edges and instance i of a batch of B:
 * feat[(e B + i) 22 + j] the features, spec[(e B + i) 128 + j] the
 * eigenvalues (zero beyond dim A), chi[e B + i] the rank kept.  acc[i] (B
 * entries) receives sum_e of the discarded share sum_{j >= chi} lam_j /
 * sum_j lam_j over all edges of the batch.  Recording does not change ranks
 * unless learned_chi = 1.  The buffers must stay valid until tn_logz.      */
tn_status tn_rank_record(tn_ctx_t* ctx, float* feat_dev, double* spec_dev, int32_t* chi_dev,
                         double* acc_dev, int64_t cap_edges);

/* After a tn_contract_approx with learned_chi = 2 (synchronous): used[i] = 1
 * where instance i kept the learned-rank run, 0 where the uniform run.      */
tn_status tn_rank_judged(tn_ctx_t* ctx, int32_t* used_learned_host, int32_t n_inst);

/* Training labels: for every pass p (edges pass_start[p] .. pass_start[p+1]-1,
 * at most 256 per pass; host array of n_pass + 1 entries, n_pass <= 65535)
 * and instance i, greedy water-filling of the pass budget sum_e min(
 * chi_uniform, cap[e]) over the pass's edges, each chi_e in [1, cap[e]] (cap
 * host, n_edges entries: the plan ranks), minimising the summed discarded
 * share of the recorded spectra spec (device, layout of tn_rank_record).
 * Starting from 1 everywhere, each step raises the edge whose next
 * eigenvalue has the largest share of its spectrum (ties: lowest edge).
 * Writes chi_dev[e B + i] (device).  When feat_dev (device, layout of
 * tn_rank_record) is set, features 20 and 21 of every edge are rewritten for
 * the labelled allocation.  Synchronous.                                    */
tn_status tn_rank_labels(tn_ctx_t* ctx, const double* spec_dev, int32_t n_inst,
                         const int32_t* cap, const int32_t* pass_start, int32_t n_pass,
                         int32_t chi_uniform, int32_t* chi_dev, float* feat_dev, void* stream);

/* Mean squared error of the model (FP32 parameters w_dev, rounded to BF16 for
 * the forward pass, as at inference) over samples idx_dev[0..n) (device; NULL
 * = 0..n-1) of X_dev (rows of 22 features) against y_dev, and its gradient
 * with respect to the rounded weights: loss_dev (1 float) and grad_dev
 * (tn_rank_model_params floats) are overwritten.  Asynchronous.             */
tn_status tn_rank_model_grad(tn_ctx_t* ctx, const float* X_dev, const float* y_dev,
                             const int32_t* idx_dev, int32_t n, const float* w_dev,
                             float* grad_dev, float* loss_dev, void* stream);

/* steps Adam steps (beta 0.9, 0.999, eps 1e-8, learning rate lr) on w_dev
 * (FP32 master weights, device, updated in place), step t using the
 * minibatch idx_dev[t batch .. (t+1) batch) (device).  loss_dev[t] (device,
 * steps floats) receives step t's minibatch loss.  Asynchronous.            */
tn_status tn_rank_model_train(tn_ctx_t* ctx, const float* X_dev, const float* y_dev,
                              const int32_t* idx_dev, int32_t steps, int32_t batch, float lr,
                              float* w_dev, float* loss_dev, void* stream);

/* ------------------------------------------------------------- diagnostics
 * Kernel classes of the hot path, for launch counts and timing.            */
enum {
  TN_KC_NORM = 0,     /* site-tensor normalisation                          */
  TN_KC_FUSE = 1,     /* block fusion, contract T(v) first (Sec. 5.3)        */
  TN_KC_ENV = 2,      /* root-side memoised density matrices (Eq. dm_cache) */
  TN_KC_LOCAL = 3,    /* local blocks M_v                                    */
  TN_KC_DENSITY = 4,  /* density matrices L_v = M_v L_u M_v^T                */
  TN_KC_EIG = 5,      /* leading_eigenvectors                                */
  TN_KC_PROJECT = 6,  /* projector application U_v^T M_v                     */
  TN_KC_ROOT = 7,     /* root M_r and its normalisation                      */
  TN_KC_CLOSE = 8,    /* closing contraction of the last partition           */
  TN_KC_FACTOR = 9,   /* Cholesky factors of the memoised environments       */
  TN_KC_COUNT = 10
};
/* Options of a ctx (the paper has no counterpart; they serve tuning and the
 * tests of the failure paths):
 *   TN_OPT_EIG_ROUNDS: multisection rounds of the TN_PREC_TF32 singular
 *     value search after its shared grid round (1 .. 16, default 9, which
 *     narrows every interval to ~4e-9 of ||T_GK||).  An interval still wider
 *     than 128 eps_32 ||T_GK|| marks its instance TN_ERR_EIG_NOCONV.
 *   TN_OPT_WAIT_PROBE: for the next tn_contract_approx only (value != 0),
 *     every tensor-core contraction first waits, bounded (~2^14 polls), on
 *     a device flag that nothing sets.  The expired wait takes the kernel's
 *     error path (bounded drain of its copies in flight, tensor memory
 *     released) and the batch reports TN_ERR_TIMEOUT from tn_logz; the ctx
 *     stays usable.  It exercises the timeout handling without a fault.
 *   TN_OPT_VALUE_PATH: accumulation of the mixed-precision value path
 *     (M_v = P_{v-1} Y_v, P_v = U_v^T M_v): 1 (default) compensated FP32
 *     (Kahan, about FP64-accumulation accuracy), 0 plain FP32 FFMA (faster;
 *     its rounding, amplified through the chain of projections, leaves
 *     ~1e-6 of ln Z on 3D lattices).
 *   TN_OPT_GROUPED: a mixed-precision batch of more than eight plan
 *     structures, all from the general planner, runs grouped: every
 *     operation is one launch over the problems of several buckets, each
 *     with its own pointers and shape (FP32 FFMA contractions, factored SVD
 *     or Gram form per pass); the buckets advance in lockstep (global
 *     step, pass section, tree vertex).  1 (default): on; 0: one launch
 *     sequence per bucket on a pool of streams.                             */
enum { TN_OPT_EIG_ROUNDS = 1, TN_OPT_WAIT_PROBE = 2, TN_OPT_VALUE_PATH = 3, TN_OPT_GROUPED = 4 };
/* Diagnostics read from the environment (none changes a result):
 *   TN_FAULT_ALLOC_AT=n  the n-th device allocation of the process fails
 *                        without a CUDA call (TN_ERR_OOM), for failure tests;
 *   TN_GROUPED_CHECK=1   a grouped batch checks every descriptor's operand
 *                        ranges on the host and launches nothing (the call
 *                        returns TN_ERR_INVALID with a summary);
 *   TN_GROUPED_GUARD=1   a grouped batch runs on one stream with every global
 *                        access checked against the batch's allocations, a
 *                        synchronisation after each launch, and the first
 *                        access outside them reported (TN_ERR_INVALID).      */
tn_status tn_ctx_set_option(tn_ctx_t* ctx, int32_t option, int64_t value);

/* Turn per-launch CUDA-event timing on (1) or off (0) for later batches of
 * ctx.  Launch counting is always on.  Timing adds two events per launch,
 * so timed numbers of a batch run with profiling on are diagnostics only. */
tn_status tn_ctx_set_profiling(tn_ctx_t* ctx, int32_t on);
/* Per class (n_classes <= TN_KC_COUNT entries, host arrays): kernel
 * launches and, when profiling was on, summed launch durations in ms
 * (CUDA events on the launching stream), since the last call.  Waits for
 * the ctx's stream, then resets the counters.  ms_host may be NULL.        */
tn_status tn_ctx_profile(tn_ctx_t* ctx, double* ms_host, int64_t* launches_host,
                         int32_t n_classes);

/* Arithmetic peaks of device (the paper has no counterpart: these are the
 * roofline denominators of the kernels that are not bandwidth bound),
 * measured by short burst kernels, best of three, TFLOP/s into tflops[0..3]
 * (host): FP32 FMA, FP32 packed-pair FMA, FP64 FMA, and the tcgen05 tensor
 * pipe in kind::tf32 (0 on devices other than sm_103).  Synchronous; takes
 * well under a second; allocates and frees a few KB of device memory.
 * TN_ERR_TIMEOUT if the tensor-pipe burst's bounded wait expired.          */
tn_status tn_measure_peaks(int32_t device, double* tflops);

/* One-line reason for the last non-OK status returned on this thread (ctx
 * may be NULL for calls that have none).  Valid until the next call.       */
const char* tn_last_error(const tn_ctx_t* ctx);

#ifdef __cplusplus
}
#endif
#endif /* TN_DMTREE_H */
