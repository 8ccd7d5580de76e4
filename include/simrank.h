/*
 * simrank.h - C ABI of libsimrank, incremental all-pairs SimRank on one GB300.
 *
 * Method: Yu, Lin, Zhang, McCann, "Dynamical SimRank Search on Time-Varying
 * Networks".  SimRank here is Li et al.'s model (§3.1, Eq. 1):
 *     S = C Q S Q^T + (1 - C) I,
 * with Q the backward transition matrix, [Q]_{a,b} = 1/in-degree(a) when there
 * is an edge b -> a.  An edge (i, j) means i -> j.  After an edge update the
 * change of S solves a low-rank Sylvester equation (Thm 2, Eq. 13-14) whose
 * K-truncated series is sum_k xi_k eta_k^T + eta_k xi_k^T (Eq. 16a, Alg 1).
 *
 * Conventions shared by every entry point:
 *  - The caller owns every buffer it passes; the library copies what it needs
 *    and never keeps a caller pointer after a call returns.
 *  - Host pointers are plain CPU memory (pinned or not) unless an argument
 *    says "device".  Device pointers are CUDA global memory on the current
 *    device of the calling thread.
 *  - Every call is ordered on the handle's CUDA stream (simrank_config.cuda_stream,
 *    NULL = the legacy default stream).  A call that returns data in host
 *    memory synchronises that stream before it returns.
 *  - No C++ exception crosses this ABI.  Errors are reported by the status code;
 *    simrank_last_error() gives a one-line message.  A call that fails
 *    validation leaves the handle unchanged (all-or-nothing).
 *  - A handle is not thread-safe: one thread at a time per handle.
 *  - Node ids are int32 in [0, n_cur).  New nodes are named by the caller as
 *    the next ids n_cur, n_cur + 1, ... (§6 Remark); they must be contiguous
 *    and stay below n_capacity.
 */
#ifndef SIMRANK_H
#define SIMRANK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SIMRANK_ABI_VERSION 1

typedef struct simrank_ctx* simrank_t;

typedef enum simrank_status {
  SR_OK = 0,
  SR_ERR_ARG = 1,            /* bad argument, bad id, non-contiguous new ids, bad config */
  SR_ERR_EDGE_EXISTS = 2,    /* insertion of an existing edge, a self-loop, or a duplicate */
  SR_ERR_EDGE_MISSING = 3,   /* deletion of an absent edge */
  SR_ERR_CAPACITY = 4,       /* more nodes than n_capacity */
  SR_ERR_OOM = 5,            /* device or host allocation failed */
  SR_ERR_CUDA = 6,           /* a CUDA runtime call or kernel launch failed */
  SR_ERR_TIMEOUT = 7,        /* a bounded device wait ran out (status word set by a kernel) */
  SR_ERR_NOT_CONVERGED = 8,  /* batch initialisation did not reach init_tol in init_max_sweeps */
  SR_ERR_UNSUPPORTED = 9     /* valid request that this build does not implement */
} simrank_status;

/* One edge update.  op = +1 inserts (src -> dst), op = -1 deletes it.
 * weight is ignored by apply_updates (updates are on unweighted graphs, §3.1). */
typedef struct simrank_update {
  int32_t src;
  int32_t dst;
  int32_t op;
  float weight;
} simrank_update;

/* Storage / apply modes. */
enum { SR_MODE_DENSE = 0,        /* dense n_cap x n_cap S resident in HBM */
       SR_MODE_COLUMN = 1 };     /* no dense S: columns on demand (§7, O(Kn + m) memory) */
enum { SR_APPLY_UNIT = 0,        /* each update in order, one rank-one update each (Alg 1/2) */
       SR_APPLY_SINK_BLOCKS = 1, /* net update + similar-sink blocks, sequentially (§8, Alg 6, Table 2) */
       SR_APPLY_ONE_SHOT = 2 };  /* whole batch as one rank-2r update (proof of Thm 2, Eq. 23-28) */
enum { SR_SUPDATE_FUSED = 0,     /* one read-modify-write pass of S per update: S += Xi H^T + H Xi^T */
       SR_SUPDATE_PLAIN = 1 };   /* K+1 passes, one rank-2 term xi_k eta_k^T + eta_k xi_k^T each (Alg 1 as printed) */
enum { SR_INIT_SWEEPS = 0,       /* S of the initial graph by Jacobi sweeps of Eq. 1 (batch SimRank) */
       SR_INIT_FOREST = 1,       /* S of a forest of arborescences in closed form (Example 2, §1):
                                    every node has at most one in-neighbour and no cycle */
       SR_INIT_COMPONENTS = 2 }; /* S block-diagonal over the weakly connected components of the
                                    initial graph (Example 1, §1): each group of components (up to
                                    4096 nodes, or one larger component) gets its own Jacobi sweeps
                                    of Eq. 1; nodes are stored component by component */

typedef struct simrank_config {
  double C;               /* damping factor, 0 < C < 1 (Eq. 1) */
  int32_t K;              /* iterations of the xi/eta recurrence (Eq. 16a); terms k = 0..K; 0 <= K <= 1023 */
  int32_t s_precision;    /* 32: S stored in FP32; 64: S stored in FP64.  The xi/eta vectors
                             have the precision of S (FP64 also with FP32 S when vec_fp64 = 1,
                             or with chain = 1); the panels the S pass reads have the precision
                             of S. */
  int32_t mode;           /* SR_MODE_DENSE or SR_MODE_COLUMN */
  int32_t n_capacity;     /* maximum number of nodes, including nodes added later; >= n at init */
  int32_t aff;            /* 1: skip S tiles outside the affected area of Thm 4; 0: touch every tile */
  int32_t apply;          /* SR_APPLY_* */
  int32_t s_update;       /* SR_SUPDATE_* */
  int32_t tc;             /* S passes on the tensor cores: 1 = 3xTF32 split, 2 = 3xFP16 split with
                             an exact power-of-two balancing of each term (twice the tensor rate);
                             used, with FP32 S, for the one-shot batch form's pass and for the
                             pass of every unit / sink-block update (or of every group of `defer`
                             pending updates); 0 = CUDA cores */
  int32_t init_max_sweeps;/* cap on Jacobi sweeps of Eq. 1 at init / re-anchor */
  double init_tol;        /* init stops when a sweep changes S by less than this (max-abs);
                             <= 0 selects 1e-13 (sweeps stored in FP32 stop at 1e-7 or at
                             their rounding noise, below 3e-7) */
  int32_t profile;        /* 1: time every S-update launch with CUDA events (simrank_get_stats) */
  int32_t relabel;        /* 1: store nodes of in-degree 0 after the others, so that rows that no
                             update can reach (Thm 4) fill whole tiles; ids in the ABI are unchanged */
  int64_t timeout_iters;  /* bound on any device spin-wait (0 = library default) */
  void* cuda_stream;      /* cudaStream_t for all work of this handle; NULL = default stream */
  int32_t s_kernel;       /* CUDA-core S update with S in FP32: 0 = warp-specialised (math and
                             memory warps overlap), 1 = single-role kernel */
  int32_t defer;          /* dense FP32 S, unit / sink-block apply, fused update: 0 or 1 = apply
                             each rank-one update to S at once; G > 1 = keep up to G updates'
                             panels pending (the rows of S an update reads are corrected by them)
                             and apply them in one rank-2G(K+1) pass (tensor cores when tc = 1).
                             Pending updates are always applied before apply_updates returns.
                             G * (K + 1) <= 4096, else SR_ERR_ARG. */
  int32_t chain;          /* work of a rank-one update before its S pass: 0 = one cooperative
                             launch (graph patch, rows of S, gamma, all K recurrence steps, masks,
                             tile list; bounded grid barriers), 1 = one launch per step (FP64
                             vectors).  Graphs with more than 8 tiles of 128 nodes per
                             co-resident CTA take the per-step path. */
  int32_t prep_ctas;      /* chain = 0: cap on the CTAs of the fused launch (0 = as many as fit) */
  int32_t prep_cache;     /* chain = 0: column indices cached in shared memory per CTA, a
                             multiple of 4 in [0, 16384] (0 = 8192); the rest are read from L2 */
  int32_t multi_launch;   /* simrank_multi_apply: 0 = per round, one launch for the work of all
                             graphs before their S passes and one S pass over all their tiles,
                             replayed from a CUDA graph; 1 = the same kernels launched graph by
                             graph (the per-graph-launch baseline) */
  int32_t prep_item;      /* chain = 0: 0 (default) = the nonzeros of all rows split evenly over
                             the CTAs of the fused launch, two per thread (work items of 1024
                             when that does not fit); > 0 = work items of at most this many
                             nonzeros inside one 128-row tile, a tile with more split over
                             several CTAs */
  int32_t upper_only;     /* dense mode: 1 = keep only the 128 x 128 tiles of S on or above the
                             block diagonal current (S is symmetric; updates then read and write
                             half the bytes, and reads of a lower tile take its mirror); 0 = keep
                             both triangles.  Default 1. */
  int32_t vec_fp64;       /* chain = 0 with S in FP32: 1 = xi/eta vectors, gamma and the
                             recurrence in FP64; 0 (default) = in FP32.  On GB300 the FP64 form
                             makes the pre-update launch about 2.3x slower. */
  int32_t init_form;      /* SR_INIT_SWEEPS (default), SR_INIT_FOREST or SR_INIT_COMPONENTS: how
                             simrank_init computes S when S0 is NULL (dense mode).  With
                             SR_INIT_FOREST the initial graph must be a forest of arborescences
                             (else SR_ERR_ARG).  The edges left out of the initial graph (the
                             non-tree edges; the edges between blocks) are then applied as
                             updates: Examples 2 and 1's use of incremental SimRank as a batch
                             accelerator.  SR_INIT_COMPONENTS sets its own node order (relabel
                             is ignored). */
  int32_t reanchor_every; /* dense mode: 0 = off; N > 0 = after every N accepted updates of
                             apply_updates, run Jacobi sweeps of Eq. 1 from the current S
                             (the drift correction of simrank_reanchor) until a sweep changes S
                             by less than init_tol, at most reanchor_sweeps of them */
  int32_t reanchor_sweeps;/* cap on the sweeps of one automatic re-anchor (0 = 4) */
} simrank_config;

/* Fills *cfg with defaults: C = 0.6, K = 15, s_precision = 32, dense, aff = 1,
 * relabel = 1, upper_only = 1, unit apply, fused update, tc = 0, defer = 0,
 * vec_fp64 = 0, init_tol = 0 (= 1e-13), 400 init sweeps.  Host only: needs
 * no GPU. */
simrank_status simrank_default_config(simrank_config* cfg);

/* Creates a handle for the graph (src[e] -> dst[e]), e < m, on n nodes.
 * Host pointers.  weight (nullable) gives per-edge weights w_e > 0 for the
 * weighted Q (row a normalised by its total in-weight); NULL means 1/in-degree.
 * S0 (nullable, host, n x n row-major, FP32 or FP64 per cfg->s_precision) is the
 * old SimRank matrix; NULL computes it by Jacobi sweeps of Eq. 1 on the GPU
 * until the max-abs change is below cfg->init_tol.  Self-loops and duplicate
 * edges return SR_ERR_EDGE_EXISTS.  Nodes n..n_capacity-1 are pre-allocated as
 * isolated nodes (S_xx = 1 - C, a valid fixed point) and become nodes when
 * an update names them.  On success *out owns device memory until simrank_destroy. */
simrank_status simrank_init(const simrank_config* cfg, int32_t n, int64_t m,
                            const int32_t* src, const int32_t* dst, const float* weight,
                            const void* S0, simrank_t* out);

/* Applies count updates (host array) and brings S to the new graph
 * (Alg 1 / Alg 2 per update, §6 new-node cases C1-C3 through pre-allocated
 * isolated nodes, §8 batches).  All updates are validated first, in order;
 * if any is invalid nothing is applied.  Asynchronous on the handle's stream:
 * the host returns once the work is queued. */
simrank_status simrank_apply_updates(simrank_t h, const simrank_update* u, int64_t count);

/* Copies columns cols[0..ncols) of the current S (n_cur rows each) to out,
 * column-major: out[c * n_cur + a] = S[a, cols[c]].  out is device memory if
 * out_on_device != 0, else host memory (the call then synchronises).  out_fp64
 * selects double (1) or float (0) output.  In SR_MODE_COLUMN the columns are
 * computed from the graph history (Procedure 1 + Eq. 70-71). */
simrank_status simrank_columns(simrank_t h, const int32_t* cols, int32_t ncols, void* out,
                               int32_t out_on_device, int32_t out_fp64);

/* Current number of nodes n_cur (<= n_capacity). */
int32_t simrank_num_nodes(simrank_t h);

/* Message of the last failed call on h (or of the last failed simrank_init when
 * h is NULL).  The string lives until the next call on h. */
const char* simrank_last_error(simrank_t h);

/* Waits for all work queued on the handle's stream; returns SR_ERR_CUDA with a
 * message if a kernel failed, SR_ERR_TIMEOUT if a bounded wait ran out. */
simrank_status simrank_sync(simrank_t h);

/* Releases all memory of h.  NULL is ignored. */
void simrank_destroy(simrank_t h);

/* Cumulative counters since init (synchronises). */
typedef struct simrank_stats {
  int64_t updates;          /* updates accepted by apply_updates */
  int64_t rank_one_updates; /* rank-one (sink-block / unit) updates run on the GPU */
  int64_t tiles_total;      /* 128 x 128 S tiles that an unpruned update would touch */
  int64_t tiles_touched;    /* S tiles actually read and written */
  int64_t s_bytes;          /* algorithmic bytes of S read + written by S-update launches */
  int64_t panel_bytes;      /* algorithmic bytes of xi/eta panels read by S-update launches */
  int64_t s_update_launches;
  int64_t kernel_launches;  /* all libsimrank kernel launches on the handle's stream */
  double s_update_ms;       /* summed CUDA-event time of S-update launches (profile = 1 only) */
  double init_residual;     /* max-abs change of the last Jacobi sweep at init / re-anchor */
  double phase_ms[4];       /* profile = 1 only: CUDA-event time of the phases of rank-one updates:
                               [0] old-S rows + gamma (chain = 0: the whole fused launch before
                               the S pass), [1] graph patch + xi/eta recurrence (chain = 1),
                               [2] affected tile list (chain = 1) and deferred S passes,
                               [3] per-update S pass */
  int32_t init_sweeps;
  int32_t reanchors;         /* automatic re-anchors run (reanchor_every) */
  double reanchor_residual;  /* max-abs residual of Eq. 1, max |C Q S Q^T + (1-C) I - S|, at
                                the last automatic re-anchor, before it (its first sweep's change) */
  double reanchor_change;    /* max-abs change of that re-anchor's last sweep */
  int32_t reserved[2];
} simrank_stats;
simrank_status simrank_get_stats(simrank_t h, simrank_stats* out);

/* Changes the launch shape of a handle's later updates without touching its
 * state: defer, tc, prep_ctas, prep_cache, prep_item and s_kernel are taken
 * from *knobs (validated as by simrank_init; every other field is ignored).
 * Pending updates are applied first (synchronises).  The results of the
 * method do not depend on these fields beyond rounding (the tensor-core and
 * CUDA-core S passes and the FP16 / TF32 splits round differently).  This is
 * the call the autotuner (paper_1711_00121_gb300.tune) times its candidates
 * through; the paper has no counterpart. */
simrank_status simrank_set_launch(simrank_t h, const simrank_config* knobs);

/* Re-anchors S to the fixed point of Eq. 1 on the current graph by up to/* Re-anchors S to the fixed point of Eq. 1 on the current graph by up to
 * `sweeps` Jacobi sweeps started from the current S (drift correction after
 * long FP32 update streams).  *max_change (nullable) receives the max-abs
 * change of the last sweep.  Synchronises. */
simrank_status simrank_reanchor(simrank_t h, int32_t sweeps, double* max_change);

/* Loss and gradient for learning edge weights: for the K-truncated series
 * S_K = (1-C) sum_{k=0}^{K} C^k Q^k (Q^T)^k (Eq. 17; the paper defines neither
 * weights nor gradients: Q[a][b] = w_ba / sum_x w_xa with the weights given at
 * init, 1 / in-degree without them),
 *   *loss = sum_p (S_K[a_p, b_p] - target_p)^2,
 *   grad_weight[e] = dL / d w_e for the init edges e < m, in the caller's init order.
 * The gradient is the exact derivative of that truncated forward (an adjoint
 * series with its terms recomputed per block of endpoints, then an SDDMM at
 * the edges and the chain rule through the row normalisation).  Host arrays;
 * npairs pairs a, b (node ids) and targets.  Needs a handle to which no
 * updates have been applied (SR_ERR_UNSUPPORTED otherwise).  Synchronises. */
simrank_status simrank_grad(simrank_t h, const int32_t* a, const int32_t* b, const double* target,
                            int64_t npairs, double* loss, double* grad_weight);

/* Host-only planning of one batch (no GPU work, usable without a device):
 * net update by edge counts, split by sign, similar-sink partition (§8,
 * Alg 6), deletion blocks by ascending sink, then for each sink ascending its
 * old-source sub-block followed by its new-source sub-block.  n_old is |V|
 * before the batch.  Writes up to max_blocks blocks: block b covers
 * sources block_src[block_off[b] .. block_off[b+1]) into sink block_sink[b]
 * with block_op[b] = +1/-1.  *nblocks receives the number of blocks;
 * block_off needs max_blocks + 1 entries and block_src `count` entries.
 * Returns SR_ERR_ARG for a net count outside {-1, 0, +1}. */
simrank_status simrank_plan_batch(const simrank_update* u, int64_t count, int32_t n_old,
                                  int32_t max_blocks, int32_t* nblocks, int32_t* block_sink,
                                  int32_t* block_op, int64_t* block_off, int32_t* block_src);

/* ---------------------------------------------------------------------------
 * Many independent graphs advanced together.  Each graph has its own dense S
 * (cfg->s_precision), adjacency and caller ids, exactly as a simrank_t of its
 * own; all graphs share C, K and the stream.  simrank_multi_apply applies
 * every graph's updates in order, one rank-one update (Alg 1, Thm 3 / Thm 9,
 * new nodes as in simrank_apply_updates) per graph per round; a round is one
 * launch for the work of all graphs before their S passes (one CTA per graph)
 * and one S pass over the affected tiles of all graphs (cfg->multi_launch).
 * This batching is not in the paper: the graphs are independent problems.
 * ------------------------------------------------------------------------- */
typedef struct simrank_multi* simrank_multi_t;

/* Creates ngraphs graphs: graph g has n[g] nodes (n_capacity[g] >= n[g] with
 * the nodes beyond n[g] pre-allocated as isolated nodes; n_capacity NULL
 * means n) and the edges src[e] -> dst[e] for edge_offsets[g] <= e <
 * edge_offsets[g+1] (host arrays; edge_offsets has ngraphs + 1 entries).
 * Every S starts at the fixed point of Eq. 1 (Jacobi sweeps on the GPU to
 * cfg->init_tol).  cfg: dense mode, SR_APPLY_UNIT, fused S update, defer
 * 0 or 1, n_capacity ignored (per graph instead), at most 65536 nodes per
 * graph.  With cfg->tc != 0 and FP32 S each round's S pass runs on the tensor
 * cores (TF32 split), the operands of all graphs in one shared pair of arrays.  Errors: SR_ERR_ARG, SR_ERR_EDGE_EXISTS, SR_ERR_OOM, SR_ERR_CUDA,
 * SR_ERR_UNSUPPORTED; the message is simrank_last_error(NULL). */
simrank_status simrank_multi_init(const simrank_config* cfg, int32_t ngraphs, const int32_t* n,
                                  const int32_t* n_capacity, const int64_t* edge_offsets,
                                  const int32_t* src, const int32_t* dst, simrank_multi_t* out);

/* Applies the updates u[update_offsets[g] .. update_offsets[g+1]) to graph g,
 * in order, for every g (host arrays).  Every graph's updates are validated
 * first, as by simrank_apply_updates; if any is invalid nothing is applied
 * and simrank_multi_last_error names the graph.  Asynchronous on the stream. */
simrank_status simrank_multi_apply(simrank_multi_t h, const simrank_update* u,
                                   const int64_t* update_offsets);

/* simrank_columns for graph g (caller ids of that graph). */
simrank_status simrank_multi_columns(simrank_multi_t h, int32_t g, const int32_t* cols,
                                     int32_t ncols, void* out, int32_t out_on_device,
                                     int32_t out_fp64);
int32_t simrank_multi_num_graphs(simrank_multi_t h);
int32_t simrank_multi_num_nodes(simrank_multi_t h, int32_t g);
/* Waits for the stream; reports SR_ERR_TIMEOUT if a bounded device wait ran out. */
simrank_status simrank_multi_sync(simrank_multi_t h);
/* Totals over all graphs of the apply calls (updates, rank_one_updates,
 * tiles_touched, s_bytes, panel_bytes, kernel_launches); with cfg->profile = 1
 * also s_update_ms, s_update_launches and phase_ms[0] (work before the S
 * passes) / phase_ms[3] (S passes), from CUDA events (profiled calls are
 * launched directly, not from a CUDA graph). */
simrank_status simrank_multi_get_stats(simrank_multi_t h, simrank_stats* out);
const char* simrank_multi_last_error(simrank_multi_t h);
void simrank_multi_destroy(simrank_multi_t h);

/* One edge update of a caller-owned dense S and graph, allocating nothing.
 * The paper has no counterpart: this is for callers that cannot allocate
 * device memory when they apply an update - code embedded in a host
 * application whose device memory is owned by another allocator (a
 * framework's caching pool, a budget enforced by the host), or latency-bound
 * loops that must not stall on cudaMalloc / cudaFree.  It calls no
 * cudaMalloc, cudaFree or other allocating routine: its scratch lives in one
 * fixed __device__ array of this library (6.2 MiB, held by every GPU
 * that loads the library until the process exits), which limits it to
 * n <= 8192 nodes and K <= 31; larger sizes return SR_ERR_ARG.
 *
 * Applies the insertion (op = +1) or deletion (op = -1) of the edge i -> j
 * (0 <= i, j < n, i != j) to S in place: the same change at truncation K that
 * simrank_apply_updates makes to a dense handle (fused S update, tiles outside
 * the affected area skipped).
 *  S: device, FP32 or FP64 (s_precision = 32 / 64), row-major with row pitch
 *     ld elements; ld is a multiple of 128 and >= n rounded up to 128, S holds
 *     that many rows, and the padding rows and columns are zero.  On entry S
 *     is the SimRank matrix of the old graph (the fixed point of Eq. 1).
 *  old_row_ptr[n+1] (int64), old_col: device CSR of the in-lists of the old
 *     graph (row a lists every b with an edge b -> a); new_row_ptr / new_col
 *     the same for the graph after the update.  d_j is the old in-degree of j.
 *  cuda_stream: the stream all work is queued on (NULL = default stream).
 * Returns once the work is queued; argument and launch errors are reported
 * by the status and simrank_last_error(NULL).  The kernels of this entry
 * point wait on nothing on the device (no grid barrier, no mbarrier), so no
 * timeout can arise; an error while they run shows at the caller's next
 * synchronisation of cuda_stream.  All calls share the one scratch array, which
 * keeps the last call's contents (the parts that must start at zero are
 * cleared by each call): calls whose work overlaps on the GPU, from any
 * thread or stream, race and give wrong results.  The first call on each
 * device looks up the array's device address once (cudaGetSymbolAddress);
 * make that first call before any stream capture. */
simrank_status simrank_update_noalloc(int32_t n, int64_t ld, void* S, int32_t s_precision,
                                      const int64_t* old_row_ptr, const int32_t* old_col,
                                      const int64_t* new_row_ptr, const int32_t* new_col,
                                      int32_t i, int32_t j, int32_t op, int32_t d_j, double C,
                                      int32_t K, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* SIMRANK_H */
