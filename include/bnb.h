/*
 * bnb.h -- C ABI of the B300 (sm_103a) l0-l2 branch-and-bound library.
 *
 * Problem (Eq. original, Eq. perspective of arxiv 2602.04551):
 *     min_beta 1/2 ||y - X beta||^2 + lambda0 ||beta||_0 + lambda2 ||beta||^2,
 *     |beta_i| <= M  (big-M of the perspective formulation, Section 2.1).
 *
 * Conventions
 *   - Every function returns an int status: BNB_OK (0) or a negative BNB_E*
 *     code.  No function aborts or exits.  bnb_last_error() gives a message.
 *   - X is column-major: element (i, j) (sample i, feature j) at X[i + j*n].
 *   - Node fixings are int8 rows of length p: -1 free, 0 fixed to zero
 *     (z_i = 0, the set F0), 1 fixed to one (z_i = 1, the set F1).
 *   - Batched node arrays are node-major: row k of a K x p array is node k.
 *   - Host-pointer entry points copy inputs in and results out (the copies are
 *     part of the call); *_device entry points take device pointers on the
 *     handle's device and stream.  Output buffers are owned by the caller.
 *   - A handle owns all device memory it allocates; it is not thread-safe.
 *     Distinct handles are independent and may run on different streams.
 *   - Objective values follow Eq. original; every lower bound returned is an
 *     FP64 dual bound of Proposition 1 evaluated on the caller's data, so it
 *     is valid whatever the precision of the ADMM iterations.
 */
#ifndef BNB_H
#define BNB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BNB_OK 0
#define BNB_EINVAL (-1)   /* bad argument (sizes, lambdas, M, options) */
#define BNB_ENOMEM (-2)   /* device allocation failed */
#define BNB_ECUDA (-3)    /* a CUDA call failed (message in bnb_last_error) */
#define BNB_ETIMEOUT (-4) /* time limit reached inside a call */
#define BNB_EQUEUE (-5)   /* node pool capacity reached */
#define BNB_ENODEV (-6)   /* no CUDA device / not an sm_103 device */

/* ADMM arithmetic of the node solves (certificates and polish are FP64 always) */
#define BNB_PREC_FP64 0   /* plain FP64 everywhere: the comparator path */
#define BNB_PREC_FP32 1   /* FP32 state and contractions */
#define BNB_PREC_BF16 2   /* BF16 operands on tcgen05 tensor cores, FP32 accumulate/state */
#define BNB_PREC_TC3 3    /* hi/lo BF16 pairs on tcgen05 (three products): FP32-class */
#define BNB_PREC_BF16X2 4 /* X stored as one BF16 term, the ADMM iterates as hi/lo pairs
                             (two products; G^-1 T with three): BF16 data, FP32-class
                             iterates; certificates and polish use the FP64 data */

/* bnb_solve status */
#define BNB_STATUS_OPTIMAL 0     /* open-node set exhausted: UB is optimal */
#define BNB_STATUS_GAP 1         /* (UB - LB) / UB <= requested gap */
#define BNB_STATUS_TIME_LIMIT 2
#define BNB_STATUS_QUEUE_FULL 3
#define BNB_STATUS_NODE_LIMIT 4
#define BNB_STATUS_DEPTH_LIMIT 5  /* a node deeper than options.max_depth was needed; its
                                     bound stays in LB, so LB remains valid */
#define BNB_STATUS_SUPPORT_LIMIT 6 /* a leaf (no free index) whose support has more than
                                      options.support_max elements could not be evaluated;
                                      its bound stays in LB, so LB remains valid */

typedef struct bnb_handle bnb_handle;

typedef struct {
  double M;              /* big-M bound, > 0 (required: no default) */
  double rho;            /* ADMM penalty (Eq. ADMM2), default 1.0 */
  double node_tol;       /* relative primal-dual gap to stop a node solve, default 1e-4 */
  int max_admm_iter;     /* ADMM iteration cap per node visit, default 400 */
  int check_every;       /* ADMM iterations between stop tests (one "round"), default 10 */
  int batch_K;           /* node slots solved together, default 512 */
  int precision;         /* BNB_PREC_*, default BNB_PREC_TC3 */
  int use_graphs;        /* capture each round in a CUDA graph, default 1 */
  double time_limit_s;   /* bnb_solve wall-clock limit, default 3600 */
  long long max_nodes;   /* bnb_solve node limit, default 1e9 */
  long long queue_capacity; /* open-node pool capacity, default 1<<20 */
  long long warm_capacity;  /* warm-start store entries (parent beta, v), default auto */
  int support_max;       /* largest candidate support for the upper bound, default 200 */
  int ub_max_iter;       /* projected-gradient iterations per candidate, default 200 */
  int device;            /* CUDA device ordinal, default 0 */
  void* stream;          /* cudaStream_t to run on; NULL = a stream owned by the handle */
  double relax_alpha;    /* ADMM over-relaxation in [1, 1.9]; 1 = the plain update order of
                            Eq. admm-update (default); alpha > 1 uses alpha b + (1 - alpha)
                            beta in the beta- and v-updates.  Bounds are valid for any alpha. */
  int root_heuristic;    /* 1 (default): seed the incumbent with the matching-pursuit
                            heuristic (Appendix A.2) polished exactly in FP64 */
  int max_depth;         /* deepest node kept (fixings stored per open node), default 256,
                            in [8, 4096]; the pool takes queue_capacity x max_depth x 4 bytes */
  int lockstep;          /* 0 (default): a freed slot is refilled with the best open node at
                            the next round; 1: the batches of Algorithm 1 -- select up to K
                            nodes, solve them all, then branch/prune and select again */
  int mv_crossover;      /* tensor-core precisions: a round whose active slots are at most this
                            many runs the ADMM products as coalesced matrix-vector kernels on
                            CUDA cores (FP32) instead of tensor-core tiles; -1 (default) = 16,
                            0 = never, at most 32.  Chosen per round on the device. */
  int fused_shape;       /* tensor-core precisions, the fused X^T U' product: 0 (default) =
                            the fastest shape measured at creation; 1 = one CTA per output
                            tile; 2 = clusters of two CTAs sharing the X tile; 3 = the
                            transposed product on CTA pairs (tcgen05 cta_group::2, 256 node
                            slots per pair tile); 4 = the product on CTA pairs untransposed
                            (256 features per pair tile; not for BNB_PREC_BF16X2).  A shape
                            the device or the problem cannot run fails bnb_create with
                            BNB_EINVAL. */
  int u_shape;           /* tensor-core precisions, the product U' = H W'^T: 0 (default) =
                            the fastest of the forms measured at creation; 1 = K split
                            over the CTAs of a thread-block cluster, reduced in distributed
                            shared memory; 2 = 256 x 256 tiles on CTA pairs with K split into
                            chunks whose partial products a second kernel adds in order
                            (BNB_PREC_TC3 and BNB_PREC_BF16 only; needs at least two chunks
                            per tile to fill the GPU); 3 = 256 x 128 tiles, each on a
                            cluster of 4 (else 2) CTA pairs that split K and add their
                            partial tiles in distributed shared memory (BNB_PREC_TC3 and
                            BNB_PREC_BF16 only).  Otherwise as fused_shape. */
  int ub_polish;         /* bnb_upper_batch: 1 (default) re-solves each support exactly in FP64
                            after the projected-gradient method; 0 returns the projected-
                            gradient solution itself (ADMM precision, upcast) with its FP64
                            objective.  bnb_solve always polishes its candidate incumbents. */
  int fused_width;       /* tensor-core precisions, the fused X^T U' product: 0 (default) =
                            the tile width measured fastest at creation; otherwise only
                            shapes of this width compete (with fused_shape: the pair forms
                            offer 128 and 144 transposed, 80, 96, 128 and 176 untransposed;
                            one CTA per tile 64, 80, 96, 128).  A width no shape offers
                            fails bnb_create with BNB_EINVAL. */
  int fused_select;      /* 1: a round's best-first selection runs as one cooperative launch
                            whose blocks meet at (bounded) grid barriers, where the device
                            supports it; 0 (default): as seven separate launches.  The same
                            selection either way; the slot refill follows in a launch of its
                            own. */
  int exact_bounds;      /* bnb_solve's certificates: 0 (default) takes the exact FP64 nu terms
                            only where they can change the prune decision, so a branched
                            node keeps the cheaper screened bound (certified, but lower than
                            the exact value at r); 1 takes them for every node it does not
                            prune, so the bound passed to the children and to the global
                            lower bound is the exact value of Proposition 1 at r.  Pruning
                            is the same either way. */
  int log_nodes;         /* tracing: record the first log_nodes nodes certified in each solve
                            (fixings, FP64 residual, certified bound; bnb_get_node_log), in
                            [0, 65536], default 0 (off); takes log_nodes x (p + 8 n + 80)
                            bytes of device memory */
  int early_branch;      /* bnb_solve's node stop: 1 also retires a node at a stop test where
                            its estimated relaxation objective P(beta) (an upper bound on the
                            node's relaxation value, beta being feasible) lies below the
                            prune threshold t = UB (1 - gap) by more than
                            10 node_tol max(1, |t|) (with an incumbent): no
                            accuracy could then prune it, so it is certified (a valid, looser
                            FP64 bound) and branched at once; 0 (default) iterates every
                            node to the node gap, as the paper does (Section 5.1).  Exactness
                            is the same either way. */
} bnb_options;

/* Fill *opt with defaults (M is set to 0: the caller must set it). */
int bnb_options_default(bnb_options* opt);

/*
 * Create a solve handle (per-tree setup): copies X (n x p, column-major,
 * FP64 host array) and y (n) to the device, keeps X in FP64 (certificates,
 * polish) and in the ADMM precision, forms c = X^T y and the inverse of
 * G = X X^T + rho I (b-update of Eq. b_update via the Woodbury identity,
 * Section 3.1.2, with the 1/rho coefficient).  lambda0 >= 0, lambda2 > 0.
 * On success *out owns all device memory; release it with bnb_destroy.
 */
int bnb_create(const double* X_colmajor, const double* y, int n, int p,
               double lambda0, double lambda2, const bnb_options* opt,
               bnb_handle** out);

/* Device memory (bytes) that bnb_create would hold for an n x p problem with
 * these options (its allocations, staging and setup temporaries); used to admit
 * solves under an HBM budget.  Allocates nothing. */
int bnb_footprint(int n, int p, const bnb_options* opt, size_t* bytes);

/* Same as bnb_create with X and y already on the device (FP64, column-major).
 * The data are copied; the caller's buffers may be freed after the call. */
int bnb_create_device(const double* dX_colmajor, const double* dy, int n, int p,
                      double lambda0, double lambda2, const bnb_options* opt,
                      bnb_handle** out);

/*
 * Batched node relaxation (Sections 3.1-3.2; Eqs. batched_b_update ..
 * batched_v_update; dual bound of Proposition 1).
 *   K            number of nodes, 1 <= K <= opt.batch_K
 *   fix          K x p int8 fixings (host)
 *   warm_beta    K x p FP32 warm start for beta, or NULL (zeros)
 *   warm_v       K x p FP32 warm start for the ADMM dual v, or NULL (zeros)
 *   max_iter     ADMM iterations cap (<= 0: opt.max_admm_iter)
 * Outputs (host, any may be NULL except lb):
 *   lb           K certified FP64 lower bounds D(r), r = y - X b
 *   beta_out     K x p final beta
 *   v_out        K x p final v
 *   z_out        K x p relaxed z (Appendix A.1 recovery)
 *   branch_idx   K most-fractional free index (-1: no free index)
 *   node_gap     K FP32-estimated relative primal-dual gap at exit
 *   iters        K ADMM iterations run
 */
int bnb_relax_batch(bnb_handle* h, int K, const int8_t* fix, const float* warm_beta,
                    const float* warm_v, int max_iter, double* lb, float* beta_out,
                    float* v_out, float* z_out, int* branch_idx, double* node_gap, int* iters);

/* Device-pointer form of bnb_relax_batch (all pointers on the handle's device;
 * runs asynchronously on the handle's stream; outputs valid after a sync). */
int bnb_relax_batch_device(bnb_handle* h, int K, const int8_t* fix, const float* warm_beta,
                           const float* warm_v, int max_iter, double* lb, float* beta_out,
                           float* v_out, float* z_out, int* branch_idx, double* node_gap,
                           int* iters);

/*
 * FP64 dual bound of Proposition 1 for caller-supplied residuals:
 *   lb[k] = -1/2 ||r_k||^2 + y^T r_k - sum_i nu_i(|X_i^T r_k|)   (Eqs. dual, nudef)
 * with the fixings of row k.  r is K x n FP64 (host), node-major.
 */
int bnb_dual_bound(bnb_handle* h, int K, const int8_t* fix, const double* r, double* lb);

/*
 * Allocation-free dual bound.  The paper has no counterpart: this is a service
 * entry point for callers that must not allocate device memory (for example code
 * that runs under another framework which already owns the GPU's memory budget
 * through its own allocator, or latency-critical loops that cannot afford
 * cudaMalloc's implicit synchronisation or an allocation failure mid-run).
 * Computes the same bound as bnb_dual_bound, without a handle:
 *   lb[k] = -1/2 ||r_k||^2 + y^T r_k - sum_i nu_i(|X_i^T r_k|),   k < K,
 * all in FP64.  Every pointer is device memory on the current device:
 *   dX  n x p FP64 column-major;  dy  n;  dfix  K x p int8 (-1 free, 0 F0, 1 F1);
 *   dr  K x n FP64 residuals (node-major);  dlb  K outputs.
 * Runs asynchronously on `stream` (cudaStream_t, NULL = default stream).
 * Scratch: a fixed 8 MiB device array inside the library (every GPU that loads the
 * library keeps it until the process exits); a call needs K * (ceil(p/256) + 2)
 * doubles of it and returns BNB_EINVAL beyond 2^20 doubles (or K > 65535).
 * The first call on a device (and in each further context a caller makes current
 * on it) looks up the array's device address once, with that device current; make
 * that first call before any stream capture.  The CUDA runtime loads the array's
 * module lazily, so that first call is also when the 8 MiB are reserved on the
 * device: it can synchronise the device and can fail with BNB_ECUDA when no memory
 * is left; later calls only launch two kernels.  All calls on a device share the
 * array: calls whose kernels overlap on the GPU race on it, so order them (one
 * stream, or events).  No cudaMalloc, cudaFree or other allocating call is made.
 */
int bnb_dual_bound_static(const double* dX, const double* dy, int n, int p, double lambda0,
                          double lambda2, double M, int K, const int8_t* dfix, const double* dr,
                          double* dlb, void* stream);

/*
 * Batched upper bound (Sections 3.3-3.4, Eq. upperboundbeta): for each of K
 * supports (K x p uint8 mask, host), projected gradient with t/(t+3)
 * extrapolation and Armijo backtracking in the ADMM precision, then (unless
 * options.ub_polish is 0) an FP64 re-solve of the box ridge on the support
 * (exact active set).  Returns
 *   ub[k]        FP64 objective of Eq. original at the returned solution (lambda0
 *                counted once per nonzero)
 *   beta_out     K x p FP64 solutions (or NULL)
 * Supports larger than opt.support_max return ub = +inf.
 */
int bnb_upper_batch(bnb_handle* h, int K, const uint8_t* support, double* ub, double* beta_out);

/*
 * Full branch-and-bound (Algorithm 1 with a device-resident node pool,
 * continuous slot refill, best-first selection, branching on the most
 * fractional z_i, pruning when LB >= UB (1 - rel_gap)).
 *   beta_out   p FP64 incumbent (host, may be NULL)
 *   ub, lb     final global bounds: lb is the smallest certified bound over the open
 *              nodes, never above ub (the incumbent is feasible), and equals ub once
 *              the tree is closed
 *   nodes      nodes solved
 *   status     BNB_STATUS_*
 */
int bnb_solve(bnb_handle* h, double rel_gap, double* beta_out, double* ub, double* lb,
              long long* nodes, int* status);

/*
 * Stepping form of bnb_solve, for callers that interleave several solves on
 * one GPU (each handle runs on its own stream):
 *   bnb_solve_start   initialise the node pool with the root and capture one
 *                     round (refill, ADMM iterations, certificates, upper
 *                     bounds, prune/branch) as a CUDA graph;
 *   bnb_solve_launch  enqueue `rounds` rounds on the handle's stream and return
 *                     at once (rounds after the tree is closed do no work);
 *   bnb_solve_poll    wait for the enqueued rounds and report progress; sets
 *                     done/status when the gap, the time or node limit, or the
 *                     pool capacity ends the solve;
 *   bnb_solve_finish  copy the incumbent and the final bounds out.
 * bnb_solve is start + (launch 1, poll) until done + finish.
 */
typedef struct {
  double ub, lb;            /* global bounds after the last completed round */
  long long nodes;          /* nodes certified so far */
  long long open_nodes;     /* nodes in the pool plus nodes in slots */
  long long active_slots;   /* nodes in slots */
  long long rounds;         /* rounds completed */
  double seconds;           /* wall time since bnb_solve_start */
  int done;                 /* 1 once the solve has stopped */
  int status;               /* BNB_STATUS_* once done */
} bnb_progress;

int bnb_solve_start(bnb_handle* h, double rel_gap);
int bnb_solve_launch(bnb_handle* h, int rounds);
int bnb_solve_poll(bnb_handle* h, bnb_progress* out);
int bnb_solve_finish(bnb_handle* h, double* beta_out, double* ub, double* lb, long long* nodes,
                     int* status);

/*
 * Matching-pursuit root heuristic (Section 3.5, Appendix A.2): greedy forward /
 * backward single-coordinate moves from beta = 0 (scores in the ADMM precision),
 * then the exact FP64 box ridge on the support it ends on.  Writes that solution
 * (p FP64, host) and its objective of Eq. original.  Overwrites the handle's
 * incumbent (bnb_solve re-initialises it).
 */
int bnb_root_heuristic(bnb_handle* h, double* beta_out, double* ub_out);

/* The CUDA stream the handle runs on (cudaStream_t as void*). */
void* bnb_stream(const bnb_handle* h);

/*
 * Diagnostics: run one round of the started solve outside the CUDA graph with
 * CUDA events around each stage on the handle's stream.  stage_ms[k] receives
 * the mean duration of stage k in milliseconds and stage_launches[k] how many
 * times it ran; stages in order: select/refill, X W^T, split-K reduce,
 * G^-1 T, U finalise, X^T U + fused prox/v, check X beta^T, stop test,
 * certificate, branch pick, upper bound, push, status, and inside the certificate
 * its FP32 screen and its exact FP64 part (15 stages).
 */
int bnb_profile_round(bnb_handle* h, double* stage_ms, int* stage_launches, int nstages);

typedef struct {
  long long nodes;          /* nodes solved (retired with an FP64 certificate) */
  long long rounds;         /* device rounds run */
  long long admm_iters;     /* ADMM batch iterations run */
  long long slot_iters;     /* sum over nodes of ADMM iterations */
  long long pruned;         /* nodes closed by their bound */
  long long ub_polished;    /* FP64 polishes of candidate incumbents */
  long long pool_peak;      /* largest open-node count */
  int max_depth;
  double solve_seconds;     /* wall time of the last bnb_solve */
  double setup_seconds;     /* wall time of bnb_create */
  double final_ub, final_lb;
  int round_kernels;        /* kernels in one captured round (CUDA graph) */
  /* tensor-core shapes chosen at creation (0 for the CUDA-core precisions): output tile
     width and cluster size of the product H W'^T, tile width of the fused X^T U' product,
     the number of two-CTA clusters sharing the X tile it runs in (0: one CTA per tile),
     the number of CTA pairs it runs on (0: none), and 1 when the pair product is taken
     transposed (256 slots x width features per pair tile; else 256 features x width
     slots) */
  int xw_tile_width, xw_cluster, fused_tile_width, fused_clusters, fused_pairs, fused_transposed;
  int u_split;              /* K chunks of U' = H W'^T on CTA pairs (0: the cluster-reduced form) */
  int u_cluster_pairs;      /* CTA pairs per cluster of U' = H W'^T in its pair-in-cluster form
                               (u_shape 3; 0: another form) */
} bnb_stats;

int bnb_get_stats(const bnb_handle* h, bnb_stats* out);

/* Histograms of the nodes solved since the last bnb_solve / bnb_solve_start (host
 * arrays, caller-owned): depth_hist[d] = nodes solved at depth d (the bin at index
 * max_depth also counts anything deeper), support_hist[s] = nodes whose rounded support
 * S = F1 + {free i : z_i >= 1/2} (the upper-bound candidate, Section 3.3) has s
 * elements (the bin at support_max + 1 counts larger supports).  Bins beyond those are
 * written as 0.  Synchronises the handle's stream.  Measurement aid for the tree-shape
 * reports; the paper has no counterpart call. */
int bnb_get_histograms(bnb_handle* h, long long* depth_hist, int ndepth, long long* support_hist,
                       int nsupport);

/*
 * Node log (tracing; options.log_nodes = L > 0): the first L nodes certified since the
 * last bnb_solve / bnb_solve_start, in retirement order.  Copies min(*count, max_entries)
 * entries to the host arrays (each may be NULL):
 *   fix   entries x p int8 fixings of the node
 *   r     entries x n FP64 residual r = y - U the certificate used (Proposition 1)
 *   rec   entries x 10 doubles: [0] the certified bound at r (exact, or screened: the
 *         rigorous upper values of the unsettled nu terms), [1] 1 when every nu term was
 *         taken in FP64, [2] width: D(r) - bound lies in [0, width] (0 when exact),
 *         [3] the node's bound in the tree (max with the parent's), [4] the parent's
 *         bound, [5] the prune threshold UB (1 - gap) it was decided against, [6] depth,
 *         [7] ADMM iterations of the visit, [8] FP32 estimate of D(r) at the stop test,
 *         [9] FP32 estimate of the primal value.
 * *count receives the number of nodes recorded.  Synchronises the handle's stream.
 * Measurement aid (re-checking certificates against an independent evaluation); the
 * paper has no counterpart call.
 */
int bnb_get_node_log(bnb_handle* h, int max_entries, int8_t* fix, double* r, double* rec,
                     int* count);

/* Message of the last failed call on h (or of the last failed create when h is
 * NULL).  Valid until the next call on the same handle. */
const char* bnb_last_error(const bnb_handle* h);

/* Release every device resource of h (NULL is accepted). */
void bnb_destroy(bnb_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* BNB_H */
