// engine.cuh -- device workspace of one solve handle and the stage launchers.
//
// One handle = one design matrix X (n x p) shared by every node of the tree
// (Section 3.2: one copy of X, c = X^T y and the b-update operator for all
// nodes), K node slots whose ADMM state is held node-major in HBM, a device
// node pool for the open nodes, and the incumbent.
//
// Template parameter R is the arithmetic of the ADMM state and contractions
// (float for the mixed-precision path, double for the plain FP64 comparator).
// Certificates (Proposition 1) and upper-bound polishing are FP64 for both.
#pragma once
#include <cuda_bf16.h>
#include <vector>
#include "common.cuh"

namespace bnb {

constexpr int UB_SEEN = 1 << 16;  // supports remembered per solve (upper bound already taken)
constexpr int MV_MAX = 32;      // most active slots the matrix-vector round form handles
constexpr int MV_ZMAX = 96;     // most contraction chunks of its partial products
constexpr int SEL_BINS = 2048;  // radix-select histogram width
constexpr int UE_NB = 8;        // blocks per node of the FP64 upper-bound evaluation
constexpr int PUSH_NB = 8;      // blocks per branched node of the warm-start copy
constexpr int REFILL_NB = 8;    // blocks per refilled slot

struct Status {                 // copied to the host after every round
  double ub, lb;
  long long pool_count;         // open nodes in the pool
  int active_slots;
  int retired;                  // nodes retired this round
  int pruned;                   // nodes closed this round
  int polished;
  int free_top;                 // free pool entries
  int warm_free;
  int error;                    // bits (the node is kept as a lost bound): 1 depth limit,
                                // 2 pool full, 4 a leaf support above support_max
  int max_depth;
  double lost_lb;
  long long nodes_total;        // nodes certified since the solve started
  long long rounds_total;
};

// Optional per-stage CUDA-event timing of a round (bnb_profile_round).
enum ProfKind {
  PK_SELECT = 0, PK_GEMM_XW, PK_REDUCE_T, PK_GEMM_GT, PK_FINAL_U, PK_GEMM_XTU, PK_CHECK, PK_STOP,
  PK_CERT, PK_BRANCH, PK_UB, PK_PUSH, PK_STATUS, PK_CERT_SCREEN, PK_CERT_EXACT, PK_COUNT
};
struct Profiler {
  std::vector<int> kind;
  std::vector<cudaEvent_t> ev;    // two per mark
  std::vector<cudaEvent_t> open;  // begin events of the intervals still open (nesting)
};
inline void prof_begin(Profiler* pf, cudaStream_t st) {
  if (!pf) return;
  cudaEvent_t e0;
  cudaEventCreate(&e0);
  cudaEventRecord(e0, st);
  pf->open.push_back(e0);
}
inline void prof_end(Profiler* pf, cudaStream_t st, int kind) {
  if (!pf || pf->open.empty()) return;
  cudaEvent_t e1;
  cudaEventCreate(&e1);
  cudaEventRecord(e1, st);
  pf->kind.push_back(kind);
  pf->ev.push_back(pf->open.back());
  pf->ev.push_back(e1);
  pf->open.pop_back();
}

// fields of a node-log record (doubles), see bnb_get_node_log
enum LogField {
  LOG_LB = 0,        // certified bound of Proposition 1 at the node's r (exact or screened)
  LOG_EXACT,         // 1: every nu term in FP64; 0: screened (rigorous upper values)
  LOG_WIDTH,         // D(r) - LOG_LB lies in [0, LOG_WIDTH]
  LOG_NODE_LB,       // max(LOG_LB, parent bound): the node's bound in the tree
  LOG_PARENT_LB,
  LOG_THRESHOLD,     // prune threshold UB (1 - gap) the certificate decided against
  LOG_DEPTH,
  LOG_ITERS,         // ADMM iterations of this visit
  LOG_EST_DUAL,      // FP32 estimate of D(r) at the stop test
  LOG_EST_PRIMAL,    // FP32 estimate of the primal value P(beta)
  LOG_REC
};

template <class R>
struct Engine {
  Prob P{};
  int n = 0, p = 0, K = 0;
  int smax = 200, ub_iters = 200;
  int s1 = 1, s2 = 1;           // split-K depth of the X W^T and G^-1 T products
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::vector<void*> allocs;

  // problem data
  double *X64 = nullptr, *y64 = nullptr, *c64 = nullptr, *xnorm = nullptr;
  float* X32 = nullptr;         // FP32 copy (certificate screen)
  R *XR = nullptr, *yR = nullptr, *cR = nullptr, *Ginv = nullptr;
  // shift of the b-update (formed once in FP64): b_c = D c, u_c = G^-1 X c = X b_c.
  // The iteration runs on W' = rho beta - V, so b = b_c + D W' and U = u_c + G^-1 X W'.
  R *bcR = nullptr, *rbcR = nullptr, *ucR = nullptr;   // b_c, rho b_c (p), u_c (n)
  R* Up = nullptr;              // U' = G^-1 X W'^T (n x K), the X^T U' operand
  double yy = 0.0;              // y^T y

  // ADMM state, node-major K x p
  R *beta = nullptr, *V = nullptr;
  int8_t* fix = nullptr;
  R *Tpart = nullptr, *T = nullptr, *Upart = nullptr, *U = nullptr;   // n x K (+ splits)
  R *XBpart = nullptr;          // check product X beta^T partials
  R* g3part = nullptr;          // [4][nbm3][K] per-block stats of the fused epilogue
  int nbm3 = 0;
  R* rstat = nullptr;           // [2][K]  ||y - U||^2, y^T (y - U)

  // slots
  int *slot_active = nullptr, *slot_iters = nullptr, *slot_depth = nullptr, *slot_nfix = nullptr;
  int dmax = 256;               // deepest node (fixings kept per open node)
  int lockstep = 0;             // 1: refill only when every slot is free (Algorithm 1 batches)
  int sel_blocks = 0;           // > 0: selection + refill as one cooperative launch of this many blocks
  unsigned long long* ub_seen = nullptr;  // [UB_SEEN] keys of evaluated supports (0: empty)
  int* sup_size = nullptr;      // [K] rounded-support size of each retired node (-1: > smax)
  int* hist_depth = nullptr;    // [dmax + 1] solved nodes by depth (last bin: deeper)
  int* hist_sup = nullptr;      // [smax + 2] solved nodes by rounded-support size
  int* slot_fixl = nullptr;     // K x dmax encoded fixings (idx << 1 | dir)
  double *slot_lbp = nullptr, *slot_gap = nullptr, *slot_dual = nullptr, *slot_primal = nullptr;
  int* slot_retire = nullptr;
  int *ret_slot = nullptr, *ret_active = nullptr, *ret_count = nullptr;

  // certificate
  double *r64 = nullptr, *cert_rr = nullptr, *cert_yr = nullptr, *cert_rn = nullptr;
  double *cert_lb = nullptr, *node_lb = nullptr;
  R* rS = nullptr;              // residual in screen precision, K x n
  float* gscr = nullptr;        // screened X_i^T r, K x p
  uint8_t* cflag = nullptr;     // K x p: 1 = exact FP64 term (F1), 2 = free, unsettled by the screen
  double* cx_part = nullptr;    // [2][K][8] exact certificate terms per p slice (F1, unsettled)
  double* cx_base = nullptr;    // [K] -1/2 ||r||^2 + y^T r - F1 terms
  uint8_t* cx_need = nullptr;   // [K] unsettled terms needed exactly
  double* cpart = nullptr;      // [2][row tiles of the screen][K] screen partial sums
  int* flist = nullptr;         // K x p flagged index lists

  // branching / upper bound
  int *br_idx = nullptr, *sup_cnt = nullptr, *sup = nullptr, *nfree = nullptr;
  R *Qg = nullptr, *qv = nullptr, *ubb = nullptr;   // K x smax^2, K x smax, K x smax
  double *Q64 = nullptr, *L64 = nullptr, *ubb64 = nullptr, *ub_val = nullptr;
  int* pol_flag = nullptr;
  double* ue_part = nullptr;   // k_ub_eval: per-node partial residual sums [K][UE_NB]
  int* ue_cnt = nullptr;       // k_ub_eval: blocks of a node done (zero between launches)
  int* push_w = nullptr;       // k_push: warm-store row of each retired node's children, or -1
  double* inc_beta = nullptr;   // p, FP64 incumbent
  double* inc_ub = nullptr;     // scalar
  double* inc_snap = nullptr;   // the incumbent when the round's certificate decides (scalar)
  float* zbuf = nullptr;        // K x p (relax outputs)

  // node pool
  long long qcap = 0, wcap = 0;
  double* pool_lb = nullptr;
  unsigned* pool_key = nullptr;
  uint8_t* pool_valid = nullptr;
  int *pool_depth = nullptr, *pool_warm = nullptr, *pool_fix = nullptr;
  int *free_stack = nullptr, *free_top = nullptr, *pool_hw = nullptr;
  R *warm_beta = nullptr, *warm_V = nullptr;
  int *warm_ref = nullptr, *warm_stack = nullptr, *warm_top = nullptr;
  unsigned* sel = nullptr;      // [3][SEL_BINS] histograms + scalars
  int* sel_state = nullptr;     // see queue.cu
  int *popped = nullptr, *free_slots = nullptr;
  unsigned long long* poolmin = nullptr;
  Status* status_d = nullptr;
  Status* status_h = nullptr;   // pinned host mirror
  double* params_d = nullptr;   // [0] gap target used by pruning

  Profiler* prof = nullptr;     // non-null only inside bnb_profile_round

  // tensor-core path (float engines): 0 = CUDA cores, 1 = BF16, 2 = BF16 data with hi/lo
  // iterates (2 products), 3 = hi/lo BF16 (3 products)
  int tc_mode = 0;
  float* H32 = nullptr;         // H = G^-1 X, n x p column-major (U' = H W' in one product)
  __nv_bfloat16 *ht_hi = nullptr, *ht_lo = nullptr;   // H row-major     (n x ldp)
  long long ldn = 0, ldp = 0;   // leading dimensions padded to multiples of 8 elements
  __nv_bfloat16 *xc_hi = nullptr, *xc_lo = nullptr;   // X column-major  (p x ldn)
  __nv_bfloat16 *xt_hi = nullptr, *xt_lo = nullptr;   // X row-major     (n x ldp)
  __nv_bfloat16 *gi_hi = nullptr, *gi_lo = nullptr;   // G^-1            (n x ldn)
  __nv_bfloat16 *w_hi = nullptr, *w_lo = nullptr;     // W operand       (K x ldp)
  __nv_bfloat16 *b_hi = nullptr, *b_lo = nullptr;     // beta operand    (K x ldp)
  __nv_bfloat16 *t_hi = nullptr, *t_lo = nullptr;     // T operand       (K x ldn)
  __nv_bfloat16 *u_hi = nullptr, *u_lo = nullptr;     // U operand       (K x ldn)
  int* tc_err = nullptr;        // pipeline error word of the tensor-core kernels
  int tc_s1 = 1, tc_s1n = 1, tc_s2 = 1, tc_s2n = 1;
  int tc_c1 = 0, tc_c2 = 0;     // cluster sizes of the cluster-reduced X W'^T / G^-1 T (0: split-K buffers)
  int tc_bn1 = 256, tc_bn2 = 256; // their output tile widths (128 or 256)
  int tc_bn3 = 64;              // tile width of the fused X^T U' product (64, 80, 96, 128)
  int tc_mc3 = 0;               // > 0: it runs in clusters of two sharing the X tile (this many)
  int tc_pair3 = 0;             // > 0: it runs on this many CTA pairs
  int tc_pairnt = 0;            // 1: the pair product untransposed (256 features x 176 slots)
  int u_kind = 0;               // U' = H W'^T: 0 measured, 1 cluster-reduced, 2 pairs split-K
  int tc_usplit = 0;            // > 0: U' on CTA pairs in this many K chunks (k_u_reduce)
  int tc_upairs = 0;            // CTA pairs the split form runs on
  int tc_ucs = 0;               // > 0: U' on 256 x 128 tiles, clusters of this many CTA pairs
                                // splitting K (tc_gemm_cpair_kernel)
  int usplit_max = 0;           // most K chunks the partial buffer holds
  float* upart = nullptr;       // [usplit_max][K][n] partial products of U'
  int fused_kind = 0;           // requested shape: 0 measured, 1 single, 2 clusters of two,
                                // 3 pairs transposed, 4 pairs untransposed
  int fused_width = 0;          // requested tile width of that product (0: measured)
  float* tc_stat = nullptr;     // [3][nbt][K] per-tile column sums: ||y-U||^2, y^T(y-U), ||y-X beta||^2
  int nbt = 0;                  // row tiles of the n x K products
  int sms = 148;                // multiprocessors of the device (persistent grids)
  // narrow batches: matrix-vector round form (admm_mv.cu)
  int mv_cross = 0;             // use it while the active slots are <= mv_cross (0: never)
  int mv_hint = -1;             // active slots known on the host (-1: read from the device)
  int* act_list = nullptr;      // [K] active slots in order
  int* act_count = nullptr;
  float* mv_part = nullptr;     // [MV_ZMAX][MV_MAX][n] partial products
  float* g3mv = nullptr;        // [4][ceil(p / 32)][MV_MAX] per-32-column stop-test sums
  cudaStream_t st_side = nullptr;  // capture of the conditional bodies
  cudaStream_t st_aux = nullptr;   // the upper-bound branch of a round, beside the certificate
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int mv_body_kernels = 0, tc_body_kernels = 0;

  // node log (tracing, options.log_nodes): the first log_cap nodes certified in a solve,
  // each with its fixings, its FP64 residual r = y - U and a record of LOG_REC doubles
  long long log_cap = 0;
  int* log_count = nullptr;     // nodes recorded so far (device scalar, <= log_cap)
  int8_t* log_fix = nullptr;    // log_cap x p
  double* log_r = nullptr;      // log_cap x n
  double* log_rec = nullptr;    // log_cap x LOG_REC (fields: LogField)
  double* cert_width = nullptr; // [K] D(r) - certified bound is in [0, width] (0: exact)

  // counters (host)
  long long nodes = 0, rounds = 0, admm_iters = 0, pruned = 0, polished = 0, pool_peak = 0;
  long long slot_iters_sum = 0;
  int max_depth = 0;
};

// ---- stage launchers (all asynchronous on e.st) ----
template <class R> int setup_data(Engine<R>& e, const double* dX, const double* dy);
// use_incumbent: 0 none; 1 a node whose dual estimate passes the prune threshold stops
// early; 2 also a node whose primal estimate lies below it (it is branched whatever the
// accuracy)
template <class R> int admm_round(Engine<R>& e, int iters, int max_iter, double node_tol,
                                  int use_incumbent);
template <class R> int certify(Engine<R>& e, const double* r_given /* K x n or null */,
                               bool use_threshold);
template <class R> int certify_screen(Engine<R>& e, const double* r_given);
template <class R> int certify_exact(Engine<R>& e, int use_threshold, const double* inc);
template <class R> int node_log(Engine<R>& e, const double* inc);
template <class R> int branch_support(Engine<R>& e, bool write_z, bool memo = false,
                                      bool defer_fallback = false);
template <class R> int branch_fallback(Engine<R>& e);
template <class R> int upper_bound(Engine<R>& e, int force_polish);
template <class R> int queue_push(Engine<R>& e);
template <class R> int queue_select_refill(Engine<R>& e);
template <class R> int queue_fused_select_blocks();
template <class R> int queue_init(Engine<R>& e);
template <class R> int queue_status(Engine<R>& e);
template <class R> int ub_from_masks(Engine<R>& e, const uint8_t* dmask, int K);
int admm_iterations_tc(Engine<float>& e, int iters);
int admm_iterations_mv(Engine<float>& e, int iters);
int mv_setup(Engine<float>& e);
int act_list(Engine<float>& e);
int capture_mv_or_tc(Engine<float>& e, int iters);
template <class R> int root_heuristic(Engine<R>& e, int max_moves);
int setup_tc(Engine<float>& e);

}  // namespace bnb
