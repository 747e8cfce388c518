// api.cu -- the C ABI declared in include/bnb.h.
//
// A handle owns one Engine<float> (mixed-precision path: FP32 ADMM state and
// contractions, FP64 certificates and polish) or one Engine<double> (plain
// FP64 path).  bnb_solve runs Algorithm 1 as device "rounds":
//   refill free slots from the pool (best-first) -> check_every ADMM iterations
//   -> stop test -> FP64 certificates of retired nodes -> branch pick + rounded
//   support -> batched upper bound (+ FP64 polish) -> prune / push children
//   -> status word to the host.
// With use_graphs a round is captured once into a CUDA graph and replayed; the
// host only reads the status word between rounds.
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <string>
#include <vector>

#include "bnb.h"
#include "engine.cuh"
#include "gemm_simt.cuh"
#include "tc_host.cuh"

namespace bnb {

static thread_local std::string g_err;

void set_cuda_error(const char* what, cudaError_t e, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  g_err = buf;
}

static int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

// When non-null, allocations are only counted (footprint query), not made.
static thread_local size_t* g_count_only = nullptr;

template <class R>
static int dalloc(Engine<R>& e, void** ptr, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (g_count_only) {
    *g_count_only += (bytes + 511) / 512 * 512;
    *ptr = nullptr;
    return 0;
  }
  cudaError_t rc = cudaMalloc(ptr, bytes);
  if (rc != cudaSuccess) {
    cudaGetLastError();
    return fail(BNB_ENOMEM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(rc));
  }
  e.allocs.push_back(*ptr);
  return 0;
}
#define ALLOC(ptr, count)                                                                 \
  do {                                                                                    \
    if (int _rc = dalloc(e, (void**)&(ptr), sizeof(*(ptr)) * (size_t)(count))) return _rc; \
  } while (0)

template <class R>
static void free_all(Engine<R>& e) {
  for (void* p : e.allocs) cudaFree(p);
  e.allocs.clear();
  if (e.status_h) cudaFreeHost(e.status_h);
  e.status_h = nullptr;
  if (e.st_side) cudaStreamDestroy(e.st_side);
  e.st_side = nullptr;
  if (e.st_aux) cudaStreamDestroy(e.st_aux);
  e.st_aux = nullptr;
  if (e.ev_fork) cudaEventDestroy(e.ev_fork);
  if (e.ev_join) cudaEventDestroy(e.ev_join);
  e.ev_fork = e.ev_join = nullptr;
  if (e.own_stream && e.st) cudaStreamDestroy(e.st);
  e.st = nullptr;
}

static int pick_splits(int m, int nn, int kred, int bm, int bn, int bk) {
  const int tiles = ((m + bm - 1) / bm) * ((nn + bn - 1) / bn);
  int s = (2 * 148 + tiles - 1) / tiles;
  const int smax = kred / (8 * bk);
  if (s > smax) s = smax;
  return s < 1 ? 1 : s;
}

template <class R>
static int allocate(Engine<R>& e) {
  using C = TileCfg<R>;
  const long long n = e.n, p = e.p, K = e.K, sm = e.smax;
  e.s1 = gemm_simt_splits<R>(e.p, pick_splits(e.n, e.K, e.p, C::BM, C::BN, C::BK));
  e.s2 = gemm_simt_splits<R>(e.n, pick_splits(e.n, e.K, e.n, C::BM, C::BN, C::BK));
  e.nbm3 = (e.p + C::BM - 1) / C::BM;
  long long s1cap = e.s1, s2cap = e.s2;
  if constexpr (sizeof(R) == 4) {
    if (e.tc_mode) {
      e.ldn = (n + 7) / 8 * 8;
      e.ldp = (p + 7) / 8 * 8;
      const int st1 = (e.p + tc::BK - 1) / tc::BK, st2 = (e.n + tc::BK - 1) / tc::BK;
      e.tc_s1 = tc_splits_for(e.n, e.K, 256, e.p);
      if (e.tc_s1 > st1 / 4) e.tc_s1 = st1 / 4 > 0 ? st1 / 4 : 1;
      e.tc_s2 = tc_splits_for(e.n, e.K, 256, e.n);
      if (e.tc_s2 > st2 / 4) e.tc_s2 = st2 / 4 > 0 ? st2 / 4 : 1;
      tc_chunk(e.p, e.tc_s1, &e.tc_s1n);
      tc_chunk(e.n, e.tc_s2, &e.tc_s2n);
      // cluster-reduced split-K for the n x K products: enough clusters of <= 8 CTAs to
      // cover the SMs, each CTA with >= 2 K steps (setup_tc clamps to what the device
      // can co-schedule); no split-K partial buffers are needed then
      e.nbt = (int)((n + tc::BM - 1) / tc::BM);
      const int tiles = e.nbt * (int)((K + 255) / 256);
      auto cl = [&](int steps) {
        int c = 148 / tiles;
        if (c > 8) c = 8;
        if (c > steps / 2) c = steps / 2;
        return c < 1 ? 1 : c;
      };
      e.tc_c1 = cl(st1);
      e.tc_c2 = cl(st2);
      ALLOC(e.tc_stat, 3LL * e.nbt * K);
      s1cap = s2cap = 0;
      ALLOC(e.act_list, K);
      ALLOC(e.act_count, 1);
      ALLOC(e.mv_part, (long long)MV_ZMAX * MV_MAX * n);
      {   // K chunks of the split pair form of U' = H W'^T (74 pairs on a B300)
        const long long tiles = ((n + 255) / 256) * ((K + 255) / 256);
        e.usplit_max = (int)(tiles > 0 ? (74 / tiles > 16 ? 16 : 74 / tiles) : 0);
        if (e.usplit_max >= 2) ALLOC(e.upart, (long long)e.usplit_max * K * n);
        else e.usplit_max = 0;
      }
      ALLOC(e.g3mv, 4LL * MV_MAX * ((p + 31) / 32));
      const bool xlo = e.tc_mode == 3;   // X as a hi/lo pair (3 terms)
      const bool lo = e.tc_mode >= 2;    // iterates and G^-1 as pairs (2 and 3 terms)
      ALLOC(e.xc_hi, p * e.ldn);
      ALLOC(e.xt_hi, n * e.ldp);
      ALLOC(e.gi_hi, n * e.ldn);
      ALLOC(e.w_hi, K * e.ldp);
      ALLOC(e.b_hi, K * e.ldp);
      ALLOC(e.t_hi, K * e.ldn);
      ALLOC(e.u_hi, K * e.ldn);
      ALLOC(e.H32, n * p);
      ALLOC(e.ht_hi, n * e.ldp);
      if (xlo) {
        ALLOC(e.xc_lo, p * e.ldn);
        ALLOC(e.xt_lo, n * e.ldp);
        ALLOC(e.ht_lo, n * e.ldp);
      }
      if (lo) {
        ALLOC(e.gi_lo, n * e.ldn);
        ALLOC(e.w_lo, K * e.ldp);
        ALLOC(e.b_lo, K * e.ldp);
        ALLOC(e.t_lo, K * e.ldn);
        ALLOC(e.u_lo, K * e.ldn);
      }
      ALLOC(e.tc_err, 1);
      if (!g_count_only) BNB_CUDA_OK(cudaMemsetAsync(e.tc_err, 0, sizeof(int), e.st));
      __nv_bfloat16* bufs[] = {e.xc_hi, e.xt_hi, e.gi_hi, e.w_hi, e.b_hi, e.t_hi, e.u_hi,
                               e.xc_lo, e.xt_lo, e.gi_lo, e.w_lo, e.b_lo, e.t_lo, e.u_lo};
      const long long cnt[] = {p * e.ldn, n * e.ldp, n * e.ldn, K * e.ldp, K * e.ldp, K * e.ldn,
                               K * e.ldn};
      for (int i = 0; i < 14; ++i)
        if (bufs[i] && !g_count_only) BNB_CUDA_OK(cudaMemsetAsync(bufs[i], 0, 2 * cnt[i % 7], e.st));
    }
  }
  ALLOC(e.X64, n * p);
  ALLOC(e.X32, n * p);
  if constexpr (sizeof(R) == 4) e.XR = (R*)e.X32; else e.XR = (R*)e.X64;
  ALLOC(e.y64, n);
  ALLOC(e.c64, p);
  ALLOC(e.xnorm, p);
  ALLOC(e.yR, n);
  ALLOC(e.cR, p);
  ALLOC(e.bcR, p);
  ALLOC(e.rbcR, p);
  ALLOC(e.ucR, n);
  ALLOC(e.Up, n * K);
  ALLOC(e.Ginv, n * n);
  ALLOC(e.beta, K * p);
  ALLOC(e.V, K * p);
  ALLOC(e.fix, K * p);
  ALLOC(e.Tpart, s1cap * n * K);
  ALLOC(e.T, n * K);
  ALLOC(e.Upart, s2cap * n * K);
  ALLOC(e.U, n * K);
  ALLOC(e.XBpart, s1cap * n * K);
  ALLOC(e.g3part, 4LL * e.nbm3 * K);
  ALLOC(e.rstat, 2 * K);
  ALLOC(e.slot_active, K);
  ALLOC(e.slot_iters, K);
  ALLOC(e.slot_depth, K);
  ALLOC(e.slot_nfix, K);
  ALLOC(e.slot_fixl, K * e.dmax);
  ALLOC(e.slot_lbp, K);
  ALLOC(e.slot_gap, K);
  ALLOC(e.slot_dual, K);
  ALLOC(e.slot_primal, K);
  ALLOC(e.slot_retire, K);
  ALLOC(e.ret_slot, K);
  ALLOC(e.ret_active, K);
  ALLOC(e.ret_count, 1);
  ALLOC(e.r64, K * n);
  ALLOC(e.rS, K * n);
  ALLOC(e.gscr, K * p);
  ALLOC(e.cflag, K * p);
  ALLOC(e.cpart, 2 * ((p + 31) / 32) * K);   // screen tiles of 32 (FP32) or 64 (FP64) rows
  ALLOC(e.cx_part, 2LL * K * 8);
  ALLOC(e.cx_base, K);
  ALLOC(e.cx_need, K);
  ALLOC(e.cert_rr, K);
  ALLOC(e.cert_yr, K);
  ALLOC(e.cert_rn, K);
  ALLOC(e.cert_lb, K);
  ALLOC(e.cert_width, K);
  if (e.log_cap > 0) {
    ALLOC(e.log_count, 1);
    ALLOC(e.log_fix, e.log_cap * p);
    ALLOC(e.log_r, e.log_cap * n);
    ALLOC(e.log_rec, e.log_cap * LOG_REC);
  }
  ALLOC(e.node_lb, K);
  ALLOC(e.br_idx, K);
  ALLOC(e.sup_cnt, K);
  ALLOC(e.nfree, K);
  ALLOC(e.sup, K * sm);
  ALLOC(e.Qg, K * sm * sm);
  ALLOC(e.qv, K * sm);
  ALLOC(e.ubb, K * sm);
  ALLOC(e.Q64, K * sm * sm);
  ALLOC(e.L64, K * sm * sm);
  ALLOC(e.ubb64, K * 2 * sm);
  ALLOC(e.ub_val, K);
  ALLOC(e.pol_flag, K);
  ALLOC(e.ue_part, K * UE_NB);
  ALLOC(e.ue_cnt, K);
  ALLOC(e.push_w, K);
  ALLOC(e.inc_beta, p);
  ALLOC(e.inc_ub, 1);
  ALLOC(e.inc_snap, 1);
  ALLOC(e.zbuf, K * p);
  ALLOC(e.pool_lb, e.qcap);
  ALLOC(e.pool_key, e.qcap);
  ALLOC(e.pool_valid, e.qcap);
  ALLOC(e.pool_depth, e.qcap);
  ALLOC(e.pool_warm, e.qcap);
  ALLOC(e.pool_fix, e.qcap * e.dmax);
  ALLOC(e.ub_seen, UB_SEEN);
  ALLOC(e.sup_size, K);
  ALLOC(e.hist_depth, e.dmax + 1);
  ALLOC(e.hist_sup, e.smax + 2);
  ALLOC(e.free_stack, e.qcap);
  ALLOC(e.free_top, 1);
  ALLOC(e.pool_hw, 1);
  ALLOC(e.warm_beta, e.wcap * p);
  ALLOC(e.warm_V, e.wcap * p);
  ALLOC(e.warm_ref, e.wcap);
  ALLOC(e.warm_stack, e.wcap);
  ALLOC(e.warm_top, 1);
  ALLOC(e.sel, 3 * SEL_BINS);
  ALLOC(e.sel_state, 16);
  ALLOC(e.popped, K);
  ALLOC(e.free_slots, K);
  ALLOC(e.poolmin, 2);
  ALLOC(e.status_d, 1);
  ALLOC(e.params_d, 4);
  if (g_count_only) return 0;
  if (cudaMallocHost((void**)&e.status_h, sizeof(Status)) != cudaSuccess)
    return fail(BNB_ENOMEM, "pinned status allocation failed");
  BNB_CUDA_OK(cudaMemsetAsync(e.beta, 0, sizeof(R) * K * p, e.st));
  BNB_CUDA_OK(cudaMemsetAsync(e.V, 0, sizeof(R) * K * p, e.st));
  BNB_CUDA_OK(cudaMemsetAsync(e.fix, 0xff, K * p, e.st));
  BNB_CUDA_OK(cudaMemsetAsync(e.slot_active, 0, sizeof(int) * K, e.st));
  BNB_CUDA_OK(cudaMemsetAsync(e.sel_state, 0, sizeof(int) * 16, e.st));
  BNB_CUDA_OK(cudaMemsetAsync(e.ue_cnt, 0, sizeof(int) * K, e.st));
  return 0;
}

// ----------------------------------------------------------------- small kernels

template <class R>
__global__ void k_load_nodes(int K, int p, const int8_t* __restrict__ fix_in,
                             const float* __restrict__ wb, const float* __restrict__ wv,
                             int8_t* __restrict__ fix, R* __restrict__ beta, R* __restrict__ V) {
  const long long m = (long long)K * p;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m;
       i += (long long)gridDim.x * blockDim.x) {
    const int f = fix_in[i];
    fix[i] = (int8_t)f;
    R b = wb ? (R)wb[i] : R(0);
    if (f == 0) b = R(0);
    beta[i] = b;
    V[i] = wv ? (R)wv[i] : R(0);
  }
}

__global__ void k_init_slots(int K, int Kact, int* slot_active, int* slot_iters, double* slot_lbp,
                             int* slot_depth, int* ret_slot, int* ret_active, int* ret_count,
                             int set_ret) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < K; s += gridDim.x * blockDim.x) {
    slot_active[s] = (s < Kact && !set_ret) ? 1 : 0;
    slot_iters[s] = 0;
    slot_lbp[s] = -INFINITY;
    slot_depth[s] = 0;
    if (set_ret) {
      ret_slot[s] = s;
      ret_active[s] = s < Kact ? 1 : 0;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && set_ret) *ret_count = Kact;
}

// per-slot results of the nodes retired this round (relax_batch)
__global__ void k_scatter_relax(const int* __restrict__ ret_slot, const int* __restrict__ ret_count,
                                const double* __restrict__ cert_lb, const int* __restrict__ br_idx,
                                double* out_lb, int* out_br) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= *ret_count) return;
  const int s = ret_slot[q];
  out_lb[s] = cert_lb[q];
  out_br[s] = br_idx[q];
}

__global__ void k_count_active(int K, const int* __restrict__ a, int* out) {
  __shared__ int sh[32];
  int c = 0;
  for (int s = threadIdx.x; s < K; s += blockDim.x) c += a[s];
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    *out = t;
  }
}

template <class R>
__global__ void k_to_float(const R* __restrict__ a, float* __restrict__ b, long long m) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

__global__ void k_scatter_ub(int K, int p, int smax, const int* __restrict__ sup,
                             const int* __restrict__ sup_cnt, const double* __restrict__ ubb64,
                             double* __restrict__ out) {
  const int q = blockIdx.x;
  if (q >= K) return;
  for (int i = threadIdx.x; i < p; i += blockDim.x) out[(long long)q * p + i] = 0.0;
  __syncthreads();
  const int s = sup_cnt[q];
  for (int a = threadIdx.x; a < s; a += blockDim.x)
    out[(long long)q * p + sup[(long long)q * smax + a]] = ubb64[(long long)q * 2 * smax + a];
}

static inline int g1d(long long m) {
  long long g = (m + 255) / 256;
  return (int)(g > 148 * 16 ? 148 * 16 : (g < 1 ? 1 : g));
}

}  // namespace bnb

using namespace bnb;

template <class R>
static int mp_moves(const Engine<R>& e) {
  const int m = 2 * e.smax + 16;
  return m < 4 * e.p ? m : 4 * e.p;
}

struct SolveState {
  bool started = false, done = false;
  long long launched = 0;       // rounds enqueued since bnb_solve_start
  int status = BNB_STATUS_OPTIMAL;
  double gap = 0.0;
  std::chrono::steady_clock::time_point t0;
  cudaGraphExec_t exec = nullptr;
  Status last{};
};

struct bnb_handle {
  bnb_options opt{};
  int n = 0, p = 0;
  double lam0 = 0, lam2 = 0;
  Engine<float>* ef = nullptr;
  Engine<double>* ed = nullptr;
  std::string err;
  bnb_stats stats{};
  // per-call staging (device)
  double *d_lb = nullptr, *d_rgiven = nullptr, *d_gap = nullptr;
  int *d_br = nullptr, *d_cnt = nullptr, *h_cnt = nullptr;
  float* d_stage = nullptr;
  double* d_ubbeta = nullptr;
  cudaGraphExec_t graph = nullptr;
  SolveState* solve = nullptr;
};

static int set_err(bnb_handle* h, int rc) {
  if (h) h->err = g_err;
  return rc;
}

extern "C" int bnb_options_default(bnb_options* o) {
  if (!o) return BNB_EINVAL;
  memset(o, 0, sizeof(*o));
  o->M = 0.0;
  o->rho = 1.0;
  o->node_tol = 1e-4;
  o->max_admm_iter = 400;
  o->check_every = 10;
  o->batch_K = 512;
  o->precision = BNB_PREC_TC3;
  o->use_graphs = 1;
  o->time_limit_s = 3600.0;
  o->max_nodes = 1000000000LL;
  o->queue_capacity = 1LL << 20;
  o->warm_capacity = 0;
  o->support_max = 200;
  o->ub_max_iter = 200;
  o->device = 0;
  o->stream = nullptr;
  o->relax_alpha = 1.0;
  o->root_heuristic = 1;
  o->max_depth = 256;
  o->lockstep = 0;
  o->mv_crossover = -1;
  o->fused_shape = 0;
  o->u_shape = 0;
  o->ub_polish = 1;
  o->log_nodes = 0;
  o->fused_width = 0;
  o->fused_select = 0;
  o->exact_bounds = 0;
  o->early_branch = 0;
  return BNB_OK;
}

template <class R>
static int engine_create(bnb_handle* h, Engine<R>*& e, const double* dX, const double* dy) {
  e = new Engine<R>();
  const bnb_options& o = h->opt;
  e->n = h->n;
  e->p = h->p;
  e->K = o.batch_K;
  e->dmax = o.max_depth;
  e->lockstep = o.lockstep ? 1 : 0;
  e->fused_kind = o.fused_shape;
  e->fused_width = o.fused_width;
  e->u_kind = o.u_shape;
  e->smax = o.support_max;
  e->ub_iters = o.ub_max_iter;
  e->qcap = o.queue_capacity;
  e->log_cap = o.log_nodes;
  long long wdef = (4LL << 30) / (2LL * h->p * (long long)sizeof(R));
  if (wdef > e->qcap / 2) wdef = e->qcap / 2;
  if (wdef < 64) wdef = 64;
  e->wcap = o.warm_capacity > 0 ? o.warm_capacity : wdef;
  Prob& P = e->P;
  P.n = h->n;
  P.p = h->p;
  P.lam0 = h->lam0;
  P.lam2 = h->lam2;
  P.M = o.M;
  P.rho = o.rho;
  P.s0 = std::sqrt(h->lam0 / h->lam2);
  P.linear = P.s0 > o.M ? 1 : 0;
  P.ridge_scale = o.rho / (o.rho + 2.0 * h->lam2);
  P.thr_soft = 2.0 * std::sqrt(h->lam0 * h->lam2) / o.rho;
  P.tau = P.thr_soft + P.s0;
  P.c_lin = h->lam0 / o.M + h->lam2 * o.M;
  P.thr_lin = P.c_lin / o.rho;
  P.c_soft = 2.0 * std::sqrt(h->lam0 * h->lam2);
  P.x0 = P.linear ? P.c_lin : P.c_soft;
  P.sqrt_l2_l0 = h->lam0 > 0 ? std::sqrt(h->lam2 / h->lam0) : INFINITY;
  P.alpha = o.relax_alpha;
  if (o.stream) {
    e->st = (cudaStream_t)o.stream;
  } else {
    BNB_CUDA_OK(cudaStreamCreateWithFlags(&e->st, cudaStreamNonBlocking));
    e->own_stream = true;
  }
  if constexpr (sizeof(R) == 4) {
    if (o.precision == BNB_PREC_BF16) e->tc_mode = 1;
    if (o.precision == BNB_PREC_BF16X2) e->tc_mode = 2;
    if (o.precision == BNB_PREC_TC3) e->tc_mode = 3;
  }
  e->sel_blocks = o.fused_select ? queue_fused_select_blocks<R>() : 0;
  if (int rc = allocate(*e)) return rc;
  if (int rc = setup_data(*e, dX, dy)) return rc;
  BNB_CUDA_OK(cudaStreamCreateWithFlags(&e->st_aux, cudaStreamNonBlocking));
  BNB_CUDA_OK(cudaEventCreateWithFlags(&e->ev_fork, cudaEventDisableTiming));
  BNB_CUDA_OK(cudaEventCreateWithFlags(&e->ev_join, cudaEventDisableTiming));
  if constexpr (sizeof(R) == 4) {
    if (e->tc_mode) {
      if (int rc = setup_tc(*e))
        return rc == BNB_EINVAL ? fail(BNB_EINVAL, "fused_shape %d / fused_width %d / u_shape %d: "
                                                    "no such shape runs here", o.fused_shape,
                                       o.fused_width, o.u_shape)
                                : rc;
      e->mv_cross = o.mv_crossover < 0 ? 16 : (o.mv_crossover > MV_MAX ? MV_MAX : o.mv_crossover);
      if (int rc = mv_setup(*e)) return rc;
      BNB_CUDA_OK(cudaStreamCreateWithFlags(&e->st_side, cudaStreamNonBlocking));
      BNB_CUDA_OK(cudaStreamSynchronize(e->st));
    }
  }
  return 0;
}

static int check_device(int dev) {
  cudaGetLastError();  // a failure left by unrelated earlier work must not be reported here
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count <= 0) {
    cudaGetLastError();
    return fail(BNB_ENODEV, "no CUDA device available");
  }
  if (dev < 0 || dev >= count) return fail(BNB_EINVAL, "device %d out of range", dev);
  cudaDeviceProp pr;
  if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) return fail(BNB_ECUDA, "device query failed");
  if (pr.major != 10) return fail(BNB_ENODEV, "device %d is sm_%d%d, this library is built for sm_103a", dev, pr.major, pr.minor);
  if (cudaSetDevice(dev) != cudaSuccess) return fail(BNB_ECUDA, "cudaSetDevice failed");
  return 0;
}

static int create_common(const double* dX, const double* dy, int n, int p, double lam0,
                         double lam2, const bnb_options* opt, bnb_handle** out) {
  if (!out) return fail(BNB_EINVAL, "out is NULL");
  *out = nullptr;
  if (n <= 0 || p <= 0) return fail(BNB_EINVAL, "n and p must be positive");
  if (!(lam0 >= 0.0) || !(lam2 > 0.0)) return fail(BNB_EINVAL, "need lambda0 >= 0 and lambda2 > 0");
  bnb_options o;
  if (opt) o = *opt; else bnb_options_default(&o);
  if (!(o.M > 0.0)) return fail(BNB_EINVAL, "options.M must be > 0");
  if (!(o.rho > 0.0)) return fail(BNB_EINVAL, "options.rho must be > 0");
  if (o.batch_K < 1 || o.batch_K > 65536) return fail(BNB_EINVAL, "batch_K out of range");
  if (o.support_max < 1 || o.support_max > 256) return fail(BNB_EINVAL, "support_max must be in [1, 256]");
  if (o.check_every < 1) return fail(BNB_EINVAL, "check_every must be >= 1");
  if (o.max_depth < 8 || o.max_depth > 4096) return fail(BNB_EINVAL, "max_depth must be in [8, 4096]");
  if (o.mv_crossover < -1 || o.mv_crossover > 32) return fail(BNB_EINVAL, "mv_crossover must be in [-1, 32]");
  if (o.fused_shape < 0 || o.fused_shape > 4) return fail(BNB_EINVAL, "fused_shape must be in [0, 4]");
  if (o.u_shape < 0 || o.u_shape > 3) return fail(BNB_EINVAL, "u_shape must be in [0, 3]");
  if (!(o.relax_alpha >= 1.0 && o.relax_alpha <= 1.9)) return fail(BNB_EINVAL, "relax_alpha must be in [1, 1.9]");
  if (o.queue_capacity < 4LL * o.batch_K + 8 || o.queue_capacity > (1LL << 30))
    return fail(BNB_EINVAL, "queue_capacity must be in [4 K + 8, 2^30]");
  if (o.ub_polish != 0 && o.ub_polish != 1) return fail(BNB_EINVAL, "ub_polish must be 0 or 1");
  if (o.log_nodes < 0 || o.log_nodes > (1 << 16)) return fail(BNB_EINVAL, "log_nodes must be in [0, 65536]");
  if (o.fused_width < 0 || o.fused_width > 256) return fail(BNB_EINVAL, "fused_width must be in [0, 256]");
  if (o.fused_select != 0 && o.fused_select != 1) return fail(BNB_EINVAL, "fused_select must be 0 or 1");
  if (o.exact_bounds != 0 && o.exact_bounds != 1) return fail(BNB_EINVAL, "exact_bounds must be 0 or 1");
  if (o.early_branch != 0 && o.early_branch != 1) return fail(BNB_EINVAL, "early_branch must be 0 or 1");
  if (o.precision < BNB_PREC_FP64 || o.precision > BNB_PREC_BF16X2)
    return fail(BNB_EINVAL, "unknown precision %d", o.precision);
  if (int rc = check_device(o.device)) return rc;
  auto t0 = std::chrono::steady_clock::now();
  bnb_handle* h = new bnb_handle();
  h->opt = o;
  h->n = n;
  h->p = p;
  h->lam0 = lam0;
  h->lam2 = lam2;
  int rc = (o.precision == BNB_PREC_FP64) ? engine_create<double>(h, h->ed, dX, dy)
                                          : engine_create<float>(h, h->ef, dX, dy);
  if (rc) {
    std::string msg = g_err;
    bnb_destroy(h);
    g_err = msg;
    return rc;
  }
  const int K = o.batch_K;
  cudaError_t ce = cudaSuccess;
  ce = ce ? ce : cudaMalloc(&h->d_lb, sizeof(double) * K);
  ce = ce ? ce : cudaMalloc(&h->d_gap, sizeof(double) * K);
  ce = ce ? ce : cudaMalloc(&h->d_br, sizeof(int) * K);
  ce = ce ? ce : cudaMalloc(&h->d_cnt, sizeof(int));
  ce = ce ? ce : cudaMallocHost(&h->h_cnt, sizeof(int));
  ce = ce ? ce : cudaMalloc(&h->d_rgiven, sizeof(double) * (size_t)K * n);
  ce = ce ? ce : cudaMalloc(&h->d_stage, sizeof(float) * (size_t)K * p);
  ce = ce ? ce : cudaMalloc(&h->d_ubbeta, sizeof(double) * (size_t)K * p);
  if (ce != cudaSuccess) {
    bnb_destroy(h);
    return fail(BNB_ENOMEM, "staging allocation failed: %s", cudaGetErrorString(ce));
  }
  h->stats.setup_seconds =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (h->ef && h->ef->tc_mode) {
    h->stats.xw_tile_width = h->ef->tc_bn1;
    h->stats.xw_cluster = h->ef->tc_c1;
    h->stats.fused_tile_width = h->ef->tc_bn3;
    h->stats.fused_clusters = h->ef->tc_mc3;
    h->stats.fused_pairs = h->ef->tc_pair3;
    h->stats.fused_transposed = h->ef->tc_pair3 > 0 && !h->ef->tc_pairnt ? 1 : 0;
    h->stats.u_split = h->ef->tc_usplit;
    h->stats.u_cluster_pairs = h->ef->tc_ucs;
  }
  *out = h;
  return BNB_OK;
}

template <class R>
static size_t footprint_of(int n, int p, const bnb_options& o) {
  Engine<R> e;
  e.n = n;
  e.p = p;
  e.K = o.batch_K;
  e.smax = o.support_max;
  e.dmax = o.max_depth;
  e.qcap = o.queue_capacity;
  e.log_cap = o.log_nodes;
  long long wdef = (4LL << 30) / (2LL * p * (long long)sizeof(R));
  if (wdef > e.qcap / 2) wdef = e.qcap / 2;
  if (wdef < 64) wdef = 64;
  e.wcap = o.warm_capacity > 0 ? o.warm_capacity : wdef;
  if constexpr (sizeof(R) == 4) {
    if (o.precision == BNB_PREC_BF16) e.tc_mode = 1;
    if (o.precision == BNB_PREC_BF16X2) e.tc_mode = 2;
    if (o.precision == BNB_PREC_TC3) e.tc_mode = 3;
  }
  size_t bytes = 0;
  g_count_only = &bytes;
  allocate(e);
  g_count_only = nullptr;
  // per-handle staging, setup temporaries (G, Newton-Schulz iterates) and input copies
  const size_t Kz = (size_t)o.batch_K;
  bytes += Kz * (8 + 8 + 4) + Kz * n * 8 + Kz * p * (4 + 8);
  bytes += (size_t)n * n * (8 + 3 * 4) + (sizeof(R) == 8 ? (size_t)n * n * 24 : 0);
  bytes += (size_t)n * p * 8 + (size_t)n * 8;
  return bytes;
}

extern "C" int bnb_footprint(int n, int p, const bnb_options* opt, size_t* bytes) {
  if (!bytes || n <= 0 || p <= 0) return fail(BNB_EINVAL, "bad arguments");
  bnb_options o;
  if (opt) o = *opt; else bnb_options_default(&o);
  *bytes = (o.precision == BNB_PREC_FP64) ? footprint_of<double>(n, p, o) : footprint_of<float>(n, p, o);
  return BNB_OK;
}

extern "C" int bnb_create(const double* X, const double* y, int n, int p, double lambda0,
                          double lambda2, const bnb_options* opt, bnb_handle** out) {
  if (!X || !y) return fail(BNB_EINVAL, "X or y is NULL");
  if (n <= 0 || p <= 0) return fail(BNB_EINVAL, "n and p must be positive");
  int dev = opt ? opt->device : 0;
  if (int rc = check_device(dev)) return rc;
  double *dX = nullptr, *dy = nullptr;
  if (cudaMalloc(&dX, sizeof(double) * (size_t)n * p) != cudaSuccess ||
      cudaMalloc(&dy, sizeof(double) * n) != cudaSuccess) {
    cudaFree(dX);
    return fail(BNB_ENOMEM, "input staging allocation failed");
  }
  int rc = BNB_OK;
  if (cudaMemcpy(dX, X, sizeof(double) * (size_t)n * p, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dy, y, sizeof(double) * n, cudaMemcpyHostToDevice) != cudaSuccess)
    rc = fail(BNB_ECUDA, "input upload failed");
  if (!rc) rc = create_common(dX, dy, n, p, lambda0, lambda2, opt, out);
  cudaFree(dX);
  cudaFree(dy);
  return rc;
}

extern "C" int bnb_create_device(const double* dX, const double* dy, int n, int p,
                                 double lambda0, double lambda2, const bnb_options* opt,
                                 bnb_handle** out) {
  if (!dX || !dy) return fail(BNB_EINVAL, "X or y is NULL");
  return create_common(dX, dy, n, p, lambda0, lambda2, opt, out);
}

extern "C" void bnb_destroy(bnb_handle* h) {
  if (!h) return;
  if (h->graph) cudaGraphExecDestroy(h->graph);
  if (h->solve) {
    if (h->solve->exec) cudaGraphExecDestroy(h->solve->exec);
    delete h->solve;
  }
  if (h->ef) { free_all(*h->ef); delete h->ef; }
  if (h->ed) { free_all(*h->ed); delete h->ed; }
  cudaFree(h->d_lb);
  cudaFree(h->d_gap);
  cudaFree(h->d_br);
  cudaFree(h->d_cnt);
  cudaFreeHost(h->h_cnt);
  cudaFree(h->d_rgiven);
  cudaFree(h->d_stage);
  cudaFree(h->d_ubbeta);
  delete h;
}

extern "C" const char* bnb_last_error(const bnb_handle* h) {
  if (h && !h->err.empty()) return h->err.c_str();
  return g_err.c_str();
}

// ------------------------------------------------------------------- relax batch

template <class R>
static int relax_impl(bnb_handle* h, Engine<R>& e, int K, const int8_t* dfix, const float* dwb,
                      const float* dwv, int max_iter, double* lb, float* beta_out, float* v_out,
                      float* z_out, int* br, double* gap, int* iters) {
  cudaStream_t st = e.st;
  const bnb_options& o = h->opt;
  if (max_iter <= 0) max_iter = o.max_admm_iter;
  const long long Kp = (long long)K * e.p;
  k_load_nodes<R><<<g1d(Kp), 256, 0, st>>>(K, e.p, dfix, dwb, dwv, e.fix, e.beta, e.V);
  k_init_slots<<<g1d(e.K), 256, 0, st>>>(e.K, K, e.slot_active, e.slot_iters, e.slot_lbp,
                                         e.slot_depth, e.ret_slot, e.ret_active, e.ret_count, 0);
  BNB_CUDA_OK(cudaGetLastError());
  double inf = INFINITY;
  BNB_CUDA_OK(cudaMemcpyAsync(e.inc_ub, &inf, sizeof(double), cudaMemcpyHostToDevice, st));
  int rounds = 0;
  const int max_rounds = (max_iter + o.check_every - 1) / o.check_every + 1;
  e.mv_hint = K;                      // active slots, known exactly on the host here
  while (true) {
    if (int rc = admm_round(e, o.check_every, max_iter, o.node_tol, 0)) return rc;
    if (int rc = certify(e, nullptr, false)) return rc;
    if (int rc = branch_support(e, true)) return rc;
    k_scatter_relax<<<(e.K + 255) / 256, 256, 0, st>>>(e.ret_slot, e.ret_count, e.cert_lb,
                                                       e.br_idx, h->d_lb, h->d_br);
    k_count_active<<<1, 1024, 0, st>>>(e.K, e.slot_active, h->d_cnt);
    BNB_CUDA_OK(cudaGetLastError());
    BNB_CUDA_OK(cudaMemcpyAsync(h->h_cnt, h->d_cnt, sizeof(int), cudaMemcpyDeviceToHost, st));
    BNB_CUDA_OK(cudaStreamSynchronize(st));
    ++rounds;
    e.mv_hint = *h->h_cnt;
    if (*h->h_cnt == 0) break;
    if (rounds > max_rounds + 2) return fail(BNB_ETIMEOUT, "relax_batch did not retire all nodes");
  }
  e.mv_hint = -1;
  // outputs
  BNB_CUDA_OK(cudaMemcpyAsync(lb, h->d_lb, sizeof(double) * K, cudaMemcpyDefault, st));
  if (br) BNB_CUDA_OK(cudaMemcpyAsync(br, h->d_br, sizeof(int) * K, cudaMemcpyDefault, st));
  if (gap) BNB_CUDA_OK(cudaMemcpyAsync(gap, e.slot_gap, sizeof(double) * K, cudaMemcpyDefault, st));
  if (iters) BNB_CUDA_OK(cudaMemcpyAsync(iters, e.slot_iters, sizeof(int) * K, cudaMemcpyDefault, st));
  if (beta_out) {
    k_to_float<R><<<g1d(Kp), 256, 0, st>>>(e.beta, h->d_stage, Kp);
    BNB_CUDA_OK(cudaMemcpyAsync(beta_out, h->d_stage, sizeof(float) * Kp, cudaMemcpyDefault, st));
  }
  if (v_out) {
    BNB_CUDA_OK(cudaStreamSynchronize(st));
    k_to_float<R><<<g1d(Kp), 256, 0, st>>>(e.V, h->d_stage, Kp);
    BNB_CUDA_OK(cudaMemcpyAsync(v_out, h->d_stage, sizeof(float) * Kp, cudaMemcpyDefault, st));
  }
  if (z_out) BNB_CUDA_OK(cudaMemcpyAsync(z_out, e.zbuf, sizeof(float) * Kp, cudaMemcpyDefault, st));
  BNB_CUDA_OK(cudaStreamSynchronize(st));
  e.rounds += rounds;
  return 0;
}

template <class F>
static int dispatch(bnb_handle* h, F&& f) {
  if (!h) return fail(BNB_EINVAL, "handle is NULL");
  cudaSetDevice(h->opt.device);
  int rc = h->ef ? f(*h->ef) : f(*h->ed);
  if (rc) set_err(h, rc);
  return rc;
}

static int relax_common(bnb_handle* h, int K, const int8_t* fix, const float* wb, const float* wv,
                        int max_iter, double* lb, float* beta_out, float* v_out, float* z_out,
                        int* br, double* gap, int* iters, bool host) {
  if (!h) return fail(BNB_EINVAL, "handle is NULL");
  if (K < 1 || K > h->opt.batch_K) return set_err(h, fail(BNB_EINVAL, "K=%d outside [1, %d]", K, h->opt.batch_K));
  if (!fix || !lb) return set_err(h, fail(BNB_EINVAL, "fix and lb are required"));
  const size_t Kp = (size_t)K * h->p;
  return dispatch(h, [&](auto& e) -> int {
    const int8_t* dfix = fix;
    const float *dwb = wb, *dwv = wv;
    int8_t* tfix = nullptr;
    float *twb = nullptr, *twv = nullptr;
    if (host) {
      BNB_CUDA_OK(cudaMallocAsync(&tfix, Kp, e.st));
      BNB_CUDA_OK(cudaMemcpyAsync(tfix, fix, Kp, cudaMemcpyHostToDevice, e.st));
      dfix = tfix;
      if (wb) {
        BNB_CUDA_OK(cudaMallocAsync(&twb, Kp * 4, e.st));
        BNB_CUDA_OK(cudaMemcpyAsync(twb, wb, Kp * 4, cudaMemcpyHostToDevice, e.st));
        dwb = twb;
      }
      if (wv) {
        BNB_CUDA_OK(cudaMallocAsync(&twv, Kp * 4, e.st));
        BNB_CUDA_OK(cudaMemcpyAsync(twv, wv, Kp * 4, cudaMemcpyHostToDevice, e.st));
        dwv = twv;
      }
    }
    int rc = relax_impl(h, e, K, dfix, dwb, dwv, max_iter, lb, beta_out, v_out, z_out, br, gap, iters);
    if (tfix) cudaFreeAsync(tfix, e.st);
    if (twb) cudaFreeAsync(twb, e.st);
    if (twv) cudaFreeAsync(twv, e.st);
    cudaStreamSynchronize(e.st);
    return rc;
  });
}

extern "C" int bnb_relax_batch(bnb_handle* h, int K, const int8_t* fix, const float* wb,
                               const float* wv, int max_iter, double* lb, float* beta_out,
                               float* v_out, float* z_out, int* br, double* gap, int* iters) {
  return relax_common(h, K, fix, wb, wv, max_iter, lb, beta_out, v_out, z_out, br, gap, iters, true);
}

extern "C" int bnb_relax_batch_device(bnb_handle* h, int K, const int8_t* fix, const float* wb,
                                      const float* wv, int max_iter, double* lb, float* beta_out,
                                      float* v_out, float* z_out, int* br, double* gap, int* iters) {
  return relax_common(h, K, fix, wb, wv, max_iter, lb, beta_out, v_out, z_out, br, gap, iters, false);
}

// -------------------------------------------------------------------- dual bound

extern "C" int bnb_dual_bound(bnb_handle* h, int K, const int8_t* fix, const double* r, double* lb) {
  if (!h) return fail(BNB_EINVAL, "handle is NULL");
  if (K < 1 || K > h->opt.batch_K) return set_err(h, fail(BNB_EINVAL, "K out of range"));
  if (!fix || !r || !lb) return set_err(h, fail(BNB_EINVAL, "NULL argument"));
  return dispatch(h, [&](auto& e) -> int {
    const size_t Kp = (size_t)K * e.p;
    BNB_CUDA_OK(cudaMemcpyAsync(e.fix, fix, Kp, cudaMemcpyHostToDevice, e.st));
    BNB_CUDA_OK(cudaMemcpyAsync(h->d_rgiven, r, sizeof(double) * (size_t)K * e.n,
                                cudaMemcpyHostToDevice, e.st));
    k_init_slots<<<g1d(e.K), 256, 0, e.st>>>(e.K, K, e.slot_active, e.slot_iters, e.slot_lbp,
                                             e.slot_depth, e.ret_slot, e.ret_active, e.ret_count, 1);
    BNB_CUDA_OK(cudaGetLastError());
    if (int rc = certify(e, h->d_rgiven, false)) return rc;
    BNB_CUDA_OK(cudaMemcpyAsync(lb, e.cert_lb, sizeof(double) * K, cudaMemcpyDeviceToHost, e.st));
    BNB_CUDA_OK(cudaStreamSynchronize(e.st));
    return 0;
  });
}

// ------------------------------------------------------------------- upper bound

extern "C" int bnb_upper_batch(bnb_handle* h, int K, const uint8_t* support, double* ub,
                               double* beta_out) {
  if (!h) return fail(BNB_EINVAL, "handle is NULL");
  if (K < 1 || K > h->opt.batch_K) return set_err(h, fail(BNB_EINVAL, "K out of range"));
  if (!support || !ub) return set_err(h, fail(BNB_EINVAL, "NULL argument"));
  return dispatch(h, [&](auto& e) -> int {
    const size_t Kp = (size_t)K * e.p;
    BNB_CUDA_OK(cudaMemcpyAsync(e.cflag, support, Kp, cudaMemcpyHostToDevice, e.st));
    k_init_slots<<<g1d(e.K), 256, 0, e.st>>>(e.K, K, e.slot_active, e.slot_iters, e.slot_lbp,
                                             e.slot_depth, e.ret_slot, e.ret_active, e.ret_count, 1);
    BNB_CUDA_OK(cudaGetLastError());
    if (int rc = ub_from_masks(e, e.cflag, K)) return rc;
    double inf = INFINITY;
    BNB_CUDA_OK(cudaMemcpyAsync(e.inc_ub, &inf, sizeof(double), cudaMemcpyHostToDevice, e.st));
    if (int rc = upper_bound(e, h->opt.ub_polish ? 1 : -1)) return rc;
    BNB_CUDA_OK(cudaMemcpyAsync(ub, e.ub_val, sizeof(double) * K, cudaMemcpyDeviceToHost, e.st));
    if (beta_out) {
      k_scatter_ub<<<K, 256, 0, e.st>>>(K, e.p, e.smax, e.sup, e.sup_cnt, e.ubb64, h->d_ubbeta);
      BNB_CUDA_OK(cudaGetLastError());
      BNB_CUDA_OK(cudaMemcpyAsync(beta_out, h->d_ubbeta, sizeof(double) * Kp,
                                  cudaMemcpyDeviceToHost, e.st));
    }
    BNB_CUDA_OK(cudaStreamSynchronize(e.st));
    return 0;
  });
}

// ------------------------------------------------------------------------- solve

__global__ void k_copy_scalar(const double* __restrict__ src, double* __restrict__ dst) {
  if (threadIdx.x == 0) *dst = *src;
}

// One round: refill, ADMM iterations, certificate, branching and upper bound, push,
// status.  After the ADMM iterations the round forks: branching and the upper bound run
// on the auxiliary stream while the certificate (FP32 screen, exact terms) runs on the
// handle's stream -- they share no buffer; the certificate decides against the
// incumbent as it was before this round's upper bound (copied at the fork, as in the
// sequential order), and the rare branching decisions that need the screened X^T r
// (every free z integral) are deferred to k_branch_fallback after the join; the push
// waits for both.  Inside a capture the fork and join become graph edges.  A profiled
// round (per-stage events on one stream) runs the stages in order.
template <class R>
static int round_body(bnb_handle* h, Engine<R>& e) {
  const bnb_options& o = h->opt;
  Profiler* pf = e.prof;
  prof_begin(pf, e.st);
  if (int rc = queue_select_refill(e)) return rc;
  prof_end(pf, e.st, PK_SELECT);
  if (int rc = admm_round(e, o.check_every, o.max_admm_iter, o.node_tol, o.early_branch ? 2 : 1))
    return rc;
  if (pf) {
    prof_begin(pf, e.st);
    if (int rc = certify_screen(e, nullptr)) return rc;
    if (int rc = certify_exact(e, o.exact_bounds ? 2 : 1, e.inc_ub)) return rc;
    if (int rc = node_log(e, e.inc_ub)) return rc;
    prof_end(pf, e.st, PK_CERT);
    prof_begin(pf, e.st);
    if (int rc = branch_support(e, false, true)) return rc;
    prof_end(pf, e.st, PK_BRANCH);
    prof_begin(pf, e.st);
    if (int rc = upper_bound(e, 0)) return rc;
    prof_end(pf, e.st, PK_UB);
  } else {
    k_copy_scalar<<<1, 32, 0, e.st>>>(e.inc_ub, e.inc_snap);
    BNB_CUDA_OK(cudaGetLastError());
    BNB_CUDA_OK(cudaEventRecord(e.ev_fork, e.st));
    BNB_CUDA_OK(cudaStreamWaitEvent(e.st_aux, e.ev_fork, 0));
    cudaStream_t main_st = e.st;
    e.st = e.st_aux;
    int rc = branch_support(e, false, true, true);
    if (!rc) rc = upper_bound(e, 0);
    e.st = main_st;
    const cudaError_t ce = cudaEventRecord(e.ev_join, e.st_aux);
    if (rc) return rc;
    BNB_CUDA_OK(ce);
    if (int rc2 = certify_screen(e, nullptr)) return rc2;
    if (int rc2 = certify_exact(e, o.exact_bounds ? 2 : 1, e.inc_snap)) return rc2;
    if (int rc2 = node_log(e, e.inc_snap)) return rc2;
    BNB_CUDA_OK(cudaStreamWaitEvent(e.st, e.ev_join, 0));
    if (int rc2 = branch_fallback(e)) return rc2;
  }
  prof_begin(pf, e.st);
  if (int rc = queue_push(e)) return rc;
  prof_end(pf, e.st, PK_PUSH);
  prof_begin(pf, e.st);
  if (int rc = queue_status(e)) return rc;
  prof_end(pf, e.st, PK_STATUS);
  return 0;
}

// One round of the current solve outside the graph, with CUDA events around
// every stage on the handle's stream; returns per-stage mean milliseconds and
// launch counts.
template <class R>
static int profile_round(bnb_handle* h, Engine<R>& e, double* ms, int* counts, int nk) {
  Profiler pf;
  e.prof = &pf;
  int rc = round_body(h, e);
  e.prof = nullptr;
  if (rc) return rc;
  BNB_CUDA_OK(cudaStreamSynchronize(e.st));
  for (int k = 0; k < nk; ++k) {
    ms[k] = 0.0;
    counts[k] = 0;
  }
  for (size_t i = 0; i < pf.kind.size(); ++i) {
    float t = 0.f;
    cudaEventElapsedTime(&t, pf.ev[2 * i], pf.ev[2 * i + 1]);
    const int k = pf.kind[i];
    if (k < nk) {
      ms[k] += t;
      counts[k] += 1;
    }
  }
  for (cudaEvent_t ev : pf.ev) cudaEventDestroy(ev);
  for (int k = 0; k < nk; ++k)
    if (counts[k]) ms[k] /= counts[k];
  return 0;
}




template <class R>
static int solve_start(bnb_handle* h, Engine<R>& e, SolveState& S, double gap) {
  const bnb_options& o = h->opt;
  if (S.exec) {
    cudaGraphExecDestroy(S.exec);
    S.exec = nullptr;
  }
  S = SolveState{};
  S.gap = gap;
  S.t0 = std::chrono::steady_clock::now();
  double params[4] = {gap, 0, 0, 0};
  BNB_CUDA_OK(cudaMemcpyAsync(e.params_d, params, sizeof(params), cudaMemcpyHostToDevice, e.st));
  if (int rc = queue_init(e)) return rc;
  if (e.log_count) BNB_CUDA_OK(cudaMemsetAsync(e.log_count, 0, sizeof(int), e.st));
  BNB_CUDA_OK(cudaMemsetAsync(e.inc_beta, 0, sizeof(double) * e.p, e.st));
  if (o.root_heuristic) {
    if (int rc = root_heuristic(e, mp_moves(e))) return rc;
  }
  BNB_CUDA_OK(cudaStreamSynchronize(e.st));
  e.nodes = e.rounds = e.admm_iters = e.pruned = e.polished = e.pool_peak = 0;
  e.max_depth = 0;
  {   // the status before the first round: the root alone in the pool, the incumbent of
      // the root heuristic (or none); a poll before any round reads this, never a stale word
    double ub0 = INFINITY;
    BNB_CUDA_OK(cudaMemcpy(&ub0, e.inc_ub, sizeof(double), cudaMemcpyDeviceToHost));
    Status s0{};
    s0.ub = ub0;
    s0.lb = -INFINITY;
    s0.pool_count = 1;
    s0.free_top = (int)(e.qcap - 1);
    s0.lost_lb = INFINITY;
    *e.status_h = s0;
  }
  if (o.use_graphs) {
    cudaGraph_t g;
    BNB_CUDA_OK(cudaStreamBeginCapture(e.st, cudaStreamCaptureModeThreadLocal));
    int rc = round_body(h, e);
    cudaError_t ce = cudaStreamEndCapture(e.st, &g);
    if (rc) return rc;
    if (ce != cudaSuccess) return fail(BNB_ECUDA, "graph capture failed: %s", cudaGetErrorString(ce));
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(g, nodes.data(), &nn);
    int kern = 0;
    for (auto nd : nodes) {
      cudaGraphNodeType t;
      cudaGraphNodeGetType(nd, &t);
      kern += (t == cudaGraphNodeTypeKernel) ? 1 : 0;
    }
    // a round with both ADMM forms runs one body of its conditional node: count the
    // tensor-core body (the form of wide batches)
    if constexpr (sizeof(R) == 4) kern += e.tc_body_kernels;
    h->stats.round_kernels = kern;
    ce = cudaGraphInstantiate(&S.exec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return fail(BNB_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(ce));
  }
  S.started = true;
  return 0;
}

template <class R>
static int solve_launch(bnb_handle* h, Engine<R>& e, SolveState& S, int rounds) {
  if (!S.started) return fail(BNB_EINVAL, "bnb_solve_start was not called");
  for (int r = 0; r < rounds; ++r) {
    if (S.exec) {
      BNB_CUDA_OK(cudaGraphLaunch(S.exec, e.st));
    } else if (int rc = round_body(h, e)) {
      return rc;
    }
    ++S.launched;
  }
  return 0;
}

template <class R>
static int solve_poll(bnb_handle* h, Engine<R>& e, SolveState& S, bnb_progress* out) {
  const bnb_options& o = h->opt;
  if (!S.started) return fail(BNB_EINVAL, "bnb_solve_start was not called");
  BNB_CUDA_OK(cudaStreamSynchronize(e.st));
  const Status s = *e.status_h;
  S.last = s;
  e.rounds = s.rounds_total;
  e.nodes = s.nodes_total;
  if (s.pool_count > e.pool_peak) e.pool_peak = s.pool_count;
  e.max_depth = s.max_depth;
  const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - S.t0).count();
  if (s.error & 8) {
    S.done = true;
    return fail(BNB_ECUDA, "a grid barrier of the fused selection timed out (device blocks "
                           "not co-resident)");
  }
  if (!S.done && S.launched > 0) {   // no round has run yet: nothing can have ended
    if (s.active_slots == 0 && s.pool_count == 0) {
      S.done = true;
      S.status = (s.error & 2) ? BNB_STATUS_QUEUE_FULL
                 : (s.error & 1) ? BNB_STATUS_DEPTH_LIMIT
                 : (s.error & 4) ? BNB_STATUS_SUPPORT_LIMIT : BNB_STATUS_OPTIMAL;
      if (s.error && std::isfinite(s.ub) && (s.ub - s.lb) <= S.gap * std::fabs(s.ub))
        S.status = BNB_STATUS_GAP;
    } else if (std::isfinite(s.ub) && (s.ub - s.lb) <= S.gap * std::fabs(s.ub)) {
      S.done = true;
      S.status = BNB_STATUS_GAP;
    } else if (s.error & 2) {
      S.done = true;
      S.status = BNB_STATUS_QUEUE_FULL;
    } else if (s.error & 4) {
      S.done = true;
      S.status = BNB_STATUS_SUPPORT_LIMIT;
    } else if (el > o.time_limit_s) {
      S.done = true;
      S.status = BNB_STATUS_TIME_LIMIT;
    } else if (e.nodes >= o.max_nodes) {
      S.done = true;
      S.status = BNB_STATUS_NODE_LIMIT;
    } else if (s.free_top < 2 * e.K + 2) {
      S.done = true;
      S.status = BNB_STATUS_QUEUE_FULL;
    }
  }
  if (out) {
    out->ub = s.ub;
    out->lb = (S.done && s.active_slots == 0 && s.pool_count == 0 && !s.error) ? s.ub : s.lb;
    out->nodes = s.nodes_total;
    out->open_nodes = s.pool_count + s.active_slots;
    out->active_slots = s.active_slots;
    out->rounds = s.rounds_total;
    out->seconds = el;
    out->done = S.done ? 1 : 0;
    out->status = S.status;
  }
  return 0;
}

template <class R>
static int solve_finish(bnb_handle* h, Engine<R>& e, SolveState& S, double* beta_out, double* ub,
                        double* lb, long long* nodes, int* status) {
  if (!S.started) return fail(BNB_EINVAL, "bnb_solve_start was not called");
  bnb_progress pr{};
  if (int rc = solve_poll(h, e, S, &pr)) return rc;
  if (beta_out)
    BNB_CUDA_OK(cudaMemcpy(beta_out, e.inc_beta, sizeof(double) * e.p, cudaMemcpyDeviceToHost));
  if (ub) *ub = pr.ub;
  if (lb) *lb = pr.lb;
  if (nodes) *nodes = pr.nodes;
  if (status) *status = S.done ? S.status : BNB_STATUS_TIME_LIMIT;
  bnb_stats& st = h->stats;
  st.nodes = pr.nodes;
  st.rounds = pr.rounds;
  st.admm_iters = pr.rounds * h->opt.check_every;
  st.pruned = S.last.pruned;
  st.ub_polished = S.last.polished;
  st.pool_peak = e.pool_peak;
  st.max_depth = e.max_depth;
  st.final_ub = pr.ub;
  st.final_lb = pr.lb;
  st.solve_seconds = pr.seconds;
  if (S.exec) {
    cudaGraphExecDestroy(S.exec);
    S.exec = nullptr;
  }
  S.started = false;
  return 0;
}

static SolveState& state_of(bnb_handle* h) {
  if (!h->solve) h->solve = new SolveState();
  return *h->solve;
}

extern "C" int bnb_solve_start(bnb_handle* h, double rel_gap) {
  if (!h) return fail(BNB_EINVAL, "handle is NULL");
  if (!(rel_gap >= 0.0) || rel_gap >= 1.0) return set_err(h, fail(BNB_EINVAL, "rel_gap must be in [0, 1)"));
  return dispatch(h, [&](auto& e) -> int { return solve_start(h, e, state_of(h), rel_gap); });
}

extern "C" int bnb_solve_launch(bnb_handle* h, int rounds) {
  if (!h) return fail(BNB_EINVAL, "handle is NULL");
  if (rounds < 0) return set_err(h, fail(BNB_EINVAL, "rounds must be >= 0"));
  return dispatch(h, [&](auto& e) -> int { return solve_launch(h, e, state_of(h), rounds); });
}

extern "C" int bnb_solve_poll(bnb_handle* h, bnb_progress* out) {
  if (!h) return fail(BNB_EINVAL, "handle is NULL");
  return dispatch(h, [&](auto& e) -> int { return solve_poll(h, e, state_of(h), out); });
}

extern "C" int bnb_solve_finish(bnb_handle* h, double* beta_out, double* ub, double* lb,
                                long long* nodes, int* status) {
  if (!h) return fail(BNB_EINVAL, "handle is NULL");
  return dispatch(h, [&](auto& e) -> int {
    return solve_finish(h, e, state_of(h), beta_out, ub, lb, nodes, status);
  });
}

extern "C" int bnb_solve(bnb_handle* h, double rel_gap, double* beta_out, double* ub, double* lb,
                         long long* nodes, int* status) {
  if (int rc = bnb_solve_start(h, rel_gap)) return rc;
  bnb_progress pr{};
  while (true) {
    if (int rc = bnb_solve_launch(h, 1)) return rc;
    if (int rc = bnb_solve_poll(h, &pr)) return rc;
    if (pr.done) break;
  }
  return bnb_solve_finish(h, beta_out, ub, lb, nodes, status);
}

extern "C" int bnb_profile_round(bnb_handle* h, double* stage_ms, int* stage_launches, int nstages) {
  if (!h || !stage_ms || !stage_launches) return fail(BNB_EINVAL, "NULL argument");
  return dispatch(h, [&](auto& e) -> int {
    if (!state_of(h).started) return fail(BNB_EINVAL, "bnb_solve_start was not called");
    return profile_round(h, e, stage_ms, stage_launches, nstages);
  });
}

extern "C" int bnb_root_heuristic(bnb_handle* h, double* beta_out, double* ub_out) {
  if (!h) return fail(BNB_EINVAL, "handle is NULL");
  return dispatch(h, [&](auto& e) -> int {
    double inf = INFINITY;
    BNB_CUDA_OK(cudaMemcpyAsync(e.inc_ub, &inf, sizeof(double), cudaMemcpyHostToDevice, e.st));
    BNB_CUDA_OK(cudaMemsetAsync(e.inc_beta, 0, sizeof(double) * e.p, e.st));
    if (int rc = root_heuristic(e, mp_moves(e))) return rc;
    if (beta_out)
      BNB_CUDA_OK(cudaMemcpyAsync(beta_out, e.inc_beta, sizeof(double) * e.p, cudaMemcpyDeviceToHost, e.st));
    if (ub_out) BNB_CUDA_OK(cudaMemcpyAsync(ub_out, e.inc_ub, sizeof(double), cudaMemcpyDeviceToHost, e.st));
    BNB_CUDA_OK(cudaStreamSynchronize(e.st));
    return 0;
  });
}

extern "C" void* bnb_stream(const bnb_handle* h) {
  if (!h) return nullptr;
  return h->ef ? (void*)h->ef->st : (h->ed ? (void*)h->ed->st : nullptr);
}

template <class R>
static int read_histograms(Engine<R>& e, long long* depth_hist, int ndepth,
                           long long* support_hist, int nsupport) {
  std::vector<int> d(e.dmax + 1), s(e.smax + 2);
  BNB_CUDA_OK(cudaMemcpyAsync(d.data(), e.hist_depth, sizeof(int) * d.size(),
                              cudaMemcpyDeviceToHost, e.st));
  BNB_CUDA_OK(cudaMemcpyAsync(s.data(), e.hist_sup, sizeof(int) * s.size(),
                              cudaMemcpyDeviceToHost, e.st));
  BNB_CUDA_OK(cudaStreamSynchronize(e.st));
  for (int i = 0; i < ndepth; ++i) depth_hist[i] = i < (int)d.size() ? d[i] : 0;
  for (int i = 0; i < nsupport; ++i) support_hist[i] = i < (int)s.size() ? s[i] : 0;
  return BNB_OK;
}

extern "C" int bnb_get_histograms(bnb_handle* h, long long* depth_hist, int ndepth,
                                  long long* support_hist, int nsupport) {
  if (!h || (!depth_hist && ndepth > 0) || (!support_hist && nsupport > 0) || ndepth < 0 ||
      nsupport < 0)
    return fail(BNB_EINVAL, "bad histogram arguments");
  int rc = h->ef ? read_histograms(*h->ef, depth_hist, ndepth, support_hist, nsupport)
                 : read_histograms(*h->ed, depth_hist, ndepth, support_hist, nsupport);
  return set_err(h, rc);
}

template <class R>
static int read_node_log(Engine<R>& e, int max_entries, int8_t* fix, double* r, double* rec,
                         int* count) {
  int c = 0;
  if (e.log_count) {
    BNB_CUDA_OK(cudaMemcpyAsync(&c, e.log_count, sizeof(int), cudaMemcpyDeviceToHost, e.st));
    BNB_CUDA_OK(cudaStreamSynchronize(e.st));
  }
  *count = c;
  const long long m = c < max_entries ? c : max_entries;
  if (m <= 0) return BNB_OK;
  if (fix) BNB_CUDA_OK(cudaMemcpyAsync(fix, e.log_fix, (size_t)m * e.p, cudaMemcpyDeviceToHost, e.st));
  if (r) BNB_CUDA_OK(cudaMemcpyAsync(r, e.log_r, sizeof(double) * m * e.n, cudaMemcpyDeviceToHost, e.st));
  if (rec)
    BNB_CUDA_OK(cudaMemcpyAsync(rec, e.log_rec, sizeof(double) * m * LOG_REC,
                                cudaMemcpyDeviceToHost, e.st));
  BNB_CUDA_OK(cudaStreamSynchronize(e.st));
  return BNB_OK;
}

extern "C" int bnb_get_node_log(bnb_handle* h, int max_entries, int8_t* fix, double* r,
                                double* rec, int* count) {
  if (!h || !count || max_entries < 0) return fail(BNB_EINVAL, "bad node-log arguments");
  return dispatch(h, [&](auto& e) -> int { return read_node_log(e, max_entries, fix, r, rec, count); });
}

extern "C" int bnb_get_stats(const bnb_handle* h, bnb_stats* out) {
  if (!h || !out) return fail(BNB_EINVAL, "NULL argument");
  *out = h->stats;
  return BNB_OK;
}
