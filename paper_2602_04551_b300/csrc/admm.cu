// admm.cu -- batched ADMM iterations over the node slots (Sections 3.1-3.2).
//
// Per iteration, for all K slots at once (Eqs. batched_b_update,
// batched_beta_update, beta_update_vector, batched_v_update):
//   W' = rho beta - V                          (formed while loading, never stored)
//   T  = X W'^T                 n x K           contraction over p
//   U' = G^{-1} T               n x K           U = u_c + U' = X b exactly (X (X^T X + rho I)^{-1}
//                                                = (X X^T + rho I)^{-1} X)
//   P  = X^T U'                 p x K           contraction over n, fused epilogue:
//        b    = b_c + (W' - P) / rho           (b = D (c + W'), Woodbury with 1/rho;
//                                               b_c = D c formed once in FP64)
//        bt   = b + V / rho
//        beta = prox(bt)                       (Eq. minbetalower, masks of the fixings)
//        V    = V + rho (b - beta)             (Eq. v_i-update)
//        and per slot: sum psi(beta), sum nu(|rho b_c - P|) (= nu(|X^T r|), r = y - U),
//        ||beta_new - beta_old||^2, ||b - beta_new||^2.
// Every check_every iterations a check product X beta^T gives the primal
// value of Eq. relaxnode2, and the node stop rule (relative primal-dual gap,
// Section 5.1 "BnB Settings") retires slots.  These FP32/FP64 estimates only
// decide when to stop; the bound used for pruning is recomputed in FP64 (cert.cu).
#include "engine.cuh"
#include "gemm_simt.cuh"

namespace bnb {

template <class R>
struct BW {  // B(k = feature j, n = slot) = W'_sj = rho beta_sj - V_sj
  const R* __restrict__ beta;
  const R* __restrict__ V;
  R rho;
  long long p;
  __device__ __forceinline__ R operator()(int k, int n) const {
    long long o = (long long)n * p + k;
    return rho * beta[o] - V[o];
  }
};

template <class R>
struct EpiAdmm {
  const R* __restrict__ bc;     // b_c = D c
  const R* __restrict__ rbc;    // rho b_c = c - X^T u_c
  R* __restrict__ beta;
  R* __restrict__ V;
  const int8_t* __restrict__ fix;
  const int* __restrict__ active;
  R* __restrict__ g3part;  // [4][nbm][K]
  Prob P;
  long long p;
  int nbm, K;
  int stats;   // 1 on the round's last iteration: per-slot stop-test sums
  template <int TM, int TN, int TX, int TY>
  __device__ __forceinline__ void apply(R (&acc)[TM][TN], int m0, int n0, int tm, int tn, int M,
                                        int N) const {
    const R rho = (R)P.rho, irho = R(1) / (R)P.rho;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int n = n0 + tn + j * TY;
      R s_psi = 0, s_nu = 0, s_db = 0, s_pr = 0;
      if (n < N && active[n]) {
#pragma unroll
        for (int i = 0; i < TM; ++i) {
          const int m = m0 + tm + i * TX;
          if (m < M) {
            const long long o = (long long)n * p + m;
            const R bo = beta[o], v = V[o], pp = acc[i][j];
            const int f = fix[o];
            const R w = rho * bo - v;                      // W'
            const R b = bc[m] + (w - pp) * irho;           // b = b_c + D W'
            const R bh = (R)P.alpha * b + (R(1) - (R)P.alpha) * bo;   // over-relaxed b
            const R bt = bh + v * irho;
            const R bn = prox_coord<R>(bt, f, P);
            beta[o] = bn;
            V[o] = v + rho * (bh - bn);
            if (stats) {
              s_psi += psi_coord<R>(bn, f, P);
              s_nu += nu_coord<R>(fabs(rbc[m] - pp), f, P);   // X^T r = rho b_c - P'
              s_db += (bn - bo) * (bn - bo);
              s_pr += (b - bn) * (b - bn);
            }
          }
        }
      }
      if (!stats) continue;
      // the TX (=16) threads sharing tn are 16 consecutive lanes
#pragma unroll
      for (int o = TX / 2; o > 0; o >>= 1) {
        s_psi += __shfl_xor_sync(0xffffffffu, s_psi, o);
        s_nu += __shfl_xor_sync(0xffffffffu, s_nu, o);
        s_db += __shfl_xor_sync(0xffffffffu, s_db, o);
        s_pr += __shfl_xor_sync(0xffffffffu, s_pr, o);
      }
      if (tm == 0 && n < N) {
        const long long base = (long long)blockIdx.x * K + n, q = (long long)nbm * K;
        g3part[base] = s_psi;
        g3part[q + base] = s_nu;
        g3part[2 * q + base] = s_db;
        g3part[3 * q + base] = s_pr;
      }
    }
  }
};

template <class R>
__global__ void k_reduce_splits(const R* __restrict__ part, int S, R* __restrict__ out, int n,
                                int K, const int* __restrict__ active) {
  const long long m = (long long)n * K, zs = m;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < m;
       idx += (long long)gridDim.x * blockDim.x) {
    int s = (int)(idx / n);
    if (!active[s]) continue;
    R acc = part[idx];
    for (int z = 1; z < S; ++z) acc += part[z * zs + idx];
    out[idx] = acc;
  }
}

// U' = sum of split partials, U = u_c + U'; per slot ||y - U||^2 and y^T (y - U)
template <class R>
__global__ void k_finalize_u(const R* __restrict__ Upart, int S, R* __restrict__ U,
                             R* __restrict__ Up, const R* __restrict__ uc,
                             const R* __restrict__ y, int n, int K, const int* __restrict__ active,
                             R* __restrict__ rstat) {
  __shared__ R sh[32];
  const int s = blockIdx.x;
  if (!active[s]) return;
  const long long zs = (long long)n * K, base = (long long)s * n;
  R rr = 0, yr = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    R up = Upart[base + i];
    for (int z = 1; z < S; ++z) up += Upart[z * zs + base + i];
    Up[base + i] = up;
    const R u = uc[i] + up;
    U[base + i] = u;
    R r = y[i] - u;
    rr += r * r;
    yr += y[i] * r;
  }
  rr = block_sum(rr, sh);
  yr = block_sum(yr, sh);
  if (threadIdx.x == 0) {
    rstat[s] = rr;
    rstat[K + s] = yr;
  }
}

// Node stop rule per slot, one warp per slot (8 slots per 256-thread block): the slot's
// partial sums are read lane-strided and added by butterfly shuffles, so no block barrier
// separates the seven sums.
template <class R>
__global__ void k_stop(const R* __restrict__ XBpart, int S, const R* __restrict__ y, int n, int K,
                       const R* __restrict__ g3part, int nbm, const R* __restrict__ rstat,
                       int* __restrict__ slot_active, int* __restrict__ slot_iters,
                       int* __restrict__ slot_retire, double* __restrict__ slot_gap,
                       double* __restrict__ slot_dual, double* __restrict__ slot_primal, int iters,
                       int max_iter, double node_tol, const double* __restrict__ inc_ub,
                       const double* __restrict__ params, int use_inc,
                       const float* __restrict__ tstat, int nbt) {
  const int lane = threadIdx.x & 31;
  const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (s >= K) return;
  if (!slot_active[s]) {
    if (lane == 0) slot_retire[s] = 0;
    return;
  }
  R xr = 0;
  R rs[2] = {0, 0};
  if (tstat) {
    // per-tile column sums of the cluster-reduced products
    R a[3] = {0, 0, 0};
    for (int b = lane; b < nbt; b += 32)
#pragma unroll
      for (int t = 0; t < 3; ++t) a[t] += (R)tstat[((long long)t * nbt + b) * K + s];
    rs[0] = warp_sum(a[0]);
    rs[1] = warp_sum(a[1]);
    xr = warp_sum(a[2]);
  } else {
    const long long zs = (long long)n * K, base = (long long)s * n;
    for (int i = lane; i < n; i += 32) {
      R xb = XBpart[base + i];
      for (int z = 1; z < S; ++z) xb += XBpart[z * zs + base + i];
      R r = y[i] - xb;
      xr += r * r;
    }
    xr = warp_sum(xr);
    rs[0] = rstat[s];
    rs[1] = rstat[K + s];
  }
  R q[4] = {0, 0, 0, 0};
  for (int b = lane; b < nbm; b += 32)
#pragma unroll
    for (int t = 0; t < 4; ++t) q[t] += g3part[((long long)t * nbm + b) * K + s];
#pragma unroll
  for (int t = 0; t < 4; ++t) q[t] = warp_sum(q[t]);
  if (lane == 0) {
    const double primal = 0.5 * (double)xr + (double)q[0];
    const double dual = -0.5 * (double)rs[0] + (double)rs[1] - (double)q[1];
    const double gap = (primal - dual) / fmax(1.0, fabs(primal));
    const int it = slot_iters[s] + iters;
    slot_iters[s] = it;
    slot_gap[s] = gap;
    slot_dual[s] = dual;
    slot_primal[s] = primal;
    int ret = (gap <= node_tol) || (it >= max_iter);
    if (use_inc) {
      const double thr = inc_ub[0] * (1.0 - params[0]);
      if (dual > thr + 1e-12 * fabs(thr)) ret = 1;
      // P(beta) >= the node's relaxation value (beta is feasible for it): a primal estimate
      // clearly below the threshold means no accuracy can prune the node
      if (use_inc == 2 && isfinite(thr) && primal < thr - 10.0 * node_tol * fmax(1.0, fabs(thr)))
        ret = 1;
    }
    slot_retire[s] = ret;
  }
}

// Ordered compaction of retired slots (single block).  Retired slots leave the
// active set; their state stays in place for the certificate and branching.
__global__ void k_retired_list(int K, int* __restrict__ slot_retire, int* __restrict__ slot_active,
                               int* __restrict__ ret_slot, int* __restrict__ ret_active,
                               int* __restrict__ ret_count) {
  __shared__ int wsum[32];
  __shared__ int base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int s0 = 0; s0 < K; s0 += blockDim.x) {
    const int s = s0 + threadIdx.x;
    const int f = (s < K) ? slot_retire[s] : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    const int pre = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    int off = 0;
    for (int t = 0; t < w; ++t) off += wsum[t];
    if (f) {
      ret_slot[base + off + pre] = s;
      slot_active[s] = 0;
      slot_retire[s] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int t = 0; t < nw; ++t) tot += wsum[t];
      base += tot;
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < K; q += blockDim.x) ret_active[q] = q < base ? 1 : 0;
  if (threadIdx.x == 0) *ret_count = base;
}

template <class R>
int admm_round(Engine<R>& e, int iters, int max_iter, double node_tol, int use_inc) {
  using C = TileCfg<R>;
  const int n = e.n, p = e.p, K = e.K;
  cudaStream_t st = e.st;
  const long long nK = (long long)n * K;
  const int red_grid = (int)((nK + 255) / 256 > 4096 ? 4096 : (nK + 255) / 256);
  int S_check = e.s1;
  bool tc = false;
  if constexpr (sizeof(R) == 4) tc = e.tc_mode != 0;
  if (tc) {
    if constexpr (sizeof(R) == 4) {
      if (e.mv_cross > 0) {
        // narrow or wide form, chosen from the active-slot count: on the device inside a
        // captured round (conditional node), else on the host
        if (int rc = act_list(e)) return rc;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        BNB_CUDA_OK(cudaStreamIsCapturing(st, &cs));
        if (cs == cudaStreamCaptureStatusActive) {
          if (int rc = capture_mv_or_tc(e, iters)) return rc;
        } else {
          int a = e.mv_hint;
          if (a < 0) {
            BNB_CUDA_OK(cudaMemcpyAsync(&a, e.act_count, sizeof(int), cudaMemcpyDeviceToHost, st));
            BNB_CUDA_OK(cudaStreamSynchronize(st));
          }
          if (int rc = a <= e.mv_cross ? admm_iterations_mv(e, iters) : admm_iterations_tc(e, iters))
            return rc;
        }
      } else {
        if (int rc = admm_iterations_tc(e, iters)) return rc;
      }
      S_check = e.tc_s1n;
    }
  } else {
    for (int it = 0; it < iters; ++it) {
      // T = X W^T
      prof_begin(e.prof, st);
      BNB_CUDA_OK((gemm_simt<R, false, false>(st, e.XR, n, n, K, p, e.s1, e.slot_active,
                                              BW<R>{e.beta, e.V, (R)e.P.rho, p},
                                              EpiStore<R>{e.Tpart, n, nK})));
      prof_end(e.prof, st, PK_GEMM_XW);
      prof_begin(e.prof, st);
      k_reduce_splits<R><<<red_grid, 256, 0, st>>>(e.Tpart, e.s1, e.T, n, K, e.slot_active);
      prof_end(e.prof, st, PK_REDUCE_T);
      // U = G^{-1} T
      prof_begin(e.prof, st);
      BNB_CUDA_OK((gemm_simt<R, false, false>(st, e.Ginv, n, n, K, n, e.s2, e.slot_active,
                                              BPlainK<R>{e.T, n}, EpiStore<R>{e.Upart, n, nK})));
      prof_end(e.prof, st, PK_GEMM_GT);
      prof_begin(e.prof, st);
      k_finalize_u<R><<<K, 256, 0, st>>>(e.Upart, e.s2, e.U, e.Up, e.ucR, e.yR, n, K,
                                         e.slot_active, e.rstat);
      prof_end(e.prof, st, PK_FINAL_U);
      // P = X^T U, fused b / prox / v epilogue
      prof_begin(e.prof, st);
      BNB_CUDA_OK((gemm_simt<R, true, false>(
          st, e.XR, n, p, K, n, 1, e.slot_active, BPlainK<R>{e.Up, n},
          EpiAdmm<R>{e.bcR, e.rbcR, e.beta, e.V, e.fix, e.slot_active, e.g3part, e.P, p, e.nbm3,
                     K, it + 1 == iters ? 1 : 0})));
      prof_end(e.prof, st, PK_GEMM_XTU);
    }
    // check: X beta^T for the primal value of Eq. relaxnode2
    prof_begin(e.prof, st);
    BNB_CUDA_OK((gemm_simt<R, false, false>(st, e.XR, n, n, K, p, e.s1, e.slot_active,
                                            BPlainK<R>{e.beta, p}, EpiStore<R>{e.XBpart, n, nK})));
    prof_end(e.prof, st, PK_CHECK);
  }
  e.admm_iters += iters;
  prof_begin(e.prof, st);
  k_stop<R><<<(K + 7) / 8, 256, 0, st>>>(e.XBpart, S_check, e.yR, n, K, e.g3part, e.nbm3, e.rstat,
                               e.slot_active, e.slot_iters, e.slot_retire, e.slot_gap, e.slot_dual,
                               e.slot_primal, iters, max_iter, node_tol, e.inc_ub, e.params_d,
                               use_inc, e.tc_c1 > 0 ? e.tc_stat : nullptr, e.nbt);
  k_retired_list<<<1, 1024, 0, st>>>(K, e.slot_retire, e.slot_active, e.ret_slot, e.ret_active,
                                     e.ret_count);
  prof_end(e.prof, st, PK_STOP);
  BNB_CUDA_OK(cudaGetLastError());
  (void)C::BM;
  return 0;
}

template int admm_round<float>(Engine<float>&, int, int, double, int);
template int admm_round<double>(Engine<double>&, int, int, double, int);

}  // namespace bnb
