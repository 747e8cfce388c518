// cert.cu -- FP64 dual certificate of Proposition 1 for retired node slots.
//
//   LB(r) = -1/2 ||r||^2 + y^T r - sum_i nu_i(|X_i^T r|),   r = y - X b   (Eqs. dual, nudef)
// is a valid lower bound for EVERY r (Proposition 1.1), so r may come from
// low-precision iterations; the bound itself is evaluated in FP64 on the
// caller's FP64 data.
//
// B300 has little FP64 throughput, so the p products X_i^T r are not all taken
// in FP64.  A screening product a_i = fl32(X32_i^T r32) runs on CUDA cores in
// FP32 (one rounding per fused multiply-add, K-chunked in order), and
//   |a_i - X_i^T r| <= e_i = (gamma_n (1+u)^2 + 2u(1+u)) ||X_i|| ||r|| (1 + 1e-3),
//   u = 2^-24, gamma_n = n u / (1 - n u)
// (standard bound for a sum of n products, Higham, "Accuracy and Stability of
// Numerical Algorithms", Sec. 3.1, plus the rounding of X and r to FP32, and
// Cauchy-Schwarz).  For a free coordinate nu_i(x) = 0 exactly when x <= x0
// (x0 = 2 sqrt(l0 l2), or l0/M + l2 M in the linear regime), so |a_i| + e_i <= x0
// proves the term is zero.  Every other coordinate (all of F1, and the free
// coordinates the screen cannot settle) gets its X_i^T r in FP64.  F0 terms are
// zero.  The FP64 path (R = double) screens in FP64 with u = 2^-53.
#include <cfloat>
#include "engine.cuh"
#include "gemm_simt.cuh"

namespace bnb {

template <class R>
__global__ void k_cert_prep(const double* __restrict__ y64, const R* __restrict__ U,
                            const double* __restrict__ r_given, int n, const int* __restrict__ ret_slot,
                            const int* __restrict__ ret_count, double* __restrict__ r64,
                            R* __restrict__ rS, double* __restrict__ cert_rr,
                            double* __restrict__ cert_yr, double* __restrict__ cert_rn) {
  __shared__ double sh[32];
  const int q = blockIdx.x;
  if (q >= *ret_count) return;
  const int slot = ret_slot[q];
  const long long rb = (long long)q * n, ub = (long long)slot * n;
  double rr = 0.0, yr = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double r = r_given ? r_given[rb + i] : y64[i] - (double)U[ub + i];
    r64[rb + i] = r;
    rS[rb + i] = (R)r;
    rr = fma(r, r, rr);
    yr = fma(y64[i], r, yr);
  }
  rr = block_sum(rr, sh);
  yr = block_sum(yr, sh);
  if (threadIdx.x == 0) {
    cert_rr[q] = rr;
    cert_yr[q] = yr;
    cert_rn[q] = sqrt(rr);
  }
}

template <class R>
struct EpiScreen {
  const int8_t* __restrict__ fix;
  const int* __restrict__ ret_slot;
  const int* __restrict__ ret_active;
  const double* __restrict__ xnorm;
  const double* __restrict__ cert_rn;
  float* __restrict__ gscr;
  uint8_t* __restrict__ cflag;
  double errc, x0;
  long long p;
  template <int TM, int TN, int TX, int TY>
  __device__ __forceinline__ void apply(R (&acc)[TM][TN], int m0, int n0, int tm, int tn, int M,
                                        int N) const {
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int q = n0 + tn + j * TY;
      if (q >= N || !ret_active[q]) continue;
      const long long slot = ret_slot[q];
      const double rn = cert_rn[q];
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        const int m = m0 + tm + i * TX;
        if (m >= M) continue;
        const int f = fix[slot * p + m];
        const double a = (double)acc[i][j];
        uint8_t need;
        if (f == 0) need = 0;
        else if (f == 1) need = 1;
        else need = (fabs(a) + errc * xnorm[m] * rn + 1e-30 > x0) ? 1 : 0;
        gscr[(long long)q * p + m] = (float)a;
        cflag[(long long)q * p + m] = need;
      }
    }
  }
};

// Exact FP64 terms for the flagged coordinates, then the bound (one block per node).
__global__ void k_cert_exact(const double* __restrict__ X64, const double* __restrict__ r64,
                             const int8_t* __restrict__ fix, const uint8_t* __restrict__ cflag,
                             int n, int p, Prob P, const int* __restrict__ ret_slot,
                             const int* __restrict__ ret_count, const double* __restrict__ cert_rr,
                             const double* __restrict__ cert_yr, const double* __restrict__ slot_lbp,
                             double* __restrict__ cert_lb, double* __restrict__ node_lb) {
  __shared__ int list[256];
  __shared__ int wcnt[8];
  __shared__ int cnt;
  __shared__ double wacc[8];
  const int q = blockIdx.x;
  if (q >= *ret_count) return;
  const int slot = ret_slot[q];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;  // 8 warps
  const double* r = r64 + (long long)q * n;
  double nu_w = 0.0;  // this warp's running sum, taken in a fixed order
  for (int i0 = 0; i0 < p; i0 += blockDim.x) {
    const int i = i0 + threadIdx.x;
    const int f = (i < p) ? cflag[(long long)q * p + i] : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wcnt[w] = __popc(bal);
    __syncthreads();
    int off = 0;
    for (int t = 0; t < w; ++t) off += wcnt[t];
    if (f) list[off + __popc(bal & ((1u << lane) - 1u))] = i;
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int t = 0; t < nw; ++t) tot += wcnt[t];
      cnt = tot;
    }
    __syncthreads();
    for (int t = w; t < cnt; t += nw) {
      const int col = list[t];
      const double* x = X64 + (long long)col * n;
      double d = 0.0;
      for (int k = lane; k < n; k += 32) d = fma(x[k], r[k], d);
      d = warp_sum(d);
      nu_w += nu_coord<double>(fabs(d), fix[(long long)slot * p + col], P);
    }
    __syncthreads();
  }
  if (lane == 0) wacc[w] = nu_w;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int t = 0; t < nw; ++t) s += wacc[t];
    const double lb = -0.5 * cert_rr[q] + cert_yr[q] - s;
    cert_lb[q] = lb;
    const double lp = slot_lbp[slot];
    node_lb[q] = lb > lp ? lb : lp;
  }
}

template <class R>
int certify(Engine<R>& e, const double* r_given) {
  const int n = e.n, p = e.p, K = e.K;
  cudaStream_t st = e.st;
  k_cert_prep<R><<<K, 256, 0, st>>>(e.y64, e.U, r_given, n, e.ret_slot, e.ret_count, e.r64, e.rS,
                                    e.cert_rr, e.cert_yr, e.cert_rn);
  BNB_CUDA_OK(cudaGetLastError());
  const double u = (sizeof(R) == 4) ? 5.9604644775390625e-08 : 1.1102230246251565e-16;
  const double nu_ = (double)(n + 2) * u;
  const double gam = nu_ / (1.0 - nu_);
  const double errc = (sizeof(R) == 4 ? (gam * (1 + u) * (1 + u) + 2 * u * (1 + u))
                                      : (gam * (1 + u) * (1 + u) + 2 * u)) * (1.0 + 1e-3);
  const double x0 = e.P.x0;
  const R* Xs;
  if constexpr (sizeof(R) == 4) Xs = (const R*)e.X32; else Xs = (const R*)e.X64;
  BNB_CUDA_OK((gemm_simt<R, true, false>(
      st, Xs, n, p, K, n, 1, e.ret_active, BPlainK<R>{e.rS, n},
      EpiScreen<R>{e.fix, e.ret_slot, e.ret_active, e.xnorm, e.cert_rn, e.gscr, e.cflag, errc, x0, p})));
  k_cert_exact<<<K, 256, 0, st>>>(e.X64, e.r64, e.fix, e.cflag, n, p, e.P, e.ret_slot, e.ret_count,
                                  e.cert_rr, e.cert_yr, e.slot_lbp, e.cert_lb, e.node_lb);
  BNB_CUDA_OK(cudaGetLastError());
  return 0;
}

template int certify<float>(Engine<float>&, const double*);
template int certify<double>(Engine<double>&, const double*);

}  // namespace bnb
