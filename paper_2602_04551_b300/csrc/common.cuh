// common.cuh -- shared device-side definitions of the branch-and-bound kernels.
//
// Coordinate-wise closed forms of the node relaxation (arxiv 2602.04551):
//   psi_i      Eq. psi (Section 3.1)
//   prox       Eq. minbetalower with the operator T of Eq. Tdef (free coordinates
//              test the regime sqrt(l0/l2) > M first, as in Appendix A.1 case 4)
//   h, nu_i    Eqs. hdef, nudef (Proposition 1)
//   z_i        Appendix A.1 recovery of z from beta
// Fixing codes: -1 free, 0 = F0 (z_i = 0), 1 = F1 (z_i = 1).
#pragma once

#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>
#include <math.h>

#include "bnb.h"

namespace bnb {

// Per-tree scalar parameters, computed once on the host in FP64.
struct Prob {
  int n, p;
  double lam0, lam2, M, rho;
  int linear;        // 1 when sqrt(l0/l2) > M (psi linear on the whole box)
  double ridge_scale;  // rho / (rho + 2 l2)
  double thr_soft;   // 2 sqrt(l0 l2) / rho          (T threshold, regime sqrt(l0/l2) <= M)
  double tau;        // thr_soft + sqrt(l0/l2)        (switch to the ridge branch)
  double thr_lin;    // (l0/M + l2 M) / rho           (T threshold, linear regime)
  double s0;         // sqrt(l0/l2)
  double c_lin;      // l0/M + l2 M                   (slope of psi in the linear regime)
  double c_soft;     // 2 sqrt(l0 l2)                 (slope of psi near 0)
  double x0;         // nu_i(x) = 0 for free i iff x <= x0
  double sqrt_l2_l0; // sqrt(l2/l0) (z recovery), +inf when l0 = 0
  double alpha;      // ADMM over-relaxation (1 = plain)
};

template <class T>
__device__ __forceinline__ T box_soft(T t, T a, T m) {
  // Eq. Tdef: 0 if |t| <= a; (|t| - a) sign(t) if a < |t| <= a + m; m sign(t) otherwise
  T s = fabs(t) - a;
  s = s > T(0) ? s : T(0);
  s = s < m ? s : m;
  return copysign(s, t);
}

template <class T>
__device__ __forceinline__ T prox_coord(T bt, int f, const Prob& P) {
  if (f == 0) return T(0);
  const T M = (T)P.M;
  T ridge = bt * (T)P.ridge_scale;
  ridge = ridge > M ? M : (ridge < -M ? -M : ridge);
  if (f == 1) return ridge;
  if (P.linear) return box_soft<T>(bt, (T)P.thr_lin, M);
  if (fabs(bt) >= (T)P.tau) return ridge;
  return box_soft<T>(bt, (T)P.thr_soft, M);
}

// FP32 copies of the constants the FP32 prox needs, rounded once on the host exactly as
// the (float) conversions inside prox_coord<float> round them, so the two agree bit for
// bit; the hot epilogue then converts nothing.
struct ProbF {
  float rho, irho, alpha, one_minus_alpha, M, ridge_scale, thr_lin, tau, thr_soft;
  int linear;
};

inline ProbF prob_f32(const Prob& P) {
  ProbF f;
  f.rho = (float)P.rho;
  f.irho = 1.0f / f.rho;
  f.alpha = (float)P.alpha;
  f.one_minus_alpha = 1.0f - f.alpha;
  f.M = (float)P.M;
  f.ridge_scale = (float)P.ridge_scale;
  f.thr_lin = (float)P.thr_lin;
  f.tau = (float)P.tau;
  f.thr_soft = (float)P.thr_soft;
  f.linear = P.linear;
  return f;
}

__device__ __forceinline__ float prox_coord_f(float bt, int f, const ProbF& P) {
  if (f == 0) return 0.0f;
  float ridge = bt * P.ridge_scale;
  ridge = ridge > P.M ? P.M : (ridge < -P.M ? -P.M : ridge);
  if (f == 1) return ridge;
  if (P.linear) return box_soft<float>(bt, P.thr_lin, P.M);
  if (fabsf(bt) >= P.tau) return ridge;
  return box_soft<float>(bt, P.thr_soft, P.M);
}

template <class T>
__device__ __forceinline__ T psi_coord(T b, int f, const Prob& P) {
  if (f == 0) return T(0);
  T ab = fabs(b);
  if (f == 1) return (T)P.lam0 + (T)P.lam2 * b * b;
  if (P.linear) return (T)P.c_lin * ab;
  if (ab <= (T)P.s0) return (T)P.c_soft * ab;
  return (T)P.lam0 + (T)P.lam2 * b * b;
}

template <class T>
__device__ __forceinline__ T h_fun(T x, const Prob& P) {
  const T M = (T)P.M, l0 = (T)P.lam0, l2 = (T)P.lam2;
  return x <= T(2) * M * l2 ? x * x / (T(4) * l2) - l0 : M * x - l0 - l2 * M * M;
}

template <class T>
__device__ __forceinline__ T nu_coord(T x, int f, const Prob& P) {
  if (f == 0) return T(0);
  if (f == 1) return h_fun<T>(x, P);
  if (P.linear) {
    T v = (T)P.M * x - (T)P.lam0 - (T)P.lam2 * (T)P.M * (T)P.M;
    return v > T(0) ? v : T(0);
  }
  T v = h_fun<T>(x, P);
  return v > T(0) ? v : T(0);
}

template <class T>
__device__ __forceinline__ T z_coord(T b, int f, const Prob& P) {
  if (f == 0) return T(0);
  if (f == 1) return T(1);
  T ab = fabs(b);
  if (P.lam0 == 0.0) return ab > T(0) ? T(1) : T(0);
  T z1 = ab / (T)P.M, z2 = (T)P.sqrt_l2_l0 * ab;
  T z = z1 > z2 ? z1 : z2;
  return z < T(1) ? z : T(1);
}

// ---------------------------------------------------------------- reductions

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum in a fixed order (deterministic); all threads get the result.
template <class T>
__device__ T block_sum(T v, T* sh /* >= 32 */) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  T t = T(0);
  if (w == 0) {
    t = lane < nw ? sh[lane] : T(0);
    t = warp_sum(t);
    if (lane == 0) sh[0] = t;
  }
  __syncthreads();
  t = sh[0];
  __syncthreads();
  return t;
}

// Order-preserving maps for atomic min over doubles / floats.
__device__ __forceinline__ unsigned long long dkey(double x) {
  unsigned long long u = (unsigned long long)__double_as_longlong(x);
  return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_inv(unsigned long long k) {
  unsigned long long u = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)u);
}
__device__ __forceinline__ unsigned int fkey(float x) {
  unsigned int u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

}  // namespace bnb

#define BNB_CUDA_OK(expr)                                                            \
  do {                                                                               \
    cudaError_t _e = (expr);                                                         \
    if (_e != cudaSuccess) {                                                         \
      ::bnb::set_cuda_error(#expr, _e, __FILE__, __LINE__);                          \
      return BNB_ECUDA;                                                              \
    }                                                                                \
  } while (0)

namespace bnb {
void set_cuda_error(const char* what, cudaError_t e, const char* file, int line);
}
