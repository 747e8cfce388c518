// cert.cu -- FP64 dual certificate of Proposition 1 for retired node slots.
//
//   LB(r) = -1/2 ||r||^2 + y^T r - sum_i nu_i(|X_i^T r|),   r = y - X b   (Eqs. dual, nudef)
// is a valid lower bound for EVERY r (Proposition 1.1), so r may come from
// low-precision iterations; the bound itself is evaluated in FP64 on the
// caller's FP64 data.
//
// B300 has little FP64 throughput, so the p products X_i^T r are not all taken
// in FP64.  A screening product a_i = fl32(X32_i^T r32) runs on CUDA cores in
// FP32 (one rounding per fused multiply-add, blocked summation), and
//   |a_i - X_i^T r| <= e_i = (gamma_d (1+u)^2 + 2u(1+u)) ||X_i|| ||r|| (1 + 1e-3),
//   u = 2^-24, gamma_d = d u / (1 - d u)
// (standard bound for a sum of products in which no product meets more than d
// roundings, Higham, "Accuracy and Stability of Numerical Algorithms", Secs. 3.1 and
// 4.2, plus the rounding of X and r to FP32, and Cauchy-Schwarz; d is the depth of the
// blocked sum plus two, screen_depth(n) + 2, about 37 + n / 128).  For a free
// coordinate nu_i(x) = 0 exactly when x <= x0
// (x0 = 2 sqrt(l0 l2), or l0/M + l2 M in the linear regime), so |a_i| + e_i <= x0
// proves the term is zero.  An F1 coordinate (nu_i = h) and a free coordinate the
// screen cannot settle have |X_i^T r| in [|a_i| - e_i, |a_i| + e_i]; both nu_i are
// nondecreasing in |x|, so nu_i(|a_i| + e_i) bounds the term from above and
// nu_i(|a_i| - e_i) from below.  During a solve the bound with the upper values is kept
// whenever the exact FP64 terms could not change the prune decision (k_cert_decide);
// otherwise, and always for bnb_relax_batch and bnb_dual_bound, those coordinates get
// their X_i^T r in FP64.  F0 terms are zero.  The FP64 path (R = double) screens in
// FP64 with u = 2^-53 and d = n + 2.
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
  double* __restrict__ cpart;   // [2][nbm][K]: sum nu(|a|+e), sum nu(|a|+e) - nu(|a|-e)
  Prob P;
  double errc, x0;
  long long p;
  int nbm, K;
  template <int TM, int TN, int TX, int TY>
  __device__ __forceinline__ void apply(R (&acc)[TM][TN], int m0, int n0, int tm, int tn, int M,
                                        int N) const {
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int q = n0 + tn + j * TY;
      const bool col = q < N && ret_active[q];
      double su = 0.0, ss = 0.0;
      if (col) {
        const long long slot = ret_slot[q];
        const double rn = cert_rn[q];
#pragma unroll
        for (int i = 0; i < TM; ++i) {
          const int m = m0 + tm + i * TX;
          if (m >= M) continue;
          const int f = fix[slot * p + m];
          const double a = (double)acc[i][j];
          const double e = errc * xnorm[m] * rn + 1e-30;
          uint8_t need = 0;
          if (f == 1 || (f == -1 && fabs(a) + e > x0)) {
            // F1 (nu = h) or a free coordinate the screen cannot settle: both terms are
            // nondecreasing in |X_i^T r|, so they enter through their rigorous interval
            need = f == 1 ? 1 : 2;
            const double up = nu_coord<double>(fabs(a) + e, f, P);
            const double lo = nu_coord<double>(fmax(0.0, fabs(a) - e), f, P);
            su += up;
            ss += up - lo;
          }
          gscr[(long long)q * p + m] = (float)a;
          cflag[(long long)q * p + m] = need;
        }
      }
#pragma unroll
      for (int o = TX / 2; o > 0; o >>= 1) {
        su += __shfl_xor_sync(0xffffffffu, su, o);
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
      }
      if (tm == 0 && col) {
        cpart[(long long)blockIdx.x * K + q] = su;
        cpart[((long long)nbm + blockIdx.x) * K + q] = ss;
      }
    }
  }
};

// Screening product of the FP32 engine, a[q][m] = fl32(X32_m^T r32_q) for the retired
// columns q < R, followed by the EpiScreen bookkeeping.  The shape is tall and skinny
// (p features x a few dozen retired nodes, contraction n), so the tiles are 32 x 32
// (about one tile per SM at R <= 32) and the contraction is split over the four 64-thread
// groups of a CTA (4 x 4 outputs per thread, 32-wide k steps); the four partial sums are
// added in a fixed order, so the result does not depend on scheduling.  The operand tiles
// stream through SC_NS shared-memory stages by cp.async (16-byte copies when n is a
// multiple of 4, else 4-byte ones), so SC_NS - 1 k steps are in flight while one is
// multiplied: with one CTA per SM a single step in flight left the kernel waiting on memory.
//
// The summation is blocked (Higham, Sec. 4.2): each 32-wide k step is accumulated from
// zero (SC_BK fused multiply-adds) and then added to the thread's running total, so a
// product passes through at most SC_BK + (k steps of its group) + SC_G - 1 roundings
// instead of n + SC_G - 1, and the bound of Sec. 3.1 holds with gamma of that depth
// (screen_depth); at n = 1000 that is 43 instead of 1003.
constexpr int SC_BM = 32, SC_BN = 32, SC_BK = 32, SC_G = 4, SC_LD = SC_BK + 4, SC_NS = 3;
constexpr int SC_STAGE_FLOATS = 2 * SC_G * SC_BM * SC_LD;
constexpr int SC_SMEM = SC_NS * SC_STAGE_FLOATS * (int)sizeof(float);

// the most roundings a product meets in k_screen32 at contraction length n
inline int screen_depth(int n) {
  const int nk = (n + SC_BK - 1) / SC_BK, per = (nk + SC_G - 1) / SC_G;
  return SC_BK + per + SC_G - 1;
}

__device__ __forceinline__ void cp_async16(float* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src),
               "r"(valid ? 16 : 0)
               : "memory");
}

__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src),
               "r"(valid ? 4 : 0)
               : "memory");
}

template <bool VEC>
__global__ void __launch_bounds__(256, 2) k_screen32(const float* __restrict__ X32, int n, int p,
                                                     const float* __restrict__ rS,
                                                     const int* __restrict__ ret_count,
                                                     EpiScreen<float> epi) {
  // SC_NS stages of operand tiles [stage][A|B][group][row][k]; after the k loop the first
  // bytes hold the four partial tiles
  extern __shared__ __align__(16) float sm[];
  static_assert(SC_G * SC_BM * (SC_BN + 1) <= SC_STAGE_FLOATS, "partial tiles fit");
  auto As = [&](int st, int g, int r) { return sm + st * SC_STAGE_FLOATS + (g * SC_BM + r) * SC_LD; };
  auto Bs = [&](int st, int g, int r) {
    return sm + st * SC_STAGE_FLOATS + ((SC_G + g) * SC_BM + r) * SC_LD;
  };
  auto red = reinterpret_cast<float(*)[SC_BM][SC_BN + 1]>(sm);
  const int R = *ret_count;
  const int q0 = blockIdx.y * SC_BN, m0 = blockIdx.x * SC_BM;
  if (q0 >= R) return;
  const int g = threadIdx.x >> 6, t = threadIdx.x & 63;
  const int tx = t & 7, ty = t >> 3;            // rows tx + 8i, columns ty + 8j
  const int nk = (n + SC_BK - 1) / SC_BK;
  const int per = (nk + SC_G - 1) / SC_G;
  const int kb0 = g * per;
  // copies of k step kb of this group into stage st (zero-filled outside the operands)
  auto issue = [&](int kb, int st) {
    const int k0 = kb * SC_BK;
    const bool live = kb < nk;
    if constexpr (VEC) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int e = t + 64 * i, rr = e >> 3, kk = (e & 7) * 4;
        const int k = k0 + kk, m = m0 + rr, q = q0 + rr;
        const bool va = live && k < n && m < p, vb = live && k < n && q < R;
        cp_async16(As(st, g, rr) + kk, va ? X32 + (long long)m * n + k : X32, va);
        cp_async16(Bs(st, g, rr) + kk, vb ? rS + (long long)q * n + k : rS, vb);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int e = t + 64 * i, kk = e & 31, rr = e >> 5;
        const int k = k0 + kk, m = m0 + rr, q = q0 + rr;
        const bool va = live && k < n && m < p, vb = live && k < n && q < R;
        cp_async4(As(st, g, rr) + kk, va ? X32 + (long long)m * n + k : X32, va);
        cp_async4(Bs(st, g, rr) + kk, vb ? rS + (long long)q * n + k : rS, vb);
      }
    }
  };
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll
  for (int st = 0; st < SC_NS - 1; ++st) {
    if (st < per) issue(kb0 + st, st);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  for (int it = 0; it < per; ++it) {
    // this thread's copies of step `it` are done; the barrier makes everyone's visible and
    // retires step it - 1, whose stage the next copies overwrite
    asm volatile("cp.async.wait_group %0;" ::"n"(SC_NS - 2) : "memory");
    __syncthreads();
    if (it + SC_NS - 1 < per) issue(kb0 + it + SC_NS - 1, (it + SC_NS - 1) % SC_NS);
    asm volatile("cp.async.commit_group;" ::: "memory");
    const int st = it % SC_NS;
    float c[4][4];                                // this k step, from zero
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) c[i][j] = 0.f;
#pragma unroll
    for (int k4 = 0; k4 < SC_BK; k4 += 4) {
      float4 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = *(const float4*)(As(st, g, tx + 8 * i) + k4);
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = *(const float4*)(Bs(st, g, ty + 8 * j) + k4);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          c[i][j] = fmaf(a[i].x, b[j].x, c[i][j]);
          c[i][j] = fmaf(a[i].y, b[j].y, c[i][j]);
          c[i][j] = fmaf(a[i].z, b[j].z, c[i][j]);
          c[i][j] = fmaf(a[i].w, b[j].w, c[i][j]);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] += c[i][j];
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();                                // every stage read before red overwrites it
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) red[g][tx + 8 * i][ty + 8 * j] = acc[i][j];
  __syncthreads();
  // epilogue: warp w takes columns w, w + 8, w + 16, w + 24; lane = row
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int m = m0 + lane;
  const double xn = m < p ? epi.xnorm[m] : 0.0;
#pragma unroll 1
  for (int j = 0; j < 4; ++j) {
    const int qq = w + 8 * j, q = q0 + qq;
    if (q >= R) break;
    const float a32 = ((red[0][lane][qq] + red[1][lane][qq]) + red[2][lane][qq]) + red[3][lane][qq];
    double su = 0.0, ss = 0.0;
    if (m < p) {
      const long long slot = epi.ret_slot[q];
      const int f = epi.fix[slot * epi.p + m];
      const double a = (double)a32;
      const double e = epi.errc * xn * epi.cert_rn[q] + 1e-30;
      uint8_t need = 0;
      if (f == 1 || (f == -1 && fabs(a) + e > epi.x0)) {
        need = f == 1 ? 1 : 2;                    // F1, or free and not settled
        const double up = nu_coord<double>(fabs(a) + e, f, epi.P);
        const double lo = nu_coord<double>(fmax(0.0, fabs(a) - e), f, epi.P);
        su = up;
        ss = up - lo;
      }
      epi.gscr[(long long)q * epi.p + m] = a32;
      epi.cflag[(long long)q * epi.p + m] = need;
    }
    su = warp_sum(su);
    ss = warp_sum(ss);
    if (lane == 0) {
      epi.cpart[(long long)blockIdx.x * epi.K + q] = su;
      epi.cpart[((long long)epi.nbm + blockIdx.x) * epi.K + q] = ss;
    }
  }
}

// sum over the flagged coordinates with cflag == code of nu_i(|X_i^T r|), exact FP64,
// in a fixed order: p is taken in chunks of blockDim coordinates; each chunk's flagged
// coordinates are listed in increasing index (ballot compaction), warp w takes list
// entries w, w + nw, ... (one FP64 dot product per warp, lanes over the n samples);
// per-warp sums are combined in warp order at the end.
__device__ double exact_terms(const double* __restrict__ X64, const double* __restrict__ r,
                              const int8_t* __restrict__ fixrow, const uint8_t* __restrict__ flags,
                              int n, int i_beg, int i_end, const Prob& P, int code, int* list,
                              int* wcnt, int* cnt, double* wacc) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double nu_w = 0.0;
  for (int i0 = i_beg; i0 < i_end; i0 += blockDim.x) {
    const int i = i0 + threadIdx.x;
    const int f = (i < i_end) ? (flags[i] == code) : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wcnt[w] = __popc(bal);
    __syncthreads();
    int off = 0;
    for (int t = 0; t < w; ++t) off += wcnt[t];
    if (f) list[off + __popc(bal & ((1u << lane) - 1u))] = i;
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int t = 0; t < nw; ++t) tot += wcnt[t];
      *cnt = tot;
    }
    __syncthreads();
    const int c_n = *cnt;
    for (int t = w; t < c_n; t += nw) {
      const int c = list[t];
      const double* x = X64 + (long long)c * n;
      double d0 = 0.0, d1 = 0.0;            // two chains: more loads in flight
      int k = lane;
      for (; k + 32 < n; k += 64) {
        d0 = fma(x[k], r[k], d0);
        d1 = fma(x[k + 32], r[k + 32], d1);
      }
      if (k < n) d0 = fma(x[k], r[k], d0);
      const double d = warp_sum(d0 + d1);
      nu_w += nu_coord<double>(fabs(d), fixrow[c], P);
    }
    __syncthreads();
  }
  if (lane == 0) wacc[w] = nu_w;
  __syncthreads();
  double s = 0.0;
  for (int t = 0; t < nw; ++t) s += wacc[t];
  __syncthreads();
  return s;
}

// The bound of each retired node, base = -1/2 ||r||^2 + y^T r minus the nu terms:
//   k_cert_decide          LB_cheap = base - sum nu(|a| + e) over the F1 and unsettled free
//                          coordinates (rigorous upper values from the screen); when a
//                          prune threshold is given and LB_cheap already reaches it, or
//                          even LB_cheap plus the total interval width cannot reach it, the
//                          exact terms cannot change the decision and LB_cheap (a valid
//                          bound) is final; otherwise the node is marked;
//   k_cert_terms (code 1)  exact FP64 terms of the F1 coordinates of marked nodes, and
//   k_cert_terms (code 2)  of their unsettled free coordinates, each node spread over
//                          CX_G blocks (one per slice of p);
//   k_cert_final           LB = (base - F1 terms) - free terms for the marked nodes.
// Every sum is taken in a fixed order (slices in order, warps in order inside a slice).
constexpr int CX_G = 8;

__global__ void __launch_bounds__(256) k_cert_terms(const double* __restrict__ X64,
                                                    const double* __restrict__ r64,
                                                    const int8_t* __restrict__ fix,
                                                    const uint8_t* __restrict__ cflag, int n, int p,
                                                    Prob P, const int* __restrict__ ret_slot,
                                                    const int* __restrict__ ret_count, int code,
                                                    const uint8_t* __restrict__ need,
                                                    double* __restrict__ part) {
  __shared__ int list[256];
  __shared__ int wcnt[8];
  __shared__ int cnt;
  __shared__ double wacc[8];
  const int q = blockIdx.x, g = blockIdx.y;
  if (q >= *ret_count) return;
  if (need != nullptr && !need[q]) return;
  const int slot = ret_slot[q];
  const int per = (p + CX_G - 1) / CX_G;
  const int i_beg = g * per, i_end = min(p, i_beg + per);
  const double s = exact_terms(X64, r64 + (long long)q * n, fix + (long long)slot * p,
                               cflag + (long long)q * p, n, i_beg, i_end, P, code, list, wcnt,
                               &cnt, wacc);
  if (threadIdx.x == 0) part[(long long)q * CX_G + g] = s;
}

// one warp per retired node
__global__ void k_cert_decide(const double* __restrict__ cpart, int nbm, int K,
                              const int* __restrict__ ret_slot, const int* __restrict__ ret_count,
                              const double* __restrict__ cert_rr, const double* __restrict__ cert_yr,
                              const double* __restrict__ slot_lbp, const double* __restrict__ inc_ub,
                              const double* __restrict__ params, int use_threshold,
                              double* __restrict__ base_out, uint8_t* __restrict__ need,
                              double* __restrict__ cert_lb, double* __restrict__ node_lb,
                              double* __restrict__ width) {
  const int q = blockIdx.x, lane = threadIdx.x;
  if (q >= *ret_count) return;
  double su = 0.0, ss = 0.0;
  for (int b = lane; b < nbm; b += 32) {
    su += cpart[(long long)b * K + q];
    ss += cpart[((long long)nbm + b) * K + q];
  }
  su = warp_sum(su);
  ss = warp_sum(ss);
  if (lane != 0) return;
  const double base = -0.5 * cert_rr[q] + cert_yr[q];
  const double lb = base - su;
  bool exact = true;
  if (use_threshold) {
    // 1: the exact terms only where they can change the prune decision; 2: also for every
    // node that will be branched (its bound is then the exact value at r for its children
    // and the global bound), skipped only for nodes the cheap bound already prunes
    const double thr = inc_ub[0] * (1.0 - params[0]);
    if (lb >= thr || (use_threshold == 1 && lb + ss < thr)) exact = false;
  }
  base_out[q] = base;
  need[q] = exact ? 1 : 0;
  cert_lb[q] = lb;                    // final unless the exact terms follow
  width[q] = exact ? 0.0 : ss;
  const double lp = slot_lbp[ret_slot[q]];
  node_lb[q] = lb > lp ? lb : lp;
}

__global__ void k_cert_final(const int* __restrict__ ret_slot, const int* __restrict__ ret_count,
                             const double* __restrict__ slot_lbp, const double* __restrict__ base,
                             const uint8_t* __restrict__ need, const double* __restrict__ part1,
                             const double* __restrict__ part2, double* __restrict__ cert_lb,
                             double* __restrict__ node_lb, int K) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= K || q >= *ret_count || !need[q]) return;
  double s1 = 0.0, s2 = 0.0;
  for (int g = 0; g < CX_G; ++g) s1 += part1[(long long)q * CX_G + g];
  for (int g = 0; g < CX_G; ++g) s2 += part2[(long long)q * CX_G + g];
  const double lb = (base[q] - s1) - s2;
  cert_lb[q] = lb;
  const double lp = slot_lbp[ret_slot[q]];
  node_lb[q] = lb > lp ? lb : lp;
}

template <class R>
int certify(Engine<R>& e, const double* r_given, bool use_threshold) {
  if (int rc = certify_screen(e, r_given)) return rc;
  return certify_exact(e, use_threshold ? 1 : 0, e.inc_ub);
}

// r = y - U (or the given r) in FP64 and FP32, then the FP32 screen of X^T r with its
// rigorous error bound
template <class R>
int certify_screen(Engine<R>& e, const double* r_given) {
  using C = TileCfg<R>;
  const int n = e.n, p = e.p, K = e.K;
  cudaStream_t st = e.st;
  k_cert_prep<R><<<K, 256, 0, st>>>(e.y64, e.U, r_given, n, e.ret_slot, e.ret_count, e.r64, e.rS,
                                    e.cert_rr, e.cert_yr, e.cert_rn);
  BNB_CUDA_OK(cudaGetLastError());
  const double u = (sizeof(R) == 4) ? 5.9604644775390625e-08 : 1.1102230246251565e-16;
  const double nu_ = (double)((sizeof(R) == 4 ? screen_depth(n) : n) + 2) * u;
  const double gam = nu_ / (1.0 - nu_);
  const double errc = (sizeof(R) == 4 ? (gam * (1 + u) * (1 + u) + 2 * u * (1 + u))
                                      : (gam * (1 + u) * (1 + u) + 2 * u)) * (1.0 + 1e-3);
  const double x0 = e.P.x0;
  const int nbm = (p + (sizeof(R) == 4 ? SC_BM : C::BM) - 1) / (sizeof(R) == 4 ? SC_BM : C::BM);
  const EpiScreen<R> epi{e.fix, e.ret_slot, e.ret_active, e.xnorm, e.cert_rn, e.gscr, e.cflag,
                         e.cpart, e.P, errc, x0, p, nbm, K};
  prof_begin(e.prof, st);
  if constexpr (sizeof(R) == 4) {
    // 16-byte copies need every row of X32 and rS to start on a 16-byte boundary
    const bool vec = n % 4 == 0 && ((uintptr_t)e.X32 & 15) == 0 && ((uintptr_t)e.rS & 15) == 0;
    auto kern = vec ? k_screen32<true> : k_screen32<false>;
    BNB_CUDA_OK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SC_SMEM));
    kern<<<dim3(nbm, (K + SC_BN - 1) / SC_BN), 256, SC_SMEM, st>>>(
        (const float*)e.X32, n, p, (const float*)e.rS, e.ret_count, epi);
    BNB_CUDA_OK(cudaGetLastError());
  } else {
    BNB_CUDA_OK((gemm_simt<R, true, false>(st, (const R*)e.X64, n, p, K, n, 1, e.ret_active,
                                           BPlainK<R>{e.rS, n}, epi)));
  }
  prof_end(e.prof, st, PK_CERT_SCREEN);
  return 0;
}

// the decision per node (against the incumbent *inc), the exact FP64 terms it needs and
// the certified bound
template <class R>
int certify_exact(Engine<R>& e, int use_threshold, const double* inc) {
  using C = TileCfg<R>;
  const int n = e.n, p = e.p, K = e.K;
  cudaStream_t st = e.st;
  const int nbm = (p + (sizeof(R) == 4 ? SC_BM : C::BM) - 1) / (sizeof(R) == 4 ? SC_BM : C::BM);
  prof_begin(e.prof, st);
  const dim3 gx(K, CX_G);
  k_cert_decide<<<K, 32, 0, st>>>(e.cpart, nbm, K, e.ret_slot, e.ret_count, e.cert_rr, e.cert_yr,
                                  e.slot_lbp, inc, e.params_d, use_threshold,
                                  e.cx_base, e.cx_need, e.cert_lb, e.node_lb, e.cert_width);
  k_cert_terms<<<gx, 256, 0, st>>>(e.X64, e.r64, e.fix, e.cflag, n, p, e.P, e.ret_slot,
                                   e.ret_count, 1, e.cx_need, e.cx_part);
  k_cert_terms<<<gx, 256, 0, st>>>(e.X64, e.r64, e.fix, e.cflag, n, p, e.P, e.ret_slot,
                                   e.ret_count, 2, e.cx_need, e.cx_part + (long long)K * CX_G);
  k_cert_final<<<(K + 127) / 128, 128, 0, st>>>(e.ret_slot, e.ret_count, e.slot_lbp, e.cx_base,
                                                e.cx_need, e.cx_part,
                                                e.cx_part + (long long)K * CX_G, e.cert_lb,
                                                e.node_lb, K);
  prof_end(e.prof, st, PK_CERT_EXACT);
  BNB_CUDA_OK(cudaGetLastError());
  return 0;
}

// Node log: the retired nodes of this round, in retirement order, fill the next free
// records (up to log_cap); k_node_log_advance then moves the count.
template <class R>
__global__ void k_node_log(int n, int p, long long cap, const int* __restrict__ log_count,
                           const int* __restrict__ ret_slot, const int* __restrict__ ret_count,
                           const int8_t* __restrict__ fix, const double* __restrict__ r64,
                           const double* __restrict__ cert_lb, const uint8_t* __restrict__ need,
                           const double* __restrict__ width, const double* __restrict__ node_lb,
                           const double* __restrict__ slot_lbp, const double* __restrict__ inc,
                           const double* __restrict__ params, const int* __restrict__ slot_depth,
                           const int* __restrict__ slot_iters, const double* __restrict__ slot_dual,
                           const double* __restrict__ slot_primal, int8_t* __restrict__ log_fix,
                           double* __restrict__ log_r, double* __restrict__ log_rec) {
  const int q = blockIdx.x;
  if (q >= *ret_count) return;
  const long long idx = (long long)*log_count + q;
  if (idx >= cap) return;
  const int slot = ret_slot[q];
  for (int i = threadIdx.x; i < p; i += blockDim.x)
    log_fix[idx * p + i] = fix[(long long)slot * p + i];
  for (int i = threadIdx.x; i < n; i += blockDim.x) log_r[idx * n + i] = r64[(long long)q * n + i];
  if (threadIdx.x == 0) {
    double* rec = log_rec + idx * LOG_REC;
    rec[LOG_LB] = cert_lb[q];
    rec[LOG_EXACT] = need[q] ? 1.0 : 0.0;
    rec[LOG_WIDTH] = width[q];
    rec[LOG_NODE_LB] = node_lb[q];
    rec[LOG_PARENT_LB] = slot_lbp[slot];
    rec[LOG_THRESHOLD] = inc ? inc[0] * (1.0 - params[0]) : INFINITY;
    rec[LOG_DEPTH] = slot_depth[slot];
    rec[LOG_ITERS] = slot_iters[slot];
    rec[LOG_EST_DUAL] = slot_dual[slot];
    rec[LOG_EST_PRIMAL] = slot_primal[slot];
  }
}

__global__ void k_node_log_advance(long long cap, int* __restrict__ log_count,
                                   const int* __restrict__ ret_count) {
  if (threadIdx.x == 0) {
    const long long c = (long long)*log_count + *ret_count;
    *log_count = (int)(c < cap ? c : cap);
  }
}

template <class R>
int node_log(Engine<R>& e, const double* inc) {
  if (e.log_cap <= 0) return 0;
  k_node_log<R><<<e.K, 256, 0, e.st>>>(e.n, e.p, e.log_cap, e.log_count, e.ret_slot, e.ret_count,
                                       e.fix, e.r64, e.cert_lb, e.cx_need, e.cert_width,
                                       e.node_lb, e.slot_lbp, inc, e.params_d, e.slot_depth,
                                       e.slot_iters, e.slot_dual, e.slot_primal, e.log_fix,
                                       e.log_r, e.log_rec);
  k_node_log_advance<<<1, 32, 0, e.st>>>(e.log_cap, e.log_count, e.ret_count);
  BNB_CUDA_OK(cudaGetLastError());
  return 0;
}

template int node_log<float>(Engine<float>&, const double*);
template int node_log<double>(Engine<double>&, const double*);
template int certify<float>(Engine<float>&, const double*, bool);
template int certify<double>(Engine<double>&, const double*, bool);
template int certify_screen<float>(Engine<float>&, const double*);
template int certify_screen<double>(Engine<double>&, const double*);
template int certify_exact<float>(Engine<float>&, int, const double*);
template int certify_exact<double>(Engine<double>&, int, const double*);

}  // namespace bnb
