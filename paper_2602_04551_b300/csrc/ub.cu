// ub.cu -- branching choice and upper bounds for retired node slots.
//
// Branch pick (Algorithm 1 "Select j"; reading: most fractional z_i, ties to the
// lowest index; z from beta by Appendix A.1).  When every free z_i is integral the
// free index with the largest |X_i^T r| is taken.  A node with no free index is a
// leaf (-1).
// Rounding (Section 3.3): S = F1 + {free i : z_i >= 1/2}.
// Upper bound on S (Eq. upperboundbeta), batched over nodes (Section 3.4):
//   accelerated projected gradient with extrapolation t/(t+3) (Eq. fpg_extrapolate),
//   gradient of Eq. fpg_grad, projected step (Eq. fpg_step) and per-node step
//   size alpha shrunk by 1/2 until the Armijo test of Eq. fpg_armijo holds.
//   It runs on the Gram form: with Q = X_S^T X_S + 2 lambda2 I and q = X_S^T y,
//   U_S(beta) = 1/2 y^T y - q^T beta + 1/2 beta^T Q beta and grad = Q beta - q,
//   the same iterates as the X_S matvec form at s^2 instead of 2ns work per step.
// Every candidate is then evaluated in FP64 on the FP64 data (Eq. original with
// lambda0 per nonzero): the value of a feasible point, hence a valid upper bound.
// Candidates that may improve the incumbent are re-solved exactly in FP64 on S
// (feasible primal active-set method for the bound-constrained strictly convex
// QP, Nocedal and Wright, Numerical Optimization, Algorithm 16.3, with dense
// Cholesky solves), so the incumbent is accurate to FP64 rounding.
#include "engine.cuh"

namespace bnb {

__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}

__device__ unsigned long long block_max_u64(unsigned long long v, unsigned long long* sh) {
  for (int o = 16; o > 0; o >>= 1) v = umax64(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = 0;
    for (int t = 0; t < nw; ++t) m = umax64(m, sh[t]);
    sh[0] = m;
  }
  __syncthreads();
  unsigned long long r = sh[0];
  __syncthreads();
  return r;
}

// Order-independent 64-bit key of a support set: the sum (mod 2^64) of a splitmix64-style
// mix of each index (a published integer hash finalizer, Steele, Lea and Flood, OOPSLA 2014).
__device__ __forceinline__ unsigned long long support_mix(int i) {
  unsigned long long z = (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (int t = 0; t < nw; ++t) s += sh[t];
    sh[0] = s;
  }
  __syncthreads();
  const unsigned long long r = sh[0];
  __syncthreads();
  return r;
}

// Open-addressed set of support keys (0 = empty slot; key 0 is mapped to 1): true when the
// key was present, else inserted (or the probe sequence is full: treated as new).
__device__ bool support_seen(unsigned long long* table, int mask, unsigned long long key) {
  if (key == 0) key = 1;
  unsigned idx = (unsigned)(key ^ (key >> 32)) & (unsigned)mask;
  for (int probe = 0; probe < 16; ++probe) {
    const unsigned long long cur = atomicCAS(&table[idx], 0ull, key);
    if (cur == 0ull) return false;      // inserted here
    if (cur == key) return true;        // already evaluated
    idx = (idx + 1) & (unsigned)mask;
  }
  return false;
}

// one block (1024 threads) per retired node.  Without gscr (the screened X^T r) a node whose
// free z are all integral gets br_idx = BR_DEFERRED, decided later by k_branch_fallback.
constexpr int BR_DEFERRED = -3;

template <class R>
__global__ void k_branch_support(const R* __restrict__ beta, const int8_t* __restrict__ fix,
                                 const float* __restrict__ gscr, int p, Prob P,
                                 const int* __restrict__ ret_slot, const int* __restrict__ ret_count,
                                 int smax, int* __restrict__ br_idx, int* __restrict__ sup,
                                 int* __restrict__ sup_cnt, int* __restrict__ nfree,
                                 float* __restrict__ zbuf, unsigned long long* __restrict__ seen,
                                 int seen_mask, int* __restrict__ sup_size) {
  __shared__ unsigned long long shk[32];
  __shared__ int wcnt[32];
  __shared__ double shd[32];
  const int q = blockIdx.x;
  if (q >= *ret_count) return;
  const long long slot = ret_slot[q];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // warp w takes the contiguous range [i_beg, i_end) of the p indices, so the support list
  // (increasing index) is the warps' lists in warp order: one pass counts, a barrier and a
  // prefix over the 32 counts give each warp its offset, and a second pass writes
  const int C = ((p + nw - 1) / nw + 31) & ~31;
  const int i_beg = min(p, w * C), i_end = min(p, i_beg + C);
  auto in_support = [&](int i, float& z, int& f) {
    f = fix[slot * p + i];
    z = (float)z_coord<R>(beta[slot * p + i], f, P);
    return f == -1 ? z >= 0.5f : f == 1;
  };
  unsigned long long kf = 0, kg = 0, hsum = 0;
  int nf = 0, cnt = 0;
  for (int i0 = i_beg; i0 < i_end; i0 += 32) {
    const int i = i0 + lane;
    int insup = 0;
    if (i < i_end) {
      float z;
      int f;
      insup = in_support(i, z, f);
      if (zbuf) zbuf[slot * p + i] = z;
      if (f == -1) {
        ++nf;
        const float fr = fminf(z, 1.0f - z);
        const unsigned long long key =
            ((unsigned long long)__float_as_uint(fr) << 32) | (unsigned)(0x7fffffff - i);
        kf = umax64(kf, key);
        if (gscr) {
          const float g = fabsf(gscr[(long long)q * p + i]);
          const unsigned long long kg2 =
              ((unsigned long long)__float_as_uint(g) << 32) | (unsigned)(0x7fffffff - i);
          kg = umax64(kg, kg2);
        }
      }
    }
    if (insup) hsum += support_mix(i);
    cnt += __popc(__ballot_sync(0xffffffffu, insup));
  }
  if (lane == 0) wcnt[w] = cnt;
  __syncthreads();
  int off = 0, base = 0;
  for (int t = 0; t < nw; ++t) {
    off += t < w ? wcnt[t] : 0;
    base += wcnt[t];
  }
  for (int i0 = i_beg; i0 < i_end && off < smax; i0 += 32) {
    const int i = i0 + lane;
    float z;
    int f;
    const int insup = i < i_end ? in_support(i, z, f) : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, insup);
    const int pos = off + __popc(bal & ((1u << lane) - 1u));
    if (insup && pos < smax) sup[(long long)q * smax + pos] = i;
    off += __popc(bal);
  }
  kf = block_max_u64(kf, shk);
  kg = block_max_u64(kg, shk);
  const unsigned long long hs = block_sum_u64(hsum, shk);
  const double nft = block_sum<double>((double)nf, shd);
  if (threadIdx.x == 0) {
    const int nfi = (int)nft;
    nfree[q] = nfi;
    int j = -1;
    if (nfi > 0) {
      const float fr = __uint_as_float((unsigned)(kf >> 32));
      if (fr > 0.0f || gscr) {
        const unsigned long long k = fr > 0.0f ? kf : kg;
        j = 0x7fffffff - (int)(unsigned)(k & 0xffffffffu);
      } else {
        j = BR_DEFERRED;   // every free z integral: k_branch_fallback decides from |X_i^T r|
      }
    }
    br_idx[q] = j;
    int sc = base <= smax ? base : -1;
    if (sup_size) sup_size[q] = sc;
    // a support whose upper bound was already taken in this solve cannot improve the
    // incumbent: -2 makes the upper-bound kernels skip it (like an oversized one)
    if (seen != nullptr && sc > 0 && support_seen(seen, seen_mask, hs)) sc = -2;
    sup_cnt[q] = sc;
  }
}

// the deferred branching decisions: the free index with the largest |X_i^T r| (screened,
// FP32), ties to the lowest index -- the rule k_branch_support applies when it has gscr
__global__ void k_branch_fallback(const int8_t* __restrict__ fix, const float* __restrict__ gscr,
                                  int p, const int* __restrict__ ret_slot,
                                  const int* __restrict__ ret_count, int* __restrict__ br_idx) {
  __shared__ unsigned long long shk[32];
  const int q = blockIdx.x;
  if (q >= *ret_count || br_idx[q] != BR_DEFERRED) return;
  const long long slot = ret_slot[q];
  unsigned long long kg = 0;
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    if (fix[slot * p + i] != -1) continue;
    const float g = fabsf(gscr[(long long)q * p + i]);
    kg = umax64(kg, ((unsigned long long)__float_as_uint(g) << 32) | (unsigned)(0x7fffffff - i));
  }
  kg = block_max_u64(kg, shk);
  if (threadIdx.x == 0) br_idx[q] = 0x7fffffff - (int)(unsigned)(kg & 0xffffffffu);
}

// Q = X_S^T X_S + 2 lambda2 I, q = X_S^T y in the ADMM precision (one block per node)
template <class R>
__global__ void k_ub_gram(const R* __restrict__ XR, const R* __restrict__ yR, int n, int smax,
                          double lam2, const int* __restrict__ sup, const int* __restrict__ sup_cnt,
                          const int* __restrict__ ret_count, R* __restrict__ Qg, R* __restrict__ qv) {
  const int q = blockIdx.x;
  if (q >= *ret_count) return;
  const int s = sup_cnt[q];
  if (s <= 0) return;
  const int* S = sup + (long long)q * smax;
  R* Q = Qg + (long long)q * smax * smax;
  const int npair = s * (s + 1) / 2;
  // one warp per entry: lanes stride over the n samples, fixed-order butterfly sum
  // the node's entries are spread over the gridDim.y blocks of its row of the grid
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int t = blockIdx.y * nw + w; t < npair + s; t += nw * gridDim.y) {
    if (t < npair) {
      // unrank t -> (a, b), a >= b
      int a = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
      while ((a + 1) * (a + 2) / 2 <= t) ++a;
      while (a * (a + 1) / 2 > t) --a;
      const int b = t - a * (a + 1) / 2;
      const R* xa = XR + (long long)S[a] * n;
      const R* xb = XR + (long long)S[b] * n;
      R d = 0;
#pragma unroll 8
      for (int k = lane; k < n; k += 32) d = fma(xa[k], xb[k], d);
      d = warp_sum(d);
      if (lane == 0) {
        if (a == b) d += (R)(2.0 * lam2);
        Q[a * s + b] = d;
        Q[b * s + a] = d;
      }
    } else {
      const int a = t - npair;
      const R* xa = XR + (long long)S[a] * n;
      R d = 0;
#pragma unroll 8
      for (int k = lane; k < n; k += 32) d = fma(xa[k], yR[k], d);
      d = warp_sum(d);
      if (lane == 0) qv[(long long)q * smax + a] = d;
    }
  }
}

// The projected-gradient iteration of k_ub_fista for a support of at most 32 on one warp:
// lane a holds coordinate a and row a of Q in registers, Q x takes x_b from lane b by
// shuffle (the same products in the same order b = 0, 1, ... as the block form), and the
// sums are butterfly shuffles, which leave the identical value in every lane, so every
// branch below is uniform over the warp.  No block barrier is involved.
template <class R>
__device__ void fista_warp(const R* __restrict__ Q, const R* __restrict__ qq, int s, R M,
                           int max_iter, double rtol, R* __restrict__ out) {
  const int a = threadIdx.x & 31;
  const bool own = a < s;
  R qrow[32];
#pragma unroll
  for (int b = 0; b < 32; ++b) qrow[b] = (own && b < s) ? Q[a * s + b] : R(0);
  const R qa = own ? qq[a] : R(0);
  auto matvec = [&](R x) {
    R v = 0;
#pragma unroll
    for (int b = 0; b < 32; ++b) v = fma(qrow[b], __shfl_sync(0xffffffffu, x, b), v);
    return v;
  };
  R ext = own ? R(1) : R(0);
  R lam = R(1);
  for (int it = 0; it < 12; ++it) {
    const R v = matvec(ext);
    const R nrm2 = warp_sum<R>(v * v);
    const R dot = warp_sum<R>(v * ext);
    const R e2 = warp_sum<R>(ext * ext);
    lam = dot / e2;
    const R inv = R(1) / sqrt(nrm2 > R(0) ? nrm2 : R(1));
    ext = own ? v * inv : R(0);
  }
  R alpha = R(1) / lam;
  R cur = R(0), prev = R(0), fcur = R(0);
  for (int t = 0; t < max_iter; ++t) {
    const R mom = (R)t / (R)(t + 3);
    const R e = own ? cur + mom * (cur - prev) : R(0);
    const R Qe = matvec(e);
    const R g = own ? Qe - qa : R(0);
    const R fext = warp_sum<R>(own ? e * (R(0.5) * Qe - qa) : R(0));
    R fnew = 0, x = 0;
    for (int bt = 0; bt < 40; ++bt) {
      x = own ? e - alpha * g : R(0);
      x = x > M ? M : (x < -M ? -M : x);
      const R Qn = matvec(x);
      const R d = x - e;
      fnew = warp_sum<R>(own ? x * (R(0.5) * Qn - qa) : R(0));
      const R gd = warp_sum<R>(g * d);
      const R dd = warp_sum<R>(d * d);
      const R slack = R(8) * (R)(sizeof(R) == 4 ? 1.2e-7 : 2.3e-16) * (fabs(fext) + R(1));
      if (fnew <= fext + gd + dd / (R(2) * alpha) + slack) break;
      alpha *= R(0.5);
    }
    prev = cur;
    cur = x;
    const bool done = t > 0 && fabs(fcur - fnew) <= (R)rtol * (fabs(fnew) + R(1));
    fcur = fnew;
    if (done) break;
  }
  if (own) out[a] = cur;
}

// Batched projected gradient with t/(t+3) extrapolation and Armijo backtracking.
// One block per node: a support of at most 32 runs on the block's first warp
// (fista_warp), a larger one on the whole block, one thread per support coordinate
// (s <= blockDim.x).
template <class R>
__global__ void k_ub_fista(const R* __restrict__ Qg, const R* __restrict__ qv, int smax, double M_,
                           const int* __restrict__ sup_cnt, const int* __restrict__ ret_count,
                           int max_iter, double rtol, R* __restrict__ ubb) {
  extern __shared__ unsigned char smem_raw[];
  R* sm = reinterpret_cast<R*>(smem_raw);
  __shared__ R red[32];
  const int q = blockIdx.x;
  if (q >= *ret_count) return;
  const int s = sup_cnt[q];
  if (s <= 0) return;
  if (s <= 32) {
    if (threadIdx.x < 32)
      fista_warp<R>(Qg + (long long)q * smax * smax, qv + (long long)q * smax, s, (R)M_,
                    max_iter, rtol, ubb + (long long)q * smax);
    return;
  }
  R* cur = sm;
  R* prev = sm + smax;
  R* ext = sm + 2 * smax;
  R* nw = sm + 3 * smax;
  const R* Q = Qg + (long long)q * smax * smax;
  const R* qq = qv + (long long)q * smax;
  const int a = threadIdx.x;
  const bool own = a < s;
  const R M = (R)M_;
  // step size from a power-iteration estimate of lambda_max(Q); Armijo corrects it
  if (own) ext[a] = R(1);
  __syncthreads();
  R lam = R(1);
  for (int it = 0; it < 12; ++it) {
    R v = 0;
    if (own)
      for (int b = 0; b < s; ++b) v = fma(Q[a * s + b], ext[b], v);
    const R nrm2 = block_sum<R>(own ? v * v : R(0), red);
    const R dot = block_sum<R>(own ? v * ext[a] : R(0), red);
    const R e2 = block_sum<R>(own ? ext[a] * ext[a] : R(0), red);
    lam = dot / e2;
    const R inv = R(1) / sqrt(nrm2 > R(0) ? nrm2 : R(1));
    if (own) ext[a] = v * inv;
    __syncthreads();
  }
  R alpha = R(1) / lam;
  if (own) {
    cur[a] = R(0);
    prev[a] = R(0);
  }
  __syncthreads();
  R fcur = R(0);  // f(beta) = -q^T beta + 1/2 beta^T Q beta (the constant 1/2 y^T y dropped)
  for (int t = 0; t < max_iter; ++t) {
    const R mom = (R)t / (R)(t + 3);
    if (own) ext[a] = cur[a] + mom * (cur[a] - prev[a]);
    __syncthreads();
    R Qe = 0;
    if (own)
      for (int b = 0; b < s; ++b) Qe = fma(Q[a * s + b], ext[b], Qe);
    const R g = own ? Qe - qq[a] : R(0);
    const R fext = block_sum<R>(own ? ext[a] * (R(0.5) * Qe - qq[a]) : R(0), red);
    R fnew = 0;
    for (int bt = 0; bt < 40; ++bt) {
      R x = own ? ext[a] - alpha * g : R(0);
      x = x > M ? M : (x < -M ? -M : x);
      if (own) nw[a] = x;
      __syncthreads();
      R Qn = 0;
      if (own)
        for (int b = 0; b < s; ++b) Qn = fma(Q[a * s + b], nw[b], Qn);
      const R d = own ? x - ext[a] : R(0);
      fnew = block_sum<R>(own ? x * (R(0.5) * Qn - qq[a]) : R(0), red);
      const R gd = block_sum<R>(g * d, red);
      const R dd = block_sum<R>(d * d, red);
      const R slack = R(8) * (R)(sizeof(R) == 4 ? 1.2e-7 : 2.3e-16) * (fabs(fext) + R(1));
      if (fnew <= fext + gd + dd / (R(2) * alpha) + slack) break;
      alpha *= R(0.5);
    }
    if (own) {
      prev[a] = cur[a];
      cur[a] = nw[a];
    }
    __syncthreads();
    const bool done = t > 0 && fabs(fcur - fnew) <= (R)rtol * (fabs(fnew) + R(1));
    fcur = fnew;
    if (done) break;
  }
  if (own) ubb[(long long)q * smax + a] = cur[a];
}

// FP64 value of Eq. original at the candidate.  UE_NB blocks per node (grid K x UE_NB),
// block z taking the samples of its slice of n; each writes its partial ||y - X_S b||^2
// and the last of a node's blocks to finish (counted in ue_cnt, which it resets) adds the
// UE_NB partials in slice order, so the value does not depend on which block ends last.
template <class R>
__global__ void k_ub_eval(const double* __restrict__ X64, const double* __restrict__ y64, int n,
                          int smax, double lam0, double lam2, double M, const int* __restrict__ sup,
                          const int* __restrict__ sup_cnt, const int* __restrict__ ret_count,
                          const R* __restrict__ ubb, double* __restrict__ ubb64,
                          double* __restrict__ ub_val, int* __restrict__ pol_flag,
                          const double* __restrict__ inc_ub, int force, double* __restrict__ part,
                          int* __restrict__ cnt) {
  __shared__ double sh[32];
  __shared__ double bs[256];
  __shared__ int sS[256];
  __shared__ int last;
  const int q = blockIdx.x, z = blockIdx.y, nz = gridDim.y;
  if (q >= *ret_count) return;
  const int s = sup_cnt[q];
  if (s < 0) {
    if (z == 0 && threadIdx.x == 0) {
      ub_val[q] = INFINITY;
      pol_flag[q] = 0;
    }
    return;
  }
  const int* S = sup + (long long)q * smax;
  double* b64 = ubb64 + (long long)q * 2 * smax;
  // the point clipped to the FP64 box: the ADMM-precision clip uses M rounded to that
  // precision, which may lie just outside the box, and the value must be a feasible one
  for (int a = threadIdx.x; a < s; a += blockDim.x) {
    bs[a] = fmin(M, fmax(-M, (double)ubb[(long long)q * smax + a]));
    sS[a] = S[a];
    if (z == 0) b64[a] = bs[a];
  }
  __syncthreads();
  // the support indices come from shared memory, so the s column loads of a sample do not
  // wait on one another; only the FMA chain on r is sequential
  const int chunk = (n + nz - 1) / nz, i0 = z * chunk, i1 = min(n, i0 + chunk);
  double rr = 0.0;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    double r = y64[i];
#pragma unroll 8
    for (int a = 0; a < s; ++a) r = fma(-X64[(long long)sS[a] * n + i], bs[a], r);
    rr = fma(r, r, rr);
  }
  rr = block_sum(rr, sh);
  if (threadIdx.x == 0) {
    part[(long long)q * nz + z] = rr;
    __threadfence();
    last = atomicAdd(&cnt[q], 1) == nz - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double bb = 0.0, nzc = 0.0;
  for (int a = threadIdx.x; a < s; a += blockDim.x) {
    bb = fma(bs[a], bs[a], bb);
    nzc += bs[a] != 0.0 ? 1.0 : 0.0;
  }
  bb = block_sum(bb, sh);
  nzc = block_sum(nzc, sh);
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int t = 0; t < nz; ++t) tot += __ldcg(&part[(long long)q * nz + t]);
    cnt[q] = 0;
    const double v = 0.5 * tot + lam0 * nzc + lam2 * bb;
    ub_val[q] = v;
    // force: 1 polish every candidate, -1 none, 0 those within 1e-6 of the incumbent
    pol_flag[q] = (s > 0) && force >= 0 && (force || v < inc_ub[0] * (1.0 + 1e-6));
  }
}

// dense Cholesky solve A x = b in place (A nf x nf, leading dim nf), one block
__device__ void block_chol_solve(double* A, double* x, int nf) {
  for (int k = 0; k < nf; ++k) {
    if (threadIdx.x == 0) A[k * nf + k] = sqrt(A[k * nf + k]);
    __syncthreads();
    const double d = A[k * nf + k];
    for (int i = k + 1 + threadIdx.x; i < nf; i += blockDim.x) A[i * nf + k] /= d;
    __syncthreads();
    const int m = nf - k - 1;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      const int i = k + 1 + t / m, j = k + 1 + t % m;
      if (j <= i) A[i * nf + j] -= A[i * nf + k] * A[j * nf + k];
    }
    __syncthreads();
  }
  // L y = b
  for (int k = 0; k < nf; ++k) {
    if (threadIdx.x == 0) x[k] /= A[k * nf + k];
    __syncthreads();
    const double xk = x[k];
    for (int i = k + 1 + threadIdx.x; i < nf; i += blockDim.x) x[i] -= A[i * nf + k] * xk;
    __syncthreads();
  }
  // L^T x = y
  for (int k = nf - 1; k >= 0; --k) {
    if (threadIdx.x == 0) x[k] /= A[k * nf + k];
    __syncthreads();
    const double xk = x[k];
    for (int i = threadIdx.x; i < k; i += blockDim.x) x[i] -= A[k * nf + i] * xk;
    __syncthreads();
  }
}

// Exact FP64 box ridge on S by a feasible primal active-set method (one block per node)
__global__ void k_ub_polish(const double* __restrict__ X64, const double* __restrict__ y64, int n,
                            int smax, double lam0, double lam2, double M,
                            const int* __restrict__ sup, const int* __restrict__ sup_cnt,
                            const int* __restrict__ ret_count, const int* __restrict__ pol_flag,
                            double* __restrict__ Q64, double* __restrict__ L64,
                            double* __restrict__ ubb64, double* __restrict__ ub_val,
                            int* __restrict__ n_polished) {
  __shared__ double sh[32];
  __shared__ int Fidx[256];
  __shared__ int W[256];
  __shared__ double bt[256], tgt[256], rhs[256];
  __shared__ int nf_s, state;
  const int q = blockIdx.x;
  if (q >= *ret_count || !pol_flag[q]) return;
  const int s = sup_cnt[q];
  const int* S = sup + (long long)q * smax;
  double* Q = Q64 + (long long)q * smax * smax;
  double* A = L64 + (long long)q * smax * smax;
  double* b64 = ubb64 + (long long)q * 2 * smax;
  double* qv = b64 + smax;
  // Gram and right-hand side in FP64
  const int npair = s * (s + 1) / 2;
  for (int t = threadIdx.x; t < npair + s; t += blockDim.x) {
    if (t < npair) {
      int a = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
      while ((a + 1) * (a + 2) / 2 <= t) ++a;
      while (a * (a + 1) / 2 > t) --a;
      const int b = t - a * (a + 1) / 2;
      const double* xa = X64 + (long long)S[a] * n;
      const double* xb = X64 + (long long)S[b] * n;
      double d = 0.0;
      for (int k = 0; k < n; ++k) d = fma(xa[k], xb[k], d);
      if (a == b) d += 2.0 * lam2;
      Q[a * s + b] = d;
      Q[b * s + a] = d;
    } else {
      const int a = t - npair;
      const double* xa = X64 + (long long)S[a] * n;
      double d = 0.0;
      for (int k = 0; k < n; ++k) d = fma(xa[k], y64[k], d);
      qv[a] = d;
    }
  }
  // feasible start: the projected-gradient point, coordinates on the box held there
  for (int a = threadIdx.x; a < s; a += blockDim.x) {
    double v = b64[a];
    v = v > M ? M : (v < -M ? -M : v);
    int wv = 0;
    if (v >= M * (1.0 - 1e-12)) { wv = 1; v = M; }
    if (v <= -M * (1.0 - 1e-12)) { wv = -1; v = -M; }
    bt[a] = v;
    W[a] = wv;
  }
  __syncthreads();
  double qscale = 0.0;
  for (int a = threadIdx.x; a < s; a += blockDim.x) qscale = fmax(qscale, fabs(qv[a]));
  // block max via sum of a one-hot is awkward; use shared atomics on a key instead
  __shared__ unsigned long long qmax_k;
  if (threadIdx.x == 0) qmax_k = 0;
  __syncthreads();
  atomicMax(&qmax_k, (unsigned long long)__double_as_longlong(qscale));
  __syncthreads();
  qscale = __longlong_as_double((long long)qmax_k);
  const int max_it = 3 * s + 10;
  for (int it = 0; it < max_it; ++it) {
    if (threadIdx.x == 0) {
      int c = 0;
      for (int a = 0; a < s; ++a)
        if (W[a] == 0) Fidx[c++] = a;
      nf_s = c;
    }
    __syncthreads();
    const int nf = nf_s;
    // rhs_F = q_F - Q_{F,W} beta_W ;  A = Q_FF
    for (int t = threadIdx.x; t < nf; t += blockDim.x) {
      const int a = Fidx[t];
      double r = qv[a];
      for (int b = 0; b < s; ++b)
        if (W[b] != 0) r -= Q[a * s + b] * bt[b];
      rhs[t] = r;
    }
    for (int t = threadIdx.x; t < nf * nf; t += blockDim.x)
      A[t] = Q[Fidx[t / nf] * s + Fidx[t % nf]];
    __syncthreads();
    if (nf > 0) block_chol_solve(A, rhs, nf);
    for (int a = threadIdx.x; a < s; a += blockDim.x) tgt[a] = bt[a];
    __syncthreads();
    for (int t = threadIdx.x; t < nf; t += blockDim.x) tgt[Fidx[t]] = rhs[t];
    __syncthreads();
    if (threadIdx.x == 0) {
      double dmax = 0.0;
      for (int a = 0; a < s; ++a) dmax = fmax(dmax, fabs(tgt[a] - bt[a]));
      if (dmax <= 1e-15 * fmax(1.0, M)) {
        // multipliers of the active bounds
        int j = -1;
        double lmin = 0.0;
        for (int a = 0; a < s; ++a) {
          if (W[a] == 0) continue;
          double g = -qv[a];
          for (int b = 0; b < s; ++b) g += Q[a * s + b] * bt[b];
          const double lam = W[a] == 1 ? -g : g;
          if (j < 0 || lam < lmin) { j = a; lmin = lam; }
        }
        if (j < 0 || lmin >= -1e-13 * fmax(1.0, qscale)) state = 1;  // optimal
        else { W[j] = 0; state = 0; }
      } else {
        double alpha = 1.0;
        int blk = -1, dir = 0;
        for (int a = 0; a < s; ++a) {
          if (W[a] != 0) continue;
          const double d = tgt[a] - bt[a];
          if (d == 0.0) continue;
          const double lim = d > 0 ? (M - bt[a]) / d : (-M - bt[a]) / d;
          if (lim < alpha) { alpha = lim; blk = a; dir = d > 0 ? 1 : -1; }
        }
        for (int a = 0; a < s; ++a)
          if (W[a] == 0) bt[a] += alpha * (tgt[a] - bt[a]);
        if (blk >= 0) {
          W[blk] = dir;
          bt[blk] = dir * M;
        }
        state = 0;
      }
    }
    __syncthreads();
    if (state == 1) break;
  }
  // FP64 objective at the polished point
  double rr = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double r = y64[i];
    for (int a = 0; a < s; ++a) r = fma(-X64[(long long)S[a] * n + i], bt[a], r);
    rr = fma(r, r, rr);
  }
  rr = block_sum(rr, sh);
  double bb = 0.0, nz = 0.0;
  for (int a = threadIdx.x; a < s; a += blockDim.x) {
    double v = bt[a];
    v = v > M ? M : (v < -M ? -M : v);
    bb = fma(v, v, bb);
    nz += v != 0.0 ? 1.0 : 0.0;
  }
  bb = block_sum(bb, sh);
  nz = block_sum(nz, sh);
  if (threadIdx.x == 0) {
    const double v = 0.5 * rr + lam0 * nz + lam2 * bb;
    if (v <= ub_val[q]) {
      ub_val[q] = v;
      for (int a = 0; a < s; ++a) b64[a] = fmin(M, fmax(-M, bt[a]));
    }
    atomicAdd(n_polished, 1);
  }
}

// Incumbent update: smallest candidate value, ties to the lowest node (single block)
__global__ void k_ub_update(int p, int smax, const int* __restrict__ sup,
                            const int* __restrict__ sup_cnt, const int* __restrict__ ret_count,
                            const double* __restrict__ ub_val, const double* __restrict__ ubb64,
                            double* __restrict__ inc_ub, double* __restrict__ inc_beta) {
  __shared__ int best_q;
  __shared__ double best_v;
  if (threadIdx.x < 32) {
    // the smallest value below the incumbent, the lowest q among equal ones: each lane
    // scans q = lane, lane + 32, ... (keeping its first strict minimum), then a butterfly
    // over (value, q) pairs; only supports evaluated in this call count (empty or skipped
    // ones left ub_val untouched)
    const int R = *ret_count;
    double v = inc_ub[0];
    int bq = -1;
    for (int q = threadIdx.x; q < R; q += 32)
      if (sup_cnt[q] > 0 && ub_val[q] < v) {
        v = ub_val[q];
        bq = q;
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int oq = __shfl_xor_sync(0xffffffffu, bq, o);
      const bool take = oq >= 0 && (bq < 0 || ov < v || (ov == v && oq < bq));
      if (take) {
        v = ov;
        bq = oq;
      }
    }
    if (threadIdx.x == 0) {
      best_q = bq;
      best_v = v;
    }
  }
  __syncthreads();
  const int q = best_q;
  if (q < 0) return;
  for (int i = threadIdx.x; i < p; i += blockDim.x) inc_beta[i] = 0.0;
  __syncthreads();
  const int s = sup_cnt[q];
  for (int a = threadIdx.x; a < s; a += blockDim.x)
    inc_beta[sup[(long long)q * smax + a]] = ubb64[(long long)q * 2 * smax + a];
  if (threadIdx.x == 0) inc_ub[0] = best_v;
}

// supports given as K x p masks (bnb_upper_batch): ordered index lists, one block per row
__global__ void k_sup_from_mask(const uint8_t* __restrict__ mask, int p, int smax, int K,
                                int* __restrict__ sup, int* __restrict__ sup_cnt) {
  __shared__ int wcnt[8];
  __shared__ int base;
  const int q = blockIdx.x;
  if (q >= K) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int i0 = 0; i0 < p; i0 += blockDim.x) {
    const int i = i0 + threadIdx.x;
    const int f = (i < p) ? (mask[(long long)q * p + i] != 0) : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wcnt[w] = __popc(bal);
    __syncthreads();
    int off = base;
    for (int t = 0; t < w; ++t) off += wcnt[t];
    const int pos = off + __popc(bal & ((1u << lane) - 1u));
    if (f && pos < smax) sup[(long long)q * smax + pos] = i;
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int t = 0; t < nw; ++t) tot += wcnt[t];
      base += tot;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) sup_cnt[q] = base <= smax ? base : -1;
}

template <class R>
int branch_support(Engine<R>& e, bool write_z, bool memo, bool defer_fallback) {
  k_branch_support<R><<<e.K, 1024, 0, e.st>>>(e.beta, e.fix, defer_fallback ? nullptr : e.gscr,
                                             e.p, e.P, e.ret_slot,
                                             e.ret_count, e.smax, e.br_idx, e.sup, e.sup_cnt,
                                             e.nfree, write_z ? e.zbuf : nullptr,
                                             memo ? e.ub_seen : nullptr, UB_SEEN - 1, e.sup_size);
  BNB_CUDA_OK(cudaGetLastError());
  return 0;
}

// force_polish: 1 polish every candidate in FP64, -1 none (the projected-gradient
// solutions are kept), 0 those within 1e-6 of the incumbent (a solve)
template <class R>
int upper_bound(Engine<R>& e, int force_polish) {
  cudaStream_t st = e.st;
  const int K = e.K;
  k_ub_gram<R><<<dim3(K, 16), 256, 0, st>>>(e.XR, e.yR, e.n, e.smax, e.P.lam2, e.sup, e.sup_cnt,
                                  e.ret_count, e.Qg, e.qv);
  const size_t sm = sizeof(R) * 4 * e.smax;
  k_ub_fista<R><<<K, 256, sm, st>>>(e.Qg, e.qv, e.smax, e.P.M, e.sup_cnt, e.ret_count,
                                    e.ub_iters, sizeof(R) == 4 ? 1e-7 : 1e-13, e.ubb);
  k_ub_eval<R><<<dim3(K, UE_NB), 256, 0, st>>>(e.X64, e.y64, e.n, e.smax, e.P.lam0, e.P.lam2,
                                               e.P.M, e.sup, e.sup_cnt, e.ret_count, e.ubb,
                                               e.ubb64, e.ub_val, e.pol_flag, e.inc_ub,
                                               force_polish, e.ue_part, e.ue_cnt);
  k_ub_polish<<<K, 256, 0, st>>>(e.X64, e.y64, e.n, e.smax, e.P.lam0, e.P.lam2, e.P.M, e.sup,
                                 e.sup_cnt, e.ret_count, e.pol_flag, e.Q64, e.L64, e.ubb64,
                                 e.ub_val, e.sel_state + 8);
  k_ub_update<<<1, 256, 0, st>>>(e.p, e.smax, e.sup, e.sup_cnt, e.ret_count, e.ub_val, e.ubb64,
                                 e.inc_ub, e.inc_beta);
  BNB_CUDA_OK(cudaGetLastError());
  return 0;
}

template <class R>
int ub_from_masks(Engine<R>& e, const uint8_t* dmask, int K) {
  k_sup_from_mask<<<K, 256, 0, e.st>>>(dmask, e.p, e.smax, K, e.sup, e.sup_cnt);
  BNB_CUDA_OK(cudaGetLastError());
  return 0;
}

template <class R>
int branch_fallback(Engine<R>& e) {
  k_branch_fallback<<<e.K, 256, 0, e.st>>>(e.fix, e.gscr, e.p, e.ret_slot, e.ret_count, e.br_idx);
  BNB_CUDA_OK(cudaGetLastError());
  return 0;
}

template int branch_support<float>(Engine<float>&, bool, bool, bool);
template int branch_support<double>(Engine<double>&, bool, bool, bool);
template int branch_fallback<float>(Engine<float>&);
template int branch_fallback<double>(Engine<double>&);
template int upper_bound<float>(Engine<float>&, int);
template int upper_bound<double>(Engine<double>&, int);
template int ub_from_masks<float>(Engine<float>&, const uint8_t*, int);
template int ub_from_masks<double>(Engine<double>&, const uint8_t*, int);

}  // namespace bnb
