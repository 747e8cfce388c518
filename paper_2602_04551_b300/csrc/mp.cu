// mp.cu -- matching-pursuit root heuristic (Section 3.5, Appendix A.2) on the GPU.
//
// Greedy single-coordinate moves on Eq. original from beta = 0, residual r = y - X beta:
//   forward   j not in S:  c_j = X_j^T r, D_j = ||X_j||^2 + 2 lambda2,
//             beta_j = clip(c_j / D_j, [-M, M]),
//             Delta_j = -beta_j c_j + 1/2 D_j beta_j^2 + lambda0;
//   backward  j in S:      Delta_j = beta_j c_j + (1/2 ||X_j||^2 - lambda2) beta_j^2 - lambda0;
// a forward move is taken while one improves (smallest Delta, ties to the lowest
// index), otherwise one improving backward move, otherwise the heuristic stops.
// Each move is one scoring kernel over all columns (a warp per column, per-block
// argmin) and one single-block step kernel; a device flag turns the remaining
// enqueued moves into no-ops once it stops.  The support it ends on is then solved
// exactly in FP64 (box ridge, the upper-bound polish) to seed the incumbent.
#include "engine.cuh"

namespace bnb {

struct MpState {
  int done, moves, s;
};

template <class R>
__global__ void k_mp_init(const R* __restrict__ y, int n, int p, double* __restrict__ beta,
                          double* __restrict__ r, uint8_t* __restrict__ in, MpState* st) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < p) {
    beta[t] = 0.0;
    in[t] = 0;
  }
  if (t < n) r[t] = (double)y[t];
  if (t == 0) {
    st->done = 0;
    st->moves = 0;
    st->s = 0;
  }
}

// key = (Delta, j) ordered lexicographically as (order-preserving Delta key, j)
__device__ __forceinline__ unsigned long long mp_key(double d, int j) {
  // 40 high bits of the order-preserving key of Delta, 24 bits of index (p < 2^24)
  return (dkey(d) & 0xFFFFFFFFFF000000ull) | (unsigned long long)(j & 0xFFFFFF);
}

template <class R>
__global__ void k_mp_scores(const R* __restrict__ X, const double* __restrict__ xsq, int n, int p,
                            const double* __restrict__ r, const double* __restrict__ beta,
                            const uint8_t* __restrict__ in, double lam0, double lam2, double M,
                            const MpState* st, double* __restrict__ cval,
                            unsigned long long* __restrict__ part_f,
                            unsigned long long* __restrict__ part_b) {
  __shared__ unsigned long long sf[8], sb[8];
  if (st->done) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long kf = ~0ull, kb = ~0ull;
  for (int j = blockIdx.x * 8 + w; j < p; j += gridDim.x * 8) {
    const R* x = X + (long long)j * n;
    double c = 0.0;
    for (int i = lane; i < n; i += 32) c = fma((double)x[i], r[i], c);
    c = warp_sum(c);
    if (lane == 0) {
      cval[j] = c;
      const double dj = xsq[j] + 2.0 * lam2;
      if (!in[j]) {
        double b = c / dj;
        b = b > M ? M : (b < -M ? -M : b);
        const double d = -b * c + 0.5 * dj * b * b + lam0;
        const unsigned long long k = mp_key(d, j);
        kf = k < kf ? k : kf;
      } else {
        const double b = beta[j];
        const double d = b * c + (0.5 * xsq[j] - lam2) * b * b - lam0;
        const unsigned long long k = mp_key(d, j);
        kb = k < kb ? k : kb;
      }
    }
  }
  if (lane == 0) {
    sf[w] = kf;
    sb[w] = kb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int t = 1; t < 8; ++t) {
      kf = sf[t] < kf ? sf[t] : kf;
      kb = sb[t] < kb ? sb[t] : kb;
    }
    kf = sf[0] < kf ? sf[0] : kf;
    kb = sb[0] < kb ? sb[0] : kb;
    part_f[blockIdx.x] = kf;
    part_b[blockIdx.x] = kb;
  }
}

__device__ __forceinline__ bool key_negative(unsigned long long k) {
  // order-preserving key of a negative double has its top bit clear
  return k != ~0ull && !(k & 0x8000000000000000ull);
}

template <class R>
__global__ void k_mp_step(const R* __restrict__ X, const double* __restrict__ xsq, int n, int nb,
                          const unsigned long long* __restrict__ part_f,
                          const unsigned long long* __restrict__ part_b,
                          const double* __restrict__ cval, double lam2, double M,
                          double* __restrict__ beta, double* __restrict__ r,
                          uint8_t* __restrict__ in, MpState* st, int max_moves) {
  __shared__ unsigned long long kf_s, kb_s;
  __shared__ int act, jsel;
  __shared__ double bsel;
  if (st->done) return;
  if (threadIdx.x == 0) {
    unsigned long long kf = ~0ull, kb = ~0ull;
    for (int t = 0; t < nb; ++t) {
      kf = part_f[t] < kf ? part_f[t] : kf;
      kb = part_b[t] < kb ? part_b[t] : kb;
    }
    kf_s = kf;
    kb_s = kb;
    act = 0;
    if (st->moves >= max_moves) {
      st->done = 1;
    } else if (key_negative(kf)) {
      const int j = (int)(kf & 0xFFFFFF);
      double b = cval[j] / (xsq[j] + 2.0 * lam2);
      b = b > M ? M : (b < -M ? -M : b);
      act = 1;
      jsel = j;
      bsel = b;
      beta[j] = b;
      in[j] = 1;
      st->s += 1;
      st->moves += 1;
    } else if (key_negative(kb)) {
      const int j = (int)(kb & 0xFFFFFF);
      act = 2;
      jsel = j;
      bsel = beta[j];
      beta[j] = 0.0;
      in[j] = 0;
      st->s -= 1;
      st->moves += 1;
    } else {
      st->done = 1;
    }
  }
  __syncthreads();
  if (act == 0) return;
  const R* x = X + (long long)jsel * n;
  const double sgn = act == 1 ? -bsel : bsel;   // add: r -= x b ; remove: r += x b
  for (int i = threadIdx.x; i < n; i += blockDim.x) r[i] = fma((double)x[i], sgn, r[i]);
}

// support list (ascending) into candidate slot 0 for the exact polish
__global__ void k_mp_support(const uint8_t* __restrict__ in, int p, int smax, int* __restrict__ sup,
                             int* __restrict__ sup_cnt, int* __restrict__ ret_count) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int s = 0;
  for (int j = 0; j < p; ++j)
    if (in[j]) {
      if (s < smax) sup[s] = j;
      ++s;
    }
  sup_cnt[0] = s <= smax ? s : -1;
  *ret_count = 1;
}

__global__ void k_col_sq_from(const double* __restrict__ xnorm, int p, double* __restrict__ xsq) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < p) xsq[j] = xnorm[j] * xnorm[j];
}

template <class R>
int root_heuristic(Engine<R>& e, int max_moves) {
  cudaStream_t st = e.st;
  const int n = e.n, p = e.p;
  const int nb = 296;
  double *mbeta = nullptr, *mr = nullptr, *mc = nullptr, *xsq = nullptr;
  uint8_t* in = nullptr;
  unsigned long long *pf = nullptr, *pb = nullptr;
  MpState* ms = nullptr;
  BNB_CUDA_OK(cudaMallocAsync(&mbeta, sizeof(double) * p, st));
  BNB_CUDA_OK(cudaMallocAsync(&mr, sizeof(double) * n, st));
  BNB_CUDA_OK(cudaMallocAsync(&mc, sizeof(double) * p, st));
  BNB_CUDA_OK(cudaMallocAsync(&xsq, sizeof(double) * p, st));
  BNB_CUDA_OK(cudaMallocAsync(&in, p, st));
  BNB_CUDA_OK(cudaMallocAsync(&pf, sizeof(unsigned long long) * nb, st));
  BNB_CUDA_OK(cudaMallocAsync(&pb, sizeof(unsigned long long) * nb, st));
  BNB_CUDA_OK(cudaMallocAsync(&ms, sizeof(MpState), st));
  const int g = ((n > p ? n : p) + 255) / 256;
  k_mp_init<R><<<g, 256, 0, st>>>(e.yR, n, p, mbeta, mr, in, ms);
  k_col_sq_from<<<(p + 255) / 256, 256, 0, st>>>(e.xnorm, p, xsq);
  for (int m = 0; m < max_moves; ++m) {
    k_mp_scores<R><<<nb, 256, 0, st>>>(e.XR, xsq, n, p, mr, mbeta, in, e.P.lam0, e.P.lam2, e.P.M,
                                       ms, mc, pf, pb);
    k_mp_step<R><<<1, 256, 0, st>>>(e.XR, xsq, n, nb, pf, pb, mc, e.P.lam2, e.P.M, mbeta, mr, in,
                                    ms, max_moves);
  }
  k_mp_support<<<1, 32, 0, st>>>(in, p, e.smax, e.sup, e.sup_cnt, e.ret_count);
  BNB_CUDA_OK(cudaGetLastError());
  if (int rc = upper_bound(e, 1)) return rc;
  BNB_CUDA_OK(cudaFreeAsync(mbeta, st));
  BNB_CUDA_OK(cudaFreeAsync(mr, st));
  BNB_CUDA_OK(cudaFreeAsync(mc, st));
  BNB_CUDA_OK(cudaFreeAsync(xsq, st));
  BNB_CUDA_OK(cudaFreeAsync(in, st));
  BNB_CUDA_OK(cudaFreeAsync(pf, st));
  BNB_CUDA_OK(cudaFreeAsync(pb, st));
  BNB_CUDA_OK(cudaFreeAsync(ms, st));
  return 0;
}

template int root_heuristic<float>(Engine<float>&, int);
template int root_heuristic<double>(Engine<double>&, int);

}  // namespace bnb
