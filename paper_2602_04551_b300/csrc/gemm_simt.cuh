// gemm_simt.cuh -- register-blocked CUDA-core GEMM with fused operand/epilogue hooks.
//
//   C[m, n] = sum_{k in chunk z} A[m, k] * B(k, n),   m < M, n < N, k < Kred
//
// A is a plain array, M-major (A[m + k*lda]) or K-major (A[k + m*lda]).  B is read
// through a functor B(k, n) so that operands formed on the fly (W = c + rho beta - V
// of the batched b-update) never touch memory; its natural layout is K-major
// (consecutive k adjacent), or N-major when B_NMAJOR.  The epilogue functor receives
// the accumulator tile and the coordinates of each element.  blockIdx.z selects a
// split-K chunk of length kchunk.  Columns n with active[n] == 0 belong to empty
// node slots: a block whose columns are all empty returns at once.
//
// This kernel is the CUDA-core path (FP32 and FP64); the bulk BF16 contractions
// use the tcgen05 kernel instead.
#pragma once
#include "common.cuh"

namespace bnb {

template <typename T, int BM, int BN, int BK, int TM, int TN, bool A_KMAJOR, bool B_NMAJOR,
          class BLoad, class Epi>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
gemm_simt_kernel(const T* __restrict__ A, long long lda, int M, int N, int Kred, int kchunk,
                 const int* __restrict__ active, BLoad bload, Epi epi) {
  constexpr int TX = BM / TM;  // threads along m
  constexpr int TY = BN / TN;  // threads along n
  constexpr int NT = TX * TY;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tm = tid % TX, tn = tid / TX;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  if (active != nullptr) {
    int any = 0;
    for (int j = tid; j < BN; j += NT)
      if (n0 + j < N && active[n0 + j]) any = 1;
    if (!__syncthreads_or(any)) return;
  }
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(Kred, kbeg + kchunk);
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    if (!A_KMAJOR) {
      for (int e = tid; e < BM * BK; e += NT) {
        int mm = e % BM, kk = e / BM, m = m0 + mm, k = k0 + kk;
        As[kk][mm] = (m < M && k < kend) ? A[(long long)k * lda + m] : T(0);
      }
    } else {
      for (int e = tid; e < BM * BK; e += NT) {
        int kk = e % BK, mm = e / BK, m = m0 + mm, k = k0 + kk;
        As[kk][mm] = (m < M && k < kend) ? A[(long long)m * lda + k] : T(0);
      }
    }
    if (!B_NMAJOR) {
      for (int e = tid; e < BN * BK; e += NT) {
        int kk = e % BK, nn = e / BK, n = n0 + nn, k = k0 + kk;
        Bs[kk][nn] = (n < N && k < kend) ? bload(k, n) : T(0);
      }
    } else {
      for (int e = tid; e < BN * BK; e += NT) {
        int nn = e % BN, kk = e / BN, n = n0 + nn, k = k0 + kk;
        Bs[kk][nn] = (n < N && k < kend) ? bload(k, n) : T(0);
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][tm + i * TX];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tn + j * TY];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  epi.template apply<TM, TN, TX, TY>(acc, m0, n0, tm, tn, M, N);
}

// ----------------------------------------------------------------- common hooks

// B(k, n) = Bm[k + n * ldb]  (K-major plain array)
template <typename T>
struct BPlainK {
  const T* __restrict__ B;
  long long ldb;
  __device__ __forceinline__ T operator()(int k, int n) const { return B[k + (long long)n * ldb]; }
};

// B(k, n) = Bm[n + k * ldb]  (N-major plain array; use with B_NMAJOR)
template <typename T>
struct BPlainN {
  const T* __restrict__ B;
  long long ldb;
  __device__ __forceinline__ T operator()(int k, int n) const { return B[n + (long long)k * ldb]; }
};

// C (+ z * zstride) [m + n * ldc] = acc   (split-K partial or plain store), M-major output
template <typename T>
struct EpiStore {
  T* __restrict__ C;
  long long ldc;
  long long zstride;
  template <int TM, int TN, int TX, int TY>
  __device__ __forceinline__ void apply(T (&acc)[TM][TN], int m0, int n0, int tm, int tn, int M,
                                        int N) const {
    T* Cz = C + (long long)blockIdx.z * zstride;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int n = n0 + tn + j * TY;
      if (n >= N) continue;
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        int m = m0 + tm + i * TX;
        if (m < M) Cz[m + (long long)n * ldc] = acc[i][j];
      }
    }
  }
};

// Launch helper.  Tile: 128 x 128 (8 x 8 per thread, 256 threads), BK 16 for FP32;
// 64 x 64 (4 x 4, 256 threads), BK 8 for FP64.
template <typename T>
struct TileCfg;
template <>
struct TileCfg<float> {
  static constexpr int BM = 128, BN = 128, BK = 16, TM = 8, TN = 8;
};
template <>
struct TileCfg<double> {
  static constexpr int BM = 64, BN = 64, BK = 8, TM = 4, TN = 4;
};

template <typename T, bool A_KMAJOR, bool B_NMAJOR, class BLoad, class Epi>
inline cudaError_t gemm_simt(cudaStream_t st, const T* A, long long lda, int M, int N, int Kred,
                             int splits, const int* active, BLoad bl, Epi ep) {
  using C = TileCfg<T>;
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (splits < 1) splits = 1;
  int kchunk = (Kred + splits - 1) / splits;
  kchunk = ((kchunk + C::BK - 1) / C::BK) * C::BK;
  if (kchunk <= 0) kchunk = C::BK;
  splits = (Kred + kchunk - 1) / kchunk;
  if (splits < 1) splits = 1;
  dim3 grid((M + C::BM - 1) / C::BM, (N + C::BN - 1) / C::BN, splits);
  dim3 block((C::BM / C::TM) * (C::BN / C::TN));
  gemm_simt_kernel<T, C::BM, C::BN, C::BK, C::TM, C::TN, A_KMAJOR, B_NMAJOR, BLoad, Epi>
      <<<grid, block, 0, st>>>(A, lda, M, N, Kred, kchunk, active, bl, ep);
  return cudaGetLastError();
}

// Number of split-K chunks gemm_simt will actually use (the partial-buffer depth).
template <typename T>
inline int gemm_simt_splits(int Kred, int splits) {
  using C = TileCfg<T>;
  if (splits < 1) splits = 1;
  int kchunk = (Kred + splits - 1) / splits;
  kchunk = ((kchunk + C::BK - 1) / C::BK) * C::BK;
  if (kchunk <= 0) kchunk = C::BK;
  int s = (Kred + kchunk - 1) / kchunk;
  return s < 1 ? 1 : s;
}

}  // namespace bnb
