// diag.cu -- diagnostics entry points (libbnb_diag.so, declared in include/bnb_diag.h):
// the tcgen05 contractions on their own, the bounded mbarrier wait on its own, and the
// TMA operand ring on its own (how fast operand tiles reach an SM).
//
// bnb_tc_gemm_check runs C = A B^T for FP64 inputs split into BF16 operands
// (1 term: hi only; 3 terms: hi/lo pairs), K-major A (M x Kred) and B (N x Kred),
// with split-K over `splits` chunks summed in order, and writes C (M x N,
// column-major FP32).  Used by the tests to check the tensor-core kernel against
// a plain product before it is used inside the ADMM iteration.
#include <cuda_bf16.h>
#include "bnb.h"
#include "bnb_diag.h"
#include "tc_host.cuh"

namespace bnb {

__global__ void k_sum_splits_f32(const float* __restrict__ part, int S, long long m,
                                 float* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m;
       i += (long long)gridDim.x * blockDim.x) {
    float a = part[i];
    for (int z = 1; z < S; ++z) a += part[z * m + i];
    out[i] = a;
  }
}

template <int BN, int NS>
static int run_check(cudaStream_t st, const TcOperand& A, const TcOperand& B, int M, int N, int Kd,
                     int splits, float* part, int* err, int* ns_out) {
  int ns = 1;
  tc_chunk(Kd, splits, &ns);
  *ns_out = ns;
  return tc_gemm<BN, NS>(st, A, B, M, N, Kd, splits, nullptr, err,
                         TcEpiStore{part, (long long)M, (long long)M * N});
}

// plain FP32 store of the cluster-reduced product, C[m + n M]
struct TcEpiPlain4 {
  static constexpr int NSTAT = 0;
  float* __restrict__ C;
  int stats;
  __device__ __forceinline__ void put4(int m, int n, float4 a, int M, int, float*) const {
    const float v[4] = {a.x, a.y, a.z, a.w};
    for (int j = 0; j < 4 && m + j < M; ++j) C[(long long)n * M + m + j] = v[j];
  }
  __device__ __forceinline__ void col(int, int, const float*) const {}
};

template <int NS>
static int run_check_cluster(cudaStream_t st, const TcOperand& A, const TcOperand& B, int M, int N,
                             int Kd, int cluster, float* C, int* err) {
  if (tc_cred_active_clusters<256, NS, TcEpiPlain4>(cluster) < 1) return BNB_EINVAL;
  return tc_gemm_cred<256, NS>(st, A, B, M, N, Kd, cluster, nullptr, err, TcEpiPlain4{C, 0});
}

// plain FP32 store of the CTA-pair product, C[m + n M] (pair-kernel epilogue interface)
struct TcEpiPairPlain {
  static constexpr int SMEM_FLOATS = 0;
  struct State {};
  struct Chunk {};
  float* __restrict__ C;
  __device__ __forceinline__ void begin(State&) const {}
  __device__ __forceinline__ void load(int, int, int, int, Chunk&) const {}
  __device__ __forceinline__ void operator()(int m, int n0, const float (&v)[16], int M, int N,
                                             State&, const Chunk&, float*, int) const {
    if (m >= M) return;
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (n0 + j < N) C[(long long)(n0 + j) * M + m] = v[j];
  }
  __device__ __forceinline__ void end(int, int, State&, float*) const {}
  __device__ __forceinline__ void finish(int, int, int, int, int, int, float*) const {}
};

template <int BN, int NS>
static int run_check_pair(cudaStream_t st, const TcOperand& A, const TcOperand& B, int M, int N,
                          int Kd, float* C, int* err) {
  const int cl = tc_pair_clusters<BN, NS, TcEpiPairPlain>();
  if (cl < 1) return BNB_EINVAL;
  return tc_gemm_pair<BN, NS>(st, A, B, M, N, Kd, cl, nullptr, err, TcEpiPairPlain{C});
}

// FP64 inputs -> BF16 (hi, and lo for 3 terms) K-major operands with leading dimension ld
static int make_operands(cudaStream_t st, const double* dA, const double* dB, int M, int N, int Kd,
                         long long ld, __nv_bfloat16** ah, __nv_bfloat16** al, __nv_bfloat16** bh,
                         __nv_bfloat16** bl) {
  cudaError_t ce = cudaSuccess;
  ce = ce ? ce : cudaMalloc(ah, sizeof(__nv_bfloat16) * ld * M);
  ce = ce ? ce : cudaMalloc(al, sizeof(__nv_bfloat16) * ld * M);
  ce = ce ? ce : cudaMalloc(bh, sizeof(__nv_bfloat16) * ld * N);
  ce = ce ? ce : cudaMalloc(bl, sizeof(__nv_bfloat16) * ld * N);
  if (ce != cudaSuccess) return BNB_ENOMEM;
  int rc = 0;
  if (!rc) rc = cudaMemset(*ah, 0, sizeof(__nv_bfloat16) * ld * M) == cudaSuccess ? 0 : BNB_ECUDA;
  if (!rc) rc = cudaMemset(*al, 0, sizeof(__nv_bfloat16) * ld * M) == cudaSuccess ? 0 : BNB_ECUDA;
  if (!rc) rc = cudaMemset(*bh, 0, sizeof(__nv_bfloat16) * ld * N) == cudaSuccess ? 0 : BNB_ECUDA;
  if (!rc) rc = cudaMemset(*bl, 0, sizeof(__nv_bfloat16) * ld * N) == cudaSuccess ? 0 : BNB_ECUDA;
  if (!rc) rc = split_bf16(st, dA, Kd, M, Kd, ld, false, *ah, *al);
  if (!rc) rc = split_bf16(st, dB, Kd, N, Kd, ld, false, *bh, *bl);
  return rc;
}

// One CTA waits on an mbarrier that nothing arrives on (phase 0 of a fresh barrier with an
// arrival count of 1), with the kernels' wait loop and short limits; no TMA copy and no
// MMA is issued, so nothing is in flight when the wait gives up.  Every thread waits;
// err receives the wait's code (1) from each expired wait and 2 if any wait reported
// success; elapsed receives the time thread 0 spent in the wait.
__global__ void k_wait_expiry(long long max_polls, unsigned long long max_ns, int* err,
                              unsigned long long* elapsed) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const unsigned long long t0 = tc::global_ns();
  const bool ok = tc::mbar_wait_bounded<false>(&bar, 0, err, 1, max_polls, max_ns);
  if (ok) atomicOr(err, 2);
  if (threadIdx.x == 0) *elapsed = tc::global_ns() - t0;
  __syncthreads();
}

// The operand ring on its own: a producer thread streams `reps` passes of 16 K steps of
// one stage (A hi, B hi, A lo, B lo: the tiles a CTA of the fused product's pair loads,
// 128-byte swizzle) through an S-stage ring; a consumer thread frees each stage once its
// bytes have landed (no MMA).  CTA c reads A rows 128 (c % 40) .. and B rows
// b_rows (c / 40) ..; every wait is bounded and the consumer sees every stage land, so
// no copy is in flight when the CTA exits.
constexpr int TMA_STREAM_MAX_STAGES = 8;
__global__ void __launch_bounds__(64, 1)
k_tma_stream(const __grid_constant__ CUtensorMap ah, const __grid_constant__ CUtensorMap bh,
             const __grid_constant__ CUtensorMap al, const __grid_constant__ CUtensorMap bl,
             int S, int b_rows, int reps, int* err) {
  extern __shared__ uint8_t raw[];
  __shared__ __align__(8) uint64_t full[TMA_STREAM_MAX_STAGES], empty[TMA_STREAM_MAX_STAGES];
  uint8_t* base = (uint8_t*)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
  const int A_B = tc::BM * tc::BK * 2, B_B = b_rows * tc::BK * 2, STAGE = 2 * A_B + 2 * B_B;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int arow = tc::BM * (blockIdx.x % 40), brow = b_rows * (blockIdx.x / 40);
  const long long total = 16ll * reps;
  if (threadIdx.x == 0) {
    for (long long g = 0; g < total; ++g) {
      const int s = (int)(g % S);
      if (g >= S && !tc::mbar_wait(&empty[s], (uint32_t)(((g / S) & 1) ^ 1), err, 1)) break;
      tc::mbar_expect_tx(&full[s], STAGE);
      const int k = (int)(g % 16) * tc::BK;
      uint8_t* st = base + s * STAGE;
      tc::tma_load_2d(st, &ah, &full[s], k, arow);
      tc::tma_load_2d(st + A_B, &bh, &full[s], k, brow);
      tc::tma_load_2d(st + A_B + B_B, &al, &full[s], k, arow);
      tc::tma_load_2d(st + 2 * A_B + B_B, &bl, &full[s], k, brow);
    }
  } else if (threadIdx.x == 32) {
    for (long long g = 0; g < total; ++g) {
      const int s = (int)(g % S);
      if (!tc::mbar_wait(&full[s], (uint32_t)((g / S) & 1), err, 2)) break;
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&empty[s]))
                   : "memory");
    }
  }
}

}  // namespace bnb

extern "C" int bnb_diag_tma_stream(int ctas, int stages, int b_rows, int reps, int launches,
                                   double* us_out, double* bytes_out, int* err_out) {
  using namespace bnb;
  const long long stage = 2ll * tc::BM * tc::BK * 2 + 2ll * b_rows * tc::BK * 2;
  const long long smem = stages * stage + 1024;
  if (ctas < 1 || ctas > 160 || stages < 2 || stages > TMA_STREAM_MAX_STAGES || b_rows < 8 ||
      b_rows > 256 || b_rows % 8 || reps < 1 || reps > 64 || launches < 1 || launches > 50 ||
      smem > 227 * 1024 || !us_out || !bytes_out || !err_out)
    return BNB_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return BNB_ENODEV;
  }
  if (ctas > sms) return BNB_EINVAL;
  const long long inner = 16 * tc::BK, arows = 40 * tc::BM, brows = 4ll * b_rows;
  __nv_bfloat16* buf[4] = {nullptr, nullptr, nullptr, nullptr};
  const long long elems[4] = {inner * arows, inner * brows, inner * arows, inner * brows};
  int* err = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaSuccess;
  for (int i = 0; i < 4 && ce == cudaSuccess; ++i) {
    ce = cudaMalloc(&buf[i], elems[i] * 2);
    if (ce == cudaSuccess) ce = cudaMemset(buf[i], 0, elems[i] * 2);
  }
  if (ce == cudaSuccess) ce = cudaMalloc(&err, sizeof(int));
  if (ce == cudaSuccess) ce = cudaMemset(err, 0, sizeof(int));
  if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  int rc = ce == cudaSuccess ? BNB_OK : BNB_ENOMEM;
  CUtensorMap m[4];
  for (int i = 0; i < 4 && rc == BNB_OK; ++i)
    rc = make_map_bf16(&m[i], buf[i], inner, (i % 2) ? brows : arows, inner,
                       (i % 2) ? b_rows : tc::BM);
  if (rc == BNB_OK &&
      cudaFuncSetAttribute(k_tma_stream, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess)
    rc = BNB_ECUDA;
  float best = -1.f;
  for (int it = 0; it < launches + 2 && rc == BNB_OK; ++it) {
    cudaEventRecord(e0);
    k_tma_stream<<<ctas, 64, (size_t)smem>>>(m[0], m[1], m[2], m[3], stages, b_rows, reps, err);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      rc = BNB_ECUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (it >= 2 && (best < 0.f || ms < best)) best = ms;
  }
  if (rc == BNB_OK && cudaGetLastError() != cudaSuccess) rc = BNB_ECUDA;
  if (rc == BNB_OK && cudaMemcpy(err_out, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = BNB_ECUDA;
  *us_out = best * 1e3;
  *bytes_out = (double)ctas * reps * 16 * (double)stage;
  for (int i = 0; i < 4; ++i) cudaFree(buf[i]);
  cudaFree(err);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaGetLastError();
  return rc;
}

namespace bnb {
}  // namespace bnb

extern "C" int bnb_diag_wait_expiry(long long max_polls, double max_seconds, int* err_out,
                                    double* seconds_out) {
  using namespace bnb;
  if (max_polls < 1 || max_polls > (1ll << 30) || !(max_seconds > 0.0) || max_seconds > 1.0 ||
      !err_out || !seconds_out)
    return BNB_EINVAL;
  int* err = nullptr;
  unsigned long long* el = nullptr;
  cudaError_t ce = cudaMalloc(&err, sizeof(int));
  if (ce == cudaSuccess) ce = cudaMalloc(&el, sizeof(unsigned long long));
  if (ce == cudaSuccess) ce = cudaMemset(err, 0, sizeof(int));
  if (ce == cudaSuccess) {
    k_wait_expiry<<<1, 128>>>(max_polls, (unsigned long long)(max_seconds * 1e9), err, el);
    ce = cudaGetLastError();
  }
  if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
  unsigned long long ns = 0;
  if (ce == cudaSuccess) ce = cudaMemcpy(err_out, err, sizeof(int), cudaMemcpyDeviceToHost);
  if (ce == cudaSuccess) ce = cudaMemcpy(&ns, el, sizeof(ns), cudaMemcpyDeviceToHost);
  *seconds_out = ns * 1e-9;
  cudaFree(err);
  cudaFree(el);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    return BNB_ECUDA;
  }
  return BNB_OK;
}

extern "C" int bnb_tc_gemm_check_cluster(const double* dA, const double* dB, int M, int N, int Kd,
                                         int nsplit, int cluster, float* dC, int* err_out) {
  using namespace bnb;
  if (M <= 0 || N <= 0 || Kd <= 0 || nsplit < 1 || nsplit > 3 || cluster < 1 || cluster > 8)
    return BNB_EINVAL;
  cudaStream_t st = 0;
  const long long ld = ((long long)Kd + 7) / 8 * 8;
  __nv_bfloat16 *ah = nullptr, *al = nullptr, *bh = nullptr, *bl = nullptr;
  int* err = nullptr;
  int rc = make_operands(st, dA, dB, M, N, Kd, ld, &ah, &al, &bh, &bl);
  if (!rc) rc = cudaMalloc(&err, sizeof(int)) == cudaSuccess ? 0 : BNB_ENOMEM;
  if (!rc) rc = cudaMemset(err, 0, sizeof(int)) == cudaSuccess ? 0 : BNB_ECUDA;
  TcOperand A{ah, al, M, Kd, ld}, B{bh, bl, N, Kd, ld};
  if (!rc) rc = nsplit == 3   ? run_check_cluster<3>(st, A, B, M, N, Kd, cluster, dC, err)
                : nsplit == 2 ? run_check_cluster<2>(st, A, B, M, N, Kd, cluster, dC, err)
                              : run_check_cluster<1>(st, A, B, M, N, Kd, cluster, dC, err);
  if (!rc) rc = cudaMemcpy(err_out, err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess ? 0 : BNB_ECUDA;
  if (!rc) rc = cudaDeviceSynchronize() == cudaSuccess ? 0 : BNB_ECUDA;
  cudaFree(ah);
  cudaFree(al);
  cudaFree(bh);
  cudaFree(bl);
  cudaFree(err);
  return rc;
}

extern "C" int bnb_tc_gemm_check_pair(const double* dA, const double* dB, int M, int N, int Kd,
                                      int nsplit, int bn, float* dC, int* err_out) {
  using namespace bnb;
  if (M <= 0 || N <= 0 || Kd <= 0 || M > 64 * 256 || nsplit < 1 || nsplit > 3 ||
      (bn != 128 && bn != 144 && bn != 256))
    return BNB_EINVAL;
  cudaStream_t st = 0;
  const long long ld = ((long long)Kd + 7) / 8 * 8;
  __nv_bfloat16 *ah = nullptr, *al = nullptr, *bh = nullptr, *bl = nullptr;
  int* err = nullptr;
  int rc = make_operands(st, dA, dB, M, N, Kd, ld, &ah, &al, &bh, &bl);
  if (!rc) rc = cudaMalloc(&err, sizeof(int)) == cudaSuccess ? 0 : BNB_ENOMEM;
  if (!rc) rc = cudaMemset(err, 0, sizeof(int)) == cudaSuccess ? 0 : BNB_ECUDA;
  TcOperand A{ah, al, M, Kd, ld}, B{bh, bl, N, Kd, ld};
  if (!rc) {
    const int key = bn * 4 + nsplit;
    switch (key) {
      case 128 * 4 + 1: rc = run_check_pair<128, 1>(st, A, B, M, N, Kd, dC, err); break;
      case 128 * 4 + 2: rc = run_check_pair<128, 2>(st, A, B, M, N, Kd, dC, err); break;
      case 128 * 4 + 3: rc = run_check_pair<128, 3>(st, A, B, M, N, Kd, dC, err); break;
      case 144 * 4 + 1: rc = run_check_pair<144, 1>(st, A, B, M, N, Kd, dC, err); break;
      case 144 * 4 + 2: rc = run_check_pair<144, 2>(st, A, B, M, N, Kd, dC, err); break;
      case 144 * 4 + 3: rc = run_check_pair<144, 3>(st, A, B, M, N, Kd, dC, err); break;
      case 256 * 4 + 1: rc = run_check_pair<256, 1>(st, A, B, M, N, Kd, dC, err); break;
      case 256 * 4 + 2: rc = run_check_pair<256, 2>(st, A, B, M, N, Kd, dC, err); break;
      default: rc = run_check_pair<256, 3>(st, A, B, M, N, Kd, dC, err); break;
    }
  }
  if (!rc) rc = cudaMemcpy(err_out, err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess ? 0 : BNB_ECUDA;
  if (!rc) rc = cudaDeviceSynchronize() == cudaSuccess ? 0 : BNB_ECUDA;
  cudaFree(ah);
  cudaFree(al);
  cudaFree(bh);
  cudaFree(bl);
  cudaFree(err);
  return rc;
}

extern "C" int bnb_tc_gemm_check(const double* dA, const double* dB, int M, int N, int Kd,
                                 int nsplit, int bn, int splits, float* dC, int* dev_err) {
  using namespace bnb;
  if (M <= 0 || N <= 0 || Kd <= 0 || nsplit < 1 || nsplit > 3 || (bn != 128 && bn != 256))
    return BNB_EINVAL;
  cudaStream_t st = 0;
  const long long ld = ((long long)Kd + 7) / 8 * 8;
  __nv_bfloat16 *ah = nullptr, *al = nullptr, *bh = nullptr, *bl = nullptr;
  float* part = nullptr;
  int* err = nullptr;
  const long long sp = splits < 1 ? 1 : splits;
  cudaError_t ce = cudaSuccess;
  ce = ce ? ce : cudaMalloc(&ah, sizeof(__nv_bfloat16) * ld * M);
  ce = ce ? ce : cudaMalloc(&al, sizeof(__nv_bfloat16) * ld * M);
  ce = ce ? ce : cudaMalloc(&bh, sizeof(__nv_bfloat16) * ld * N);
  ce = ce ? ce : cudaMalloc(&bl, sizeof(__nv_bfloat16) * ld * N);
  ce = ce ? ce : cudaMalloc(&part, sizeof(float) * (size_t)M * N * (sp + 1));
  ce = ce ? ce : cudaMalloc(&err, sizeof(int));
  int rc = ce == cudaSuccess ? 0 : BNB_ENOMEM;
  if (!rc) rc = cudaMemset(err, 0, sizeof(int)) == cudaSuccess ? 0 : BNB_ECUDA;
  if (!rc) rc = cudaMemset(ah, 0, sizeof(__nv_bfloat16) * ld * M) == cudaSuccess ? 0 : BNB_ECUDA;
  if (!rc) rc = cudaMemset(al, 0, sizeof(__nv_bfloat16) * ld * M) == cudaSuccess ? 0 : BNB_ECUDA;
  if (!rc) rc = cudaMemset(bh, 0, sizeof(__nv_bfloat16) * ld * N) == cudaSuccess ? 0 : BNB_ECUDA;
  if (!rc) rc = cudaMemset(bl, 0, sizeof(__nv_bfloat16) * ld * N) == cudaSuccess ? 0 : BNB_ECUDA;
  // A, B are K-major: element (k, row) of a column-major Kd x rows array
  if (!rc) rc = split_bf16(st, dA, Kd, M, Kd, ld, false, ah, al);
  if (!rc) rc = split_bf16(st, dB, Kd, N, Kd, ld, false, bh, bl);
  TcOperand A{ah, al, M, Kd, ld}, B{bh, bl, N, Kd, ld};
  int ns = 1;
  if (!rc) {
    if (bn == 128 && nsplit == 1) rc = run_check<128, 1>(st, A, B, M, N, Kd, splits, part, err, &ns);
    if (bn == 128 && nsplit == 3) rc = run_check<128, 3>(st, A, B, M, N, Kd, splits, part, err, &ns);
    if (bn == 256 && nsplit == 1) rc = run_check<256, 1>(st, A, B, M, N, Kd, splits, part, err, &ns);
    if (bn == 256 && nsplit == 3) rc = run_check<256, 3>(st, A, B, M, N, Kd, splits, part, err, &ns);
    if (bn == 128 && nsplit == 2) rc = run_check<128, 2>(st, A, B, M, N, Kd, splits, part, err, &ns);
    if (bn == 256 && nsplit == 2) rc = run_check<256, 2>(st, A, B, M, N, Kd, splits, part, err, &ns);
  }
  if (!rc) {
    k_sum_splits_f32<<<256, 256, 0, st>>>(part, ns, (long long)M * N, dC);
    rc = cudaGetLastError() == cudaSuccess ? 0 : BNB_ECUDA;
  }
  if (!rc) rc = cudaMemcpy(dev_err, err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess ? 0 : BNB_ECUDA;
  if (!rc) rc = cudaDeviceSynchronize() == cudaSuccess ? 0 : BNB_ECUDA;
  cudaFree(ah);
  cudaFree(al);
  cudaFree(bh);
  cudaFree(bl);
  cudaFree(part);
  cudaFree(err);
  return rc;
}
