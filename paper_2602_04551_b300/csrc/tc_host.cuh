// tc_host.cuh -- launch helpers for the tcgen05 contraction (host side).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include "common.cuh"
#include "tc_gemm.cuh"

namespace bnb {

int make_map_bf16(CUtensorMap* map, const void* ptr, long long inner, long long rows, long long ld,
                  int box_rows);
int split_bf16(cudaStream_t st, const double* x, long long rows, long long cols, long long ld_in,
               long long ld_out, bool transpose, __nv_bfloat16* hi, __nv_bfloat16* lo);

// Operand pair: hi (and lo for the 3-term product) BF16, K-major, rows x K.
struct TcOperand {
  const __nv_bfloat16* hi = nullptr;
  const __nv_bfloat16* lo = nullptr;
  long long rows = 0, kdim = 0, ld = 0;
};

inline int tc_splits_for(int M, int N, int BN, int Kred, int want_blocks = 2 * 148) {
  const int tiles = ((M + tc::BM - 1) / tc::BM) * ((N + BN - 1) / BN);
  int s = (want_blocks + tiles - 1) / tiles;
  const int maxs = (Kred + tc::BK - 1) / tc::BK;
  if (s > maxs) s = maxs;
  return s < 1 ? 1 : s;
}

// number of split-K chunks actually launched for a requested count (each >= 1 K step)
inline int tc_chunk(int Kred, int splits, int* nsplit) {
  int steps = (Kred + tc::BK - 1) / tc::BK;
  if (splits > steps) splits = steps;
  if (splits < 1) splits = 1;
  const int per = (steps + splits - 1) / splits;
  *nsplit = (steps + per - 1) / per;
  return per * tc::BK;
}

template <int BN, int NSPLIT, class Epi, int EPIW = tc::EPI_WARPS>
int tc_gemm(cudaStream_t st, const TcOperand& A, const TcOperand& B, int M, int N, int Kred,
            int splits, const int* active, int* err, Epi epi) {
  using G = tc::Geo<BN, NSPLIT>;
  if (M <= 0 || N <= 0 || Kred <= 0) return 0;
  CUtensorMap ah, al, bh, bl;
  if (int rc = make_map_bf16(&ah, A.hi, A.kdim, A.rows, A.ld, tc::BM)) return rc;
  if (int rc = make_map_bf16(&bh, B.hi, B.kdim, B.rows, B.ld, BN)) return rc;
  al = ah;
  bl = bh;
  if (NSPLIT == 3)
    if (int rc = make_map_bf16(&al, A.lo, A.kdim, A.rows, A.ld, tc::BM)) return rc;
  if (NSPLIT >= 2)
    if (int rc = make_map_bf16(&bl, B.lo, B.kdim, B.rows, B.ld, BN)) return rc;
  int ns = 1;
  const int kchunk = tc_chunk(Kred, splits, &ns);
  auto kern = tc::tc_gemm_kernel<BN, NSPLIT, Epi, EPIW>;
  static bool attr_set = false;
  if (!attr_set) {
    BNB_CUDA_OK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM));
    attr_set = true;
  }
  dim3 grid((M + tc::BM - 1) / tc::BM, (N + BN - 1) / BN, ns);
  kern<<<grid, 64 + 32 * EPIW, G::SMEM, st>>>(ah, al, bh, bl, M, N, Kred, kchunk, active, err, epi);
  BNB_CUDA_OK(cudaGetLastError());
  return 0;
}

// Co-resident clusters of size cs (1, 2, 4 or 8) of the cluster-reduce kernel on the
// current device (0 when none fits); cached per instantiation.
template <int BN, int NSPLIT, class Epi>
int tc_cred_active_clusters(int cs) {
  using G = tc::Geo<BN, NSPLIT>;
  static int cached[9] = {-1, -1, -1, -1, -1, -1, -1, -1, -1};
  if (cs < 1 || cs > 8) return 0;
  if (cached[cs] < 0) {
    auto kern = tc::tc_gemm_cred_kernel<BN, NSPLIT, Epi>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM) !=
        cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1, 1, cs);
    cfg.blockDim = dim3(64 + 32 * 8);
    cfg.dynamicSmemBytes = G::SMEM;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 1;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = cs;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, kern, &cfg) != cudaSuccess) {
      cudaGetLastError();
      nc = 0;
    }
    cached[cs] = nc;
  }
  return cached[cs];
}

// Cluster size for `tiles` output tiles over `steps` K steps: the size (1, 2, 4, 8, at
// most steps / 2) with the least estimated time, waves x (K steps per CTA + 2), where a
// wave is as many clusters as the device co-schedules.  0 when nothing fits.
template <int BN, int NSPLIT, class Epi>
int tc_cred_pick_cluster(int tiles, int steps) {
  int best = 0;
  long long best_t = 0;
  for (int cs = 1; cs <= 8; cs <<= 1) {
    if (cs > 1 && cs > steps / 2) break;
    const int act = tc_cred_active_clusters<BN, NSPLIT, Epi>(cs);
    if (act < 1) continue;
    const long long waves = (tiles + act - 1) / act;
    const long long t = waves * ((steps + cs - 1) / cs + 2);
    if (best == 0 || t < best_t) {
      best = cs;
      best_t = t;
    }
  }
  return best;
}

// C = A B^T over K split into `cluster` chunks reduced inside a cluster (see
// tc_gemm_cred_kernel); `cluster` must be a size tc_cred_active_clusters accepts.
template <int BN, int NSPLIT, class Epi>
int tc_gemm_cred(cudaStream_t st, const TcOperand& A, const TcOperand& B, int M, int N, int Kred,
                 int cluster, const int* active, int* err, Epi epi) {
  using G = tc::Geo<BN, NSPLIT>;
  if (M <= 0 || N <= 0 || Kred <= 0) return 0;
  if (cluster < 1 || cluster > 8) return BNB_EINVAL;
  CUtensorMap ah, al, bh, bl;
  if (int rc = make_map_bf16(&ah, A.hi, A.kdim, A.rows, A.ld, tc::BM)) return rc;
  if (int rc = make_map_bf16(&bh, B.hi, B.kdim, B.rows, B.ld, BN)) return rc;
  al = ah;
  bl = bh;
  if (NSPLIT == 3)
    if (int rc = make_map_bf16(&al, A.lo, A.kdim, A.rows, A.ld, tc::BM)) return rc;
  if (NSPLIT >= 2)
    if (int rc = make_map_bf16(&bl, B.lo, B.kdim, B.rows, B.ld, BN)) return rc;
  int ns = 1;
  const int kchunk = tc_chunk(Kred, cluster, &ns);
  auto kern = tc::tc_gemm_cred_kernel<BN, NSPLIT, Epi>;
  static bool attr_set = false;
  if (!attr_set) {
    BNB_CUDA_OK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM));
    attr_set = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((M + tc::BM - 1) / tc::BM, (N + BN - 1) / BN, ns);
  cfg.blockDim = dim3(64 + 32 * 8);
  cfg.dynamicSmemBytes = G::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 1;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = ns;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  BNB_CUDA_OK(cudaLaunchKernelEx(&cfg, kern, ah, al, bh, bl, M, N, Kred, kchunk, active, err, epi));
  return 0;
}

// Persistent launch of the heavy-epilogue product (see tc_gemm_persist_kernel): one CTA
// per SM (at most one per tile).  N must not exceed 64 BN.
template <int BN, int NSPLIT, class Epi, int EPIW = tc::EPI_WARPS>
int tc_gemm_persist(cudaStream_t st, const TcOperand& A, const TcOperand& B, int M, int N,
                    int Kred, int sms, const int* active, int* err, Epi epi) {
  using G = tc::Geo<BN, NSPLIT>;
  if (M <= 0 || N <= 0 || Kred <= 0) return 0;
  if (N > 64 * BN) return BNB_EINVAL;
  CUtensorMap ah, al, bh, bl;
  if (int rc = make_map_bf16(&ah, A.hi, A.kdim, A.rows, A.ld, tc::BM)) return rc;
  if (int rc = make_map_bf16(&bh, B.hi, B.kdim, B.rows, B.ld, BN)) return rc;
  al = ah;
  bl = bh;
  if (NSPLIT == 3)
    if (int rc = make_map_bf16(&al, A.lo, A.kdim, A.rows, A.ld, tc::BM)) return rc;
  if (NSPLIT >= 2)
    if (int rc = make_map_bf16(&bl, B.lo, B.kdim, B.rows, B.ld, BN)) return rc;
  auto kern = tc::tc_gemm_persist_kernel<BN, NSPLIT, Epi, EPIW>;
  static bool attr_set = false;
  if (!attr_set) {
    BNB_CUDA_OK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::PSMEM));
    attr_set = true;
  }
  const long long tiles = (long long)((M + tc::BM - 1) / tc::BM) * ((N + BN - 1) / BN);
  const int grid = (int)(tiles < sms ? tiles : sms);
  kern<<<grid, 64 + 32 * EPIW, G::PSMEM, st>>>(ah, al, bh, bl, M, N, Kred, active, err, epi);
  BNB_CUDA_OK(cudaGetLastError());
  return 0;
}

// Co-resident clusters of two of the multicast persistent kernel (0: none).
template <int BN, int NSPLIT, class Epi, int EPIW = tc::EPI_WARPS>
int tc_persist_mc_clusters() {
  using G = tc::Geo<BN, NSPLIT>;
  static int cached = -1;
  if (cached < 0) {
    auto kern = tc::tc_gemm_persist_mc_kernel<BN, NSPLIT, Epi, EPIW>;
    cached = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::PSMEM) !=
        cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2);
    cfg.blockDim = dim3(64 + 32 * EPIW);
    cfg.dynamicSmemBytes = G::PSMEM;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, kern, &cfg) != cudaSuccess) {
      cudaGetLastError();
      nc = 0;
    }
    cached = nc;
  }
  return cached;
}

// Persistent product in clusters of two sharing the A tile (tc_gemm_persist_mc_kernel):
// `clusters` co-resident clusters at most.
template <int BN, int NSPLIT, class Epi, int EPIW = tc::EPI_WARPS>
int tc_gemm_persist_mc(cudaStream_t st, const TcOperand& A, const TcOperand& B, int M, int N,
                       int Kred, int clusters, const int* active, int* err, Epi epi) {
  using G = tc::Geo<BN, NSPLIT>;
  if (M <= 0 || N <= 0 || Kred <= 0) return 0;
  if (N > 64 * BN || clusters < 1) return BNB_EINVAL;
  CUtensorMap ah, al, bh, bl;
  if (int rc = make_map_bf16(&ah, A.hi, A.kdim, A.rows, A.ld, tc::BM / 2)) return rc;
  if (int rc = make_map_bf16(&bh, B.hi, B.kdim, B.rows, B.ld, BN)) return rc;
  al = ah;
  bl = bh;
  if (NSPLIT == 3)
    if (int rc = make_map_bf16(&al, A.lo, A.kdim, A.rows, A.ld, tc::BM / 2)) return rc;
  if (NSPLIT >= 2)
    if (int rc = make_map_bf16(&bl, B.lo, B.kdim, B.rows, B.ld, BN)) return rc;
  auto kern = tc::tc_gemm_persist_mc_kernel<BN, NSPLIT, Epi, EPIW>;
  static bool attr_set = false;
  if (!attr_set) {
    BNB_CUDA_OK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::PSMEM));
    attr_set = true;
  }
  const long long units = (long long)((M + tc::BM - 1) / tc::BM) * (((N + BN - 1) / BN + 1) / 2);
  const int ncl = (int)(units < clusters ? units : clusters);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * ncl);
  cfg.blockDim = dim3(64 + 32 * EPIW);
  cfg.dynamicSmemBytes = G::PSMEM;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  BNB_CUDA_OK(cudaLaunchKernelEx(&cfg, kern, ah, al, bh, bl, M, N, Kred, active, err, epi));
  return 0;
}

// Co-resident clusters (CTA pairs) of the pair kernel (0: none).
template <int BN, int NSPLIT, class Epi, int EPIW = tc::EPI_WARPS>
int tc_pair_clusters() {
  using G = tc::PairGeo<BN, NSPLIT>;
  static int cached = -1;
  if (cached < 0) {
    auto kern = tc::tc_gemm_pair_kernel<BN, NSPLIT, Epi, EPIW>;
    cached = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM) !=
        cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2);
    cfg.blockDim = dim3(64 + 32 * EPIW);
    cfg.dynamicSmemBytes = G::SMEM;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, kern, &cfg) != cudaSuccess) {
      cudaGetLastError();
      nc = 0;
    }
    cached = nc;
  }
  return cached;
}

// C = A B^T on CTA pairs (tc_gemm_pair_kernel): 256 x BN tiles, at most `clusters` pairs.
// A: M rows (boxes of 128 rows, hi and, for 2 and 3 terms, lo); B: N rows (boxes of BN/2
// rows, hi and, for 3 terms, lo).  With an activity mask over the rows (row tiles with no
// active row are skipped) M <= 64 x 256.
template <int BN, int NSPLIT, class Epi, int EPIW = tc::EPI_WARPS>
int tc_gemm_pair(cudaStream_t st, const TcOperand& A, const TcOperand& B, int M, int N, int Kred,
                 int clusters, const int* active, int* err, Epi epi, int kchunk = 0) {
  using G = tc::PairGeo<BN, NSPLIT>;
  if (M <= 0 || N <= 0 || Kred <= 0) return 0;
  if ((active != nullptr && M > 64 * 256) || clusters < 1) return BNB_EINVAL;
  CUtensorMap ah, al, bh, bl;
  if (int rc = make_map_bf16(&ah, A.hi, A.kdim, A.rows, A.ld, tc::BM)) return rc;
  if (int rc = make_map_bf16(&bh, B.hi, B.kdim, B.rows, B.ld, BN / 2)) return rc;
  al = ah;
  bl = bh;
  if (NSPLIT >= 2)
    if (int rc = make_map_bf16(&al, A.lo, A.kdim, A.rows, A.ld, tc::BM)) return rc;
  if (NSPLIT == 3)
    if (int rc = make_map_bf16(&bl, B.lo, B.kdim, B.rows, B.ld, BN / 2)) return rc;
  auto kern = tc::tc_gemm_pair_kernel<BN, NSPLIT, Epi, EPIW>;
  static bool attr_set = false;
  if (!attr_set) {
    BNB_CUDA_OK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM));
    attr_set = true;
  }
  if (kchunk <= 0 || kchunk >= Kred) kchunk = (Kred + tc::BK - 1) / tc::BK * tc::BK;
  if (kchunk % tc::BK) return BNB_EINVAL;
  const long long units = (long long)((M + 255) / 256) * ((N + BN - 1) / BN) *
                          ((Kred + kchunk - 1) / kchunk);
  const int ncl = (int)(units < clusters ? units : clusters);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * ncl);
  cfg.blockDim = dim3(64 + 32 * EPIW);
  cfg.dynamicSmemBytes = G::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  BNB_CUDA_OK(cudaLaunchKernelEx(&cfg, kern, ah, al, bh, bl, M, N, Kred, kchunk, active, err,
                                 epi));
  return 0;
}

// Co-resident clusters of 2 cs CTAs (cs pairs) of the pair-in-cluster kernel (0: none);
// cached per instantiation and cs.
template <int BN, int NSPLIT, class Epi>
int tc_cpair_active_clusters(int cs) {
  using G = tc::CPairGeo<BN, NSPLIT>;
  static int cached[5] = {-1, -1, -1, -1, -1};
  if (cs < 1 || cs > 4) return 0;
  if (cached[cs] < 0) {
    cached[cs] = 0;
    auto kern = tc::tc_gemm_cpair_kernel<BN, NSPLIT, Epi>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM) !=
        cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * cs);
    cfg.blockDim = dim3(64 + 32 * tc::EPI_WARPS);
    cfg.dynamicSmemBytes = G::SMEM;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2 * cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, kern, &cfg) != cudaSuccess) {
      cudaGetLastError();
      nc = 0;
    }
    cached[cs] = nc;
  }
  return cached[cs];
}

// C = A B^T with 256 x BN tiles, each on a cluster of cs CTA pairs that split the K range
// (tc_gemm_cpair_kernel); A: M rows (boxes of 128 rows), B: N rows (boxes of BN/2 rows).
template <int BN, int NSPLIT, class Epi>
int tc_gemm_cpair(cudaStream_t st, const TcOperand& A, const TcOperand& B, int M, int N, int Kred,
                  int cs, const int* active, int* err, Epi epi) {
  using G = tc::CPairGeo<BN, NSPLIT>;
  if (M <= 0 || N <= 0 || Kred <= 0) return 0;
  if (cs < 1 || cs > 4) return BNB_EINVAL;
  CUtensorMap ah, al, bh, bl;
  if (int rc = make_map_bf16(&ah, A.hi, A.kdim, A.rows, A.ld, tc::BM)) return rc;
  if (int rc = make_map_bf16(&bh, B.hi, B.kdim, B.rows, B.ld, BN / 2)) return rc;
  al = ah;
  bl = bh;
  if (NSPLIT >= 2)
    if (int rc = make_map_bf16(&al, A.lo, A.kdim, A.rows, A.ld, tc::BM)) return rc;
  if (NSPLIT == 3)
    if (int rc = make_map_bf16(&bl, B.lo, B.kdim, B.rows, B.ld, BN / 2)) return rc;
  auto kern = tc::tc_gemm_cpair_kernel<BN, NSPLIT, Epi>;
  static bool attr_set = false;
  if (!attr_set) {
    BNB_CUDA_OK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM));
    attr_set = true;
  }
  const int steps = (Kred + tc::BK - 1) / tc::BK;
  const int kchunk = (steps + cs - 1) / cs * tc::BK;
  const long long tiles = (long long)((M + 255) / 256) * ((N + BN - 1) / BN);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * cs * tiles));
  cfg.blockDim = dim3(64 + 32 * tc::EPI_WARPS);
  cfg.dynamicSmemBytes = G::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2 * cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  BNB_CUDA_OK(cudaLaunchKernelEx(&cfg, kern, ah, al, bh, bl, M, N, Kred, kchunk, active, err, epi));
  return 0;
}

// Split-K partial store: C + z * zstride [m + n * ldc] = acc
struct TcEpiStore {
  static constexpr int SMEM_FLOATS = 0;
  float* __restrict__ C;
  long long ldc, zstride;
  __device__ __forceinline__ void finish(int, int, int, int, int, int, float*) const {}
  __device__ __forceinline__ void operator()(int m, int n0, const float (&v)[16], int M, int N, int,
                                             float*) const {
    if (m >= M) return;
    float* Cz = C + (long long)blockIdx.z * zstride;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int n = n0 + j;
      if (n < N) Cz[m + (long long)n * ldc] = v[j];
    }
  }
};

}  // namespace bnb
