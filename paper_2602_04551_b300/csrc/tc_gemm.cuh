// tc_gemm.cuh -- Blackwell (sm_103a) tensor-core contraction for the ADMM products.
//
//   C[m, n] = sum_{k in chunk z} A[m, k] B[n, k]        (both operands K-major, BF16)
//
// Tiles of 128 x BN outputs, 64-wide K steps.  One CTA = 2 + EPIW warps:
//   warp 0  (one thread)  TMA producer: cp.async.bulk.tensor 2D loads of the A and B
//                         tiles (128-byte swizzle) into an S-stage shared-memory ring,
//                         completion counted on the stage's "full" mbarrier;
//   warp 1  (one thread)  MMA issuer: tcgen05.mma kind::f16 (BF16 x BF16 -> FP32) into a
//                         128 x BN accumulator in tensor memory; tcgen05.commit frees a
//                         stage ("empty" mbarrier) and finally signals "done";
//                         the whole warp allocates / frees the TMEM columns;
//   warps 2..             epilogue: tcgen05.ld of the accumulator rows (a warp reads its
//                         32-lane quarter of TMEM, the warps of a quarter take
//                         alternate 16-column chunks), handed to the epilogue functor.
// The kernel shapes share the device helpers:
//   tc_gemm_kernel          one tile per CTA, split-K partials stored (diagnostics);
//   tc_gemm_cred_kernel     K split over the CTAs of a thread-block cluster, partial tiles
//                           summed through distributed shared memory in rank order, fused
//                           epilogue on the sum (H W'^T, the check product X beta^T);
//   tc_gemm_persist_kernel  one CTA per SM over the tiles, double-buffered accumulator so
//                           the epilogue of a tile overlaps the next tile (X^T U' with the
//                           fused ADMM update); tc_gemm_persist_mc_kernel the same in
//                           clusters of two CTAs that share the A tile by TMA multicast;
//   tc_gemm_pair_kernel     256 x BN tiles computed by a pair of CTAs on two SMs (tcgen05
//                           cta_group::2): each CTA loads 128 rows of A and half of the B
//                           columns, so the B bytes each SM receives per output are halved
//                           (X^T U' with the fused update, as features x slots or, with the
//                           roles exchanged, slots x features).
// NSPLIT = 3 uses hi/lo BF16 pairs of both operands (A = Ah + Al, B = Bh + Bl) and
// accumulates Ah Bh + Ah Bl + Al Bh: about 16 significant bits per operand, the
// FP32-class arithmetic of the ADMM path.  NSPLIT = 2 keeps one operand as a single BF16
// term (the data) and the other as a pair (the iterate): B is the pair in the one-CTA
// kernels (Ah Bh + Ah Bl), A in the pair kernel (Ah Bh + Al Bh).  NSPLIT = 1 is the plain
// BF16 product.
//
// Every mbarrier wait is bounded; on expiry the kernel records an error code in
// *err and leaves its loops, so a fault in the pipeline never hangs the GPU.
#pragma once
#include <cuda.h>
#include "common.cuh"

namespace bnb {
namespace tc {

constexpr int BM = 128;
constexpr int BK = 64;             // 64 BF16 = 128 bytes: one swizzle row
constexpr int EPI_WARPS = 8;       // default epilogue warps: two per TMEM lane quarter
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr long long WAIT_LIMIT = 1ll << 24;   // polls of one bounded mbarrier wait
constexpr unsigned long long WAIT_NS = 2000000000ull;   // and at most 2 s of it

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// bounded wait on the phase with parity `ph`: at most max_polls polls and max_ns of
// %globaltimer; false (and *err |= code) on expiry.  CLUSTER selects the cluster-scope
// acquire form (arrivals from the other CTA of a pair).  The kernels use the limits of
// mbar_wait / mbar_wait_cluster; a diagnostics kernel runs the same loop with short
// limits on a barrier nobody arrives on, to show that an expired wait returns.
template <bool CLUSTER>
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t ph, int* err, int code,
                                                  long long max_polls, uint64_t max_ns) {
  const uint32_t a = smem_u32(bar);
  const uint64_t t0 = global_ns();
  for (long long i = 0; i < max_polls; ++i) {
    uint32_t ok;
    if constexpr (CLUSTER)
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
          " selp.b32 %0, 1, 0, p;\n}\n"
          : "=r"(ok)
          : "r"(a), "r"(ph)
          : "memory");
    else
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
          " selp.b32 %0, 1, 0, p;\n}\n"
          : "=r"(ok)
          : "r"(a), "r"(ph)
          : "memory");
    if (ok) return true;
    if ((i & 255) == 255 && global_ns() - t0 > max_ns) break;
  }
  atomicOr(err, code);
  return false;
}

// the kernels' bound: WAIT_LIMIT polls and WAIT_NS (2 s)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t ph, int* err, int code) {
  return mbar_wait_bounded<false>(bar, ph, err, code, WAIT_LIMIT, WAIT_NS);
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

// shared-memory matrix descriptor: K-major tile, rows of 128 bytes, 128-byte swizzle,
// 8-row groups 1024 bytes apart (stride byte offset), descriptor version 1
__device__ __forceinline__ uint64_t smem_desc_sw128(const void* p) {
  const uint64_t addr = smem_u32(p);
  uint64_t d = 0;
  d |= (addr >> 4) & 0x3FFFull;            // start address
  d |= (uint64_t)1 << 16;                  // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset
  d |= (uint64_t)1 << 46;                  // version
  d |= (uint64_t)2 << 61;                  // layout: 128-byte swizzle
  return d;
}

// instruction descriptor: dense, D = F32, A = B = BF16, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// multicast variants (thread-block cluster): the TMA box lands at the same shared-memory
// offset in every CTA of `mask`, each CTA's mbarrier at that offset counting the bytes;
// the commit arrives on the mbarrier at the same offset in every CTA of `mask`
__device__ __forceinline__ void tma_load_2d_mc(void* dst, const CUtensorMap* map, uint64_t* bar,
                                               int c0, int c1, uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      ".multicast::cluster [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(smem_u32(bar)), "h"(mask)
      : "memory");
}
__device__ __forceinline__ void mma_commit_mc(uint64_t* bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(smem_u32(bar)), "h"(mask)
      : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
      " [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}


// ---- thread-block clusters (split-K reduction through distributed shared memory)
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_size() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
// every thread of every CTA of the cluster arrives (release) and waits (acquire)
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
// 16 bytes at the same shared-memory offset in the CTA of rank `rank`
__device__ __forceinline__ float4 ld_dsmem_f4(uint32_t local_addr, uint32_t rank) {
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(local_addr), "r"(rank));
  float4 v;
  // volatile keeps the loads after the cluster barrier; no memory clobber, so that
  // consecutive loads are not serialised by the compiler
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(ra));
  return v;
}

template <int BN, int NSPLIT>
struct Geo {
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = BN * BK * 2;
  // a stage holds [A hi | B hi], then [A lo | B lo] (3 terms) or [B lo] (2 terms)
  static constexpr int STAGE_BYTES =
      A_BYTES * (NSPLIT == 3 ? 2 : 1) + B_BYTES * (NSPLIT >= 2 ? 2 : 1);
  static constexpr int SBUDGET = BN <= 64 ? 100 * 1024 : 196 * 1024;  // <= 64: 2 CTAs per SM
  static constexpr int STAGES =
      SBUDGET / STAGE_BYTES < 2 ? 2 : (SBUDGET / STAGE_BYTES > 6 ? 6 : SBUDGET / STAGE_BYTES);
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024;  // + alignment slack
  // persistent variant (one CTA per SM): as many stages as fit in ~200 KB
  static constexpr int PSTAGES = (200 * 1024) / STAGE_BYTES < 2 ? 2 : (200 * 1024) / STAGE_BYTES;
  static constexpr int PSMEM = PSTAGES * STAGE_BYTES + 1024;
  static constexpr int TMEM_COLS = BN < 32 ? 32 : BN;
  // persistent kernel: each of its two accumulators starts at a power-of-two column
  static constexpr int PBUF = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
};

struct Maps {
  CUtensorMap a_hi, a_lo, b_hi, b_lo;
};

// Operand ring of one CTA: stage s holds [A hi | B hi | A lo | B lo] for the 3-term
// product, [A hi | B hi | B lo] for the 2-term one (A single, B a hi/lo pair), and
// [A hi | B hi] for the 1-term one.
template <int BN, int NSPLIT>
__device__ __forceinline__ uint8_t* ring_a(uint8_t* base, int s, int part) {
  using G = Geo<BN, NSPLIT>;
  return base + s * G::STAGE_BYTES + part * (G::A_BYTES + G::B_BYTES);
}
template <int BN, int NSPLIT>
__device__ __forceinline__ uint8_t* ring_blo(uint8_t* base, int s) {
  using G = Geo<BN, NSPLIT>;
  return NSPLIT == 3 ? ring_a<BN, NSPLIT>(base, s, 1) + G::A_BYTES
                     : base + s * G::STAGE_BYTES + G::A_BYTES + G::B_BYTES;
}

// TMA producer (one thread): nk K steps from kbeg, A rows m0.., B rows n0..
template <int BN, int NSPLIT>
__device__ __forceinline__ void tma_producer(const CUtensorMap* ma_hi, const CUtensorMap* ma_lo,
                                             const CUtensorMap* mb_hi, const CUtensorMap* mb_lo,
                                             uint8_t* base, uint64_t* full_bar, uint64_t* empty_bar,
                                             int nk, int kbeg, int m0, int n0, int* err) {
  using G = Geo<BN, NSPLIT>;
  constexpr int S = G::STAGES;
  for (int kb = 0; kb < nk; ++kb) {
    const int s = kb % S;
    if (kb >= S && !mbar_wait(&empty_bar[s], ((kb / S) & 1) ^ 1, err, 1)) break;
    mbar_expect_tx(&full_bar[s], G::STAGE_BYTES);
    const int k = kbeg + kb * BK;
    uint8_t* a0 = ring_a<BN, NSPLIT>(base, s, 0);
    tma_load_2d(a0, ma_hi, &full_bar[s], k, m0);
    tma_load_2d(a0 + G::A_BYTES, mb_hi, &full_bar[s], k, n0);
    if (NSPLIT >= 2) tma_load_2d(ring_blo<BN, NSPLIT>(base, s), mb_lo, &full_bar[s], k, n0);
    if (NSPLIT == 3) tma_load_2d(ring_a<BN, NSPLIT>(base, s, 1), ma_lo, &full_bar[s], k, m0);
  }
}

// MMA issuer (one thread): accumulates the nk K steps into the 128 x BN tensor-memory
// tile at `tmem`, frees each stage with a commit, and finally commits `done_bar`.
template <int BN, int NSPLIT>
__device__ __forceinline__ void mma_issuer(uint32_t tmem, uint8_t* base, uint64_t* full_bar,
                                           uint64_t* empty_bar, uint64_t* done_bar, int nk,
                                           int* err) {
  using G = Geo<BN, NSPLIT>;
  constexpr int S = G::STAGES;
  constexpr uint32_t idesc = idesc_bf16(BN);
  for (int kb = 0; kb < nk; ++kb) {
    const int s = kb % S;
    if (!mbar_wait(&full_bar[s], (kb / S) & 1, err, 2)) break;
    fence_after();
    uint8_t* a0 = ring_a<BN, NSPLIT>(base, s, 0);
    uint8_t* a1 = ring_a<BN, NSPLIT>(base, s, 1);
    uint8_t* b1 = ring_blo<BN, NSPLIT>(base, s);
#pragma unroll
    for (int kk = 0; kk < BK / 16; ++kk) {
      const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
      const uint64_t ah = smem_desc_sw128(a0 + kk * 32);
      const uint64_t bh = smem_desc_sw128(a0 + G::A_BYTES + kk * 32);
      mma_bf16(tmem, ah, bh, idesc, acc);
      if (NSPLIT >= 2) mma_bf16(tmem, ah, smem_desc_sw128(b1 + kk * 32), idesc, 1u);
      if (NSPLIT == 3) mma_bf16(tmem, smem_desc_sw128(a1 + kk * 32), bh, idesc, 1u);
    }
    mma_commit(&empty_bar[s]);
  }
  mma_commit(done_bar);
}

// Epilogue interface:
//   epi(row m, first column n0 + c, 16 accumulator values, M, N, lane quarter q, smem)
//     called by every epilogue thread for each 16-column chunk of its row;
//   epi.finish(t, nthreads, m0, n0, M, N, smem)  after the epilogue warps meet;
//   Epi::SMEM_FLOATS  shared scratch the functor needs.
template <int BN, int NSPLIT, class Epi, int EPIW>
__global__ void __launch_bounds__(64 + 32 * EPIW, EPIW == 4 ? 2 : 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap ma_hi, const __grid_constant__ CUtensorMap ma_lo,
               const __grid_constant__ CUtensorMap mb_hi, const __grid_constant__ CUtensorMap mb_lo,
               int M, int N, int Kred, int kchunk, const int* __restrict__ active, int* err, Epi epi) {
  using G = Geo<BN, NSPLIT>;
  constexpr int S = G::STAGES;
  extern __shared__ uint8_t dsm_raw[];
  __shared__ __align__(8) uint64_t full_bar[S];
  __shared__ __align__(8) uint64_t empty_bar[S];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ float epi_smem[Epi::SMEM_FLOATS > 0 ? Epi::SMEM_FLOATS : 1];
  uint8_t* base = (uint8_t*)(((uintptr_t)dsm_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  if (active != nullptr) {
    int any = 0;
    for (int j = threadIdx.x; j < BN; j += blockDim.x)
      if (n0 + j < N && active[n0 + j]) any = 1;
    if (!__syncthreads_or(any)) return;
  }
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(Kred, kbeg + kchunk);
  const int nk = (kend - kbeg + BK - 1) / BK;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(G::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    tma_producer<BN, NSPLIT>(&ma_hi, &ma_lo, &mb_hi, &mb_lo, base, full_bar, empty_bar, nk, kbeg,
                             m0, n0, err);
  } else if (warp == 1 && lane == 0) {
    mma_issuer<BN, NSPLIT>(tmem, base, full_bar, empty_bar, &done_bar, nk, err);
  } else if (warp >= 2) {
    // ---------------- epilogue: warp w owns TMEM lanes [32 (w % 4), 32 (w % 4) + 32)
    const int q = warp & 3;
    const int g = (warp - 2) >> 2;      // which of the quarter's EPIW/4 warps
    const bool ok = mbar_wait(&done_bar, 0, err, 4);
    fence_after();
    const int row = m0 + 32 * q + lane;
    if (ok) {
#pragma unroll 1
      for (int c = 16 * g; c < BN; c += 16 * (EPIW / 4)) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c, v);
        epi(row, n0 + c, v, M, N, q, epi_smem);
      }
    }
    // the epilogue warps meet (named barrier 1) before the per-tile finish
    asm volatile("bar.sync 1, %0;" ::"n"(32 * EPIW) : "memory");
    if (ok) epi.finish(threadIdx.x - 64, 32 * EPIW, m0, n0, M, N, epi_smem);
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(G::TMEM_COLS)
                 : "memory");
  }
}


// Split-K with the reduction inside a thread-block cluster.  The CTAs of a cluster
// (cluster dimension = gridDim.z) take consecutive K chunks of the same 128 x BN output
// tile.  Each copies its tensor-memory accumulator into its own (now idle) operand ring
// as a column-major 128 x BN FP32 tile; after a cluster barrier, CTA rank r sums the
// column slice [r BN / S, (r + 1) BN / S) over the S partial tiles, read through
// distributed shared memory in rank order (a fixed order: the result does not depend
// on scheduling), and hands each 4-row group to the epilogue:
//   epi.put4(m, n, {C[m..m+3][n]}, M, N, st)   accumulates Epi::NSTAT per-column sums
//   epi.col(tile_m, n, st)                     the warp totals (when epi.stats), lane 0.
// Every CTA of a cluster takes the same path (the early exit depends only on the tile),
// and every thread reaches both cluster barriers, so the barriers always complete.
template <int BN, int NSPLIT, class Epi>
__global__ void __launch_bounds__(64 + 32 * 8, 1)
tc_gemm_cred_kernel(const __grid_constant__ CUtensorMap ma_hi,
                    const __grid_constant__ CUtensorMap ma_lo,
                    const __grid_constant__ CUtensorMap mb_hi,
                    const __grid_constant__ CUtensorMap mb_lo, int M, int N, int Kred, int kchunk,
                    const int* __restrict__ active, int* err, Epi epi) {
  using G = Geo<BN, NSPLIT>;
  constexpr int S = G::STAGES;
  static_assert(S * G::STAGE_BYTES >= BN * BM * 4, "the partial tile reuses the operand ring");
  extern __shared__ uint8_t dsm_raw[];
  __shared__ __align__(8) uint64_t full_bar[S];
  __shared__ __align__(8) uint64_t empty_bar[S];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_slot;
  uint8_t* base = (uint8_t*)(((uintptr_t)dsm_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  if (active != nullptr) {
    int any = 0;
    for (int j = threadIdx.x; j < BN; j += blockDim.x)
      if (n0 + j < N && active[n0 + j]) any = 1;
    if (!__syncthreads_or(any)) return;     // the whole cluster shares this tile
  }
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(Kred, kbeg + kchunk);
  const int nk = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(G::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;
  float* part = reinterpret_cast<float*>(base);   // [BN][BM] after the main loop

  if (warp == 0 && lane == 0) {
    tma_producer<BN, NSPLIT>(&ma_hi, &ma_lo, &mb_hi, &mb_lo, base, full_bar, empty_bar, nk, kbeg,
                             m0, n0, err);
  } else if (warp == 1 && lane == 0) {
    mma_issuer<BN, NSPLIT>(tmem, base, full_bar, empty_bar, &done_bar, nk, err);
  } else if (warp >= 2) {
    // accumulator -> own partial tile (warp w: TMEM lanes 32 (w % 4) .., alternate chunks)
    const int q = warp & 3, g = (warp - 2) >> 2;
    const bool ok = mbar_wait(&done_bar, 0, err, 4);
    fence_after();
    const int row = 32 * q + lane;
#pragma unroll 1
    for (int c = 16 * g; c < BN; c += 32) {
      float v[16];
      if (ok && nk > 0) {
        tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c, v);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0.f;
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) part[(c + j) * BM + row] = v[j];
    }
  }
  cluster_sync_all();
  if (warp >= 2) {
    const uint32_t rank = cluster_rank(), cs = cluster_size();
    const int w = warp - 2;
    const int per = (BN + (int)cs - 1) / (int)cs;
    const int c0 = (int)rank * per, c1 = min(BN, c0 + per);
    const uint32_t lbase = smem_u32(part);
#pragma unroll 1
    for (int c = c0 + w; c < c1; c += 8) {
      const int n = n0 + c;
      if (n >= N) break;                         // warp-uniform; later columns are out too
      const uint32_t off = lbase + (uint32_t)(c * BM + 4 * lane) * 4u;
      // issue every rank's load before the first add (independent remote loads in
      // flight together), then add in rank order
      float4 pr[8];
#pragma unroll
      for (uint32_t r = 0; r < 8; ++r)
        if (r < cs) pr[r] = ld_dsmem_f4(off, r);
      float4 a = pr[0];
#pragma unroll
      for (uint32_t r = 1; r < 8; ++r)
        if (r < cs) {
          a.x += pr[r].x;
          a.y += pr[r].y;
          a.z += pr[r].z;
          a.w += pr[r].w;
        }
      float st[Epi::NSTAT > 0 ? Epi::NSTAT : 1];
#pragma unroll
      for (int k = 0; k < (Epi::NSTAT > 0 ? Epi::NSTAT : 1); ++k) st[k] = 0.f;
      epi.put4(m0 + 4 * lane, n, a, M, N, st);
      if constexpr (Epi::NSTAT > 0) {
        if (epi.stats) {
#pragma unroll
          for (int k = 0; k < Epi::NSTAT; ++k) st[k] = warp_sum(st[k]);
          if (lane == 0) epi.col(blockIdx.x, n, st);
        }
      }
    }
  }
  cluster_sync_all();                            // no CTA leaves while its tile is read
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(G::TMEM_COLS)
                 : "memory");
  }
}


// Persistent variant for the product whose epilogue is heavy (X^T U' with the fused
// ADMM update): one CTA per SM walks the 128 x BN output tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ... (column-tile-major, so that CTAs working at the same
// time share the B slice in L2).  The accumulator is double-buffered in tensor memory
// (2 x BN columns): while the epilogue warps drain tile i from buffer i & 1, the MMA
// issuer already accumulates tile i + 1 into the other buffer, and the TMA ring runs
// continuously across tiles.  Hand-offs:
//   tmem_full[b]   MMA -> epilogue  (tcgen05.commit after the tile's last K step)
//   tmem_empty[b]  epilogue -> MMA  (one arrive per epilogue warp once it has read b)
// Tiles whose columns are all inactive are skipped by every role alike.  The epilogue
// interface is the one of tc_gemm_kernel (per 16-column chunk, then finish per tile).
template <int BN, int NSPLIT, class Epi, int EPIW>
__global__ void __launch_bounds__(64 + 32 * EPIW, 1)
tc_gemm_persist_kernel(const __grid_constant__ CUtensorMap ma_hi,
                       const __grid_constant__ CUtensorMap ma_lo,
                       const __grid_constant__ CUtensorMap mb_hi,
                       const __grid_constant__ CUtensorMap mb_lo, int M, int N, int Kred,
                       const int* __restrict__ active, int* err, Epi epi) {
  using G = Geo<BN, NSPLIT>;
  constexpr int S = G::PSTAGES;
  constexpr int MAXNT = 64;                      // column tiles (N <= 64 BN)
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "MMA N: a multiple of 16 up to 256");
  extern __shared__ uint8_t dsm_raw[];
  __shared__ __align__(8) uint64_t full_bar[S];
  __shared__ __align__(8) uint64_t empty_bar[S];
  __shared__ __align__(8) uint64_t tfull_bar[2];
  __shared__ __align__(8) uint64_t tempty_bar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int tile_on[MAXNT];
  __shared__ float epi_smem[Epi::SMEM_FLOATS > 0 ? Epi::SMEM_FLOATS : 1];
  uint8_t* base = (uint8_t*)(((uintptr_t)dsm_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mtiles = (M + BM - 1) / BM, ntiles = (N + BN - 1) / BN;
  const int ntot = mtiles * ntiles;
  const int nk = (Kred + BK - 1) / BK;
  for (int j = threadIdx.x; j < MAXNT; j += blockDim.x) {
    int on = 0;
    if (j < ntiles) {
      for (int c = 0; c < BN && j * BN + c < N; ++c)
        if (active == nullptr || active[j * BN + c]) {
          on = 1;
          break;
        }
    }
    tile_on[j] = on;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull_bar[b], 1);
      mbar_init(&tempty_bar[b], EPIW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(2 * G::PBUF)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer: one continuous ring over all tiles of this CTA
    long long g = 0;                             // K steps issued so far
    bool ok = true;
    for (int t = blockIdx.x; t < ntot && ok; t += gridDim.x) {
      const int mt = t % mtiles, nt = t / mtiles;
      if (!tile_on[nt]) continue;
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = (int)(g % S);
        if (g >= S && !mbar_wait(&empty_bar[s], (uint32_t)(((g / S) & 1) ^ 1), err, 1)) {
          ok = false;
          break;
        }
        mbar_expect_tx(&full_bar[s], G::STAGE_BYTES);
        const int k = kb * BK;
        uint8_t* a0 = ring_a<BN, NSPLIT>(base, s, 0);
        tma_load_2d(a0, &ma_hi, &full_bar[s], k, mt * BM);
        tma_load_2d(a0 + G::A_BYTES, &mb_hi, &full_bar[s], k, nt * BN);
        if (NSPLIT >= 2)
          tma_load_2d(ring_blo<BN, NSPLIT>(base, s), &mb_lo, &full_bar[s], k, nt * BN);
        if (NSPLIT == 3)
          tma_load_2d(ring_a<BN, NSPLIT>(base, s, 1), &ma_lo, &full_bar[s], k, mt * BM);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    constexpr uint32_t idesc = idesc_bf16(BN);
    long long g = 0;
    int i = 0;                                   // tiles of this CTA so far
    bool ok = true;
    for (int t = blockIdx.x; t < ntot && ok; t += gridDim.x) {
      const int nt = t / mtiles;
      if (!tile_on[nt]) continue;
      const int b = i & 1;
      if (i >= 2 && !mbar_wait(&tempty_bar[b], (uint32_t)(((i >> 1) & 1) ^ 1), err, 8)) break;
      fence_after();
      const uint32_t acc_addr = tmem + (uint32_t)(b * G::PBUF);
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = (int)(g % S);
        if (!mbar_wait(&full_bar[s], (uint32_t)((g / S) & 1), err, 2)) {
          ok = false;
          break;
        }
        fence_after();
        uint8_t* a0 = ring_a<BN, NSPLIT>(base, s, 0);
        uint8_t* a1 = ring_a<BN, NSPLIT>(base, s, 1);
        uint8_t* b1 = ring_blo<BN, NSPLIT>(base, s);
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
          const uint64_t ah = smem_desc_sw128(a0 + kk * 32);
          const uint64_t bh = smem_desc_sw128(a0 + G::A_BYTES + kk * 32);
          mma_bf16(acc_addr, ah, bh, idesc, acc);
          if (NSPLIT >= 2) mma_bf16(acc_addr, ah, smem_desc_sw128(b1 + kk * 32), idesc, 1u);
          if (NSPLIT == 3) mma_bf16(acc_addr, smem_desc_sw128(a1 + kk * 32), bh, idesc, 1u);
        }
        mma_commit(&empty_bar[s]);
      }
      mma_commit(&tfull_bar[b]);
      ++i;
    }
  } else if (warp >= 2) {
    // ---------------- epilogue warps: warp w reads TMEM lanes 32 (w % 4) ..
    const int q = warp & 3;
    const int gq = (warp - 2) >> 2;             // which of the quarter's EPIW/4 warps
    int i = 0;
    for (int t = blockIdx.x; t < ntot; t += gridDim.x) {
      const int mt = t % mtiles, nt = t / mtiles;
      if (!tile_on[nt]) continue;
      const int b = i & 1;
      // warp-uniform, so that an epilogue using warp shuffles runs in all lanes or none
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&tfull_bar[b], (uint32_t)((i >> 1) & 1), err, 4));
      fence_after();
      const int m0 = mt * BM, n0 = nt * BN;
      const int row = m0 + 32 * q + lane;
      if (ok) {
#pragma unroll 1
        for (int c = 16 * gq; c < BN; c += 16 * (EPIW / 4)) {
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * G::PBUF + c), v);
          epi(row, n0 + c, v, M, N, q, epi_smem);
        }
      }
      fence_before();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty_bar[b]))
                     : "memory");
      // the epilogue warps meet (and agree whether every wait completed) before the
      // per-tile finish, and again before the next tile reuses the shared scratch
      uint32_t all_ok;
      asm volatile(
          "{\n .reg .pred p, r;\n setp.ne.u32 p, %1, 0;\n"
          " bar.red.and.pred r, 1, %2, p;\n selp.u32 %0, 1, 0, r;\n}\n"
          : "=r"(all_ok)
          : "r"((uint32_t)ok), "n"(32 * EPIW)
          : "memory");
      if (all_ok) epi.finish(threadIdx.x - 64, 32 * EPIW, m0, n0, M, N, epi_smem);
      asm volatile("bar.sync 1, %0;" ::"n"(32 * EPIW) : "memory");
      ++i;
      if (!all_ok) break;
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(2 * G::PBUF)
                 : "memory");
  }
}


// Persistent kernel in clusters of two CTAs that share the A tile: the cluster walks
// units (row tile mt, column-tile pair ntp); CTA rank r computes the tile (mt, 2 ntp + r),
// loads rows [64 r, 64 r + 64) of the A tile and multicasts them to both CTAs, and loads
// its own B tile.  Each A tile therefore crosses L2 once per pair of column tiles
// instead of once per column tile.  A stage is refilled only after both CTAs' MMAs
// released it (its "empty" barrier counts the two commits, which are multicast).
// Barriers are initialised on both CTAs before any remote signal (cluster barrier) and
// neither CTA leaves while the other may still signal it (cluster barrier at the end);
// every thread reaches both cluster barriers.  The A tensor maps have 64-row boxes.
template <int BN, int NSPLIT, class Epi, int EPIW>
__global__ void __launch_bounds__(64 + 32 * EPIW, 1)
tc_gemm_persist_mc_kernel(const __grid_constant__ CUtensorMap ma_hi,
                          const __grid_constant__ CUtensorMap ma_lo,
                          const __grid_constant__ CUtensorMap mb_hi,
                          const __grid_constant__ CUtensorMap mb_lo, int M, int N, int Kred,
                          const int* __restrict__ active, int* err, Epi epi) {
  using G = Geo<BN, NSPLIT>;
  constexpr int S = G::PSTAGES;
  constexpr int MAXNT = 64;
  constexpr int AH = G::A_BYTES / 2;             // 64 rows x 128 bytes
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "MMA N: a multiple of 16 up to 256");
  extern __shared__ uint8_t dsm_raw[];
  __shared__ __align__(8) uint64_t full_bar[S];
  __shared__ __align__(8) uint64_t empty_bar[S];
  __shared__ __align__(8) uint64_t tfull_bar[2];
  __shared__ __align__(8) uint64_t tempty_bar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int tile_on[MAXNT];
  __shared__ float epi_smem[Epi::SMEM_FLOATS > 0 ? Epi::SMEM_FLOATS : 1];
  uint8_t* base = (uint8_t*)(((uintptr_t)dsm_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rank = (int)cluster_rank();
  const int cid = blockIdx.x >> 1, ncl = gridDim.x >> 1;
  const int mtiles = (M + BM - 1) / BM, ntiles = (N + BN - 1) / BN;
  const int npairs = (ntiles + 1) / 2;
  const int nunits = mtiles * npairs;
  const int nk = (Kred + BK - 1) / BK;
  for (int j = threadIdx.x; j < MAXNT; j += blockDim.x) {
    int on = 0;
    if (j < ntiles) {
      for (int c = 0; c < BN && j * BN + c < N; ++c)
        if (active == nullptr || active[j * BN + c]) {
          on = 1;
          break;
        }
    }
    tile_on[j] = on;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 2);             // both CTAs' MMA commits
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull_bar[b], 1);
      mbar_init(&tempty_bar[b], EPIW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(2 * G::PBUF)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  cluster_sync_all();                            // both CTAs' barriers exist
  const uint32_t tmem = tmem_slot;
  auto unit_on = [&](int ntp) {
    return tile_on[2 * ntp] || (2 * ntp + 1 < ntiles && tile_on[2 * ntp + 1]);
  };

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    long long g = 0;
    bool ok = true;
    for (int u = cid; u < nunits && ok; u += ncl) {
      const int mt = u % mtiles, ntp = u / mtiles;
      if (!unit_on(ntp)) continue;
      const int nt = 2 * ntp + rank;
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = (int)(g % S);
        if (g >= S && !mbar_wait(&empty_bar[s], (uint32_t)(((g / S) & 1) ^ 1), err, 1)) {
          ok = false;
          break;
        }
        mbar_expect_tx(&full_bar[s], G::STAGE_BYTES);
        const int k = kb * BK;
        uint8_t* a0 = ring_a<BN, NSPLIT>(base, s, 0);
        tma_load_2d_mc(a0 + rank * AH, &ma_hi, &full_bar[s], k, mt * BM + 64 * rank, 3);
        tma_load_2d(a0 + G::A_BYTES, &mb_hi, &full_bar[s], k, nt * BN);
        if (NSPLIT >= 2)
          tma_load_2d(ring_blo<BN, NSPLIT>(base, s), &mb_lo, &full_bar[s], k, nt * BN);
        if (NSPLIT == 3)
          tma_load_2d_mc(ring_a<BN, NSPLIT>(base, s, 1) + rank * AH, &ma_lo, &full_bar[s], k,
                         mt * BM + 64 * rank, 3);
      }
    }
    // every copy this CTA issued has landed before the cluster may be left (after an
    // error the MMA may not have consumed them); bounded like every wait
    for (long long j = g - S < 0 ? 0 : g - S; j < g; ++j)
      mbar_wait(&full_bar[(int)(j % S)], (uint32_t)((j / S) & 1), err, 16);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    constexpr uint32_t idesc = idesc_bf16(BN);
    long long g = 0;
    int i = 0;
    bool ok = true;
    for (int u = cid; u < nunits && ok; u += ncl) {
      const int ntp = u / mtiles;
      if (!unit_on(ntp)) continue;
      const int b = i & 1;
      if (i >= 2 && !mbar_wait(&tempty_bar[b], (uint32_t)(((i >> 1) & 1) ^ 1), err, 8)) break;
      fence_after();
      const uint32_t acc_addr = tmem + (uint32_t)(b * G::PBUF);
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = (int)(g % S);
        if (!mbar_wait(&full_bar[s], (uint32_t)((g / S) & 1), err, 2)) {
          ok = false;
          break;
        }
        fence_after();
        uint8_t* a0 = ring_a<BN, NSPLIT>(base, s, 0);
        uint8_t* a1 = ring_a<BN, NSPLIT>(base, s, 1);
        uint8_t* b1 = ring_blo<BN, NSPLIT>(base, s);
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
          const uint64_t ah = smem_desc_sw128(a0 + kk * 32);
          const uint64_t bh = smem_desc_sw128(a0 + G::A_BYTES + kk * 32);
          mma_bf16(acc_addr, ah, bh, idesc, acc);
          if (NSPLIT >= 2) mma_bf16(acc_addr, ah, smem_desc_sw128(b1 + kk * 32), idesc, 1u);
          if (NSPLIT == 3) mma_bf16(acc_addr, smem_desc_sw128(a1 + kk * 32), bh, idesc, 1u);
        }
        mma_commit_mc(&empty_bar[s], 3);         // frees stage s in both CTAs
      }
      mma_commit(&tfull_bar[b]);
      ++i;
    }
  } else if (warp >= 2) {
    // ---------------- epilogue warps (own tile of each unit)
    const int q = warp & 3;
    const int gq = (warp - 2) >> 2;
    int i = 0;
    for (int u = cid; u < nunits; u += ncl) {
      const int mt = u % mtiles, ntp = u / mtiles;
      if (!unit_on(ntp)) continue;
      const int nt = 2 * ntp + rank;
      const int b = i & 1;
      // warp-uniform, so that an epilogue using warp shuffles runs in all lanes or none
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&tfull_bar[b], (uint32_t)((i >> 1) & 1), err, 4));
      fence_after();
      const int m0 = mt * BM, n0 = nt * BN;
      const int row = m0 + 32 * q + lane;
      if (ok && n0 < N) {
#pragma unroll 1
        for (int c = 16 * gq; c < BN; c += 16 * (EPIW / 4)) {
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * G::PBUF + c), v);
          epi(row, n0 + c, v, M, N, q, epi_smem);
        }
      }
      fence_before();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty_bar[b]))
                     : "memory");
      uint32_t all_ok;
      asm volatile(
          "{\n .reg .pred p, r;\n setp.ne.u32 p, %1, 0;\n"
          " bar.red.and.pred r, 1, %2, p;\n selp.u32 %0, 1, 0, r;\n}\n"
          : "=r"(all_ok)
          : "r"((uint32_t)ok), "n"(32 * EPIW)
          : "memory");
      if (all_ok && n0 < N) epi.finish(threadIdx.x - 64, 32 * EPIW, m0, n0, M, N, epi_smem);
      asm volatile("bar.sync 1, %0;" ::"n"(32 * EPIW) : "memory");
      ++i;
      if (!all_ok) break;
    }
  }
  fence_before();
  __syncthreads();
  cluster_sync_all();                            // no remote signal can still arrive
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(2 * G::PBUF)
                 : "memory");
  }
}


// ---- CTA pairs (tcgen05 cta_group::2): one 256 x BN tile on two SMs
//
// The two CTAs of a cluster of two form the pair; rank 0 (the leader) issues the MMAs.
// A tile's rows [256 mt, 256 mt + 256) split as 128 per CTA (A operand and the
// accumulator: each CTA's tensor memory holds its 128 rows x BN columns); its columns
// [BN nt, BN nt + BN) split as BN/2 per CTA for the B operand, which the MMA reads from
// both CTAs' shared memory.  Both CTAs load their halves with TMA into the same ring
// offsets; the completion of both is counted on the leader's "full" barrier.

__device__ __forceinline__ uint32_t mapa_u32(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

// TMA load into this CTA's shared memory, completion counted on the mbarrier at the
// shared::cluster address `bar` (the leader's)
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map, uint32_t bar,
                                                 int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.cta_group::2"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

// instruction descriptor: dense, D = F32, A = B = BF16, both K-major, M = 256 (the pair),
// N = n
__host__ __device__ constexpr uint32_t idesc_bf16_pair(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(256 >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16_pair(uint32_t tmem, uint64_t ad, uint64_t bd,
                                              uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
      : "memory");
}

// arrives on the mbarrier at the same offset in both CTAs once the leader's MMAs so far
// have completed
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(smem_u32(bar)), "h"((uint16_t)3)
      : "memory");
}

// arrive (release, cluster scope) on the mbarrier at shared::cluster address `bar`
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar)
               : "memory");
}

// bounded wait with cluster-scope acquire (arrivals from the other CTA of the pair)
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* bar, uint32_t ph, int* err, int code) {
  return mbar_wait_bounded<true>(bar, ph, err, code, WAIT_LIMIT, WAIT_NS);
}

template <int BN, int NSPLIT>
struct PairGeo {
  static constexpr int A_BYTES = BM * BK * 2;              // this CTA's 128 rows of A
  static constexpr int B_BYTES = (BN / 2) * BK * 2;        // this CTA's BN/2 rows of B
  // a stage holds [A hi | B hi], then [A lo] (2 and 3 terms), then [B lo] (3 terms): the
  // 2-term product keeps B (the data) as one BF16 term and A (the iterate) as a pair
  static constexpr int STAGE_BYTES =
      A_BYTES * (NSPLIT >= 2 ? 2 : 1) + B_BYTES * (NSPLIT == 3 ? 2 : 1);
  static constexpr int STAGES =
      (200 * 1024) / STAGE_BYTES > 8 ? 8 : (200 * 1024) / STAGE_BYTES;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024;
  // 256 tensor-memory columns per CTA: two accumulators up to 128 columns wide, else one
  static constexpr int BUF = BN <= 128 ? 128 : 256;
  static constexpr int NBUF = 256 / BUF;
  static_assert(STAGES >= 2, "at least two stages");
};

// Persistent product on CTA pairs: cluster c walks the units u = c, c + clusters, ...
// (K chunk z = u / tiles of kchunk elements, row tile mt and column tile nt of u % tiles,
// rows fastest); units whose 256 rows are all inactive are skipped by every role of both
// CTAs alike.  With one chunk (kchunk >= Kred) a unit is a whole output tile; with several
// the epilogue receives the partial product of chunk z.
//   full[s]      leader: both CTAs' TMA bytes of stage s (expect_tx by the leader)
//   empty[s]     each CTA: the leader's MMAs have read stage s (multicast commit)
//   tfull[b]     each CTA: accumulator b holds the tile (multicast commit)
//   tempty[b]    leader: all epilogue warps of both CTAs have read accumulator b
//   fin          each CTA: every MMA of the leader has completed (before teardown)
// Tensor memory is allocated for the pair (cta_group::2, 256 columns in each CTA); the
// CTAs check that they hold the same address and otherwise skip all work and report it.
// Epilogue interface (rows = A rows, e.g. node slots; columns = B rows, e.g. features):
//   typename Epi::State st; epi.begin(st);
//   typename Epi::Chunk ck; epi.load(row, first column, M, N, ck)   the chunk's other
//                                 inputs (issued for the first chunk before the wait)
//   epi(row, first column, 16 accumulator values, M, N, st, ck, smem, z)  per 16-column
//                                 chunk of the partial product of K chunk z
//   epi.end(r, gq, st, smem)      after the thread's last chunk of the tile (r = row in CTA)
//   epi.finish(t, nthreads, first row of the CTA, nt, M, N, smem)  after the warps meet
template <int BN, int NSPLIT, class Epi, int EPIW>
__global__ void __launch_bounds__(64 + 32 * EPIW, 1)
tc_gemm_pair_kernel(const __grid_constant__ CUtensorMap ma_hi,
                    const __grid_constant__ CUtensorMap ma_lo,
                    const __grid_constant__ CUtensorMap mb_hi,
                    const __grid_constant__ CUtensorMap mb_lo, int M, int N, int Kred,
                    int kchunk, const int* __restrict__ active, int* err, Epi epi) {
  using G = PairGeo<BN, NSPLIT>;
  constexpr int S = G::STAGES;
  constexpr int MAXMT = 64;                      // row tiles with an activity mask (M <= 64 x 256)
  static_assert(BN % 16 == 0 && BN >= 32 && BN <= 256, "pair MMA N: a multiple of 16 up to 256");
  static_assert(EPIW % 4 == 0, "epilogue warps cover the four lane quarters");
  extern __shared__ uint8_t dsm_raw[];
  __shared__ __align__(8) uint64_t full_bar[S];
  __shared__ __align__(8) uint64_t empty_bar[S];
  __shared__ __align__(8) uint64_t tfull_bar[2];
  __shared__ __align__(8) uint64_t tempty_bar[2];
  __shared__ __align__(8) uint64_t fin_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int tile_on[MAXMT];
  __shared__ float epi_smem[Epi::SMEM_FLOATS > 0 ? Epi::SMEM_FLOATS : 1];
  uint8_t* base = (uint8_t*)(((uintptr_t)dsm_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const int cid = blockIdx.x >> 1, ncl = gridDim.x >> 1;
  const int mtiles = (M + 255) / 256, ntiles = (N + BN - 1) / BN;
  const int ntile = mtiles * ntiles;
  const int nz = (Kred + kchunk - 1) / kchunk;   // K chunks: unit u takes chunk u / ntile
  const int nunits = ntile * nz;
  // K steps of a unit's chunk
  auto unit_nk = [&](int z) {
    const int kb = z * kchunk, ke = min(Kred, kb + kchunk);
    return (ke - kb + BK - 1) / BK;
  };
  for (int j = threadIdx.x; j < MAXMT; j += blockDim.x) {
    int on = 0;
    if (j < mtiles && active != nullptr) {
      for (int r = 0; r < 256 && j * 256 + r < M; ++r)
        if (active[j * 256 + r]) {
          on = 1;
          break;
        }
    }
    tile_on[j] = on;
  }
  auto row_tile_on = [&](int mt) { return active == nullptr || tile_on[mt] != 0; };
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull_bar[b], 1);
      mbar_init(&tempty_bar[b], 2 * EPIW);
    }
    mbar_init(&fin_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(256)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  cluster_sync_all();                            // both CTAs' barriers and TMEM exist
  const uint32_t tmem = tmem_slot;
  uint32_t peer_tmem;
  asm volatile("ld.shared::cluster.u32 %0, [%1];"
               : "=r"(peer_tmem)
               : "r"(mapa_u32(smem_u32(&tmem_slot), rank ^ 1u))
               : "memory");
  const bool pair_ok = peer_tmem == tmem;
  if (!pair_ok && threadIdx.x == 0) atomicOr(err, 32);
  const uint32_t full_l = mapa_u32(smem_u32(&full_bar[0]), 0);     // the leader's barriers
  const uint32_t tempty_l = mapa_u32(smem_u32(&tempty_bar[0]), 0);

  if (pair_ok && warp == 0 && lane == 0) {
    // ---------------- TMA producer (both CTAs): this CTA's halves of every stage
    long long g = 0;
    bool ok = true;
    for (int u = cid; u < nunits && ok; u += ncl) {
      const int z = u / ntile, mt = (u % ntile) % mtiles, nt = (u % ntile) / mtiles;
      if (!row_tile_on(mt)) continue;
      const int arow = mt * 256 + 128 * (int)rank, brow = nt * BN + (BN / 2) * (int)rank;
      const int nk = unit_nk(z);
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = (int)(g % S);
        if (g >= S && !mbar_wait(&empty_bar[s], (uint32_t)(((g / S) & 1) ^ 1), err, 1)) {
          ok = false;
          break;
        }
        if (leader) mbar_expect_tx(&full_bar[s], 2 * G::STAGE_BYTES);
        const int k = z * kchunk + kb * BK;
        const uint32_t fb = full_l + 8u * (uint32_t)s;
        uint8_t* st0 = base + s * G::STAGE_BYTES;
        tma_load_2d_pair(st0, &ma_hi, fb, k, arow);
        tma_load_2d_pair(st0 + G::A_BYTES, &mb_hi, fb, k, brow);
        if (NSPLIT >= 2) tma_load_2d_pair(st0 + G::A_BYTES + G::B_BYTES, &ma_lo, fb, k, arow);
        if (NSPLIT == 3)
          tma_load_2d_pair(st0 + 2 * G::A_BYTES + G::B_BYTES, &mb_lo, fb, k, brow);
      }
    }
    // the leader's last stages count both CTAs' copies: they have all landed before the
    // pair may be left (bounded like every wait)
    if (leader)
      for (long long j = g - S < 0 ? 0 : g - S; j < g; ++j)
        mbar_wait(&full_bar[(int)(j % S)], (uint32_t)((j / S) & 1), err, 16);
  } else if (pair_ok && warp == 1 && lane == 0 && leader) {
    // ---------------- MMA issuer (leader)
    constexpr uint32_t idesc = idesc_bf16_pair(BN);
    long long g = 0;
    int i = 0;
    bool ok = true;
    for (int u = cid; u < nunits && ok; u += ncl) {
      const int z = u / ntile, mt = (u % ntile) % mtiles;
      if (!row_tile_on(mt)) continue;
      const int nk = unit_nk(z);
      const int b = i % G::NBUF, use = i / G::NBUF;
      if (use >= 1 && !mbar_wait_cluster(&tempty_bar[b], (uint32_t)((use & 1) ^ 1), err, 8)) break;
      fence_after();
      const uint32_t acc_addr = tmem + (uint32_t)(b * G::BUF);
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = (int)(g % S);
        if (!mbar_wait(&full_bar[s], (uint32_t)((g / S) & 1), err, 2)) {
          ok = false;
          break;
        }
        fence_after();
        uint8_t* st0 = base + s * G::STAGE_BYTES;
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
          const uint64_t ah = smem_desc_sw128(st0 + kk * 32);
          const uint64_t bh = smem_desc_sw128(st0 + G::A_BYTES + kk * 32);
          mma_bf16_pair(acc_addr, ah, bh, idesc, acc);
          if (NSPLIT >= 2)
            mma_bf16_pair(acc_addr, smem_desc_sw128(st0 + G::A_BYTES + G::B_BYTES + kk * 32), bh,
                          idesc, 1u);
          if (NSPLIT == 3)
            mma_bf16_pair(acc_addr, ah,
                          smem_desc_sw128(st0 + 2 * G::A_BYTES + G::B_BYTES + kk * 32), idesc, 1u);
        }
        mma_commit_pair(&empty_bar[s]);          // stage s free in both CTAs
      }
      if (!ok) break;
      mma_commit_pair(&tfull_bar[b]);
      ++i;
    }
    mma_commit_pair(&fin_bar);                   // after every MMA issued above
  } else if (pair_ok && warp >= 2) {
    // ---------------- epilogue warps (both CTAs): warp w reads TMEM lanes 32 (w % 4) ..
    const int q = warp & 3;
    const int gq = (warp - 2) >> 2;
    int i = 0;
    for (int u = cid; u < nunits; u += ncl) {
      const int z = u / ntile, mt = (u % ntile) % mtiles, nt = (u % ntile) / mtiles;
      if (!row_tile_on(mt)) continue;
      const int b = i % G::NBUF, use = i / G::NBUF;
      const int m0 = mt * 256 + 128 * (int)rank;
      const int row = m0 + 32 * q + lane;
      // the node state of the thread's first chunk is loaded before the accumulator is
      // ready, so that its latency overlaps the tile's MMAs
      typename Epi::Chunk ck;
      const int cf = 16 * gq;
      if (cf < BN) epi.load(row, nt * BN + cf, M, N, ck);
      // warp-uniform, so that an epilogue using warp shuffles runs in all lanes or none
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&tfull_bar[b], (uint32_t)(use & 1), err, 4));
      fence_after();
      typename Epi::State es;
      epi.begin(es);
      if (ok) {
#pragma unroll 1
        for (int c = cf; c < BN; c += 16 * (EPIW / 4)) {
          if (c != cf) epi.load(row, nt * BN + c, M, N, ck);
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * G::BUF + c), v);
          epi(row, nt * BN + c, v, M, N, es, ck, epi_smem, z);
        }
      }
      fence_before();
      if (lane == 0) mbar_arrive_cluster(tempty_l + 8u * (uint32_t)b);
      epi.end(32 * q + lane, gq, es, epi_smem);
      uint32_t all_ok;
      asm volatile(
          "{\n .reg .pred p, r;\n setp.ne.u32 p, %1, 0;\n"
          " bar.red.and.pred r, 1, %2, p;\n selp.u32 %0, 1, 0, r;\n}\n"
          : "=r"(all_ok)
          : "r"((uint32_t)ok), "n"(32 * EPIW)
          : "memory");
      if (all_ok) epi.finish(threadIdx.x - 64, 32 * EPIW, m0, nt, M, N, epi_smem);
      asm volatile("bar.sync 1, %0;" ::"n"(32 * EPIW) : "memory");
      ++i;
      if (!all_ok) break;
    }
  }
  // teardown: every MMA of the leader (which writes both CTAs' tensor memory) has
  // completed, no remote signal can still arrive, then the pair frees its columns
  if (pair_ok && warp == 1) {
    if (lane == 0) mbar_wait(&fin_bar, 0u, err, 64);
    __syncwarp();
  }
  fence_before();
  __syncthreads();
  cluster_sync_all();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256)
                 : "memory");
  }
}

// ---- CTA pairs inside a split-K cluster: one 256 x BN tile per cluster
//
// A cluster of 2 cs CTAs computes one 256 x BN output tile: CTA rank r is half h = r & 1
// of pair z = r >> 1, and pair z accumulates the K chunk [z kchunk, (z + 1) kchunk) with
// cta_group::2 MMAs issued by its even CTA (rows [0, 128) of the tile in the even CTA's
// tensor memory, [128, 256) in the odd one's; B rows [BN/2 h, BN/2 (h + 1)) loaded by
// half h).  Against the cluster-reduced kernel (128 x BN tiles, one CTA per K chunk), each
// CTA loads half the B rows per output, so the operand bytes each SM receives drop by a
// quarter at BN = 128.  The partial tiles are then summed through distributed shared
// memory: the cs CTAs of half h each own BN / cs columns, add the pairs' partials in
// pair order (deterministic) and hand each 4-row group to the epilogue (put4 / col as
// for tc_gemm_cred_kernel, col's row tile = 2 mt + h in 128-row tiles).
template <int BN, int NSPLIT>
struct CPairGeo {
  static constexpr int A_BYTES = BM * BK * 2;              // this CTA's 128 rows of A
  static constexpr int B_BYTES = (BN / 2) * BK * 2;        // this CTA's BN/2 rows of B
  static constexpr int STAGE_BYTES =
      A_BYTES * (NSPLIT >= 2 ? 2 : 1) + B_BYTES * (NSPLIT == 3 ? 2 : 1);
  static constexpr int STAGES =
      (196 * 1024) / STAGE_BYTES > 8 ? 8 : (196 * 1024) / STAGE_BYTES;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024;
  static constexpr int TMEM_COLS = BN < 32 ? 32 : BN;
  static_assert(STAGES >= 2, "at least two stages");
  static_assert(STAGES * STAGE_BYTES >= BN * BM * 4, "the partial tile reuses the operand ring");
};

// the leader's commit arrives on the mbarrier at this offset in both CTAs of its pair
// (cluster ranks `first` and first + 1)
__device__ __forceinline__ void mma_commit_pair_at(uint64_t* bar, uint32_t first) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(smem_u32(bar)), "h"((uint16_t)(3u << first))
      : "memory");
}

template <int BN, int NSPLIT, class Epi>
__global__ void __launch_bounds__(64 + 32 * EPI_WARPS, 1)
tc_gemm_cpair_kernel(const __grid_constant__ CUtensorMap ma_hi,
                     const __grid_constant__ CUtensorMap ma_lo,
                     const __grid_constant__ CUtensorMap mb_hi,
                     const __grid_constant__ CUtensorMap mb_lo, int M, int N, int Kred,
                     int kchunk, const int* __restrict__ active, int* err, Epi epi) {
  using G = CPairGeo<BN, NSPLIT>;
  constexpr int S = G::STAGES;
  static_assert(BN % 16 == 0 && BN >= 32 && BN <= 256, "pair MMA N: a multiple of 16 up to 256");
  extern __shared__ uint8_t dsm_raw[];
  __shared__ __align__(8) uint64_t full_bar[S];
  __shared__ __align__(8) uint64_t empty_bar[S];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_slot;
  uint8_t* base = (uint8_t*)(((uintptr_t)dsm_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank(), cs2 = cluster_size();
  const uint32_t h = rank & 1u, z = rank >> 1, first = rank & ~1u;
  const bool leader = h == 0;
  const int tile = (int)(blockIdx.x / cs2);
  const int mtiles = (M + 255) / 256;
  const int mt = tile % mtiles, nt = tile / mtiles;
  const int m0 = mt * 256 + 128 * (int)h;                  // this CTA's first output row
  const int nb = nt * BN;                                  // the tile's first column
  if (active != nullptr) {
    int any = 0;
    for (int j = threadIdx.x; j < BN; j += blockDim.x)
      if (nb + j < N && active[nb + j]) any = 1;
    if (!__syncthreads_or(any)) return;     // the whole cluster shares this tile
  }
  const int kbeg = (int)z * kchunk;
  const int kend = min(Kred, kbeg + kchunk);
  const int nk = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(G::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  cluster_sync_all();                            // every CTA's barriers and TMEM exist
  const uint32_t tmem = tmem_slot;
  uint32_t peer_tmem;
  asm volatile("ld.shared::cluster.u32 %0, [%1];"
               : "=r"(peer_tmem)
               : "r"(mapa_u32(smem_u32(&tmem_slot), rank ^ 1u))
               : "memory");
  const bool pair_ok = peer_tmem == tmem;
  if (!pair_ok && threadIdx.x == 0) atomicOr(err, 32);
  const uint32_t full_l = mapa_u32(smem_u32(&full_bar[0]), first);   // the pair leader's
  float* part = reinterpret_cast<float*>(base);   // [BN][BM] after the main loop

  if (pair_ok && warp == 0 && lane == 0) {
    // ---------------- TMA producer (both CTAs of the pair): this CTA's halves of each stage
    const int brow = nb + (BN / 2) * (int)h;
    long long g = 0;
    for (int kb = 0; kb < nk; ++kb, ++g) {
      const int s = kb % S;
      if (kb >= S && !mbar_wait(&empty_bar[s], (uint32_t)(((kb / S) & 1) ^ 1), err, 1)) break;
      if (leader) mbar_expect_tx(&full_bar[s], 2 * G::STAGE_BYTES);
      const int k = kbeg + kb * BK;
      const uint32_t fb = full_l + 8u * (uint32_t)s;
      uint8_t* st0 = base + s * G::STAGE_BYTES;
      tma_load_2d_pair(st0, &ma_hi, fb, k, m0);
      tma_load_2d_pair(st0 + G::A_BYTES, &mb_hi, fb, k, brow);
      if (NSPLIT >= 2) tma_load_2d_pair(st0 + G::A_BYTES + G::B_BYTES, &ma_lo, fb, k, m0);
      if (NSPLIT == 3) tma_load_2d_pair(st0 + 2 * G::A_BYTES + G::B_BYTES, &mb_lo, fb, k, brow);
    }
    // the leader's last stages count both CTAs' copies: they have all landed before the
    // ring is reused for the partial tile
    if (leader)
      for (long long j = g - S < 0 ? 0 : g - S; j < g; ++j)
        mbar_wait(&full_bar[(int)(j % S)], (uint32_t)((j / S) & 1), err, 16);
  } else if (pair_ok && warp == 1 && lane == 0 && leader) {
    // ---------------- MMA issuer (the pair's even CTA)
    constexpr uint32_t idesc = idesc_bf16_pair(BN);
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % S;
      if (!mbar_wait(&full_bar[s], (uint32_t)((kb / S) & 1), err, 2)) break;
      fence_after();
      uint8_t* st0 = base + s * G::STAGE_BYTES;
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
        const uint64_t ah = smem_desc_sw128(st0 + kk * 32);
        const uint64_t bh = smem_desc_sw128(st0 + G::A_BYTES + kk * 32);
        mma_bf16_pair(tmem, ah, bh, idesc, acc);
        if (NSPLIT >= 2)
          mma_bf16_pair(tmem, smem_desc_sw128(st0 + G::A_BYTES + G::B_BYTES + kk * 32), bh, idesc,
                        1u);
        if (NSPLIT == 3)
          mma_bf16_pair(tmem, ah, smem_desc_sw128(st0 + 2 * G::A_BYTES + G::B_BYTES + kk * 32),
                        idesc, 1u);
      }
      mma_commit_pair_at(&empty_bar[s], first);   // stage s free in both CTAs of the pair
    }
    mma_commit_pair_at(&done_bar, first);         // after every MMA issued above
  } else if (pair_ok && warp >= 2) {
    // ---------------- accumulator -> own partial tile (warp w: TMEM lanes 32 (w % 4) ..)
    const int q = warp & 3, g = (warp - 2) >> 2;
    const bool ok = mbar_wait_cluster(&done_bar, 0, err, 4);
    fence_after();
    const int row = 32 * q + lane;
#pragma unroll 1
    for (int c = 16 * g; c < BN; c += 16 * (EPI_WARPS / 4)) {
      float v[16];
      if (ok && nk > 0) {
        tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c, v);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0.f;
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) part[(c + j) * BM + row] = v[j];
    }
  }
  cluster_sync_all();
  if (pair_ok && warp >= 2) {
    // ---------------- this CTA's columns of its half: the pairs' partials added in order
    const int cs = (int)(cs2 >> 1);
    const int w = warp - 2;
    const int per = (BN + cs - 1) / cs;
    const int c0 = (int)z * per, c1 = min(BN, c0 + per);
    const uint32_t lbase = smem_u32(part);
#pragma unroll 1
    for (int c = c0 + w; c < c1; c += EPI_WARPS) {
      const int n = nb + c;
      if (n >= N) break;                         // warp-uniform; later columns are out too
      const uint32_t off = lbase + (uint32_t)(c * BM + 4 * lane) * 4u;
      float4 pr[4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (r < cs) pr[r] = ld_dsmem_f4(off, 2u * (uint32_t)r + h);
      float4 a = pr[0];
#pragma unroll
      for (int r = 1; r < 4; ++r)
        if (r < cs) {
          a.x += pr[r].x;
          a.y += pr[r].y;
          a.z += pr[r].z;
          a.w += pr[r].w;
        }
      float st[Epi::NSTAT > 0 ? Epi::NSTAT : 1];
#pragma unroll
      for (int k = 0; k < (Epi::NSTAT > 0 ? Epi::NSTAT : 1); ++k) st[k] = 0.f;
      epi.put4(m0 + 4 * lane, n, a, M, N, st);
      if constexpr (Epi::NSTAT > 0) {
        if (epi.stats && m0 < M) {
#pragma unroll
          for (int k = 0; k < Epi::NSTAT; ++k) st[k] = warp_sum(st[k]);
          if (lane == 0) epi.col(2 * mt + (int)h, n, st);
        }
      }
    }
  }
  // teardown: every MMA of the pair has completed, no CTA leaves while its tile is read,
  // then the pair frees its columns
  if (pair_ok && warp == 1) {
    if (lane == 0) mbar_wait_cluster(&done_bar, 0, err, 64);
    __syncwarp();
  }
  cluster_sync_all();
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(G::TMEM_COLS)
                 : "memory");
  }
}

}  // namespace tc
}  // namespace bnb
