// admm_mv.cu -- the batched ADMM iteration for narrow node batches: coalesced
// matrix-vector products on CUDA cores instead of tensor-core tiles.
//
// Same iteration and the same state as admm_tc.cu (Sections 3.1-3.2, the shifted
// Woodbury b-update: W' = rho beta - V, U' = G^{-1} X W' = H W', b = b_c + (W' - X^T U')/rho,
// prox, v-update), in FP32 on FP32 data, for the active slots listed by k_act_list
// (at most MV_MAX of them).  With a few active nodes a 128-wide tensor-core tile is
// almost all padding, while these kernels read X once per product and do only the
// useful work:
//   k_mv_part     Y_c = A v_c over a chunk of the contraction (lanes over 4 output rows
//                 each with float4 loads of the column-major A, the chunk's columns over
//                 8 warps with eight in flight each, the vectors of 16 slots staged in
//                 shared memory, warp partials added in order); A = H = G^-1 X for
//                 U' = H W', A = X for the check product X beta; partial sums per chunk
//   k_mv_reduce   sum of the chunks in order, plus the product's epilogue (T; U', U and
//                 the stop-test sums of r = y - U; the check ||y - X beta||^2)
//   k_mv_prox     X^T U' for 32 feature columns per block: a warp takes four columns,
//                 lanes over the samples (float4), U' of 16 slots in shared memory
//                 (asynchronous copies); the 64 dot products of a warp are reduce-scattered so that
//                 each lane ends with two (column, slot) totals and applies the
//                 coordinate update of Eq. minbetalower and the v-update to them
//   k_mv_fold     the per-32-column stop-test sums folded into the per-128-column
//                 layout the stop test reads (last iteration only)
// They write exactly what the tensor-core round writes (beta, V, U, the per-tile sums
// read by the stop test), so the stop test, the certificate and the node pool do not
// depend on which form ran.  The choice is made per round on the device (a CUDA-graph
// conditional node on the active-slot count) or, outside a graph, by the host.
#include <vector>
#include "engine.cuh"

namespace bnb {

constexpr int MV_G = 16;     // slots per group
constexpr int MV_PC = 32;    // feature columns per block of k_mv_prox

// ordered list of the active slots (single block)
__global__ void k_act_list(int K, const int* __restrict__ slot_active, int* __restrict__ act_list,
                           int* __restrict__ act_count) {
  __shared__ int wsum[32];
  __shared__ int base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int s0 = 0; s0 < K; s0 += blockDim.x) {
    const int s = s0 + threadIdx.x;
    const int f = (s < K) ? (slot_active[s] != 0) : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    int off = base;
    for (int t = 0; t < w; ++t) off += wsum[t];
    if (f) act_list[off + __popc(bal & ((1u << lane) - 1u))] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int t = 0; t < nw; ++t) tot += wsum[t];
      base += tot;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *act_count = base;
}

// condition of the round's IF node: 1 = matrix-vector form
__global__ void k_set_mv_cond(cudaGraphConditionalHandle h, const int* __restrict__ act_count,
                              int cross) {
  if (threadIdx.x == 0) cudaGraphSetConditional(h, *act_count <= cross ? 1u : 0u);
}

// Vector c of the group for contraction index j:
//   MODE 0: W'_s = rho beta_s - V_s;  MODE 1: beta_s;  MODE 2: src_s (slot-major, ld ldv)
template <int MODE>
__device__ __forceinline__ float mv_vec(int s, long long j, const float* beta, const float* V,
                                        float rho, const float* src, long long ldv) {
  const long long o = (long long)s * ldv + j;
  if (MODE == 0) return rho * beta[o] - V[o];
  if (MODE == 1) return beta[o];
  return src[o];
}

// part[z][c][i] = sum_{j in chunk z} A[i + j lda] v_c[j],  c = compact slot index.
// A block takes 32 R rows (lanes over the rows, R per lane: float4 loads for R = 4, which
// needs lda and M multiples of 4) and the chunk's columns interleaved over its 8 warps
// (eight columns in flight per warp); the warps' partial sums are added in warp order in
// shared memory.  grid (ceil(M / (32 R)), Z, MV_MAX / MV_G); block 256; dynamic shared
// memory (MV_G zchunk + 8 MV_G 32 R) floats: the chunk's vectors, then the partials.
template <int MODE, int R>
__global__ void __launch_bounds__(256) k_mv_part(const float* __restrict__ A, long long lda, int M,
                                                 int L, int zchunk,
                                                 const int* __restrict__ act_list,
                                                 const int* __restrict__ act_count,
                                                 const float* __restrict__ beta,
                                                 const float* __restrict__ V, float rho,
                                                 const float* __restrict__ src, long long ldv,
                                                 float* __restrict__ part) {
  extern __shared__ float smv[];
  constexpr int RB = 32 * R;                              // rows of the block
  float* vs = smv;                                        // [MV_G][zchunk]
  float* red = smv + MV_G * zchunk;                       // [8][MV_G][RB]
  const int a = min(*act_count, MV_MAX);
  const int c0 = blockIdx.z * MV_G;
  if (c0 >= a) return;
  const int nc = min(MV_G, a - c0);
  const int j0 = blockIdx.y * zchunk, jn = min(L, j0 + zchunk) - j0;
  for (int e = threadIdx.x; e < MV_G * zchunk; e += blockDim.x) {
    const int c = e / zchunk, jj = e % zchunk;
    vs[e] = (c < nc && jj < jn) ? mv_vec<MODE>(act_list[c0 + c], j0 + jj, beta, V, rho, src, ldv)
                                : 0.f;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i0 = blockIdx.x * RB + lane * R;
  float acc[R][MV_G];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < MV_G; ++c) acc[r][c] = 0.f;
  if (i0 < M) {
    const float* ap = A + (long long)j0 * lda + i0;
    int jj = w;                                           // this warp: columns w, w + 8, ...
    for (; jj + 56 < jn; jj += 64) {
      float x[8][R];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float* q = ap + (long long)(jj + 8 * u) * lda;
        if constexpr (R == 4) {
          const float4 t = *reinterpret_cast<const float4*>(q);
          x[u][0] = t.x;
          x[u][1] = t.y;
          x[u][2] = t.z;
          x[u][3] = t.w;
        } else {
          x[u][0] = q[0];
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int c = 0; c < MV_G; ++c) {
          const float wv = vs[c * zchunk + jj + 8 * u];
#pragma unroll
          for (int r = 0; r < R; ++r) acc[r][c] = fmaf(x[u][r], wv, acc[r][c]);
        }
    }
    for (; jj < jn; jj += 8) {
      const float* q = ap + (long long)jj * lda;
      float x[R];
      if constexpr (R == 4) {
        const float4 t = *reinterpret_cast<const float4*>(q);
        x[0] = t.x;
        x[1] = t.y;
        x[2] = t.z;
        x[3] = t.w;
      } else {
        x[0] = q[0];
      }
#pragma unroll
      for (int c = 0; c < MV_G; ++c) {
        const float wv = vs[c * zchunk + jj];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r][c] = fmaf(x[r], wv, acc[r][c]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < MV_G; ++c)
#pragma unroll
    for (int r = 0; r < R; ++r) red[(w * MV_G + c) * RB + lane * R + r] = acc[r][c];
  __syncthreads();
  for (int e = threadIdx.x; e < nc * RB; e += blockDim.x) {
    const int c = e / RB, rr = e % RB;
    const int i = blockIdx.x * RB + rr;
    if (i < M) {
      float sum = 0.f;
#pragma unroll
      for (int ww = 0; ww < 8; ++ww) sum += red[(ww * MV_G + c) * RB + rr];
      part[((long long)blockIdx.y * MV_MAX + c0 + c) * M + i] = sum;
    }
  }
}

// Sum of the Z chunks in order, per (128-row block, compact slot); block 128.
//   MODE 0 (T):     out[s n + i] = sum
//   MODE 1 (U'):    out[s n + i] = U';  with stats also U = u_c + U' and the per-block sums
//                   ||y - U||^2 -> stat[0], y^T (y - U) -> stat[1]
//   MODE 2 (check): per-block sums ||y - X beta||^2 -> stat[2]
template <int MODE>
__global__ void __launch_bounds__(128) k_mv_reduce(const float* __restrict__ part, int Z, int M,
                                                   const int* __restrict__ act_list,
                                                   const int* __restrict__ act_count,
                                                   float* __restrict__ out, float* __restrict__ U,
                                                   const float* __restrict__ uc,
                                                   const float* __restrict__ y, int stats,
                                                   float* __restrict__ stat, int nbt, int K) {
  __shared__ float sh[32];
  const int c = blockIdx.y;
  if (c >= min(*act_count, MV_MAX)) return;
  const int s = act_list[c];
  const int i = blockIdx.x * 128 + threadIdx.x;
  float v = 0.f;
  if (i < M)
#pragma unroll 8
    for (int z = 0; z < Z; ++z) v += part[((long long)z * MV_MAX + c) * M + i];
  float r0 = 0.f, r1 = 0.f;
  if (i < M) {
    if (MODE == 0) {
      out[(long long)s * M + i] = v;
    } else if (MODE == 1) {
      out[(long long)s * M + i] = v;
      if (stats) {
        const float u = uc[i] + v;
        U[(long long)s * M + i] = u;
        const float r = y[i] - u;
        r0 = r * r;
        r1 = y[i] * r;
      }
    } else {
      const float r = y[i] - v;
      r0 = r * r;
    }
  }
  if (MODE == 1 && stats) {
    r0 = block_sum(r0, sh);
    r1 = block_sum(r1, sh);
    if (threadIdx.x == 0) {
      stat[(0LL * nbt + blockIdx.x) * K + s] = r0;
      stat[(1LL * nbt + blockIdx.x) * K + s] = r1;
    }
  } else if (MODE == 2) {
    r0 = block_sum(r0, sh);
    if (threadIdx.x == 0) stat[(2LL * nbt + blockIdx.x) * K + s] = r0;
  }
}

// One reduce-scatter step over 2H values: the lanes with bit H set keep the upper half,
// the others the lower half, each adding the partner lane's copy of the half it keeps.
template <int H>
__device__ __forceinline__ void rs_step(float* v, int lane) {
  const bool up = (lane & H) != 0;
#pragma unroll
  for (int k = 0; k < H; ++k) {
    const float send = up ? v[k] : v[k + H];
    const float keep = up ? v[k + H] : v[k];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, H);
  }
}
// 32 per-lane values -> lane l holds the warp total of value l (31 shuffles)
__device__ __forceinline__ float reduce_scatter32(float* v, int lane) {
  rs_step<16>(v, lane);
  rs_step<8>(v, lane);
  rs_step<4>(v, lane);
  rs_step<2>(v, lane);
  rs_step<1>(v, lane);
  return v[0];
}

// X^T U' for MV_PC feature columns per block, fused with the coordinate update.
// grid (ceil(p / MV_PC), MV_MAX / MV_G); block 256 (8 warps x 4 columns); dynamic shared
// memory MV_G x nu floats (U' of the group's slots, nu = n rounded up to 4, zero
// padded), staged with asynchronous 16-byte copies when n is a multiple of 4.
// W = 4: float4 loads along the samples (n a multiple of 4), else 1.  Lane l owns the
// totals (column l / 16, slot l % 16) and (column 2 + l / 16, slot l % 16) of its
// warp's four columns.  With stats (the round's last iteration) the per-slot sums of
// psi(beta), nu(|X^T r|), ||beta - beta_prev||^2, ||b - beta||^2 over the block's
// columns go to g3mv[stat][block][compact slot index].
template <int W>
__global__ void __launch_bounds__(256) k_mv_prox(const float* __restrict__ X, int n, int p,
                                                 const float* __restrict__ Up,
                                                 const int* __restrict__ act_list,
                                                 const int* __restrict__ act_count,
                                                 const float* __restrict__ bc,
                                                 const float* __restrict__ rbc,
                                                 float* __restrict__ beta, float* __restrict__ V,
                                                 const int8_t* __restrict__ fix, Prob P, ProbF PF,
                                                 int stats, float* __restrict__ g3mv, int nb32) {
  extern __shared__ float us[];            // [MV_G][nu]
  __shared__ float wst[8][4][MV_G];        // per-warp stop-test sums
  const int a = min(*act_count, MV_MAX);
  const int c0 = blockIdx.y * MV_G;
  if (c0 >= a) return;
  const int nc = min(MV_G, a - c0);
  const int nu = (n + 3) & ~3;
  if constexpr (W == 4) {
    // nu == n: every 16-byte chunk of a slot's row is copied without waiting in between
    const int q4 = n / 4;
    for (int e = threadIdx.x; e < MV_G * q4; e += blockDim.x) {
      const int c = e / q4, i4 = e % q4;
      float* dst = us + c * nu + 4 * i4;
      if (c < nc) {
        const float* src = Up + (long long)act_list[c0 + c] * n + 4 * i4;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(dst)),
                     "l"(src)
                     : "memory");
      } else {
        *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
  } else {
    for (int e = threadIdx.x; e < MV_G * nu; e += blockDim.x) {
      const int c = e / nu, i = e % nu;
      us[e] = (c < nc && i < n) ? Up[(long long)act_list[c0 + c] * n + i] : 0.f;
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int cs = lane & 15;                               // the lane's slot in the group
  const int s_l = cs < nc ? act_list[c0 + cs] : 0;
  float st0 = 0.f, st1 = 0.f, st2 = 0.f, st3 = 0.f;
  const int jb = blockIdx.x * MV_PC + w * 4;              // this warp's columns jb .. jb + 3
  if (jb < p) {                                           // warp-uniform
    const float* xc[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) xc[t] = X + (long long)min(jb + t, p - 1) * n;
    float acc[4 * MV_G];
#pragma unroll
    for (int k = 0; k < 4 * MV_G; ++k) acc[k] = 0.f;
#pragma unroll 4
    for (int i = W * lane; i < n; i += 32 * W) {
      float x[4][W];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if constexpr (W == 4) {
          const float4 v4 = *reinterpret_cast<const float4*>(xc[t] + i);
          x[t][0] = v4.x;
          x[t][1] = v4.y;
          x[t][2] = v4.z;
          x[t][3] = v4.w;
        } else {
          x[t][0] = xc[t][i];
        }
      }
#pragma unroll
      for (int c = 0; c < MV_G; ++c) {
        float u[W];
        if constexpr (W == 4) {
          const float4 u4 = *reinterpret_cast<const float4*>(us + c * nu + i);
          u[0] = u4.x;
          u[1] = u4.y;
          u[2] = u4.z;
          u[3] = u4.w;
        } else {
          u[0] = us[c * nu + i];
        }
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
          for (int r = 0; r < W; ++r) acc[t * MV_G + c] = fmaf(x[t][r], u[r], acc[t * MV_G + c]);
      }
    }
    float tot[2];
    tot[0] = reduce_scatter32(acc, lane);                 // (column lane / 16, slot cs)
    tot[1] = reduce_scatter32(acc + 32, lane);            // (column 2 + lane / 16, slot cs)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = jb + 2 * h + (lane >> 4);
      if (cs < nc && j < p) {
        const float mine = tot[h];
        const long long o = (long long)s_l * p + j;
        const float bo = beta[o], vv = V[o];
        const int ff = fix[o];
        const float wv = PF.rho * bo - vv;
        const float b = bc[j] + (wv - mine) * PF.irho;
        const float bh = PF.alpha * b + PF.one_minus_alpha * bo;
        const float bn = prox_coord_f(bh + vv * PF.irho, ff, PF);
        const float vn = vv + PF.rho * (bh - bn);
        beta[o] = bn;
        V[o] = vn;
        if (stats) {
          st0 += psi_coord<float>(bn, ff, P);
          st1 += nu_coord<float>(fabsf(rbc[j] - mine), ff, P);
          st2 += (bn - bo) * (bn - bo);
          st3 += (b - bn) * (b - bn);
        }
      }
    }
  }
  if (!stats) return;
  // lanes l and l + 16 hold the same slot
  st0 += __shfl_xor_sync(0xffffffffu, st0, 16);
  st1 += __shfl_xor_sync(0xffffffffu, st1, 16);
  st2 += __shfl_xor_sync(0xffffffffu, st2, 16);
  st3 += __shfl_xor_sync(0xffffffffu, st3, 16);
  if (lane < MV_G) {
    wst[w][0][lane] = st0;
    wst[w][1][lane] = st1;
    wst[w][2][lane] = st2;
    wst[w][3][lane] = st3;
  }
  __syncthreads();
  if (threadIdx.x < 4 * MV_G) {
    const int t = threadIdx.x / MV_G, c = threadIdx.x % MV_G;
    if (c < nc) {
      float sum = 0.f;
#pragma unroll
      for (int ww = 0; ww < 8; ++ww) sum += wst[ww][t][c];
      g3mv[((long long)t * nb32 + blockIdx.x) * MV_MAX + c0 + c] = sum;
    }
  }
}

// g3part[stat][b][slot] = sum over the (up to) four 32-column blocks of the 128-column
// block b, in order.  grid (ceil(nbm / 32), MV_MAX); block 128 = 32 blocks b x 4 stats.
__global__ void k_mv_fold(const float* __restrict__ g3mv, int nb32, const int* __restrict__ act_list,
                          const int* __restrict__ act_count, float* __restrict__ g3part, int nbm,
                          int K) {
  const int c = blockIdx.y;
  const int b = blockIdx.x * 32 + (threadIdx.x >> 2), t = threadIdx.x & 3;
  if (c >= min(*act_count, MV_MAX) || b >= nbm) return;
  float sum = 0.f;
  for (int q = 0; q < 4; ++q) {
    const int b32 = 4 * b + q;
    if (b32 < nb32) sum += g3mv[((long long)t * nb32 + b32) * MV_MAX + c];
  }
  g3part[((long long)t * nbm + b) * K + act_list[c]] = sum;
}

// ----------------------------------------------------------------------------- host

// chunks of the contraction for k_mv_part: about two blocks per SM, chunks of at most
// MV_ZCOL columns (a multiple of 8: the warps' column interleave)
constexpr int MV_ZCOL = 1024;
static int mv_chunks(int M, int L, int R, int sms, int* zchunk) {
  const int rows = (M + 32 * R - 1) / (32 * R);
  int Z = (2 * sms + rows - 1) / rows;
  if (Z < (L + MV_ZCOL - 1) / MV_ZCOL) Z = (L + MV_ZCOL - 1) / MV_ZCOL;
  if (Z > MV_ZMAX) Z = MV_ZMAX;
  if (Z > (L + 7) / 8) Z = (L + 7) / 8;
  if (Z < 1) Z = 1;
  int zc = (L + Z - 1) / Z;
  zc = (zc + 7) / 8 * 8;
  *zchunk = zc;
  return (L + zc - 1) / zc;
}

static size_t mv_part_smem(int zc, int R) {
  return sizeof(float) * ((size_t)MV_G * zc + (size_t)8 * MV_G * 32 * R);
}

template <int MODE>
static void mv_part(Engine<float>& e, const float* A, int Z, int zc, int R, const float* beta,
                    const float* V, float rho) {
  const int n = e.n, p = e.p, G = MV_MAX / MV_G;
  const size_t sh = mv_part_smem(zc, R);
  if (R == 4)
    k_mv_part<MODE, 4><<<dim3((n + 127) / 128, Z, G), 256, sh, e.st>>>(
        A, n, n, p, zc, e.act_list, e.act_count, beta, V, rho, nullptr, p, e.mv_part);
  else
    k_mv_part<MODE, 1><<<dim3((n + 31) / 32, Z, G), 256, sh, e.st>>>(
        A, n, n, p, zc, e.act_list, e.act_count, beta, V, rho, nullptr, p, e.mv_part);
}

int admm_iterations_mv(Engine<float>& e, int iters) {
  const int n = e.n, p = e.p, K = e.K;
  cudaStream_t st = e.st;
  const int G = MV_MAX / MV_G;
  const int R = (n % 4 == 0) ? 4 : 1;             // float4 rows (H, X columns 16-byte aligned)
  int zc1 = 0;
  const int Z1 = mv_chunks(n, p, R, e.sms > 0 ? e.sms : 148, &zc1);   // contraction over p
  const dim3 gr((n + 127) / 128, MV_MAX);
  const ProbF PF = prob_f32(e.P);
  const size_t ush = sizeof(float) * MV_G * (size_t)((n + 3) & ~3);
  const int nb32 = (p + MV_PC - 1) / MV_PC;
  for (int it = 0; it < iters; ++it) {
    const int last = it + 1 == iters;
    // U' = H W' with H = G^-1 X (one product), then U and the stop-test sums
    prof_begin(e.prof, st);
    mv_part<0>(e, e.H32, Z1, zc1, R, e.beta, e.V, PF.rho);
    k_mv_reduce<1><<<gr, 128, 0, st>>>(e.mv_part, Z1, n, e.act_list, e.act_count, e.Up, e.U,
                                       e.ucR, e.yR, last, e.tc_stat, e.nbt, K);
    prof_end(e.prof, st, PK_GEMM_XW);
    prof_begin(e.prof, st);
    if (R == 4)
      k_mv_prox<4><<<dim3(nb32, G), 256, ush, st>>>(
          (const float*)e.X32, n, p, e.Up, e.act_list, e.act_count, e.bcR, e.rbcR, e.beta, e.V,
          e.fix, e.P, PF, last, e.g3mv, nb32);
    else
      k_mv_prox<1><<<dim3(nb32, G), 256, ush, st>>>(
          (const float*)e.X32, n, p, e.Up, e.act_list, e.act_count, e.bcR, e.rbcR, e.beta, e.V,
          e.fix, e.P, PF, last, e.g3mv, nb32);
    if (last)
      k_mv_fold<<<dim3((e.nbm3 + 31) / 32, MV_MAX), 128, 0, st>>>(
          e.g3mv, nb32, e.act_list, e.act_count, e.g3part, e.nbm3, K);
    prof_end(e.prof, st, PK_GEMM_XTU);
    BNB_CUDA_OK(cudaGetLastError());
  }
  // check product X beta
  prof_begin(e.prof, st);
  mv_part<1>(e, (const float*)e.X32, Z1, zc1, R, e.beta, nullptr, 0.f);
  k_mv_reduce<2><<<gr, 128, 0, st>>>(e.mv_part, Z1, n, e.act_list, e.act_count, nullptr, nullptr,
                                     nullptr, e.yR, 1, e.tc_stat, e.nbt, K);
  prof_end(e.prof, st, PK_CHECK);
  BNB_CUDA_OK(cudaGetLastError());
  return 0;
}

int mv_setup(Engine<float>& e) {
  const size_t ush = sizeof(float) * MV_G * (size_t)((e.n + 3) & ~3);
  if (ush > 200 * 1024) {
    e.mv_cross = 0;                               // U' of a group does not fit: no matvec form
    return 0;
  }
  const int psh = (int)mv_part_smem(MV_ZCOL, 4);  // the largest chunk
  BNB_CUDA_OK(cudaFuncSetAttribute(k_mv_part<0, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, psh));
  BNB_CUDA_OK(cudaFuncSetAttribute(k_mv_part<1, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, psh));
  BNB_CUDA_OK(cudaFuncSetAttribute(k_mv_part<0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, psh));
  BNB_CUDA_OK(cudaFuncSetAttribute(k_mv_part<1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, psh));
  BNB_CUDA_OK(cudaFuncSetAttribute(k_mv_prox<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)ush));
  BNB_CUDA_OK(cudaFuncSetAttribute(k_mv_prox<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)ush));
  return 0;
}

int act_list(Engine<float>& e) {
  k_act_list<<<1, 1024, 0, e.st>>>(e.K, e.slot_active, e.act_list, e.act_count);
  BNB_CUDA_OK(cudaGetLastError());
  return 0;
}

static int count_kernels(cudaGraph_t g) {
  size_t nn = 0;
  if (cudaGraphGetNodes(g, nullptr, &nn) != cudaSuccess) return 0;
  std::vector<cudaGraphNode_t> nodes(nn);
  cudaGraphGetNodes(g, nodes.data(), &nn);
  int k = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    cudaGraphNodeGetType(nd, &t);
    k += t == cudaGraphNodeTypeKernel ? 1 : 0;
  }
  return k;
}

// Inside a stream capture: a kernel sets a conditional handle from the active-slot
// count, and an IF/ELSE node runs the matrix-vector iterations (IF) or the tensor-core
// iterations (ELSE); the two bodies are captured on the side stream.
int capture_mv_or_tc(Engine<float>& e, int iters) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  BNB_CUDA_OK(cudaStreamGetCaptureInfo(e.st, &cs, nullptr, &g, &deps, nullptr, &nd));
  cudaGraphConditionalHandle hd;
  BNB_CUDA_OK(cudaGraphConditionalHandleCreate(&hd, g, 0, 0));
  k_set_mv_cond<<<1, 32, 0, e.st>>>(hd, e.act_count, e.mv_cross);
  BNB_CUDA_OK(cudaGetLastError());
  BNB_CUDA_OK(cudaStreamGetCaptureInfo(e.st, &cs, nullptr, &g, &deps, nullptr, &nd));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = hd;
  np.conditional.type = cudaGraphCondTypeIf;
  np.conditional.size = 2;
  cudaGraphNode_t cn;
  BNB_CUDA_OK(cudaGraphAddNode(&cn, g, deps, nullptr, nd, &np));
  cudaGraph_t bodies[2] = {np.conditional.phGraph_out[0], np.conditional.phGraph_out[1]};
  cudaStream_t main_st = e.st;
  for (int b = 0; b < 2; ++b) {
    BNB_CUDA_OK(cudaStreamBeginCaptureToGraph(e.st_side, bodies[b], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeRelaxed));
    e.st = e.st_side;
    const int rc = b == 0 ? admm_iterations_mv(e, iters) : admm_iterations_tc(e, iters);
    e.st = main_st;
    cudaGraph_t tmp = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(e.st_side, &tmp);
    if (rc) return rc;
    BNB_CUDA_OK(ce);
  }
  e.mv_body_kernels = count_kernels(bodies[0]);
  e.tc_body_kernels = count_kernels(bodies[1]);
  BNB_CUDA_OK(cudaStreamUpdateCaptureDependencies(e.st, &cn, nullptr, 1,
                                                  cudaStreamSetCaptureDependencies));
  return 0;
}

}  // namespace bnb
