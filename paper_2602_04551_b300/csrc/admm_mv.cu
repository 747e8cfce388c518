// admm_mv.cu -- the batched ADMM iteration for narrow node batches: coalesced
// matrix-vector products on CUDA cores instead of tensor-core tiles.
//
// Same iteration and the same state as admm_tc.cu (Sections 3.1-3.2, the shifted
// Woodbury b-update: W' = rho beta - V, U' = G^{-1} X W' = H W', b = b_c + (W' - X^T U')/rho,
// prox, v-update), in FP32 on FP32 data, for the active slots listed by k_act_list
// (at most MV_MAX of them).  With a few active nodes a 128-wide tensor-core tile is
// almost all padding, while these kernels read X once per product and do only the
// useful work:
//   k_mv_part     Y_c = A v_c over a chunk of the contraction (one thread per output row,
//                 A = H = G^-1 X for U' = H W', A = X for the check product X beta;
//                 coalesced column reads of the column-major A, the vectors of 8 slots
//                 staged in shared memory); partial sums per chunk
//   k_mv_reduce   sum of the chunks in order, plus the product's epilogue (T; U', U and
//                 the stop-test sums of r = y - U; the check ||y - X beta||^2)
//   k_mv_prox     X^T U' by warp-reduction dot products (one warp per feature column,
//                 lanes over the samples, U' of 8 slots in shared memory) fused with the
//                 coordinate update of Eq. minbetalower and the v-update
// They write exactly what the tensor-core round writes (beta, V, U, the per-tile sums
// read by the stop test), so the stop test, the certificate and the node pool do not
// depend on which form ran.  The choice is made per round on the device (a CUDA-graph
// conditional node on the active-slot count) or, outside a graph, by the host.
#include <vector>
#include "engine.cuh"

namespace bnb {

constexpr int MV_G = 8;      // slots per block group
constexpr int MV_TJ = 64;    // contraction step staged in shared memory

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
// grid (ceil(M / 256), Z, ceil(MV_MAX / MV_G)); block 256.
template <int MODE>
__global__ void __launch_bounds__(256) k_mv_part(const float* __restrict__ A, long long lda, int M,
                                                 int L, int zchunk,
                                                 const int* __restrict__ act_list,
                                                 const int* __restrict__ act_count,
                                                 const float* __restrict__ beta,
                                                 const float* __restrict__ V, float rho,
                                                 const float* __restrict__ src, long long ldv,
                                                 float* __restrict__ part) {
  __shared__ float vs[MV_G][MV_TJ];
  const int a = min(*act_count, MV_MAX);
  const int c0 = blockIdx.z * MV_G;
  if (c0 >= a) return;
  const int nc = min(MV_G, a - c0);
  const int i = blockIdx.x * 256 + threadIdx.x;
  const int j0 = blockIdx.y * zchunk, j1 = min(L, j0 + zchunk);
  float acc[MV_G];
#pragma unroll
  for (int c = 0; c < MV_G; ++c) acc[c] = 0.f;
  for (int jb = j0; jb < j1; jb += MV_TJ) {
    for (int e = threadIdx.x; e < MV_G * MV_TJ; e += 256) {
      const int c = e / MV_TJ, jj = e % MV_TJ, j = jb + jj;
      vs[c][jj] = (c < nc && j < j1) ? mv_vec<MODE>(act_list[c0 + c], j, beta, V, rho, src, ldv)
                                     : 0.f;
    }
    __syncthreads();
    if (i < M) {
      const int jn = min(MV_TJ, j1 - jb);
      const float* ap = A + (long long)jb * lda + i;
      int jj = 0;
      for (; jj + 4 <= jn; jj += 4) {          // four independent column loads in flight
        float x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = ap[(long long)(jj + u) * lda];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int c = 0; c < MV_G; ++c) acc[c] = fmaf(x[u], vs[c][jj + u], acc[c]);
      }
      for (; jj < jn; ++jj) {
        const float x = ap[(long long)jj * lda];
#pragma unroll
        for (int c = 0; c < MV_G; ++c) acc[c] = fmaf(x, vs[c][jj], acc[c]);
      }
    }
    __syncthreads();
  }
  if (i < M)
    for (int c = 0; c < nc; ++c) part[((long long)blockIdx.y * MV_MAX + c0 + c) * M + i] = acc[c];
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

// X^T U' by warp-reduction dot products, fused with the coordinate update.
// grid (ceil(p / 128), ceil(MV_MAX / MV_G)); block 256 (8 warps x 16 columns);
// dynamic shared memory MV_G x n floats (U' of the group's slots).
// With stats (the round's last iteration) the per-slot sums of psi(beta), nu(|X^T r|),
// ||beta - beta_prev||^2, ||b - beta||^2 over the block's 128 columns go to
// g3part[stat][block][slot] (the layout the tensor-core epilogue writes).
__global__ void __launch_bounds__(256) k_mv_prox(const float* __restrict__ X, int n, int p,
                                                 const float* __restrict__ Up,
                                                 const int* __restrict__ act_list,
                                                 const int* __restrict__ act_count,
                                                 const float* __restrict__ bc,
                                                 const float* __restrict__ rbc,
                                                 float* __restrict__ beta, float* __restrict__ V,
                                                 const int8_t* __restrict__ fix, Prob P, ProbF PF,
                                                 int stats, float* __restrict__ g3part, int nbm,
                                                 int K) {
  extern __shared__ float us[];            // [MV_G][n]
  __shared__ float wst[8][4][MV_G];        // per-warp stop-test sums
  const int a = min(*act_count, MV_MAX);
  const int c0 = blockIdx.y * MV_G;
  if (c0 >= a) return;
  const int nc = min(MV_G, a - c0);
  for (int e = threadIdx.x; e < MV_G * n; e += blockDim.x) {
    const int c = e / n, i = e % n;
    us[e] = c < nc ? Up[(long long)act_list[c0 + c] * n + i] : 0.f;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int s_l = lane < nc ? act_list[c0 + lane] : 0;   // lane c < nc updates slot c
  float st0 = 0.f, st1 = 0.f, st2 = 0.f, st3 = 0.f;
  for (int jj = 0; jj < 16; ++jj) {
    const int j = blockIdx.x * 128 + w * 16 + jj;
    if (j >= p) break;                                     // warp-uniform
    const float* xj = X + (long long)j * n;
    float acc[MV_G];
#pragma unroll
    for (int c = 0; c < MV_G; ++c) acc[c] = 0.f;
    for (int i = lane; i < n; i += 32) {
      const float x = xj[i];
#pragma unroll
      for (int c = 0; c < MV_G; ++c) acc[c] = fmaf(x, us[c * n + i], acc[c]);
    }
    float mine = 0.f;
#pragma unroll
    for (int c = 0; c < MV_G; ++c) {
      const float t = warp_sum(acc[c]);
      if (lane == c) mine = t;
    }
    if (lane < nc) {
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
  if (!stats) return;
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
      for (int ww = 0; ww < 8; ++ww) sum += wst[ww][t][c];
      g3part[((long long)t * nbm + blockIdx.x) * K + act_list[c0 + c]] = sum;
    }
  }
}

// ----------------------------------------------------------------------------- host

// chunks of the contraction for k_mv_part: enough blocks to cover the SMs
static int mv_chunks(int M, int L, int* zchunk) {
  const int rows = (M + 255) / 256;
  int Z = (2 * 148 + rows - 1) / rows;
  const int zmax = (L + MV_TJ - 1) / MV_TJ;
  if (Z > zmax) Z = zmax;
  if (Z > MV_ZMAX) Z = MV_ZMAX;
  if (Z < 1) Z = 1;
  int zc = (L + Z - 1) / Z;
  zc = (zc + MV_TJ - 1) / MV_TJ * MV_TJ;
  *zchunk = zc;
  return (L + zc - 1) / zc;
}

int admm_iterations_mv(Engine<float>& e, int iters) {
  const int n = e.n, p = e.p, K = e.K;
  cudaStream_t st = e.st;
  const int G = (MV_MAX + MV_G - 1) / MV_G;
  int zc1 = 0;
  const int Z1 = mv_chunks(n, p, &zc1);          // H W' and X beta: contraction over p
  const dim3 g1((n + 255) / 256, Z1, G);
  const dim3 gr((n + 127) / 128, MV_MAX);
  const ProbF PF = prob_f32(e.P);
  const size_t ush = sizeof(float) * MV_G * (size_t)n;
  for (int it = 0; it < iters; ++it) {
    const int last = it + 1 == iters;
    // U' = H W' with H = G^-1 X (one product), then U and the stop-test sums
    prof_begin(e.prof, st);
    k_mv_part<0><<<g1, 256, 0, st>>>(e.H32, n, n, p, zc1, e.act_list, e.act_count, e.beta, e.V,
                                     PF.rho, nullptr, p, e.mv_part);
    k_mv_reduce<1><<<gr, 128, 0, st>>>(e.mv_part, Z1, n, e.act_list, e.act_count, e.Up, e.U,
                                       e.ucR, e.yR, last, e.tc_stat, e.nbt, K);
    prof_end(e.prof, st, PK_GEMM_XW);
    prof_begin(e.prof, st);
    k_mv_prox<<<dim3((p + 127) / 128, G), 256, ush, st>>>(
        (const float*)e.X32, n, p, e.Up, e.act_list, e.act_count, e.bcR, e.rbcR, e.beta, e.V,
        e.fix, e.P, PF, last, e.g3part, e.nbm3, K);
    prof_end(e.prof, st, PK_GEMM_XTU);
    BNB_CUDA_OK(cudaGetLastError());
  }
  // check product X beta
  prof_begin(e.prof, st);
  k_mv_part<1><<<g1, 256, 0, st>>>((const float*)e.X32, n, n, p, zc1, e.act_list, e.act_count,
                                   e.beta, nullptr, 0.f, nullptr, p, e.mv_part);
  k_mv_reduce<2><<<gr, 128, 0, st>>>(e.mv_part, Z1, n, e.act_list, e.act_count, nullptr, nullptr,
                                     nullptr, e.yR, 1, e.tc_stat, e.nbt, K);
  prof_end(e.prof, st, PK_CHECK);
  BNB_CUDA_OK(cudaGetLastError());
  return 0;
}

int mv_setup(Engine<float>& e) {
  const size_t ush = sizeof(float) * MV_G * (size_t)e.n;
  if (ush > 200 * 1024) {
    e.mv_cross = 0;                               // U' of a group does not fit: no matvec form
    return 0;
  }
  BNB_CUDA_OK(cudaFuncSetAttribute(k_mv_prox, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
