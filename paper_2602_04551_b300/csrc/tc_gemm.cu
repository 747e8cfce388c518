// tc_gemm.cu -- host side of the tcgen05 contraction: tensor maps and launches,
// plus the BF16 hi/lo operand splits the 3-term product uses.
#include <cudaTypedefs.h>
#include <mutex>
#include "tc_gemm.cuh"
#include "tc_host.cuh"

namespace bnb {

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

// 2D BF16 tensor with `inner` contiguous elements per row (leading dimension `ld`
// elements, a multiple of 8) and `rows` rows; box = 64 x box_rows, 128-byte swizzle.
int make_map_bf16(CUtensorMap* map, const void* ptr, long long inner, long long rows, long long ld,
                  int box_rows) {
  auto fn = encode_fn();
  if (!fn) return BNB_ECUDA;
  if ((ld * 2) % 16 != 0 || ((uintptr_t)ptr & 15) != 0) return BNB_EINVAL;
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides,
                  box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : BNB_ECUDA;
}

// hi = bf16(x), lo = bf16(x - hi), written with leading dimension ld_out
__global__ void k_split_bf16_f64(const double* __restrict__ x, long long rows, long long cols,
                                 long long ld_in, long long ld_out, int transpose,
                                 __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const long long m = rows * cols;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < m;
       t += (long long)gridDim.x * blockDim.x) {
    const long long i = t % rows, j = t / rows;   // element (i, j) of a column-major rows x cols
    const double v = x[i + j * ld_in];
    const __nv_bfloat16 h = __double2bfloat16(v);
    const __nv_bfloat16 l = __double2bfloat16(v - (double)__bfloat162float(h));
    const long long o = transpose ? (j + i * ld_out) : (i + j * ld_out);
    hi[o] = h;
    if (lo) lo[o] = l;
  }
}

int split_bf16(cudaStream_t st, const double* x, long long rows, long long cols, long long ld_in,
               long long ld_out, bool transpose, __nv_bfloat16* hi, __nv_bfloat16* lo) {
  const long long m = rows * cols;
  long long g = (m + 255) / 256;
  if (g > 148 * 64) g = 148 * 64;
  k_split_bf16_f64<<<(int)g, 256, 0, st>>>(x, rows, cols, ld_in, ld_out, transpose ? 1 : 0, hi, lo);
  BNB_CUDA_OK(cudaGetLastError());
  return 0;
}

}  // namespace bnb
