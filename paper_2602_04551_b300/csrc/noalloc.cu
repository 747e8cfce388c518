// noalloc.cu -- allocation-free variant of the FP64 dual-bound certificate.
//
// bnb_dual_bound_static computes the same Proposition 1 bound as bnb_dual_bound
// for caller-supplied residuals, but it needs no handle and allocates nothing:
// its per-(node, column block) partial sums live in a fixed, file-scope device
// array.  It is meant for callers that must not allocate device memory: for
// example code running under another framework that already owns the GPU's
// memory budget through its own allocator, or a latency-critical loop that
// cannot afford cudaMalloc's implicit synchronisation or the risk of an
// allocation failure mid-run.
//
// When the array comes into being: the CUDA runtime loads this file's module
// lazily (the default since CUDA 12.2), so the array is reserved on a device the
// first time this entry point runs there -- the address lookup below triggers
// the load.  That first call can therefore synchronise the device and can fail
// (BNB_ECUDA) when the device has no 8 MiB left; later calls only launch.  Once
// reserved, the array stays until the process exits.
//
// Limits and sharing: the array holds SCRATCH_DOUBLES doubles (8 MiB); a call
// needs K * (ceil(p / 256) + 2) of them and is rejected with BNB_EINVAL beyond
// that.  All calls on a device share the array and it keeps the last call's
// contents; every entry a call reads is written earlier in the same call, so no
// clearing is needed, but calls whose kernels overlap on the GPU (different
// streams, no ordering between them) race on the array.
#include <mutex>
#include "bnb.h"
#include "common.cuh"

namespace bnb {

constexpr long long SCRATCH_DOUBLES = 1ll << 20;   // 8 MiB
constexpr int COLS_PER_BLOCK = 256;                 // columns of X per block (8 warps x 32)
constexpr int MAX_CONTEXTS = 64;       // cached (device, context) lookups

static __device__ __align__(256) double g_cert_scratch[SCRATCH_DOUBLES];

// Partial sums: for node k and column block b, sum of nu_i(|X_i^T r_k|) over the
// block's columns; block b == 0 also writes ||r_k||^2 and y^T r_k.
__global__ void k_cert_static_partial(const double* __restrict__ X, const double* __restrict__ y,
                                      int n, int p, Prob P, const int8_t* __restrict__ fix,
                                      const double* __restrict__ r, int nb,
                                      double* __restrict__ scratch) {
  __shared__ double wsum[8];
  __shared__ double sh[32];
  const int b = blockIdx.x, k = blockIdx.y;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const double* rk = r + (long long)k * n;
  double acc = 0.0;  // this warp's columns, in increasing order
  for (int c = b * COLS_PER_BLOCK + w; c < min(p, (b + 1) * COLS_PER_BLOCK); c += 8) {
    const double* x = X + (long long)c * n;
    double d = 0.0;
    for (int i = lane; i < n; i += 32) d = fma(x[i], rk[i], d);
    d = warp_sum(d);
    acc += nu_coord<double>(fabs(d), fix[(long long)k * p + c], P);
  }
  if (lane == 0) wsum[w] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int t = 0; t < 8; ++t) s += wsum[t];
    scratch[(long long)k * (nb + 2) + 2 + b] = s;
  }
  if (b == 0) {
    double rr = 0.0, yr = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      rr = fma(rk[i], rk[i], rr);
      yr = fma(y[i], rk[i], yr);
    }
    rr = block_sum(rr, sh);
    yr = block_sum(yr, sh);
    if (threadIdx.x == 0) {
      scratch[(long long)k * (nb + 2)] = rr;
      scratch[(long long)k * (nb + 2) + 1] = yr;
    }
  }
}

__global__ void k_cert_static_final(int K, int nb, const double* __restrict__ scratch,
                                    double* __restrict__ lb) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const double* s = scratch + (long long)k * (nb + 2);
  double nu = 0.0;
  for (int b = 0; b < nb; ++b) nu += s[2 + b];
  lb[k] = -0.5 * s[0] + s[1] - nu;
}

// Device address of g_cert_scratch, looked up once per (device, context) with that
// device current: a device address is valid only in the context it came from, so a
// caller that makes its own (non-primary) context current gets its own lookup.  The
// driver's cuCtxGetCurrent is reached through the runtime's entry-point query, so the
// library still links only the CUDA runtime.
struct ScratchEntry {
  int dev;
  void* ctx;
  double* ptr;
};
static ScratchEntry scratch_tab[MAX_CONTEXTS];
static int scratch_used = 0;
static std::mutex scratch_mu;

typedef int (*CtxGetCurrentFn)(void** ctx);

static int current_context(void** ctx) {
  static CtxGetCurrentFn fn = nullptr;
  static bool tried = false;
  if (!tried) {   // called under scratch_mu
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      fn = (CtxGetCurrentFn)f;
    else
      cudaGetLastError();
  }
  *ctx = nullptr;
  if (!fn || fn(ctx) != 0) return BNB_ECUDA;
  return 0;
}

static int scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
    cudaGetLastError();
    return BNB_ENODEV;
  }
  // with no context current yet (a thread's first CUDA call), the symbol lookup below
  // makes the device's primary context current; the context is read again after it
  std::lock_guard<std::mutex> lock(scratch_mu);
  void* ctx = nullptr;
  if (current_context(&ctx)) return BNB_ECUDA;
  for (int i = 0; ctx && i < scratch_used; ++i)
    if (scratch_tab[i].dev == dev && scratch_tab[i].ctx == ctx) {
      *out = scratch_tab[i].ptr;
      return 0;
    }
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_cert_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return BNB_ECUDA;
  }
  if (!ctx && current_context(&ctx)) return BNB_ECUDA;
  if (ctx && scratch_used < MAX_CONTEXTS) scratch_tab[scratch_used++] = ScratchEntry{dev, ctx, (double*)p};
  *out = (double*)p;
  return 0;
}

}  // namespace bnb

extern "C" int bnb_dual_bound_static(const double* dX, const double* dy, int n, int p,
                                     double lambda0, double lambda2, double M, int K,
                                     const int8_t* dfix, const double* dr, double* dlb,
                                     void* stream) {
  using namespace bnb;
  if (!dX || !dy || !dfix || !dr || !dlb) return BNB_EINVAL;
  if (n <= 0 || p <= 0 || K <= 0 || !(lambda0 >= 0.0) || !(lambda2 > 0.0) || !(M > 0.0))
    return BNB_EINVAL;
  const int nb = (p + COLS_PER_BLOCK - 1) / COLS_PER_BLOCK;
  if ((long long)K * (nb + 2) > SCRATCH_DOUBLES) return BNB_EINVAL;  // beyond the fixed scratch
  if (K > 65535) return BNB_EINVAL;                                   // grid.y limit
  double* scratch = nullptr;
  if (int rc = scratch_for_current_device(&scratch)) return rc;
  Prob P{};
  P.n = n;
  P.p = p;
  P.lam0 = lambda0;
  P.lam2 = lambda2;
  P.M = M;
  P.s0 = sqrt(lambda0 / lambda2);
  P.linear = P.s0 > M ? 1 : 0;
  cudaStream_t st = (cudaStream_t)stream;
  k_cert_static_partial<<<dim3(nb, K), 256, 0, st>>>(dX, dy, n, p, P, dfix, dr, nb, scratch);
  k_cert_static_final<<<(K + 127) / 128, 128, 0, st>>>(K, nb, scratch, dlb);
  return cudaGetLastError() == cudaSuccess ? BNB_OK : BNB_ECUDA;
}
