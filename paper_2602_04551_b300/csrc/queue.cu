// queue.cu -- device-resident open-node pool with best-first selection.
//
// Section 2.2.1 / Algorithm 1: nodes are (F0, F1, LB of the parent); the batch
// is the min(K_free, |N|) open nodes of smallest LB; a node whose LB reaches
// UB (1 - gap) is pruned; a branched node adds (F0 + {j}, F1) and (F0, F1 + {j}),
// both carrying the parent's LB.  Warm start (Section 3.1.3): both children
// take the parent's final (beta, v); the F0 child sets beta_j = 0.
//
// Layout: struct-of-arrays records in a pool of fixed capacity; free entries
// on a stack (allocation only in k_push, release only in the selection
// kernels, so no kernel both pops and pushes).  Each record stores its fixings
// as a list of (index << 1 | value) of length depth.  Parent (beta, v) rows go
// to a reference-counted warm store; when it is full the children start cold
// (beta = v = 0), which changes iteration counts but never a bound.
//
// Selection keys are the node LB rounded down to FP32 and made order-preserving
// as unsigned integers; an exact 3-pass radix select (11 + 11 + 10 bits) finds
// the threshold key, ties at the threshold are taken in arbitrary order.
#include <cfloat>
#include "engine.cuh"

namespace bnb {

// sel_state slots
enum {
  SS_TAKE_ALL = 0, SS_F = 1, SS_PREFIX = 2, SS_NEED = 3, SS_LESS = 4, SS_TAU = 5, SS_EQ = 6,
  SS_OUT = 7, SS_POLISHED = 8, SS_PRUNED = 9, SS_COUNT = 10, SS_ERROR = 11, SS_MAXDEPTH = 12,
  SS_BARCNT = 13, SS_BARGEN = 14,   // grid barrier of the fused selection (arrivals, phase)
  SS_WORDS = 16
};

__device__ __forceinline__ void warm_release(int w, int* warm_ref, int* warm_stack, int* warm_top) {
  if (w >= 0 && atomicSub(&warm_ref[w], 1) == 1) warm_stack[atomicAdd(warm_top, 1)] = w;
}

__global__ void k_queue_init(long long qcap, long long wcap, int* free_stack, int* free_top,
                             int* pool_hw, int* warm_stack, int* warm_top, uint8_t* pool_valid,
                             double* pool_lb, unsigned* pool_key, int* pool_depth, int* pool_warm,
                             double* inc_ub, double ub0) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < qcap;
       t += (long long)gridDim.x * blockDim.x) {
    free_stack[t] = (int)(qcap - 1 - t);
    pool_valid[t] = 0;
  }
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < wcap;
       t += (long long)gridDim.x * blockDim.x)
    warm_stack[t] = (int)(wcap - 1 - t);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *free_top = (int)qcap - 1;  // entry 0 goes to the root
    *warm_top = (int)wcap;
    *pool_hw = 1;
    pool_valid[0] = 1;
    pool_lb[0] = -INFINITY;
    pool_key[0] = fkey(-INFINITY);
    pool_depth[0] = 0;
    pool_warm[0] = -1;
    inc_ub[0] = ub0;
  }
}

// Prune or branch each retired node (one block per retired node).
template <class R>
__global__ void k_push(int p, int dmax, const int* __restrict__ ret_slot, const int* __restrict__ ret_count,
                       const double* __restrict__ node_lb, const int* __restrict__ br_idx,
                       const double* __restrict__ inc_ub, const double* __restrict__ params,
                       const int* __restrict__ slot_depth, const int* __restrict__ slot_fixl,
                       const R* __restrict__ beta, const R* __restrict__ V, int* free_stack,
                       int* free_top, int* pool_hw, uint8_t* pool_valid, double* pool_lb,
                       unsigned* pool_key, int* pool_depth, int* pool_warm, int* pool_fix,
                       R* warm_beta, R* warm_V, int* warm_ref, int* warm_stack, int* warm_top,
                       int* sel_state, unsigned long long* poolmin, unsigned long long* lost_key,
                       const int* __restrict__ sup_cnt, int smax, int* hist_depth,
                       int* hist_sup, int* __restrict__ push_w) {
  __shared__ int c0, c1, wslot, decision;
  const int q = blockIdx.x;
  if (q >= *ret_count) return;
  const int slot = ret_slot[q];
  const int d = slot_depth[slot];
  const double lbu = node_lb[q];
  const int j = br_idx[q];
  if (threadIdx.x == 0) {
    // solved-node histograms: depth, and size of the rounded support (smax + 1: larger)
    atomicAdd(&hist_depth[d < dmax ? d : dmax], 1);
    const int sc = sup_cnt[q];
    atomicAdd(&hist_sup[(sc < 0 || sc > smax) ? smax + 1 : sc], 1);
    const double thr = inc_ub[0] * (1.0 - params[0]);
    decision = 0;
    if (lbu >= thr) {
      atomicAdd(&sel_state[SS_PRUNED], 1);
    } else if (j < 0) {
      // a leaf is closed by its support's upper bound (taken this round, or earlier when
      // sup_cnt is -2); a leaf support larger than smax had none taken: keep its bound as
      // a lost bound and stop the solve rather than drop its objective
      if (sup_cnt[q] == -1) {
        atomicOr(&sel_state[SS_ERROR], 4);
        atomicMin(lost_key, dkey(lbu));
      } else {
        atomicAdd(&sel_state[SS_PRUNED], 1);
      }
    } else if (d + 1 > dmax) {
      atomicOr(&sel_state[SS_ERROR], 1);
      atomicMin(lost_key, dkey(lbu));
    } else {
      const int t = atomicSub(free_top, 2);
      if (t < 2) {  // pool full: keep the node's bound as a lost bound, stop the solve
        atomicAdd(free_top, 2);
        atomicOr(&sel_state[SS_ERROR], 2);
        atomicMin(lost_key, dkey(lbu));
        goto decided;
      }
      decision = 1;
      c0 = free_stack[t - 1];
      c1 = free_stack[t - 2];
      atomicMax(pool_hw, (c0 > c1 ? c0 : c1) + 1);
      const int wt = atomicSub(warm_top, 1);
      if (wt > 0) {
        wslot = warm_stack[wt - 1];
        warm_ref[wslot] = 2;
      } else {
        atomicAdd(warm_top, 1);
        wslot = -1;
      }
      const unsigned key = fkey(__double2float_rd(lbu));
      pool_lb[c0] = lbu;
      pool_lb[c1] = lbu;
      pool_key[c0] = key;
      pool_key[c1] = key;
      pool_depth[c0] = d + 1;
      pool_depth[c1] = d + 1;
      pool_warm[c0] = wslot;
      pool_warm[c1] = wslot;
      atomicMax(&sel_state[SS_MAXDEPTH], d + 1);
      // the children are open nodes for this round's global lower bound
      atomicMin(poolmin, dkey(lbu));
      atomicAdd(&sel_state[SS_COUNT], 2);
    }
  decided:;
  }
  __syncthreads();
  if (threadIdx.x == 0) push_w[q] = decision ? wslot : -1;
  if (!decision) return;
  for (int t = threadIdx.x; t < d; t += blockDim.x) {
    const int e = slot_fixl[(long long)slot * dmax + t];
    pool_fix[(long long)c0 * dmax + t] = e;
    pool_fix[(long long)c1 * dmax + t] = e;
  }
  if (threadIdx.x == 0) {
    pool_fix[(long long)c0 * dmax + d] = (j << 1) | 0;
    pool_fix[(long long)c1 * dmax + d] = (j << 1) | 1;
  }
  if (threadIdx.x == 0) {
    pool_valid[c0] = 1;
    pool_valid[c1] = 1;
  }
}

// the parent's (beta, v) rows into the warm store slot k_push gave its children (grid
// K x PUSH_NB: block z copies the z-th slice of the p values).  The rows are read next by
// the refill of a later launch, so stream order is all the synchronisation needed.
template <class R>
__global__ void k_push_copy(int p, const int* __restrict__ ret_slot,
                            const int* __restrict__ ret_count, const int* __restrict__ push_w,
                            const R* __restrict__ beta, const R* __restrict__ V,
                            R* __restrict__ warm_beta, R* __restrict__ warm_V) {
  const int q = blockIdx.x;
  if (q >= *ret_count) return;
  const int w = push_w[q];
  if (w < 0) return;
  const int chunk = (p + gridDim.y - 1) / gridDim.y;
  const int i0 = blockIdx.y * chunk, i1 = min(p, i0 + chunk);
  const long long so = (long long)ret_slot[q] * p, wo = (long long)w * p;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    warm_beta[wo + i] = beta[so + i];
    warm_V[wo + i] = V[so + i];
  }
}

__device__ __forceinline__ void sel_reset_body(unsigned* hist, int* sel_state,
                                               unsigned long long* poolmin) {
  for (int t = threadIdx.x; t < 3 * SEL_BINS; t += blockDim.x) hist[t] = 0;
  if (threadIdx.x == 0) {
    sel_state[SS_TAKE_ALL] = 0;
    sel_state[SS_PREFIX] = 0;
    sel_state[SS_NEED] = 0;
    sel_state[SS_LESS] = 0;
    sel_state[SS_TAU] = 0;
    sel_state[SS_EQ] = 0;
    sel_state[SS_OUT] = 0;
    sel_state[SS_COUNT] = 0;
    *poolmin = ~0ull;
  }
}

__global__ void k_sel_reset(unsigned* hist, int* sel_state, unsigned long long* poolmin) {
  sel_reset_body(hist, sel_state, poolmin);
}

// One histogram increment per distinct bin among a warp's lanes (bin ~0u: none).  The
// keys of a deep tree's open nodes sit in a few bins of the upper levels (children carry
// their parent's bound), so per-lane shared atomics would serialise on those bins.
__device__ __forceinline__ void warp_hist_add(unsigned* sh, unsigned bin) {
  const unsigned peers = __match_any_sync(0xffffffffu, bin);
  if (bin != ~0u && (__ffs(peers) - 1) == (int)(threadIdx.x & 31)) atomicAdd(&sh[bin], __popc(peers));
}

// Slots in a shared array for the lanes whose flag is set: one atomicAdd per warp on the
// counter, each flagged lane gets base + its rank among the flagged lanes (-1 if unflagged).
__device__ __forceinline__ int warp_claim(int* counter, bool flag) {
  const unsigned m = __ballot_sync(0xffffffffu, flag);
  const int lane = threadIdx.x & 31;
  int base = 0;
  if (m && lane == __ffs(m) - 1) base = atomicAdd(counter, __popc(m));
  base = __shfl_sync(0xffffffffu, base, __ffs(m ? m : 1u) - 1);
  return flag ? base + __popc(m & ((1u << lane) - 1u)) : -1;
}

// pass 1: drop prunable entries, count, min LB, histogram of the top 11 key bits (block
// `blk` of `nblk` in a grid-stride loop over the pool).  The loop runs over whole warps
// (entries i0 + lane, i0 a multiple of 32) so that every lane takes part in the warp-wide
// aggregation of the histogram and of the free-stack pushes.
__device__ __forceinline__ void sel_pass1_body(int blk, int nblk, const int* __restrict__ pool_hw,
                                               uint8_t* pool_valid,
                                               const double* __restrict__ pool_lb,
                                               const unsigned* __restrict__ pool_key,
                                               const int* __restrict__ pool_warm, int* free_stack,
                                               int* free_top, int* warm_ref, int* warm_stack,
                                               int* warm_top, const double* __restrict__ inc_ub,
                                               const double* __restrict__ params, unsigned* hist,
                                               int* sel_state, unsigned long long* poolmin) {
  __shared__ unsigned sh[SEL_BINS];
  const int hw = *pool_hw;
  if (blk * (int)blockDim.x >= hw) return;   // no pool entry for this block (grid-stride)
  for (int t = threadIdx.x; t < SEL_BINS; t += blockDim.x) sh[t] = 0;
  __syncthreads();
  const double thr = inc_ub[0] * (1.0 - params[0]);
  const int lane = threadIdx.x & 31;
  int cnt = 0, npruned = 0;
  unsigned long long mn = ~0ull;
  for (int i0 = blk * blockDim.x + (threadIdx.x & ~31); i0 < hw; i0 += nblk * blockDim.x) {
    const int i = i0 + lane;
    const bool live = i < hw && pool_valid[i];
    const double lb = live ? pool_lb[i] : 0.0;
    const bool prune = live && lb >= thr;
    const int slot = warp_claim(free_top, prune);
    unsigned bin = ~0u;
    if (prune) {
      pool_valid[i] = 0;
      free_stack[slot] = i;
      warm_release(pool_warm[i], warm_ref, warm_stack, warm_top);
      ++npruned;
    } else if (live) {
      ++cnt;
      const unsigned long long k = dkey(lb);
      mn = k < mn ? k : mn;
      bin = pool_key[i] >> 21;
    }
    warp_hist_add(sh, bin);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < SEL_BINS; t += blockDim.x)
    if (sh[t]) atomicAdd(&hist[t], sh[t]);
  cnt = warp_sum(cnt);
  npruned = warp_sum(npruned);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, mn, o);
    mn = y < mn ? y : mn;
  }
  if (lane == 0) {
    if (cnt) atomicAdd(&sel_state[SS_COUNT], cnt);
    if (npruned) atomicAdd(&sel_state[SS_PRUNED], npruned);
    if (mn != ~0ull) atomicMin(poolmin, mn);
  }
}

__global__ void k_sel_pass1(const int* __restrict__ pool_hw, uint8_t* pool_valid,
                            const double* __restrict__ pool_lb, const unsigned* __restrict__ pool_key,
                            const int* __restrict__ pool_warm, int* free_stack, int* free_top,
                            int* warm_ref, int* warm_stack, int* warm_top,
                            const double* __restrict__ inc_ub, const double* __restrict__ params,
                            unsigned* hist, int* sel_state, unsigned long long* poolmin) {
  sel_pass1_body(blockIdx.x, gridDim.x, pool_hw, pool_valid, pool_lb, pool_key, pool_warm,
                 free_stack, free_top, warm_ref, warm_stack, warm_top, inc_ub, params, hist,
                 sel_state, poolmin);
}

// level-L scan (single block).  Level 1 also lists the free slots in order.
// With `lockstep` (Algorithm 1's batches) nothing is selected until every slot is free;
// SS_TAKE_ALL = 2 then means "take none" for the later levels and the collection.
__device__ __forceinline__ void sel_scan_body(int level, const unsigned* __restrict__ hist,
                                              int* sel_state, int K,
                                              const int* __restrict__ slot_active,
                                              int* free_slots, int lockstep) {
  __shared__ int wcnt[32];
  __shared__ int base;
  if (level == 1) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int s0 = 0; s0 < K; s0 += blockDim.x) {
      const int s = s0 + threadIdx.x;
      const int f = (s < K) ? !slot_active[s] : 0;
      const unsigned bal = __ballot_sync(0xffffffffu, f);
      if (lane == 0) wcnt[w] = __popc(bal);
      __syncthreads();
      int off = base;
      for (int t = 0; t < w; ++t) off += wcnt[t];
      if (f) free_slots[off + __popc(bal & ((1u << lane) - 1u))] = s;
      __syncthreads();
      if (threadIdx.x == 0) {
        int tot = 0;
        for (int t = 0; t < nw; ++t) tot += wcnt[t];
        base += tot;
      }
      __syncthreads();
    }
  }
  // level decisions (all threads take part in the bin scan below)
  __shared__ int need_s, done_s;
  if (threadIdx.x == 0) {
    done_s = 0;
    if (level == 1) {
      const int F = base;
      sel_state[SS_F] = F;
      const int count = sel_state[SS_COUNT];
      if (lockstep && F < K) {
        sel_state[SS_TAKE_ALL] = 2;
        sel_state[SS_F] = 0;
        done_s = 1;
      } else if (count <= F) {
        sel_state[SS_TAKE_ALL] = 1;
        done_s = 1;
      } else {
        sel_state[SS_NEED] = F;
        sel_state[SS_LESS] = 0;
      }
    } else if (sel_state[SS_TAKE_ALL]) {
      done_s = 1;
    }
    need_s = sel_state[SS_NEED];
  }
  __syncthreads();
  if (done_s) return;
  // block-wide inclusive scan of the histogram (bins split evenly over the threads),
  // then the first bin whose cumulative count reaches `need`
  const int nbins = level == 3 ? 1024 : SEL_BINS;
  const unsigned* h = hist + (level - 1) * SEL_BINS;
  const int per = (nbins + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per;
  int local = 0;
  for (int b = b0; b < b0 + per && b < nbins; ++b) local += (int)h[b];
  // exclusive prefix of `local` over the block
  int x = local;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) >= o) x += y;
  }
  if ((threadIdx.x & 31) == 31) wcnt[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int nw = blockDim.x >> 5;
    int v = threadIdx.x < nw ? wcnt[threadIdx.x] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, v, o);
      if (threadIdx.x >= o) v += y;
    }
    if (threadIdx.x < nw) wcnt[threadIdx.x] = v;   // inclusive warp totals
  }
  __syncthreads();
  const int excl = x - local + ((threadIdx.x >> 5) > 0 ? wcnt[(threadIdx.x >> 5) - 1] : 0);
  const int need = need_s;
  if (excl < need && excl + local >= need) {
    int cum = excl, b = b0;
    for (; b < b0 + per && b < nbins; ++b) {
      if (cum + (int)h[b] >= need) break;
      cum += (int)h[b];
    }
    sel_state[SS_NEED] = need - cum;
    sel_state[SS_LESS] += cum;
    if (level == 1) sel_state[SS_PREFIX] = b;
    else if (level == 2) sel_state[SS_PREFIX] = (sel_state[SS_PREFIX] << 11) | b;
    else sel_state[SS_TAU] = (int)(((unsigned)sel_state[SS_PREFIX] << 10) | (unsigned)b);
  }
}

__global__ void k_sel_scan(int level, const unsigned* __restrict__ hist, int* sel_state, int K,
                           const int* __restrict__ slot_active, int* free_slots, int lockstep) {
  sel_scan_body(level, hist, sel_state, K, slot_active, free_slots, lockstep);
}

// levels 2 and 3: histogram of the next key bits among entries matching the prefix
// (whole-warp loop and warp-aggregated increments, as in pass 1)
__device__ __forceinline__ void sel_pass_body(int blk, int nblk, int level,
                                              const int* __restrict__ pool_hw,
                                              const uint8_t* __restrict__ pool_valid,
                                              const unsigned* __restrict__ pool_key,
                                              unsigned* hist, const int* __restrict__ sel_state) {
  if (sel_state[SS_TAKE_ALL]) return;
  __shared__ unsigned sh[SEL_BINS];
  const int hw = *pool_hw;
  if (blk * (int)blockDim.x >= hw) return;   // no pool entry for this block (grid-stride)
  for (int t = threadIdx.x; t < SEL_BINS; t += blockDim.x) sh[t] = 0;
  __syncthreads();
  const unsigned pre = (unsigned)sel_state[SS_PREFIX];
  const int lane = threadIdx.x & 31;
  for (int i0 = blk * blockDim.x + (threadIdx.x & ~31); i0 < hw; i0 += nblk * blockDim.x) {
    const int i = i0 + lane;
    unsigned bin = ~0u;
    if (i < hw && pool_valid[i]) {
      const unsigned k = pool_key[i];
      if (level == 2) {
        if ((k >> 21) == pre) bin = (k >> 10) & 2047u;
      } else {
        if ((k >> 10) == pre) bin = k & 1023u;
      }
    }
    warp_hist_add(sh, bin);
  }
  __syncthreads();
  unsigned* h = hist + (level - 1) * SEL_BINS;
  for (int t = threadIdx.x; t < SEL_BINS; t += blockDim.x)
    if (sh[t]) atomicAdd(&h[t], sh[t]);
}

__global__ void k_sel_pass(int level, const int* __restrict__ pool_hw,
                           const uint8_t* __restrict__ pool_valid,
                           const unsigned* __restrict__ pool_key, unsigned* hist,
                           const int* __restrict__ sel_state) {
  sel_pass_body(blockIdx.x, gridDim.x, level, pool_hw, pool_valid, pool_key, hist, sel_state);
}

__device__ __forceinline__ void sel_collect_body(int blk, int nblk, const int* __restrict__ pool_hw,
                                                 uint8_t* pool_valid,
                                                 const unsigned* __restrict__ pool_key,
                                                 int* free_stack, int* free_top, int* sel_state,
                                                 int* popped) {
  const int hw = *pool_hw;
  const int all = sel_state[SS_TAKE_ALL];
  if (all == 2) return;                     // lockstep: slots still busy
  const unsigned tau = (unsigned)sel_state[SS_TAU];
  const int need_eq = sel_state[SS_NEED];
  const int lane = threadIdx.x & 31;
  for (int i0 = blk * blockDim.x + (threadIdx.x & ~31); i0 < hw; i0 += nblk * blockDim.x) {
    const int i = i0 + lane;
    const bool live = i < hw && pool_valid[i];
    const unsigned k = live ? pool_key[i] : 0u;
    bool take = live && (all == 1 || k < tau);
    // entries at the threshold key: the first need_eq claims (in any order) are taken
    const int eq = warp_claim(&sel_state[SS_EQ], live && !take && k == tau);
    if (eq >= 0 && eq < need_eq) take = true;
    const int out = warp_claim(&sel_state[SS_OUT], take);
    const int fs = warp_claim(free_top, take);
    if (take) {
      popped[out] = i;
      pool_valid[i] = 0;
      free_stack[fs] = i;
    }
  }
}

__global__ void k_sel_collect(const int* __restrict__ pool_hw, uint8_t* pool_valid,
                              const unsigned* __restrict__ pool_key, int* free_stack, int* free_top,
                              int* sel_state, int* popped) {
  sel_collect_body(blockIdx.x, gridDim.x, pool_hw, pool_valid, pool_key, free_stack, free_top,
                   sel_state, popped);
}

// load popped node t into its free slot: grid K x REFILL_NB, block z writing the z-th
// slice of the slot's p values (cleared fixings, warm or zero beta and v, then the node's
// fixings that fall in the slice); block 0 also copies the fixing list and the slot's
// bookkeeping and releases the warm row (whose slot only a later k_push can reuse, so the
// other blocks of this launch still read it safely)
template <class R>
__global__ void k_refill(int p, int dmax, const int* __restrict__ sel_state, const int* __restrict__ popped,
                         const int* __restrict__ free_slots, const double* __restrict__ pool_lb,
                         const int* __restrict__ pool_depth, const int* __restrict__ pool_warm,
                         const int* __restrict__ pool_fix, const R* __restrict__ warm_beta,
                         const R* __restrict__ warm_V, int* warm_ref, int* warm_stack,
                         int* warm_top, int8_t* fix, R* beta, R* V, int* slot_active,
                         int* slot_iters, double* slot_lbp, int* slot_depth, int* slot_nfix,
                         int* slot_fixl) {
  const int t = blockIdx.x, z = blockIdx.y;
  if (t >= sel_state[SS_OUT]) return;
  const int slot = free_slots[t];
  const int idx = popped[t];
  const int d = pool_depth[idx];
  const int w = pool_warm[idx];
  const int chunk = (p + gridDim.y - 1) / gridDim.y;
  const int i0 = z * chunk, i1 = min(p, i0 + chunk);
  const long long so = (long long)slot * p;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    fix[so + i] = -1;
    beta[so + i] = w >= 0 ? warm_beta[(long long)w * p + i] : R(0);
    V[so + i] = w >= 0 ? warm_V[(long long)w * p + i] : R(0);
  }
  __syncthreads();
  for (int u = threadIdx.x; u < d; u += blockDim.x) {
    const int e = pool_fix[(long long)idx * dmax + u];
    if (z == 0) slot_fixl[(long long)slot * dmax + u] = e;
    const int i = e >> 1;
    if (i < i0 || i >= i1) continue;
    fix[so + i] = (int8_t)(e & 1);
    if ((e & 1) == 0) beta[so + i] = R(0);  // the new F0 coordinate starts at zero
  }
  if (z == 0 && threadIdx.x == 0) {
    slot_active[slot] = 1;
    slot_iters[slot] = 0;
    slot_lbp[slot] = pool_lb[idx];
    slot_depth[slot] = d;
    slot_nfix[slot] = d;
    warm_release(w, warm_ref, warm_stack, warm_top);
  }
}

// ---- the selection of a round in one cooperative launch ----
// The steps above (reset, pass 1, three scans, two passes, collection) are dependent, and
// as separate launches much of their time is launch and ramp latency; here the blocks of
// one cooperative launch (all co-resident) meet at grid barriers between the steps.  The
// refill (one block per popped node, copying its warm start) stays a launch of its own:
// with wide batches it moves K rows of p values and wants the whole GPU.  Every barrier wait is bounded (2^24 polls and 1 s): a block that gives up
// sets bit 8 of the error word and leaves, and the solve then ends with an error.

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* a) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// arrival count and phase generation live in sel_state; the last block to arrive resets
// the count and advances the generation, the others wait for the generation to change
__device__ bool coop_grid_sync(int* sel_state) {
  __shared__ int ok_s;
  unsigned* cnt = reinterpret_cast<unsigned*>(&sel_state[SS_BARCNT]);
  unsigned* gen = reinterpret_cast<unsigned*>(&sel_state[SS_BARGEN]);
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned g0 = ld_acquire_gpu(gen);
    __threadfence();                             // this block's writes before its arrival
    if (atomicAdd(cnt, 1u) + 1u == gridDim.x) {
      atomicExch(cnt, 0u);
      __threadfence();
      atomicAdd(gen, 1u);                        // release the next phase
    } else {
      const unsigned long long t0 = global_timer_ns();
      for (long long i = 0;; ++i) {
        if (ld_acquire_gpu(gen) != g0) break;
        if (i >= (1ll << 24) || ((i & 255) == 255 && global_timer_ns() - t0 > 1000000000ull)) {
          atomicOr(&sel_state[SS_ERROR], 8);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

constexpr int SELC_THREADS = 1024;   // the scans' block width
constexpr int SELC_BLOCKS = 64;      // co-resident blocks of the fused selection

__global__ void __launch_bounds__(SELC_THREADS) k_select_coop(
    int K, int lockstep, const int* __restrict__ pool_hw, uint8_t* pool_valid,
    const double* __restrict__ pool_lb, const unsigned* __restrict__ pool_key,
    const int* __restrict__ pool_warm, int* free_stack, int* free_top, int* warm_ref,
    int* warm_stack, int* warm_top, const double* __restrict__ inc_ub,
    const double* __restrict__ params, unsigned* hist, int* sel_state,
    unsigned long long* poolmin, int* free_slots, int* popped, const int* __restrict__ slot_active) {
  const int blk = blockIdx.x, nblk = gridDim.x;
  if (blk == 0) sel_reset_body(hist, sel_state, poolmin);
  if (!coop_grid_sync(sel_state)) return;
  sel_pass1_body(blk, nblk, pool_hw, pool_valid, pool_lb, pool_key, pool_warm, free_stack,
                 free_top, warm_ref, warm_stack, warm_top, inc_ub, params, hist, sel_state,
                 poolmin);
  if (!coop_grid_sync(sel_state)) return;
  for (int level = 1; level <= 3; ++level) {
    if (level > 1) {
      sel_pass_body(blk, nblk, level, pool_hw, pool_valid, pool_key, hist, sel_state);
      if (!coop_grid_sync(sel_state)) return;
    }
    if (blk == 0) sel_scan_body(level, hist, sel_state, K, slot_active, free_slots, lockstep);
    if (!coop_grid_sync(sel_state)) return;
  }
  sel_collect_body(blk, nblk, pool_hw, pool_valid, pool_key, free_stack, free_top, sel_state,
                   popped);
}

__global__ void k_status(int K, const int* __restrict__ slot_active,
                         const double* __restrict__ slot_lbp, const int* __restrict__ sel_state,
                         const unsigned long long* __restrict__ poolmin,
                         const unsigned long long* __restrict__ lost_key,
                         const double* __restrict__ inc_ub, const int* __restrict__ free_top,
                         const int* __restrict__ warm_top, const int* __restrict__ ret_count,
                         Status* st) {
  __shared__ int act_s[32];
  __shared__ unsigned long long mn_s[32];
  int act = 0;
  unsigned long long mn = ~0ull;
  for (int s = threadIdx.x; s < K; s += blockDim.x)
    if (slot_active[s]) {
      ++act;
      const unsigned long long k = dkey(slot_lbp[s]);
      mn = k < mn ? k : mn;
    }
  for (int o = 16; o > 0; o >>= 1) {
    act += __shfl_xor_sync(0xffffffffu, act, o);
    const unsigned long long m2 = __shfl_xor_sync(0xffffffffu, mn, o);
    mn = m2 < mn ? m2 : mn;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    act_s[w] = act;
    mn_s[w] = mn;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  act = 0;
  mn = ~0ull;
  for (int t = 0; t < nw; ++t) {
    act += act_s[t];
    mn = mn_s[t] < mn ? mn_s[t] : mn;
  }
  const long long pool_after = (long long)sel_state[SS_COUNT] - sel_state[SS_OUT];
  if (pool_after > 0 && *poolmin < mn) mn = *poolmin;
  if (*lost_key < mn) mn = *lost_key;
  const double ub = inc_ub[0];
  st->ub = ub;
  st->lb = (mn == ~0ull) ? ub : dkey_inv(mn);
  if (st->lb > ub) st->lb = ub;
  st->pool_count = pool_after;
  st->active_slots = act;
  st->retired = *ret_count;
  st->pruned = sel_state[SS_PRUNED];
  st->polished = sel_state[SS_POLISHED];
  st->free_top = *free_top;
  st->warm_free = *warm_top;
  st->error = sel_state[SS_ERROR];
  st->max_depth = sel_state[SS_MAXDEPTH];
  st->lost_lb = (*lost_key == ~0ull) ? INFINITY : dkey_inv(*lost_key);
  st->nodes_total += *ret_count;
  st->rounds_total += 1;
}

static inline int pool_grid(long long qcap) {
  long long g = (qcap + 255) / 256;
  return (int)(g > 148 * 8 ? 148 * 8 : (g < 1 ? 1 : g));
}

template <class R>
int queue_init(Engine<R>& e) {
  BNB_CUDA_OK(cudaMemsetAsync(e.sel_state, 0, sizeof(int) * SS_WORDS, e.st));
  BNB_CUDA_OK(cudaMemsetAsync(e.slot_active, 0, sizeof(int) * e.K, e.st));
  BNB_CUDA_OK(cudaMemsetAsync(e.poolmin + 1, 0xff, sizeof(unsigned long long), e.st));  // lost key
  BNB_CUDA_OK(cudaMemsetAsync(e.status_d, 0, sizeof(Status), e.st));
  BNB_CUDA_OK(cudaMemsetAsync(e.hist_depth, 0, sizeof(int) * (e.dmax + 1), e.st));
  BNB_CUDA_OK(cudaMemsetAsync(e.ub_seen, 0, sizeof(unsigned long long) * UB_SEEN, e.st));
  BNB_CUDA_OK(cudaMemsetAsync(e.hist_sup, 0, sizeof(int) * (e.smax + 2), e.st));
  k_queue_init<<<pool_grid(e.qcap), 256, 0, e.st>>>(e.qcap, e.wcap, e.free_stack, e.free_top,
                                                    e.pool_hw, e.warm_stack, e.warm_top,
                                                    e.pool_valid, e.pool_lb, e.pool_key,
                                                    e.pool_depth, e.pool_warm, e.inc_ub, INFINITY);
  BNB_CUDA_OK(cudaGetLastError());
  return 0;
}

template <class R>
int queue_push(Engine<R>& e) {
  k_push<R><<<e.K, 256, 0, e.st>>>(e.p, e.dmax, e.ret_slot, e.ret_count, e.node_lb, e.br_idx, e.inc_ub,
                                   e.params_d, e.slot_depth, e.slot_fixl, e.beta, e.V,
                                   e.free_stack, e.free_top, e.pool_hw, e.pool_valid, e.pool_lb,
                                   e.pool_key, e.pool_depth, e.pool_warm, e.pool_fix, e.warm_beta,
                                   e.warm_V, e.warm_ref, e.warm_stack, e.warm_top, e.sel_state,
                                   e.poolmin, e.poolmin + 1, e.sup_size, e.smax, e.hist_depth,
                                   e.hist_sup, e.push_w);
  k_push_copy<R><<<dim3(e.K, PUSH_NB), 256, 0, e.st>>>(e.p, e.ret_slot, e.ret_count, e.push_w,
                                                       e.beta, e.V, e.warm_beta, e.warm_V);
  BNB_CUDA_OK(cudaGetLastError());
  return 0;
}

// blocks of the fused selection this engine launches (0: the separate launches), from the
// device's cooperative-launch support and the kernel's occupancy
template <class R>
int queue_fused_select_blocks() {
  int dev = 0, coop = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_select_coop, SELC_THREADS,
                                                    0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (coop && per * sms >= SELC_BLOCKS) ? SELC_BLOCKS : 0;
}

template <class R>
int queue_select_refill(Engine<R>& e) {
  cudaStream_t st = e.st;
  if (e.sel_blocks > 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(e.sel_blocks);
    cfg.blockDim = dim3(SELC_THREADS);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    BNB_CUDA_OK(cudaLaunchKernelEx(
        &cfg, k_select_coop, e.K, e.lockstep, (const int*)e.pool_hw, e.pool_valid,
        (const double*)e.pool_lb, (const unsigned*)e.pool_key, (const int*)e.pool_warm,
        e.free_stack, e.free_top, e.warm_ref, e.warm_stack, e.warm_top, (const double*)e.inc_ub,
        (const double*)e.params_d, e.sel, e.sel_state, e.poolmin, e.free_slots, e.popped,
        (const int*)e.slot_active));
    k_refill<R><<<dim3(e.K, REFILL_NB), 256, 0, st>>>(
        e.p, e.dmax, e.sel_state, e.popped, e.free_slots, e.pool_lb, e.pool_depth, e.pool_warm,
        e.pool_fix, e.warm_beta, e.warm_V, e.warm_ref, e.warm_stack, e.warm_top, e.fix, e.beta,
        e.V, e.slot_active, e.slot_iters, e.slot_lbp, e.slot_depth, e.slot_nfix, e.slot_fixl);
    BNB_CUDA_OK(cudaGetLastError());
    return 0;
  }
  const int g = pool_grid(e.qcap);
  k_sel_reset<<<1, 256, 0, st>>>(e.sel, e.sel_state, e.poolmin);
  k_sel_pass1<<<g, 256, 0, st>>>(e.pool_hw, e.pool_valid, e.pool_lb, e.pool_key, e.pool_warm,
                                 e.free_stack, e.free_top, e.warm_ref, e.warm_stack, e.warm_top,
                                 e.inc_ub, e.params_d, e.sel, e.sel_state, e.poolmin);
  k_sel_scan<<<1, 1024, 0, st>>>(1, e.sel, e.sel_state, e.K, e.slot_active, e.free_slots,
                                 e.lockstep);
  k_sel_pass<<<g, 256, 0, st>>>(2, e.pool_hw, e.pool_valid, e.pool_key, e.sel, e.sel_state);
  k_sel_scan<<<1, 1024, 0, st>>>(2, e.sel, e.sel_state, e.K, e.slot_active, e.free_slots,
                                 e.lockstep);
  k_sel_pass<<<g, 256, 0, st>>>(3, e.pool_hw, e.pool_valid, e.pool_key, e.sel, e.sel_state);
  k_sel_scan<<<1, 1024, 0, st>>>(3, e.sel, e.sel_state, e.K, e.slot_active, e.free_slots,
                                 e.lockstep);
  k_sel_collect<<<g, 256, 0, st>>>(e.pool_hw, e.pool_valid, e.pool_key, e.free_stack, e.free_top,
                                   e.sel_state, e.popped);
  k_refill<R><<<dim3(e.K, REFILL_NB), 256, 0, st>>>(
      e.p, e.dmax, e.sel_state, e.popped, e.free_slots, e.pool_lb, e.pool_depth, e.pool_warm,
      e.pool_fix, e.warm_beta, e.warm_V, e.warm_ref, e.warm_stack, e.warm_top, e.fix, e.beta,
      e.V, e.slot_active, e.slot_iters, e.slot_lbp, e.slot_depth, e.slot_nfix, e.slot_fixl);
  BNB_CUDA_OK(cudaGetLastError());
  return 0;
}

template <class R>
int queue_status(Engine<R>& e) {
  k_status<<<1, 256, 0, e.st>>>(e.K, e.slot_active, e.slot_lbp, e.sel_state, e.poolmin,
                                e.poolmin + 1, e.inc_ub, e.free_top, e.warm_top, e.ret_count,
                                e.status_d);
  BNB_CUDA_OK(cudaGetLastError());
  BNB_CUDA_OK(cudaMemcpyAsync(e.status_h, e.status_d, sizeof(Status), cudaMemcpyDeviceToHost, e.st));
  return 0;
}

#define INST(R)                                      \
  template int queue_fused_select_blocks<R>();       \
  template int queue_init<R>(Engine<R>&);            \
  template int queue_push<R>(Engine<R>&);            \
  template int queue_select_refill<R>(Engine<R>&);   \
  template int queue_status<R>(Engine<R>&);
INST(float)
INST(double)
#undef INST

}  // namespace bnb
