/*
 * bnb_diag.h -- diagnostics library (libbnb_diag.so) of the B300 branch-and-bound
 * library: B300-specific kernels run on their own so that tests can check them in
 * isolation.  None of these calls is needed to solve a problem, and the paper has no
 * counterpart for any of them; they live in a library of their own so that the
 * product library (include/bnb.h, libbnb.so) exports only the solver.
 *
 * Conventions are those of bnb.h: int status (BNB_OK or a negative BNB_E* code),
 * never abort.  These calls allocate their own temporaries and synchronise the
 * current device.
 */
#ifndef BNB_DIAG_H
#define BNB_DIAG_H

#include "bnb.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Diagnostics: the tcgen05 tensor-core contraction on its own.  C = A B^T with
 * A (M x Kd) and B (N x Kd) given K-major in FP64 device memory (element (m, k)
 * at A[k + m*Kd]), split into BF16 operands (nsplit 1: hi; 2: A hi, B a hi/lo pair,
 * two products; 3: hi/lo pairs, three products), tile width bn (128 or 256), `splits`
 * split-K chunks summed
 * in order; C is M x N column-major FP32 (device).  *err_out (host) receives the
 * kernel's pipeline error word (0 when every bounded wait completed).
 */
int bnb_tc_gemm_check(const double* dA, const double* dB, int M, int N, int Kd, int nsplit, int bn,
                      int splits, float* dC, int* err_out);

/* Diagnostics: the same product through the cluster-reduced tcgen05 kernel that the
 * ADMM iteration uses for X W'^T and G^-1 T (128 x 256 tiles; the K range split over
 * `cluster` CTAs of one thread-block cluster, 1 <= cluster <= 8, whose partial tiles
 * are summed in rank order through distributed shared memory).  Arguments as for
 * bnb_tc_gemm_check; C (device, M x N column-major FP32) is written directly.
 * Returns BNB_EINVAL for bad sizes or a cluster size the device cannot co-schedule.
 * The paper has no counterpart: this checks a B300-specific kernel in isolation. */
int bnb_tc_gemm_check_cluster(const double* dA, const double* dB, int M, int N, int Kd,
                              int nsplit, int cluster, float* dC, int* err_out);

/* Diagnostics: the same product through the CTA-pair tcgen05 kernel (cta_group::2) that
 * the ADMM iteration can use for X^T U' with the roles exchanged: 256 x bn tiles
 * (bn = 128, 144 or 256), each computed by two CTAs on two SMs, the first holding rows
 * [0, 128) of the tile and B rows [0, bn/2), the second the rest.  nsplit: 1 (BF16),
 * 2 (A as a hi/lo pair, B one BF16 term: the iterate is A in that use) or 3 (both
 * pairs).  Arguments otherwise as for bnb_tc_gemm_check; C (device, M x N column-major
 * FP32) is written directly; M <= 16384.  Returns BNB_EINVAL for bad sizes or when the
 * device cannot co-schedule a pair; err_out receives the kernel's error word (0 when
 * every bounded wait completed and both CTAs of each pair held the same tensor-memory
 * columns).  The paper has no counterpart: this checks a B300-specific kernel alone. */
int bnb_tc_gemm_check_pair(const double* dA, const double* dB, int M, int N, int Kd, int nsplit,
                           int bn, float* dC, int* err_out);

/*
 * Diagnostics: the bounded mbarrier wait that every tensor-core kernel of the library
 * uses, on its own.  One thread block waits on an mbarrier that nothing arrives on,
 * with no TMA copy and no MMA in flight, using the kernels' wait loop with the limits
 * given here (max_polls in [1, 2^30] polls, max_seconds in (0, 1] of %globaltimer)
 * instead of the kernels' own (2^24 polls, 2 s).  The kernel returns once the wait
 * gives up.  *err_out receives the error word: bit 1 set by each wait that expired,
 * bit 2 if any wait wrongly reported success (so 1 is the expected value);
 * *seconds_out the time one thread spent waiting.  Returns BNB_EINVAL for out-of-range limits.
 */
int bnb_diag_wait_expiry(long long max_polls, double max_seconds, int* err_out,
                         double* seconds_out);

/*
 * Diagnostics: the TMA operand ring of the tensor-core kernels on its own, to measure
 * how fast operand tiles reach the SMs.  `ctas` CTAs (1 <= ctas <= the SM count; one per
 * SM) each stream `reps` passes (1..64) of 16 K steps; a K step is one ring stage holding
 * the four tiles one CTA of the fused product's CTA pair loads: A hi and lo (128 rows) and
 * B hi and lo (b_rows rows, a multiple of 8 up to 256), each 64 BF16 = 128 bytes wide with
 * the 128-byte swizzle, through a ring of `stages` stages (2..8, within 227 KB of shared
 * memory).  There is no MMA: a consumer thread frees each stage as soon as it has landed.
 * The four source tensors (1024 BF16 wide, zeroed, together 21 MB at b_rows = 88) are
 * allocated here and stay L2-resident.  *us_out: the shortest of `launches` (1..50)
 * launches after two warm-ups, in microseconds (CUDA events); *bytes_out: the bytes one
 * launch delivers (ctas x reps x 16 x stage bytes); *err_out: the kernel's error word (0
 * when every bounded wait completed).  Returns BNB_EINVAL for out-of-range arguments.
 * The paper has no counterpart: this measures the ceiling the operand-streaming main
 * loops of the two ADMM products run against.
 */
int bnb_diag_tma_stream(int ctas, int stages, int b_rows, int reps, int launches, double* us_out,
                        double* bytes_out, int* err_out);

#ifdef __cplusplus
}
#endif
#endif /* BNB_DIAG_H */
