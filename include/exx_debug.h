/*
 * exx_debug.h -- host-only inspection hooks of libexx_gb300, for tests.
 *
 * These run entirely on the CPU (no CUDA call), so the plan-setup mathematics and the
 * pair scheduler can be checked on a machine without a GPU.  They have no counterpart
 * in the paper beyond the steps they expose (Eqs. 6-7 for the eigen-decomposition,
 * Sec. II.B's batches of right-hand sides for the schedule).
 */
#ifndef EXX_GB300_DEBUG_H
#define EXX_GB300_DEBUG_H
#ifdef __cplusplus
extern "C" {
#endif

/* FD weights w[0..p] of the order-2p central second difference (host copy of what a plan uses). */
int exx_debug_fd_weights(int p, double *w);

/* 1D second-derivative operator (n x n column-major) as a plan assembles it. */
int exx_debug_second_derivative(int n, double h, int bc, int p, double *D);

/* The plan's symmetric eigensolver: A (n x n column-major) = V diag(lam) V^T, lam ascending. */
int exx_debug_sym_eig(int n, const double *A, double *V, double *lam);

/* Pair schedule of exx_apply.  First call with NULL arrays to get the sizes; then with
 * pairs (2 ints per pair: m, n), batches (3 ints: nfields, first block, nblocks) and
 * blocks (6 ints: I0, nI, J0, nJ, kind, field0) of at least those sizes. */
int exx_debug_schedule(int n_occ, int n_in, int aliased, int block, int max_pairs, long *npairs,
                       long *nbatches, long *nblocks, int *pairs, int *batches, int *blocks);

/* One 128 x n x k tensor-core tile (tcgen05.mma, one bf16 or tf32 piece per operand,
 * FP32 accumulation): D (128 x n, row-major) = A (128 x k, row-major) B (n x k,
 * row-major)^T.  DEVICE pointers; n, k multiples of 16 in [16, 256].  Synchronizes the
 * device.  Checks the operand layout and descriptors of the split-precision path. */
int exx_debug_tc_gemm(int tf32, int n, int k, const float *A, const float *B, float *D, int *err);

/* Quotients n[i] / d by the multiply-shift division the pass kernels use for row ->
 * (field, row in field) (Granlund & Montgomery 1994, Fig. 4.1), host-side.  d >= 1. */
int exx_debug_fastdiv(unsigned d, int count, const unsigned *n, unsigned *q);

/* The automatic BF16X7 (three-pass) layouts of an n1 x n2 x n3 grid, host-side (no device):
 * out (HOST int[16]) = supported; shared memory of pass A and pass C; pass A streams its x/y
 * matrices and their chunk width; the same for pass C; pass A pipelined; pass A staged; pass B
 * shared memory (0 = none fits); pass B K-chunks; its chunk or block width; its buffers; its
 * matrices resident; units per thread; the shared-memory limit.  share01 = 1 when x and y have
 * the same length and boundary condition (one image serves both).  Sizes in [2, 256]. */
int exx_debug_tc3_layout(int n1, int n2, int n3, int share01, int *out);

/* The base-512 digit image of the 1D matrices, host-side: C (HOST, row-major nout x nk, row n =
 * output n, column k = contraction index k) cut for a WN x Kp block of rows n0.. and indices
 * k0.. (a K-chunk when k0 > 0 or Kp < nk), decoded from the tensor-core layout back to values:
 * digits (HOST float[4][WN][Kp]) holds the four weighted digits of every entry (their sum times
 * the row's scale is the entry), scales (HOST float[WN]) the column scales.  Every row is
 * scaled by the largest entry of the whole row, so the chunks of a row share one scale.
 * WN and Kp multiples of 8. */
int exx_debug_matrix_digits(int nout, int nk, const double *C, int WN, int Kp, int n0, int k0, float *digits,
                            float *scales);

/* Failure detection without a fault: launches one kernel whose two mbarrier waits (the
 * same bounded waits the pass kernels use: the polled one of the five-pass kernels, 4096
 * polls, and the wall-time one of the three-pass kernels, here 2 ms) wait on a barrier that
 * nothing completes.  Each limit runs out, the kernel records it in an error word and
 * returns; *status_h is then EXX_ERR_TIMEOUT when both waits gave up (EXX_OK otherwise).
 * The context stays usable.  Returns EXX_ERR_CUDA without a GPU. */
int exx_debug_wait_timeout(int *status_h);

#ifdef __cplusplus
}
#endif
#endif
