// Internal declarations of libexx_gb300 (not part of the public C interface).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>

#include "../../include/exx.h"

namespace exx {

// ---- error plumbing ---------------------------------------------------------------
void set_error(const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);
#define EXX_CUDA(call)                                                     \
    do {                                                                   \
        cudaError_t _e = (call);                                           \
        if (_e != cudaSuccess) return ::exx::cuda_fail(_e, #call);         \
    } while (0)
#define EXX_LAUNCH(what)                                                   \
    do {                                                                   \
        cudaError_t _e = cudaGetLastError();                               \
        if (_e != cudaSuccess) return ::exx::cuda_fail(_e, what);          \
    } while (0)

// ---- division by an invariant 32-bit divisor ------------------------------------------
// Granlund & Montgomery, "Division by invariant integers using multiplication" (PLDI
// 1994), Fig. 4.1: with l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
//   t = mulhi(m, n),  n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0)
// exactly for every 32-bit n.  Used for row -> (field, row in field) in the pass kernels.
#ifdef __CUDACC__
#define EXX_HD __host__ __device__
#else
#define EXX_HD
#endif
struct FastDiv {
    uint32_t d, m, s1, s2;
};
inline FastDiv make_fastdiv(uint32_t d)
{
    uint32_t l = 0;
    while ((uint64_t(1) << l) < d) ++l;
    const uint64_t m = ((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1;
    return {d, uint32_t(m), l < 1 ? l : 1u, l > 0 ? l - 1 : 0u};
}
EXX_HD inline uint32_t fast_div(uint32_t n, const FastDiv &f)
{
#ifdef __CUDA_ARCH__
    const uint32_t t = __umulhi(f.m, n);
#else
    const uint32_t t = uint32_t((uint64_t(f.m) * n) >> 32);
#endif
    return (t + ((n - t) >> f.s1)) >> f.s2;
}

// ---- the five passes of one batched solve --------------------------------------------
// A grid function batch is P fields of N values.  Each pass contracts one axis with
// an n_d x n_d matrix; a pass sees a field as R = N / K rows of K values.
//   LOAD_KSLOW : element (row r, k) at k*R + r   (contracted axis slowest)
//   LOAD_KFAST : element (row r, k) at r*K + k   (contracted axis fastest)
//   LOAD_PAIR  : as KSLOW, value psi_m * psi_n of the field's orbital pair
//   STORE_NSLOW: output (row r, n) at n*R + r;  STORE_NFAST: at r*K + n
enum { LOAD_KSLOW = 0, LOAD_KFAST = 1, LOAD_PAIR = 2 };
enum { STORE_NSLOW = 0, STORE_NFAST = 1 };

// Pass table (x fastest natural layout (z,y,x); letters a,b,c are the eigen-modes):
//   P1 pair density + forward z   (z,y,x) -> (c,y,x)   KSLOW(PAIR) / NSLOW   R = n1 n2
//   P2 forward x                  (c,y,x) -> (a,c,y)   KFAST / NSLOW         R = n2 n3
//   P3 forward y, x F, inverse y  (a,c,y) -> (a,c,j)   KFAST / NFAST         R = n1 n3
//   P4 inverse x                  (a,c,j) -> (c,j,x)   KSLOW / NFAST         R = n2 n3
//   P5 inverse z                  (c,j,x) -> (z,j,x)   KSLOW / NSLOW         R = n1 n2
struct PassGeom {
    int load, store, axis, inverse, scale;
    int R, K;
};
PassGeom pass_geom(const int n[3], int pass);  // pass 0..4 (P1..P5)

// ---- pair blocks and batches (host scheduler) ----------------------------------------
// A block pairs orbital group I (occupied) with group J.
//   SYM_OFF : I != J, both occupied; pairs I x J; writes outputs of I and J
//   SYM_DIAG: I == J; pairs m <= n in I;          writes outputs of I
//   ONE_SIDE: I occupied, J output-only;          writes outputs of J
// Blocks in one batch write disjoint outputs, so the accumulation needs no atomics
// and its order is fixed.
enum { BLK_SYM_OFF = 0, BLK_SYM_DIAG = 1, BLK_ONE_SIDE = 2 };
struct Block {
    int I0, nI, J0, nJ, kind, field0;
};
struct Batch {
    int nfields;       // pairs (= fields) in this batch
    int block0, nblocks;  // range in the schedule's block list
};
struct Schedule {
    std::vector<Block> blocks;
    std::vector<int2> pairs;   // (m, n) per field, concatenated over batches
    std::vector<Batch> batches;
    std::vector<int> pair0;    // first pair index of each batch
    long unique_pairs = 0;
    int max_fields = 0;
    int max_blocks = 0;
};
Schedule build_schedule(int n_occ, int n_in, bool aliased, int block, int max_pairs);

// ---- host FP64 setup -------------------------------------------------------------------
void fd_weights(int p, double *w);                       // w[0..p]
void second_derivative(int n, double h, int bc, int p, double *D);  // n x n column-major
int sym_eig(int n, const double *A, double *V, double *lam);  // Householder + implicit QL
double kernel_f(double lam, int kernel, double omega);

// ---- the plan ----------------------------------------------------------------------------
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};
int dev_reserve(DevBuf &b, size_t bytes);
void dev_free(DevBuf &b);

// CUDA-event timing of every launch (exx_plan_set_timing)
struct TimingRec {
    int kind;
    cudaEvent_t start, stop;
};
struct Timing {
    bool on = false;
    std::vector<TimingRec> recs;
    std::vector<cudaEvent_t> pool;
};
struct Plan;
// Bracket one launch: tb = timing_begin(P, kind, s); launch; timing_end(P, tb, s).
int timing_begin(Plan &P, int kind, cudaStream_t s);
void timing_end(Plan &P, int rec, cudaStream_t s);

struct Plan {
    int n[3];
    int N;
    double h, dV, omega;
    int bc[3], fd_order, kernel;
    int prec = EXX_PREC_FP64;
    int pairs_per_batch = 0;   // 0 = default
    int block_orbitals = 0;    // 0 = default
    int shard_rank = 0, shard_world = 1;   // exx_plan_set_shard
    int device = 0;
    int num_sms = 0;
    std::vector<double> V[3], lam[3], F;   // host copies
    // FP64 path: per pass the K x K contraction matrix B[k*K + j] (output j, input k)
    DevBuf B64[6];                  // P1, P2, P3-forward, P3-inverse, P4, P5
    DevBuf F64;                     // F in the P3 layout [b][a][c]
    DevBuf F32;                     // same as two float planes, hi then lo
    // tensor path: per pass and precision the B operand pieces, canonical SMEM image
    DevBuf Btc[5][6];               // [prec][pass slot]: nblk^2 block images, (c, h) at (c nblk + h)
    int tc_nblk[5][3] = {};         // [prec][axis]: blocks the axis is cut into (1 = whole axis)
    int tc_bsz[5][3] = {};          // [prec][axis]: points per block (the last may be shorter)
    int tc_ysplit[5] = {};          // [prec]: pass 3 as two kernels (forward, inverse)
    // three-pass mode (EXX_PREC_BF16X7): per axis forward and inverse digit images (z in
    // N-blocks), f(Lambda) in the natural layout as FP32 hi and lo planes
    DevBuf t3img[3][2];
    DevBuf t3imgc[2][2];            // x and y images as K-chunks, when the slice passes stream them
    DevBuf F32n;
    int t3_share01 = 0;             // x and y have the same length and bc: one image serves both
    int t3_zwn = 0, t3_znbuf = 0;   // pass B matrix block width and buffers (0 = automatic)
    int t3_stage = -1;              // slice-pass input staging (-1 = automatic)
    int t3_pipe = -1;               // slice-pass software pipeline (-1 = automatic)
    int tuned = 0;                  // 1 = measured by exx_plan_autotune, 2 = taken from its cache
    double tune_ms = 0.0;           // the chosen setting's trial time per pair solve
    // original (non-batched) formalism: eigenvectors, f(Lambda) in the natural layout, workspace
    DevBuf orig_V, F64n, orig_ws;
    // Bloch (complex) plans: phases, eigenvalues, f, contraction matrices and workspace
    int cplx = 0;
    double theta[3] = {0.0, 0.0, 0.0};
    std::vector<double> clam[3], cF;
    DevBuf cmats, cFd, cwork, cpairs, cred, cace;
    // workspace
    DevBuf work[3];                 // batch buffers (fields x N)
    DevBuf pairs_d, blocks_d;       // schedule on the device
    DevBuf acc_hi, acc_lo, g32, psi32;  // split path accumulators and fp32 orbital copies
    DevBuf gemm_ws, small_ws, info_d, red_ws;
    DevBuf host_stage_psi, host_stage_f, host_stage_xi, host_stage_w;
    DevBuf err_d;                   // device error word of the bounded waits
    int tc_occ_off = 0;             // column of Psi_occ in the fp32 planes (0 when aliased)
    int tc_n_occ = 0;               // rows of g32's hi plane (its lo plane follows)
    float *tc_result = nullptr;     // buffer holding the last batch's solutions
    long tc_lo_off = 0;             // hi+lo intermediates: offset of the lo plane (floats)
    long launches = 0;
    Timing timing;
    // cached schedule
    int sched_key[4] = {-1, -1, -1, -1};
    uint64_t epoch = 0;   // changes whenever device data or settings that launches read change
    Schedule sched;
};

// kernels (exx_fp64.cu)
int fp64_solve_batch(Plan &P, const double *psi_occ, long ld_occ, const double *psi_in, long ld_in,
                     const int2 *pairs_d, int nfields, double *bufA, double *bufB, double **result,
                     cudaStream_t s);
int fp64_accumulate(Plan &P, const double *psi_occ, long ld_occ, const double *psi_in, long ld_in,
                    const double *f, const Block *blocks_d, int nblocks, const double *V,
                    double *out, long ld_out, cudaStream_t s);
int fp64_upload(Plan &P);

// split path (exx_tc.cu)
int tc_upload(Plan &P, int prec);
int tc_reserve_orbitals(Plan &P, int n_occ, int n_in, bool aliased);
void bump_epoch(Plan &P);
int tc_prepare_orbitals(Plan &P, const double *psi_occ, int n_occ, long ld_occ, const double *f,
                        const double *psi_in, int n_in, long ld_in, bool aliased, cudaStream_t s);
int tc_solve_batch(Plan &P, int prec, const int2 *pairs_d, int nfields, float *bufA, float *bufB,
                   cudaStream_t s);
int tc_accumulate(Plan &P, const Block *blocks_d, int nblocks, const float *V, cudaStream_t s);
int tc_finalize(Plan &P, int n_in, double *out, long ld_out, cudaStream_t s);
int tc_check_error(Plan &P, cudaStream_t s);
bool tc_is_hilo(int prec);
// original Kronecker formalism, one pair at a time (exx_original.cu)
int original_apply(Plan &P, const double *psi_occ, int n_occ, long ld_occ, const double *f, const double *psi_in,
                   int n_in, long ld_in, double *out, long ld_out, bool aliased, cudaStream_t s);
// three-pass split path (exx_tc3.cu)
bool tc3_supported(const Plan &P, std::string *why);
int tc3_upload(Plan &P);
int tc3_solve_batch(Plan &P, const int2 *pairs_d, int nfields, float *bufA, float *bufB, cudaStream_t s);
std::vector<std::pair<int, int>> tc3_z_choices(int n3);
void tc3_debug_layout(int n1, int n2, int n3, int share01, int *out);
void tc3_debug_matrix_digits(int nout, int nk, const double *C, int WN, int Kp, int n0, int k0, float *digits,
                             float *scales);
int tc_unit_gemm(int tf32, int n, int k, const float *A, const float *B, float *D, int *err);
int tc_wait_timeout_probe(int *status_h);

// reductions, GEMM, Cholesky (exx_linalg.cu)
int energy_fp64(Plan &P, const double *psi, int n, long ld, const double *f, const double *v,
                long ld_v, double *E_h, cudaStream_t s);
// D(i, j) = alpha sum_k A(i, k) B(j, k) on the tensor cores (fixed-point digits, exact
// 320-long chunks summed in FP64); A(i, k) = A[i as_i + k as_k], same for B and D.
int tc_gemm(Plan &P, int m, int n, long K, const double *A, long as_i, long as_k, const double *B, long bs_j,
            long bs_k, double alpha, double *D, long ds_i, long ds_j, cudaStream_t s);
int gemm_fp64_tn_splitk(Plan &P, int n_a, int n_b, int K, const double *A, long lda,
                        const double *B, long ldb, double alpha, double *C, int ldc, cudaStream_t s);
int gemm_fp64_nt(Plan &P, int M, int Ncols, int K, const double *A, long lda, const double *B,
                 long ldb, double alpha, double *C, long ldc, cudaStream_t s);
int gemm_fp64_nn(Plan &P, int M, int Ncols, int K, const double *A, long lda, const double *B,
                 long ldb, double alpha, double *C, long ldc, cudaStream_t s);
int cholesky_neg_sym_and_inverse(Plan &P, int n, const double *M, double *Linv, int *info_d,
                                 cudaStream_t s);

}  // namespace exx
