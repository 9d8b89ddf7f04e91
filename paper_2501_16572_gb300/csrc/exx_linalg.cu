// FP64 reductions and dense linear algebra of the path: exchange energy, the ACE
// matrices of Sec. III.A (M = dV Psi^T W, Cholesky factor of -sym(M), its inverse,
// xi = W L^{-T}) and the ACE application of Sec. III.B.
#include "exx_internal.h"

#include <algorithm>
#include <mutex>

namespace exx {

namespace {

// Neumaier-compensated accumulator (s, c)
struct KSum {
    double s, c;
};
__device__ __forceinline__ void kadd(KSum &k, double x)
{
    double t = k.s + x;
    if (fabs(k.s) >= fabs(x)) k.c += (k.s - t) + x;
    else k.c += (x - t) + k.s;
    k.s = t;
}
__device__ __forceinline__ void kmerge(KSum &a, const KSum &b)
{
    kadd(a, b.s);
    a.c += b.c;
}

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 512;

// E partial sums over a fixed grid: thread t of T sums (f_c dV / 4) psi_c(r) v_c(r) over
// the columns c in order and its points r = t, t + T, ... in plain FP64 (n N / T terms,
// about 10^2..10^4: relative rounding far below 1e-13); the threads' sums are merged with
// Neumaier compensation in a fixed tree, then the blocks' (reduce_partials_kernel).
__global__ void __launch_bounds__(kRedThreads)
energy_partial_kernel(const double *psi, int n, long ld, const double *f, const double *v, long ldv,
                      long N, double dV, KSum *partials)
{
    __shared__ KSum sh[kRedThreads];
    KSum acc{0.0, 0.0};
    const long T = long(gridDim.x) * blockDim.x;
    const long t0 = long(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t0 < N) {
        double s = 0.0;
        for (int c = 0; c < n; ++c) {
            const double *pc = psi + long(c) * ld, *vc = v + long(c) * ldv;
            const double w = 0.25 * f[c] * dV;
            for (long r = t0; r < N; r += T) s = fma(w * pc[r], vc[r], s);
        }
        acc.s = s;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int stride = kRedThreads / 2; stride > 0; stride >>= 1) {
        if (threadIdx.x < stride) kmerge(sh[threadIdx.x], sh[threadIdx.x + stride]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

// The block partials merged in a fixed tree by one block of kRedThreads threads.
__global__ void __launch_bounds__(kRedThreads) reduce_partials_kernel(const KSum *partials, int np, double *out)
{
    __shared__ KSum sh[kRedThreads];
    KSum acc{0.0, 0.0};
    for (int i = threadIdx.x; i < np; i += kRedThreads) kmerge(acc, partials[i]);
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int stride = kRedThreads / 2; stride > 0; stride >>= 1) {
        if (threadIdx.x < stride) kmerge(sh[threadIdx.x], sh[threadIdx.x + stride]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0].s + sh[0].c;
}

// ---- FP64 GEMMs (DFMA; GB300's FP64 rate makes these compute-bound) -----------------
constexpr int kTile = 64, kKt = 16, kGemmThreads = 256;

// C_z[i][j] = sum_{r in chunk z} A(r, i) B(r, j); A(r, i) = A[r + lda*i] (the columns of
// A and B are orbitals, r runs over the grid).  Partial tiles go to ws[z].
__global__ void __launch_bounds__(kGemmThreads)
gemm_tn_partial_kernel(int na, int nb, long K, long kchunk, const double *A, long lda,
                       const double *B, long ldb, double *ws)
{
    __shared__ double As[kKt][kTile + 1];
    __shared__ double Bs[kKt][kTile + 1];
    const int i0 = blockIdx.x * kTile, j0 = blockIdx.y * kTile;
    const long k_begin = long(blockIdx.z) * kchunk;
    const long k_end = min(K, k_begin + kchunk);
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    for (long k0 = k_begin; k0 < k_end; k0 += kKt) {
        for (int t = threadIdx.x; t < kKt * kTile; t += kGemmThreads) {
            int kk = t % kKt, ii = t / kKt;
            long r = k0 + kk;
            As[kk][ii] = (r < k_end && i0 + ii < na) ? A[r + lda * (i0 + ii)] : 0.0;
            Bs[kk][ii] = (r < k_end && j0 + ii < nb) ? B[r + ldb * (j0 + ii)] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kKt; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[kk][ty + 16 * u];
                b[u] = Bs[kk][tx + 16 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[u][w] = fma(a[u], b[w], acc[u][w]);
        }
        __syncthreads();
    }
    double *wz = ws + size_t(blockIdx.z) * na * nb;
    for (int u = 0; u < 4; ++u)
        for (int w = 0; w < 4; ++w) {
            int i = i0 + ty + 16 * u, j = j0 + tx + 16 * w;
            if (i < na && j < nb) wz[i + size_t(na) * j] = acc[u][w];
        }
}

__global__ void splitk_reduce_kernel(const double *ws, int nsplit, int na, int nb, double alpha,
                                     double *C, int ldc)
{
    const long e = long(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= long(na) * nb) return;
    int i = int(e % na), j = int(e / na);
    double s = 0.0;
    for (int z = 0; z < nsplit; ++z) s += ws[size_t(z) * na * nb + e];
    C[i + size_t(ldc) * j] = alpha * s;
}

// C(r, j) = alpha * sum_k A(r, k) Bop(k, j), A(r, k) = A[r + lda*k],
// Bop(k, j) = B[j*sbj + k*sbk];  r < M (grid rows), j < Nc, k < K.
__global__ void __launch_bounds__(kGemmThreads)
gemm_rows_kernel(long M, int Nc, int K, const double *A, long lda, const double *B, long sbj,
                 long sbk, double alpha, double *C, long ldc)
{
    __shared__ double As[kKt][kTile + 1];
    __shared__ double Bs[kKt][kTile + 1];
    const long r0 = long(blockIdx.x) * kTile;
    const int j0 = blockIdx.y * kTile;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += kKt) {
        for (int t = threadIdx.x; t < kKt * kTile; t += kGemmThreads) {
            int rr = t % kTile, kk = t / kTile;
            As[kk][rr] = (r0 + rr < M && k0 + kk < K) ? A[(r0 + rr) + lda * (k0 + kk)] : 0.0;
            int jj = t % kTile;
            Bs[kk][jj] = (j0 + jj < Nc && k0 + kk < K) ? B[(j0 + jj) * sbj + (k0 + kk) * sbk] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kKt; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[kk][tx + 16 * u];
                b[u] = Bs[kk][ty + 16 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[u][w] = fma(a[u], b[w], acc[u][w]);
        }
        __syncthreads();
    }
    for (int u = 0; u < 4; ++u)
        for (int w = 0; w < 4; ++w) {
            long r = r0 + tx + 16 * u;
            int j = j0 + ty + 16 * w;
            if (r < M && j < Nc) C[r + ldc * j] = alpha * acc[u][w];
        }
}

constexpr int kCholThreads = 1024;

// n <= kCholSmemMax: one CTA with everything in shared memory (column-major n x n):
// right-looking Cholesky (column j: pivot, scale, rank-1 update of the trailing lower
// triangle), then the inverse in place, columns from the right (unblocked triangular
// inverse): X_jj = 1 / L_jj and X(j+1:, j) = -X_jj X(j+1:, j+1:) L(j+1:, j), the
// triangular product into a scratch column.
constexpr int kCholSmemMax = 128;
__global__ void __launch_bounds__(kCholThreads)
cholesky_inverse_smem_kernel(int n, const double *M, double *Linv, int *info_d)
{
    extern __shared__ double S[];   // n x n, S[i + n j], then n scratch values
    double *y = S + n * n;
    __shared__ int failed;
    const int tid = threadIdx.x;
    for (int e = tid; e < n * n; e += blockDim.x) {
        const int i = e % n, j = e / n;
        S[e] = (i >= j) ? -0.5 * (M[i + size_t(n) * j] + M[j + size_t(n) * i]) : 0.0;
    }
    if (tid == 0) {
        failed = 0;
        info_d[0] = 0;
    }
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        if (tid == 0) {
            const double d = S[j + n * j];
            if (!(d > 0.0)) {
                failed = 1;
                info_d[0] = j + 1;
            } else {
                S[j + n * j] = sqrt(d);
            }
        }
        __syncthreads();
        if (failed) return;   // uniform: read after the barrier
        const double djj = S[j + n * j];
        for (int i = j + 1 + tid; i < n; i += blockDim.x) S[i + n * j] /= djj;
        __syncthreads();
        // trailing lower triangle: warps over its columns k, lanes over consecutive rows i
        for (int k = j + 1 + (tid >> 5); k < n; k += blockDim.x >> 5) {
            const double lk = S[k + n * j];
            for (int i = k + (tid & 31); i < n; i += 32) S[i + n * k] -= S[i + n * j] * lk;
        }
        __syncthreads();
    }
    for (int j = n - 1; j >= 0; --j) {
        const double xjj = 1.0 / S[j + n * j];
        // y_i = sum_{k = j+1..i} X(i, k) L(k, j), rows i > j (X(j+1:, j+1:) is final): a
        // thread per row (consecutive lanes read consecutive rows of a column), four
        // partial sums against the FMA latency
        for (int i = j + 1 + tid; i < n; i += blockDim.x) {
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
            int k = j + 1;
            for (; k + 3 <= i; k += 4) {
                s0 = fma(S[i + n * k], S[k + n * j], s0);
                s1 = fma(S[i + n * (k + 1)], S[k + 1 + n * j], s1);
                s2 = fma(S[i + n * (k + 2)], S[k + 2 + n * j], s2);
                s3 = fma(S[i + n * (k + 3)], S[k + 3 + n * j], s3);
            }
            for (; k <= i; ++k) s0 = fma(S[i + n * k], S[k + n * j], s0);
            y[i] = (s0 + s1) + (s2 + s3);
        }
        __syncthreads();
        for (int i = j + 1 + tid; i < n; i += blockDim.x) S[i + n * j] = -xjj * y[i];
        if (tid == 0) S[j + n * j] = xjj;
        __syncthreads();
    }
    for (int e = tid; e < n * n; e += blockDim.x) {
        const int i = e % n, j = e / n;
        Linv[e] = (i >= j) ? S[e] : 0.0;
    }
}

// ---- blocked Cholesky and triangular inverse for n > kCholSmemMax (many CTAs) -----------
// A = -(M + M^T)/2 is factored in place, right-looking, in column blocks of kCb:
//   diagonal block: A_kk = L_kk L_kk^T and D_k = L_kk^{-1} (one CTA, shared memory);
//   panel:          L_ik = A_ik D_k^T for the row blocks i > k (a CTA per row block);
//   trailing:       A_ij -= L_ik L_jk^T for i >= j > k (a CTA per lower 64 x 64 tile).
// Then X = L^{-1} block row by block row: X_ii = D_i (written with the factorisation),
// X_ij = -D_i sum_{k=j}^{i-1} L_ik X_kj (a CTA per block j < i).
// A failed pivot sets info_d[0] = 1 + its index; every later kernel then returns at once.
constexpr int kCb = 64;

__global__ void chol_prep_kernel(int n, const double *M, double *A, double *X, int *info_d)
{
    for (long e = long(blockIdx.x) * blockDim.x + threadIdx.x; e < long(n) * n; e += long(gridDim.x) * blockDim.x) {
        const int i = int(e % n), j = int(e / n);
        A[e] = (i >= j) ? -0.5 * (M[i + size_t(n) * j] + M[j + size_t(n) * i]) : 0.0;
        X[e] = 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) info_d[0] = 0;
}

// One CTA: the diagonal block at (k0, k0) of size b <= kCb: factor, write L_kk into A and
// D = L_kk^{-1} (lower, b x b, leading dimension kCb) into Dk and into X's diagonal block.
__global__ void __launch_bounds__(kCholThreads) chol_diag_kernel(int n, double *A, int k0, int b, double *Dk,
                                                                 double *X, int *info_d)
{
    __shared__ double S[kCb * kCb];
    __shared__ double y[kCb];
    __shared__ int failed;
    const int tid = threadIdx.x;
    if (tid == 0) failed = info_d[0] != 0;
    __syncthreads();
    if (failed) return;
    for (int e = tid; e < b * b; e += blockDim.x) {
        const int i = e % b, j = e / b;
        S[i + kCb * j] = (i >= j) ? A[(k0 + i) + size_t(n) * (k0 + j)] : 0.0;
    }
    __syncthreads();
    for (int j = 0; j < b; ++j) {
        if (tid == 0) {
            const double d = S[j + kCb * j];
            if (!(d > 0.0)) {
                failed = 1;
                info_d[0] = k0 + j + 1;
            } else {
                S[j + kCb * j] = sqrt(d);
            }
        }
        __syncthreads();
        if (failed) return;
        const double djj = S[j + kCb * j];
        for (int i = j + 1 + tid; i < b; i += blockDim.x) S[i + kCb * j] /= djj;
        __syncthreads();
        for (int k = j + 1 + (tid >> 5); k < b; k += blockDim.x >> 5) {
            const double lk = S[k + kCb * j];
            for (int i = k + (tid & 31); i < b; i += 32) S[i + kCb * k] -= S[i + kCb * j] * lk;
        }
        __syncthreads();
    }
    for (int e = tid; e < b * b; e += blockDim.x) {
        const int i = e % b, j = e / b;
        if (i >= j) A[(k0 + i) + size_t(n) * (k0 + j)] = S[i + kCb * j];
    }
    __syncthreads();
    // in-place inverse of the b x b lower triangle, columns from the right
    for (int j = b - 1; j >= 0; --j) {
        const double xjj = 1.0 / S[j + kCb * j];
        for (int i = j + 1 + tid; i < b; i += blockDim.x) {
            double acc = 0.0;
            for (int k = j + 1; k <= i; ++k) acc = fma(S[i + kCb * k], S[k + kCb * j], acc);
            y[i] = acc;
        }
        __syncthreads();
        for (int i = j + 1 + tid; i < b; i += blockDim.x) S[i + kCb * j] = -xjj * y[i];
        if (tid == 0) S[j + kCb * j] = xjj;
        __syncthreads();
    }
    for (int e = tid; e < kCb * kCb; e += blockDim.x) {
        const int i = e % kCb, j = e / kCb;
        const double v = (i < b && j < b && i >= j) ? S[i + kCb * j] : 0.0;
        Dk[e] = v;
        if (i < b && j < b) X[(k0 + i) + size_t(n) * (k0 + j)] = v;
    }
}

// C (rows r0.., columns c0.., 64 x 64 tile, leading dimension n) op= sum_t P(r, t) Q(c, t),
// P(r, t) = Pm[r + ldp t], Q(c, t) = Qm[c + ldq t], t < K; mode 0: C = alpha acc; 1: C += alpha acc.
__device__ __forceinline__ void tile_gemm_nt(int rows, int cols, int K, const double *Pm, long ldp, const double *Qm,
                                             long ldq, double alpha, double *C, long ldc, int mode)
{
    __shared__ double Ps[kKt][kTile + 1];
    __shared__ double Qs[kKt][kTile + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += kKt) {
        for (int t = threadIdx.x; t < kKt * kTile; t += kGemmThreads) {
            const int rr = t % kTile, kk = t / kTile;
            Ps[kk][rr] = (rr < rows && k0 + kk < K) ? Pm[rr + ldp * (k0 + kk)] : 0.0;
            Qs[kk][rr] = (rr < cols && k0 + kk < K) ? Qm[rr + ldq * (k0 + kk)] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kKt; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = Ps[kk][tx + 16 * u];
                b[u] = Qs[kk][ty + 16 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[u][w] = fma(a[u], b[w], acc[u][w]);
        }
        __syncthreads();
    }
    for (int u = 0; u < 4; ++u)
        for (int w = 0; w < 4; ++w) {
            const int r = tx + 16 * u, c = ty + 16 * w;
            if (r < rows && c < cols) {
                double *o = C + r + ldc * c;
                *o = mode ? *o + alpha * acc[u][w] : alpha * acc[u][w];
            }
        }
}

// panel: row block i = k0/kCb + 1 + blockIdx.x, L_ik = A_ik D_k^T (into a scratch copy first:
// the tile reads A_ik while writing it)
__global__ void __launch_bounds__(kGemmThreads) chol_panel_kernel(int n, double *A, int k0, int b, const double *Dk,
                                                                  double *scratch, const int *info_d)
{
    if (info_d[0]) return;
    const int r0 = k0 + b + blockIdx.x * kCb;
    const int rows = min(kCb, n - r0);
    double *tmp = scratch + size_t(blockIdx.x) * kCb * kCb;
    // tmp(r, c) = sum_t A(r0 + r, k0 + t) D(c, t)
    tile_gemm_nt(rows, b, b, A + r0 + size_t(n) * k0, n, Dk, kCb, 1.0, tmp, kCb, 0);
    __syncthreads();
    for (int e = threadIdx.x; e < kCb * kCb; e += blockDim.x) {
        const int r = e % kCb, c = e / kCb;
        if (r < rows && c < b) A[(r0 + r) + size_t(n) * (k0 + c)] = tmp[r + kCb * c];
    }
}

// trailing update of the lower triangle: tile (bi, bj), bi >= bj, of the part past k0 + b
__global__ void __launch_bounds__(kGemmThreads) chol_update_kernel(int n, double *A, int k0, int b, const int *info_d)
{
    if (info_d[0]) return;
    const int bi = blockIdx.x, bj = blockIdx.y;
    if (bi < bj) return;
    const int base = k0 + b;
    const int r0 = base + bi * kCb, c0 = base + bj * kCb;
    const int rows = min(kCb, n - r0), cols = min(kCb, n - c0);
    // A(r, c) -= sum_t L(r, k0 + t) L(c, k0 + t)   (the strict upper part of a diagonal tile
    // is updated too; it is never read and is cleared at the end)
    tile_gemm_nt(rows, cols, b, A + r0 + size_t(n) * k0, n, A + c0 + size_t(n) * k0, n, -1.0,
                 A + r0 + size_t(n) * c0, n, 1);
}

// block row i of X = L^{-1}: for bj < i (blockIdx.x): T = sum_{k=bj}^{i-1} L_ik X_kj, X_ij = -D_i T
__global__ void __launch_bounds__(kGemmThreads) chol_inv_row_kernel(int n, const double *A, double *X, int bi,
                                                                    const double *Dall, double *scratch,
                                                                    const int *info_d)
{
    if (info_d[0]) return;
    const int bj = blockIdx.x;
    const int r0 = bi * kCb, c0 = bj * kCb;
    const int rows = min(kCb, n - r0), cols = min(kCb, n - c0);
    double *T = scratch + size_t(blockIdx.x) * kCb * kCb;
    // T(r, c) = sum_{t = c0 .. r0-1} L(r0 + r, t) X(t, c0 + c): P = L rows, Q(c, t) = X(t, c0 + c)
    // (Q given transposed: Q(c, t) = Xm[c + ldq t] needs X^T; use the rows form instead)
    const int K = r0 - c0;
    {
        __shared__ double Ps[kKt][kTile + 1];
        __shared__ double Qs[kKt][kTile + 1];
        const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
        double acc[4][4] = {};
        for (int k = 0; k < K; k += kKt) {
            for (int t = threadIdx.x; t < kKt * kTile; t += kGemmThreads) {
                const int rr = t % kTile, kk = t / kTile;
                const int tt = c0 + k + kk;
                Ps[kk][rr] = (rr < rows && k + kk < K) ? A[(r0 + rr) + size_t(n) * tt] : 0.0;
                Qs[kk][rr] = (rr < cols && k + kk < K) ? X[tt + size_t(n) * (c0 + rr)] : 0.0;
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < kKt; ++kk) {
                double a[4], b[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    a[u] = Ps[kk][tx + 16 * u];
                    b[u] = Qs[kk][ty + 16 * u];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int w = 0; w < 4; ++w) acc[u][w] = fma(a[u], b[w], acc[u][w]);
            }
            __syncthreads();
        }
        for (int u = 0; u < 4; ++u)
            for (int w = 0; w < 4; ++w) {
                const int r = tx + 16 * u, c = ty + 16 * w;
                T[r + kCb * c] = (r < rows && c < cols) ? acc[u][w] : 0.0;
            }
    }
    __syncthreads();
    // X_ij(r, c) = -sum_t D_i(r, t) T(t, c): P = D_i (rows r), Q(c, t) = T(t, c) -> T^T
    const double *Di = Dall + size_t(bi) * kCb * kCb;
    {
        __shared__ double Ps[kKt][kTile + 1];
        __shared__ double Qs[kKt][kTile + 1];
        const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
        double acc[4][4] = {};
        for (int k = 0; k < rows; k += kKt) {
            for (int t = threadIdx.x; t < kKt * kTile; t += kGemmThreads) {
                const int rr = t % kTile, kk = t / kTile;
                Ps[kk][rr] = (k + kk < rows) ? Di[rr + kCb * (k + kk)] : 0.0;
                Qs[kk][rr] = (k + kk < rows) ? T[(k + kk) + kCb * rr] : 0.0;
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < kKt; ++kk) {
                double a[4], b[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    a[u] = Ps[kk][tx + 16 * u];
                    b[u] = Qs[kk][ty + 16 * u];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int w = 0; w < 4; ++w) acc[u][w] = fma(a[u], b[w], acc[u][w]);
            }
            __syncthreads();
        }
        for (int u = 0; u < 4; ++u)
            for (int w = 0; w < 4; ++w) {
                const int r = tx + 16 * u, c = ty + 16 * w;
                if (r < rows && c < cols) X[(r0 + r) + size_t(n) * (c0 + c)] = -acc[u][w];
            }
    }
}

}  // namespace

int energy_fp64(Plan &P, const double *psi, int n, long ld, const double *f, const double *v, long ld_v,
                double *E_h, cudaStream_t s)
{
    size_t need = kRedBlocks * sizeof(KSum) + 64;
    if (int rc = dev_reserve(P.red_ws, need)) return rc;
    KSum *parts = static_cast<KSum *>(P.red_ws.p);
    double *res = reinterpret_cast<double *>(static_cast<char *>(P.red_ws.p) + kRedBlocks * sizeof(KSum));
    int tb = timing_begin(P, EXX_TIMING_ENERGY, s);
    energy_partial_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(psi, n, ld, f, v, ld_v, P.N, P.dV, parts);
    EXX_LAUNCH("energy_partial_kernel");
    reduce_partials_kernel<<<1, kRedThreads, 0, s>>>(parts, kRedBlocks, res);
    timing_end(P, tb, s);
    EXX_LAUNCH("reduce_partials_kernel");
    P.launches += 2;
    EXX_CUDA(cudaMemcpyAsync(E_h, res, sizeof(double), cudaMemcpyDeviceToHost, s));
    EXX_CUDA(cudaStreamSynchronize(s));
    return EXX_OK;
}

int gemm_fp64_tn_splitk(Plan &P, int na, int nb, int K, const double *A, long lda, const double *B,
                        long ldb, double alpha, double *C, int ldc, cudaStream_t s)
{
    const int gx = (na + kTile - 1) / kTile, gy = (nb + kTile - 1) / kTile;
    // enough CTAs to fill the GPU twice over, each with a K chunk of at least 256
    int nsplit = std::max(1, (2 * P.num_sms + gx * gy - 1) / (gx * gy));
    long kchunk = (long(K) + nsplit - 1) / nsplit;
    kchunk = ((kchunk + kKt - 1) / kKt) * kKt;
    if (kchunk < 256) kchunk = 256;
    nsplit = int((long(K) + kchunk - 1) / kchunk);
    if (int rc = dev_reserve(P.gemm_ws, size_t(nsplit) * na * nb * sizeof(double))) return rc;
    double *ws = static_cast<double *>(P.gemm_ws.p);
    int tb = timing_begin(P, EXX_TIMING_GEMM, s);
    gemm_tn_partial_kernel<<<dim3(gx, gy, nsplit), kGemmThreads, 0, s>>>(na, nb, K, kchunk, A, lda, B,
                                                                         ldb, ws);
    EXX_LAUNCH("gemm_tn_partial_kernel");
    long tot = long(na) * nb;
    splitk_reduce_kernel<<<unsigned((tot + 255) / 256), 256, 0, s>>>(ws, nsplit, na, nb, alpha, C, ldc);
    timing_end(P, tb, s);
    EXX_LAUNCH("splitk_reduce_kernel");
    P.launches += 2;
    return EXX_OK;
}

int gemm_fp64_nt(Plan &P, int M, int Nc, int K, const double *A, long lda, const double *B, long ldb,
                 double alpha, double *C, long ldc, cudaStream_t s)
{
    // Bop(k, j) = B(j, k) = B[j + ldb*k]
    dim3 grid(unsigned((long(M) + kTile - 1) / kTile), unsigned((Nc + kTile - 1) / kTile));
    int tb = timing_begin(P, EXX_TIMING_GEMM, s);
    gemm_rows_kernel<<<grid, kGemmThreads, 0, s>>>(M, Nc, K, A, lda, B, 1, ldb, alpha, C, ldc);
    timing_end(P, tb, s);
    EXX_LAUNCH("gemm_rows_kernel");
    P.launches++;
    return EXX_OK;
}

int gemm_fp64_nn(Plan &P, int M, int Nc, int K, const double *A, long lda, const double *B, long ldb,
                 double alpha, double *C, long ldc, cudaStream_t s)
{
    // Bop(k, j) = B(k, j) = B[k + ldb*j]
    dim3 grid(unsigned((long(M) + kTile - 1) / kTile), unsigned((Nc + kTile - 1) / kTile));
    int tb = timing_begin(P, EXX_TIMING_GEMM, s);
    gemm_rows_kernel<<<grid, kGemmThreads, 0, s>>>(M, Nc, K, A, lda, B, ldb, 1, alpha, C, ldc);
    timing_end(P, tb, s);
    EXX_LAUNCH("gemm_rows_kernel");
    P.launches++;
    return EXX_OK;
}

int cholesky_neg_sym_and_inverse(Plan &P, int n, const double *M, double *Linv, int *info_d,
                                 cudaStream_t s)
{
    int tb = timing_begin(P, EXX_TIMING_CHOL, s);
    if (n <= kCholSmemMax) {
        const size_t smem = (size_t(n) * n + n) * sizeof(double);
        EXX_CUDA(cudaFuncSetAttribute(cholesky_inverse_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      int(smem)));
        cholesky_inverse_smem_kernel<<<1, kCholThreads, smem, s>>>(n, M, Linv, info_d);
        timing_end(P, tb, s);
        EXX_LAUNCH("cholesky_inverse_smem_kernel");
        P.launches++;
        return EXX_OK;
    }
    // workspace: A (n x n), the diagonal-block inverses (nbk blocks of kCb^2), tile scratch
    const int nbk = (n + kCb - 1) / kCb;
    const size_t nn = size_t(n) * n, blk = size_t(kCb) * kCb;
    if (int rc = dev_reserve(P.small_ws, (nn + 2 * size_t(nbk) * blk) * sizeof(double))) return rc;
    double *A = static_cast<double *>(P.small_ws.p);
    double *Dall = A + nn;
    double *scratch = Dall + size_t(nbk) * blk;
    const int eg = std::min(4 * P.num_sms, int((nn + 255) / 256));
    chol_prep_kernel<<<eg, 256, 0, s>>>(n, M, A, Linv, info_d);
    EXX_LAUNCH("chol_prep_kernel");
    P.launches++;
    for (int kb = 0; kb < nbk; ++kb) {
        const int k0 = kb * kCb, b = std::min(kCb, n - k0);
        chol_diag_kernel<<<1, kCholThreads, 0, s>>>(n, A, k0, b, Dall + size_t(kb) * blk, Linv, info_d);
        EXX_LAUNCH("chol_diag_kernel");
        P.launches++;
        const int rest = nbk - kb - 1;
        if (rest == 0) break;
        chol_panel_kernel<<<rest, kGemmThreads, 0, s>>>(n, A, k0, b, Dall + size_t(kb) * blk, scratch, info_d);
        EXX_LAUNCH("chol_panel_kernel");
        chol_update_kernel<<<dim3(rest, rest), kGemmThreads, 0, s>>>(n, A, k0, b, info_d);
        EXX_LAUNCH("chol_update_kernel");
        P.launches += 2;
    }
    for (int bi = 1; bi < nbk; ++bi) {
        chol_inv_row_kernel<<<bi, kGemmThreads, 0, s>>>(n, A, Linv, bi, Dall, scratch, info_d);
        EXX_LAUNCH("chol_inv_row_kernel");
        P.launches++;
    }
    timing_end(P, tb, s);
    return EXX_OK;
}

// ---------------------------------------------------------------------------------------
// Allocation-free Gram matrix M = dV Psi^T W (exx_gram_noalloc in include/exx.h).
//
// Same split-K kernels as the ACE matrix above, but the partial tiles live in a fixed
// device array that is part of the loaded library, so the call needs no cudaMalloc and
// no plan.  It exists for callers that must not allocate device memory at the point of
// the call: callers whose device memory is owned by a pool or framework allocator that
// this library cannot use, memory-capped processes that reserve everything up front, and
// loops that must not stall (cudaMalloc and cudaFree can synchronize the whole device).
namespace {

constexpr int kGramNoAllocMaxN = 128;      // largest n accepted
constexpr int kGramNoAllocMaxSplit = 8;    // K chunks (partial tiles per entry)

// One copy per GPU that loads the library (1 MiB), held until the process exits.  Host
// code must not pass this name to a kernel: on the host it is only a stand-in symbol.
static __device__ __align__(256) double g_gram_partials[kGramNoAllocMaxSplit * kGramNoAllocMaxN * kGramNoAllocMaxN];

constexpr int kMaxDevices = 64;
std::mutex g_gram_mutex;
double *g_gram_addr[kMaxDevices] = {};     // device address of g_gram_partials, per device

// Device address of the scratch array on the current device (looked up once per device).
int gram_scratch(double **out)
{
    int dev = 0;
    EXX_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("exx_gram_noalloc: device ordinal out of range");
        return EXX_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_gram_mutex);
    if (!g_gram_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_gram_partials);
        if (e != cudaSuccess) return cuda_fail(e, "exx_gram_noalloc: cudaGetSymbolAddress");
        g_gram_addr[dev] = static_cast<double *>(p);
    }
    *out = g_gram_addr[dev];
    return EXX_OK;
}

}  // namespace
}  // namespace exx

extern "C" int exx_gram_noalloc(int N, double dV, const double *Psi, int n, long ld, const double *W, long ld_w,
                                double *M, exx_stream_t stream)
{
    using namespace exx;
    if (!Psi || !W || !M) {
        set_error("exx_gram_noalloc: NULL array");
        return EXX_ERR_INVALID_ARG;
    }
    if (N < 1 || ld < N || ld_w < N) {
        set_error("exx_gram_noalloc: need N >= 1 and leading dimensions >= N");
        return EXX_ERR_INVALID_ARG;
    }
    if (n < 1 || n > kGramNoAllocMaxN) {
        set_error("exx_gram_noalloc: n must be in [1, 128] (the fixed scratch holds 8 partial 128 x 128 tiles)");
        return EXX_ERR_INVALID_ARG;
    }
    double *ws = nullptr;
    if (int rc = gram_scratch(&ws)) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int g = (n + kTile - 1) / kTile;
    long kchunk = (long(N) + kGramNoAllocMaxSplit - 1) / kGramNoAllocMaxSplit;
    kchunk = std::max<long>(256, ((kchunk + kKt - 1) / kKt) * kKt);
    const int nsplit = int((long(N) + kchunk - 1) / kchunk);   // <= kGramNoAllocMaxSplit
    // every partial tile entry (z, i < n, j < n) is rewritten below, so nothing from an
    // earlier call survives into this one and no clearing is needed
    gemm_tn_partial_kernel<<<dim3(g, g, nsplit), kGemmThreads, 0, s>>>(n, n, N, kchunk, Psi, ld, W, ld_w, ws);
    EXX_LAUNCH("gemm_tn_partial_kernel (no-alloc)");
    const long tot = long(n) * n;
    splitk_reduce_kernel<<<unsigned((tot + 255) / 256), 256, 0, s>>>(ws, nsplit, n, n, dV, M, n);
    EXX_LAUNCH("splitk_reduce_kernel (no-alloc)");
    return EXX_OK;
}
