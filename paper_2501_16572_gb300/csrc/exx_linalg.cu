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

// One CTA: A = -(M + M^T)/2 (lower part), right-looking Cholesky A = L L^T in place,
// then Linv = L^{-1} (lower).  info_d[0] = 0 or 1 + failing pivot.
constexpr int kCholThreads = 1024;
__global__ void __launch_bounds__(kCholThreads)
cholesky_inverse_kernel(int n, const double *M, double *L, double *Linv, int *info_d)
{
    __shared__ int failed;
    const int tid = threadIdx.x;
    for (long e = tid; e < long(n) * n; e += blockDim.x) {
        int i = int(e % n), j = int(e / n);
        L[e] = (i >= j) ? -0.5 * (M[i + size_t(n) * j] + M[j + size_t(n) * i]) : 0.0;
        Linv[e] = 0.0;
    }
    if (tid == 0) {
        failed = 0;
        info_d[0] = 0;
    }
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        if (tid == 0) {
            double d = L[j + size_t(n) * j];
            if (!(d > 0.0)) {
                failed = 1;
                info_d[0] = j + 1;
            } else {
                L[j + size_t(n) * j] = sqrt(d);
            }
        }
        __syncthreads();
        if (failed) return;
        const double djj = L[j + size_t(n) * j];
        for (int i = j + 1 + tid; i < n; i += blockDim.x) L[i + size_t(n) * j] /= djj;
        __syncthreads();
        // trailing update of the lower triangle, columns k in (j, n), rows i >= k
        const int m = n - j - 1;
        for (long e = tid; e < long(m) * m; e += blockDim.x) {
            int ii = int(e % m), kk = int(e / m);
            if (ii < kk) continue;
            int i = j + 1 + ii, k = j + 1 + kk;
            L[i + size_t(n) * k] -= L[i + size_t(n) * j] * L[k + size_t(n) * j];
        }
        __syncthreads();
    }
    // Linv: row by row, X(i, c) = (delta_ic - sum_{k=c}^{i-1} L(i,k) X(k,c)) / L(i,i), c <= i
    for (int i = 0; i < n; ++i) {
        const double lii = L[i + size_t(n) * i];
        for (int c = tid; c <= i; c += blockDim.x) {
            double s = (c == i) ? 1.0 : 0.0;
            for (int k = c; k < i; ++k) s -= L[i + size_t(n) * k] * Linv[k + size_t(n) * c];
            Linv[i + size_t(n) * c] = s / lii;
        }
        __syncthreads();
    }
}

// The same for n <= kCholSmemMax with everything in shared memory (column-major n x n):
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
    if (n > kCholSmemMax) {
        if (int rc = dev_reserve(P.small_ws, size_t(n) * n * sizeof(double))) return rc;
    }
    int tb = timing_begin(P, EXX_TIMING_CHOL, s);
    if (n <= kCholSmemMax) {
        const size_t smem = (size_t(n) * n + n) * sizeof(double);
        EXX_CUDA(cudaFuncSetAttribute(cholesky_inverse_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      int(smem)));
        cholesky_inverse_smem_kernel<<<1, kCholThreads, smem, s>>>(n, M, Linv, info_d);
        timing_end(P, tb, s);
        EXX_LAUNCH("cholesky_inverse_smem_kernel");
    } else {
        double *L = static_cast<double *>(P.small_ws.p);
        cholesky_inverse_kernel<<<1, kCholThreads, 0, s>>>(n, M, L, Linv, info_d);
        timing_end(P, tb, s);
        EXX_LAUNCH("cholesky_inverse_kernel");
    }
    P.launches++;
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
