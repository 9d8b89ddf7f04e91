// FP64 path of the batched Kronecker Poisson solve (Sec. II.B) and of the
// exchange accumulation (Eq. 1), on the CUDA cores.
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so these kernels are bound by
// the double-precision FMA pipe, not by memory: a mode product of length n does 2n
// flops per 8-byte element.  Each thread owns one row (a pencil along the contracted
// axis) and produces 16 outputs at a time from the K x 16 slice of the contraction
// matrix staged in shared memory (every thread of a warp reads the same entry, a
// broadcast).
#include "exx_internal.h"

namespace exx {

namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 16;

struct Fp64PassArgs {
    int nfields, R, K;
    const double *in;            // field stride N
    double *out;                 // field stride N
    long N;
    const double *B;             // K x K, B[k*K + j]
    const double *F;             // [j][r] scaling (R*K values) or null
    const double *psi_a, *psi_b; // pair prologue: psi_a[m*lda + ...], psi_b[n*ldb + ...]
    long lda, ldb;
    const int2 *pairs;
};

template <int LOAD, int STORE, bool SCALE>
__global__ void __launch_bounds__(kThreads) fp64_pass_kernel(Fp64PassArgs a)
{
    extern __shared__ double Bs[];   // [K][kChunk]
    const long rows = long(a.nfields) * a.R;
    const long g = long(blockIdx.x) * blockDim.x + threadIdx.x;
    const bool active = g < rows;
    const int p = active ? int(g / a.R) : 0;
    const int r = active ? int(g - long(p) * a.R) : 0;
    const double *in = a.in + size_t(p) * a.N;
    const double *pa = nullptr, *pb = nullptr;
    if (LOAD == LOAD_PAIR && active) {
        int2 mn = a.pairs[p];
        pa = a.psi_a + size_t(mn.x) * a.lda;
        pb = a.psi_b + size_t(mn.y) * a.ldb;
    }
    double *out = a.out + size_t(p) * a.N;
    for (int j0 = 0; j0 < a.K; j0 += kChunk) {
        __syncthreads();
        for (int i = threadIdx.x; i < a.K * kChunk; i += blockDim.x) {
            int k = i / kChunk, j = i - k * kChunk;
            Bs[i] = (j0 + j < a.K) ? a.B[size_t(k) * a.K + j0 + j] : 0.0;
        }
        __syncthreads();
        if (!active) continue;
        double acc[kChunk];
#pragma unroll
        for (int j = 0; j < kChunk; ++j) acc[j] = 0.0;
        for (int k = 0; k < a.K; ++k) {
            double x;
            if (LOAD == LOAD_PAIR) x = pa[size_t(k) * a.R + r] * pb[size_t(k) * a.R + r];
            else if (LOAD == LOAD_KSLOW) x = in[size_t(k) * a.R + r];
            else x = in[size_t(r) * a.K + k];
            const double2 *bk = reinterpret_cast<const double2 *>(Bs + k * kChunk);
#pragma unroll
            for (int j = 0; j < kChunk / 2; ++j) {
                double2 b = bk[j];
                acc[2 * j] = fma(x, b.x, acc[2 * j]);
                acc[2 * j + 1] = fma(x, b.y, acc[2 * j + 1]);
            }
        }
        const int jn = min(kChunk, a.K - j0);
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
            if (j >= jn) break;
            double v = acc[j];
            if (SCALE) v *= a.F[size_t(j0 + j) * a.R + r];
            if (STORE == STORE_NSLOW) out[size_t(j0 + j) * a.R + r] = v;
            else out[size_t(r) * a.K + j0 + j] = v;
        }
    }
}

template <int LOAD, int STORE, bool SCALE>
int launch_pass(Plan &P, int kind, const Fp64PassArgs &a, cudaStream_t s)
{
    const long rows = long(a.nfields) * a.R;
    const int grid = int((rows + kThreads - 1) / kThreads);
    const size_t smem = size_t(a.K) * kChunk * sizeof(double);
    auto kern = fp64_pass_kernel<LOAD, STORE, SCALE>;
    if (smem > 48 * 1024) EXX_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    int tb = timing_begin(P, kind, s);
    kern<<<grid, kThreads, smem, s>>>(a);
    timing_end(P, tb, s);
    EXX_LAUNCH("fp64_pass_kernel");
    return EXX_OK;
}

// out_t(r) += - sum over the block's contributions f_s psi_s(r) V_field(r), FP64.
struct Fp64AccArgs {
    long N;
    const double *psi_a, *psi_b;  // occupied (sources) / input orbitals
    long lda, ldb;
    const double *f;
    const Block *blocks;
    const double *V;              // fields of the batch
    double *out;
    long ldo;
};

__device__ __forceinline__ int diag_index(int i, int j, int nI)
{
    // index of (i <= j) in the row-major upper-triangle enumeration of an nI x nI block
    return i * nI - (i * (i - 1)) / 2 + (j - i);
}

__global__ void __launch_bounds__(kThreads) fp64_accum_kernel(Fp64AccArgs a)
{
    const Block b = a.blocks[blockIdx.y];
    const long r = long(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= a.N) return;
    const double *V = a.V + size_t(b.field0) * a.N + r;
    if (b.kind == BLK_SYM_DIAG) {
        for (int t = 0; t < b.nI; ++t) {
            double acc = 0.0;
            for (int s = 0; s < b.nI; ++s) {
                int m = b.I0 + s;
                int fi = s <= t ? diag_index(s, t, b.nI) : diag_index(t, s, b.nI);
                acc = fma(-a.f[m] * a.psi_a[size_t(m) * a.lda + r], V[size_t(fi) * a.N], acc);
            }
            double *o = a.out + size_t(b.I0 + t) * a.ldo + r;
            *o += acc;
        }
        return;
    }
    // outputs of J (both kinds): sources m in I
    for (int j = 0; j < b.nJ; ++j) {
        double acc = 0.0;
        for (int i = 0; i < b.nI; ++i) {
            int m = b.I0 + i;
            acc = fma(-a.f[m] * a.psi_a[size_t(m) * a.lda + r], V[size_t(i * b.nJ + j) * a.N], acc);
        }
        double *o = a.out + size_t(b.J0 + j) * a.ldo + r;
        *o += acc;
    }
    if (b.kind == BLK_SYM_OFF) {
        // outputs of I: sources n in J (J occupied as well, same array)
        for (int i = 0; i < b.nI; ++i) {
            double acc = 0.0;
            for (int j = 0; j < b.nJ; ++j) {
                int n = b.J0 + j;
                acc = fma(-a.f[n] * a.psi_a[size_t(n) * a.lda + r], V[size_t(i * b.nJ + j) * a.N], acc);
            }
            double *o = a.out + size_t(b.I0 + i) * a.ldo + r;
            *o += acc;
        }
    }
}

}  // namespace

int fp64_solve_batch(Plan &P, const double *psi_occ, long ld_occ, const double *psi_in, long ld_in,
                     const int2 *pairs_d, int nfields, double *bufA, double *bufB, double **result,
                     cudaStream_t s)
{
    double *src = nullptr, *dst = bufA;
    for (int pass = 0; pass < 5; ++pass) {
        PassGeom g = pass_geom(P.n, pass);
        Fp64PassArgs a{};
        a.nfields = nfields;
        a.R = g.R;
        a.K = g.K;
        a.N = P.N;
        a.psi_a = psi_occ;
        a.psi_b = psi_in;
        a.lda = ld_occ;
        a.ldb = ld_in;
        a.pairs = pairs_d;
        int rc = EXX_OK;
        if (pass == 2) {
            // forward y with the Hadamard scaling by f(Lambda), then inverse y
            a.in = src;
            a.out = dst;
            a.B = static_cast<const double *>(P.B64[2].p);
            a.F = static_cast<const double *>(P.F64.p);
            rc = launch_pass<LOAD_KFAST, STORE_NFAST, true>(P, EXX_TIMING_PASS3, a, s);
            if (rc) return rc;
            P.launches++;
            std::swap(src, dst);
            a.in = src;
            a.out = dst;
            a.B = static_cast<const double *>(P.B64[3].p);
            a.F = nullptr;
            rc = launch_pass<LOAD_KFAST, STORE_NFAST, false>(P, EXX_TIMING_PASS3, a, s);
        } else {
            a.in = src;
            a.out = dst;
            a.B = static_cast<const double *>(P.B64[pass < 2 ? pass : pass + 1].p);
            if (pass == 0) rc = launch_pass<LOAD_PAIR, STORE_NSLOW, false>(P, EXX_TIMING_PASS1, a, s);
            else if (pass == 1) rc = launch_pass<LOAD_KFAST, STORE_NSLOW, false>(P, EXX_TIMING_PASS2, a, s);
            else if (pass == 3) rc = launch_pass<LOAD_KSLOW, STORE_NFAST, false>(P, EXX_TIMING_PASS4, a, s);
            else rc = launch_pass<LOAD_KSLOW, STORE_NSLOW, false>(P, EXX_TIMING_PASS5, a, s);
        }
        if (rc) return rc;
        P.launches++;
        src = dst;
        dst = (dst == bufA) ? bufB : bufA;
    }
    *result = src;   // the solutions, natural layout
    return EXX_OK;
}

int fp64_accumulate(Plan &P, const double *psi_occ, long ld_occ, const double *psi_in, long ld_in,
                    const double *f, const Block *blocks_d, int nblocks, const double *V, double *out,
                    long ld_out, cudaStream_t s)
{
    Fp64AccArgs a{};
    a.N = P.N;
    a.psi_a = psi_occ;
    a.psi_b = psi_in;
    a.lda = ld_occ;
    a.ldb = ld_in;
    a.f = f;
    a.blocks = blocks_d;
    a.V = V;
    a.out = out;
    a.ldo = ld_out;
    dim3 grid(unsigned((P.N + kThreads - 1) / kThreads), unsigned(nblocks));
    int tb = timing_begin(P, EXX_TIMING_ACCUM, s);
    fp64_accum_kernel<<<grid, kThreads, 0, s>>>(a);
    timing_end(P, tb, s);
    EXX_LAUNCH("fp64_accum_kernel");
    P.launches++;
    return EXX_OK;
}

int fp64_upload(Plan &P)
{
    // contraction matrices: forward B[k][j] = V(k, j); inverse B[k][j] = V(j, k)
    const int axis_of[6] = {2, 0, 1, 1, 0, 2};
    const int inv_of[6] = {0, 0, 0, 1, 1, 1};
    for (int slot = 0; slot < 6; ++slot) {
        int d = axis_of[slot], nd = P.n[d];
        std::vector<double> B(size_t(nd) * nd);
        for (int k = 0; k < nd; ++k)
            for (int j = 0; j < nd; ++j)
                B[size_t(k) * nd + j] = inv_of[slot] ? P.V[d][j + size_t(nd) * k] : P.V[d][k + size_t(nd) * j];
        if (int rc = dev_reserve(P.B64[slot], B.size() * sizeof(double))) return rc;
        EXX_CUDA(cudaMemcpy(P.B64[slot].p, B.data(), B.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    // F in the P3 layout: [b][a][c] -> F(a, b, c)
    const int n1 = P.n[0], n2 = P.n[1], n3 = P.n[2];
    std::vector<double> F3(size_t(P.N));
    std::vector<float> F3f(2 * size_t(P.N));   // hi plane, then lo plane
    for (int b = 0; b < n2; ++b)
        for (int a = 0; a < n1; ++a)
            for (int c = 0; c < n3; ++c) {
                double v = P.F[a + size_t(n1) * (b + size_t(n2) * c)];
                size_t idx = size_t(b) * n1 * n3 + size_t(a) * n3 + c;
                F3[idx] = v;
                F3f[idx] = float(v);
                F3f[idx + size_t(P.N)] = float(v - double(float(v)));
            }
    if (int rc = dev_reserve(P.F64, F3.size() * sizeof(double))) return rc;
    EXX_CUDA(cudaMemcpy(P.F64.p, F3.data(), F3.size() * sizeof(double), cudaMemcpyHostToDevice));
    if (int rc = dev_reserve(P.F32, F3f.size() * sizeof(float))) return rc;
    EXX_CUDA(cudaMemcpy(P.F32.p, F3f.data(), F3f.size() * sizeof(float), cudaMemcpyHostToDevice));
    return EXX_OK;
}

}  // namespace exx
