// The original (non-batched) Kronecker product formalism of Sec. II.A, Eq. 8, on the GPU in
// FP64: every orbital pair is one linear system solved on its own with 4 n3 + 2 dense matrix
// products, each issued as its own small GEMM launch, the way a library GEMM per product
// would run it:
//   forward, per frontal slice k:  T = Vx^T B_k,  Y_k = T Vy            (2 n3 GEMMs)
//   along z:                       Z = Y Vz,  Z <- f(Lambda) (.) Z      (1 GEMM, scaled)
//   inverse along z:               Wt = Z Vz^T                          (1 GEMM)
//   inverse, per frontal slice k:  U = Vx Wt_k,  X_k = U Vy^T           (2 n3 GEMMs)
// followed by the pair's contribution to Eq. 1.  The batched path (exx_apply) is the
// production one; this exists to measure what batching buys (Sec. II.B, Figs. 1-2).
#include "exx_internal.h"

#include <algorithm>

namespace exx {

namespace {

constexpr int kT = 16;   // output tile edge and K chunk of the small GEMM

// C(i, j) = sum_k A(i, k) B(k, j), optionally times S(i, j); X(i, j) = X[i xi + j xj].
struct SmallGemm {
    int M, Nc, K;
    const double *A;
    long ai, ak;
    const double *B;
    long bk, bj;
    double *C;
    long ci, cj;
    const double *S;   // optional elementwise scale (same strides as C)
};

__global__ void __launch_bounds__(kT * kT) small_gemm_kernel(const SmallGemm g)
{
    __shared__ double sa[kT][kT + 1], sb[kT][kT + 1];
    const int ti = threadIdx.x / kT, tj = threadIdx.x % kT;
    const int i = blockIdx.y * kT + ti, j = blockIdx.x * kT + tj;
    double acc = 0.0;
    for (int k0 = 0; k0 < g.K; k0 += kT) {
        // A tile rows i, columns k0..; B tile rows k0.., columns j
        const int ka = k0 + tj, kb = k0 + ti;
        sa[ti][tj] = (i < g.M && ka < g.K) ? g.A[i * g.ai + ka * g.ak] : 0.0;
        sb[ti][tj] = (kb < g.K && j < g.Nc) ? g.B[kb * g.bk + j * g.bj] : 0.0;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kT; ++k) acc = fma(sa[ti][k], sb[k][tj], acc);
        __syncthreads();
    }
    if (i < g.M && j < g.Nc) {
        const long o = i * g.ci + j * g.cj;
        g.C[o] = g.S ? acc * g.S[o] : acc;
    }
}

__global__ void pair_density_kernel(long N, const double *a, const double *b, double *rho)
{
    for (long r = long(blockIdx.x) * blockDim.x + threadIdx.x; r < N; r += long(gridDim.x) * blockDim.x)
        rho[r] = a[r] * b[r];
}

// out_n -= f_m psi_m V; with `both`, also out_m -= f_n psi_n V (V_mn = V_nm)
__global__ void pair_accumulate_kernel(long N, const double *V, const double *psi_m, const double *f_m,
                                       double *out_n, const double *psi_n, const double *f_n, double *out_m,
                                       int both)
{
    const double fm = *f_m, fn = both ? *f_n : 0.0;
    for (long r = long(blockIdx.x) * blockDim.x + threadIdx.x; r < N; r += long(gridDim.x) * blockDim.x) {
        const double v = V[r];
        out_n[r] -= fm * psi_m[r] * v;
        if (both) out_m[r] -= fn * psi_n[r] * v;
    }
}

int gemm(Plan &P, const SmallGemm &g, cudaStream_t s)
{
    dim3 grid(unsigned((g.Nc + kT - 1) / kT), unsigned((g.M + kT - 1) / kT));
    small_gemm_kernel<<<grid, kT * kT, 0, s>>>(g);
    EXX_LAUNCH("small_gemm_kernel");
    P.launches++;
    return EXX_OK;
}

}  // namespace

// One pair's solve: rho (N) -> V (N) in place of rho, using tmp (2 N) as workspace.  The
// matrices are the plan's host eigenvectors uploaded once (orig_V) with V_d(k, c) at
// k + n_d c (column c = eigenvector c), and f(Lambda) in the natural layout (F64n).
static int solve_one(Plan &P, double *rho, double *tmp, cudaStream_t s)
{
    const int n1 = P.n[0], n2 = P.n[1], n3 = P.n[2];
    const long R = long(n1) * n2;
    const double *V1 = static_cast<const double *>(P.orig_V.p);
    const double *V2 = V1 + size_t(n1) * n1;
    const double *V3 = V2 + size_t(n2) * n2;
    const double *F = static_cast<const double *>(P.F64n.p);
    double *T = tmp, *Y = tmp + size_t(P.N);   // T: one slice (n1 x n2 values); Y: N values
    // forward, slice by slice: T(a, y) = sum_x V1(x, a) B_k(x, y); Y_k(a, b) = sum_y T(a, y) V2(y, b)
    for (int k = 0; k < n3; ++k) {
        const double *Bk = rho + size_t(k) * R;
        if (int rc = gemm(P, {n1, n2, n1, V1, long(n1), 1, Bk, 1, long(n1), T, 1, long(n1), nullptr}, s)) return rc;
        if (int rc = gemm(P, {n1, n2, n2, T, 1, long(n1), V2, 1, long(n2), Y + size_t(k) * R, 1, long(n1), nullptr}, s))
            return rc;
    }
    // along z: Z(r, c) = f(r, c) sum_k Y(r, k) V3(k, c)   (r = a + n1 b), into rho
    if (int rc = gemm(P, {int(R), n3, n3, Y, 1, R, V3, 1, long(n3), rho, 1, R, F}, s)) return rc;
    // inverse along z: Wt(r, k) = sum_c Z(r, c) V3(k, c), into Y
    if (int rc = gemm(P, {int(R), n3, n3, rho, 1, R, V3, long(n3), 1, Y, 1, R, nullptr}, s)) return rc;
    // inverse, slice by slice: U(x, b) = sum_a V1(x, a) Wt_k(a, b); X_k(x, y) = sum_b U(x, b) V2(y, b)
    for (int k = 0; k < n3; ++k) {
        const double *Wk = Y + size_t(k) * R;
        if (int rc = gemm(P, {n1, n2, n1, V1, 1, long(n1), Wk, 1, long(n1), T, 1, long(n1), nullptr}, s)) return rc;
        if (int rc = gemm(P, {n1, n2, n2, T, 1, long(n1), V2, long(n2), 1, rho + size_t(k) * R, 1, long(n1), nullptr}, s))
            return rc;
    }
    return EXX_OK;
}

int original_upload(Plan &P)
{
    const size_t nv = size_t(P.n[0]) * P.n[0] + size_t(P.n[1]) * P.n[1] + size_t(P.n[2]) * P.n[2];
    if (int rc = dev_reserve(P.orig_V, nv * sizeof(double))) return rc;
    size_t off = 0;
    for (int d = 0; d < 3; ++d) {
        EXX_CUDA(cudaMemcpy(static_cast<double *>(P.orig_V.p) + off, P.V[d].data(), P.V[d].size() * sizeof(double),
                            cudaMemcpyHostToDevice));
        off += P.V[d].size();
    }
    if (int rc = dev_reserve(P.F64n, size_t(P.N) * sizeof(double))) return rc;
    EXX_CUDA(cudaMemcpy(P.F64n.p, P.F.data(), size_t(P.N) * sizeof(double), cudaMemcpyHostToDevice));
    return EXX_OK;
}

int original_apply(Plan &P, const double *psi_occ, int n_occ, long ld_occ, const double *f, const double *psi_in,
                   int n_in, long ld_in, double *out, long ld_out, bool aliased, cudaStream_t s)
{
    if (!P.orig_V.p)
        if (int rc = original_upload(P)) return rc;
    if (int rc = dev_reserve(P.orig_ws, 3 * size_t(P.N) * sizeof(double))) return rc;
    double *rho = static_cast<double *>(P.orig_ws.p);
    double *tmp = rho + P.N;
    EXX_CUDA(cudaMemset2DAsync(out, size_t(ld_out) * sizeof(double), 0, size_t(P.N) * sizeof(double), n_in, s));
    const int blocks = std::max(1, std::min(4 * P.num_sms, int((P.N + 255) / 256)));
    // pairs in a fixed order: with aliased inputs each pair m <= n among the occupied
    // orbitals once (used for both outputs), then the occupied x unoccupied pairs
    for (int n = 0; n < n_in; ++n) {
        for (int m = 0; m < n_occ; ++m) {
            const bool sym = aliased && n < n_occ;
            if (sym && m > n) continue;
            const double *pm = psi_occ + size_t(m) * ld_occ, *pn = psi_in + size_t(n) * ld_in;
            pair_density_kernel<<<blocks, 256, 0, s>>>(P.N, pm, pn, rho);
            EXX_LAUNCH("pair_density_kernel");
            P.launches++;
            if (int rc = solve_one(P, rho, tmp, s)) return rc;
            const int both = sym && m != n;
            pair_accumulate_kernel<<<blocks, 256, 0, s>>>(P.N, rho, pm, f + m, out + size_t(n) * ld_out, pn,
                                                          f + (both ? n : m), out + size_t(both ? m : n) * ld_out, both);
            EXX_LAUNCH("pair_accumulate_kernel");
            P.launches++;
        }
    }
    return EXX_OK;
}

}  // namespace exx
