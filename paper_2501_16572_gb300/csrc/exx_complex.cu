// Complex (Bloch) path of the exchange operator: Eq. 1 with Brillouin-zone wavevectors, the
// pair problems of Eqs. 2-3 under Bloch boundary conditions at k - q along the extended
// axes (Sec. II), FP64 on the CUDA cores.
//
// A Bloch plan carries the phase theta_d across one period of every periodic axis (a grid
// function obeys u(j + n) = exp(i theta) u(j)).  The 1D FD operator of such an axis is
// Hermitian with the plane waves u_p(j) = exp(i phi_p j) / sqrt(n), phi_p = (2 pi p + theta)/n,
// as eigenvectors and w0 + 2 sum_k w_k cos(k phi_p) (over h^2) as eigenvalues, for any
// stencil radius; Dirichlet axes keep their real eigenvectors.  The solve is Eq. 8 with its
// conjugates: forward contractions with conj(U_d), f(Lambda), inverse contractions with U_d.
// Pair densities are conj(psi_m) psi_n; there is no V_mn = V_nm symmetry across k != q, so
// every ordered pair is solved.  Complex arrays are interleaved (re, im) doubles.
#include "exx_internal.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

namespace exx {

namespace {

constexpr double kPi = 3.14159265358979323846;

struct cd {
    double re, im;
};
__device__ __forceinline__ cd cmul(cd a, cd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cd cfma(cd a, cd b, cd c)   // a b + c
{
    return {fma(a.re, b.re, fma(-a.im, b.im, c.re)), fma(a.re, b.im, fma(a.im, b.re, c.im))};
}

// rho[p][r] = conj(psi_occ[m_p](r)) psi_in[n_p](r)
__global__ void c_pair_kernel(long N, int nfields, const cd *psi_occ, long ld_occ, const cd *psi_in, long ld_in,
                              const int2 *pairs, cd *rho)
{
    const long total = long(nfields) * N;
    for (long e = long(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += long(gridDim.x) * blockDim.x) {
        const long p = e / N, r = e - p * N;
        const int2 mn = pairs[p];
        const cd a = psi_occ[size_t(mn.x) * ld_occ + r], b = psi_in[size_t(mn.y) * ld_in + r];
        rho[e] = {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
    }
}

// Contraction of axis d (length nd, stride sd in the natural layout) of every field:
// out(..., o, ...) = sum_k C[k nd + o] in(..., k, ...), times S(r) when S is set (real).
__global__ void c_mode_kernel(long N, int nfields, int nd, long sd, const cd *C, const cd *in, cd *out,
                              const double *S)
{
    const long total = long(nfields) * N;
    for (long e = long(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += long(gridDim.x) * blockDim.x) {
        const long p = e / N, r = e - p * N;
        const int o = int((r / sd) % nd);
        const cd *src = in + p * N + (r - long(o) * sd);
        cd acc = {0.0, 0.0};
        for (int k = 0; k < nd; ++k) acc = cfma(C[size_t(k) * nd + o], src[size_t(k) * sd], acc);
        if (S) {
            acc.re *= S[r];
            acc.im *= S[r];
        }
        out[e] = acc;
    }
}

// out_n(r) (-)= sum_{j < cnt} f_{m_j} psi_occ[m_j](r) V_j(r) for one output column: the fields
// V_j of the batch all belong to output n, in the order of m.
__global__ void c_accum_kernel(long N, int cnt, const int2 *pairs, const cd *psi_occ, long ld_occ, const double *f,
                               const cd *V, cd *out_n, int add)
{
    for (long r = long(blockIdx.x) * blockDim.x + threadIdx.x; r < N; r += long(gridDim.x) * blockDim.x) {
        cd acc = add ? out_n[r] : cd{0.0, 0.0};
        for (int j = 0; j < cnt; ++j) {
            const int m = pairs[j].x;
            const cd t = cmul(psi_occ[size_t(m) * ld_occ + r], V[size_t(j) * N + r]);
            acc.re -= f[m] * t.re;
            acc.im -= f[m] * t.im;
        }
        out_n[r] = acc;
    }
}

// per column n: partial sums of Re conj(psi_n(r)) vx_n(r) over blocks of the grid
__global__ void c_dot_kernel(long N, const cd *psi, long ld, const cd *vx, long ld_v, double *partial)
{
    __shared__ double sh[256];
    const int n = blockIdx.y;
    double s = 0.0;
    for (long r = long(blockIdx.x) * blockDim.x + threadIdx.x; r < N; r += long(gridDim.x) * blockDim.x) {
        const cd a = psi[size_t(n) * ld + r], b = vx[size_t(n) * ld_v + r];
        s += a.re * b.re + a.im * b.im;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (int(threadIdx.x) < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[size_t(n) * gridDim.x + blockIdx.x] = sh[0];
}

// C(i, j) = alpha sum_k opA(i, k) opB(k, j) (complex; 16 x 16 tiles), with
// A(i, k) = A[i ai + k ak] conjugated when conjA, B(k, j) = B[k bk + j bj] conjugated when conjB.
struct CGemm {
    int M, Nc;
    long K;
    const cd *A;
    long ai, ak;
    int conjA;
    const cd *B;
    long bk, bj;
    int conjB;
    double alpha;
    cd *C;
    long ci, cj;
};

__global__ void __launch_bounds__(256) c_gemm_kernel(const CGemm g)
{
    __shared__ cd sa[16][17], sb[16][17];
    const int ti = threadIdx.x / 16, tj = threadIdx.x % 16;
    const int i = blockIdx.y * 16 + ti, j = blockIdx.x * 16 + tj;
    cd acc = {0.0, 0.0};
    for (long k0 = 0; k0 < g.K; k0 += 16) {
        const long ka = k0 + tj, kb = k0 + ti;
        cd a = (i < g.M && ka < g.K) ? g.A[i * g.ai + ka * g.ak] : cd{0.0, 0.0};
        cd b = (kb < g.K && j < g.Nc) ? g.B[kb * g.bk + j * g.bj] : cd{0.0, 0.0};
        if (g.conjA) a.im = -a.im;
        if (g.conjB) b.im = -b.im;
        sa[ti][tj] = a;
        sb[ti][tj] = b;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) acc = cfma(sa[ti][k], sb[k][tj], acc);
        __syncthreads();
    }
    if (i < g.M && j < g.Nc) g.C[i * g.ci + j * g.cj] = {g.alpha * acc.re, g.alpha * acc.im};
}

// One CTA, n <= kCCholMax: A = -(M + M^H)/2, A = L L^H, then Linv = L^{-1} (lower); info_d[0]
// = 0 or 1 + failing pivot.
constexpr int kCCholMax = 96;
__global__ void __launch_bounds__(1024) c_chol_kernel(int n, const cd *M, cd *Linv, int *info_d)
{
    extern __shared__ cd S[];   // n x n, S[i + n j], then n scratch values
    cd *y = S + n * n;
    __shared__ int failed;
    const int tid = threadIdx.x;
    for (int e = tid; e < n * n; e += blockDim.x) {
        const int i = e % n, j = e / n;
        const cd a = M[i + size_t(n) * j], b = M[j + size_t(n) * i];
        S[e] = (i >= j) ? cd{-0.5 * (a.re + b.re), -0.5 * (a.im - b.im)} : cd{0.0, 0.0};
    }
    if (tid == 0) {
        failed = 0;
        info_d[0] = 0;
    }
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        if (tid == 0) {
            const double d = S[j + n * j].re;
            if (!(d > 0.0)) {
                failed = 1;
                info_d[0] = j + 1;
            } else {
                S[j + n * j] = {sqrt(d), 0.0};
            }
        }
        __syncthreads();
        if (failed) return;
        const double djj = S[j + n * j].re;
        for (int i = j + 1 + tid; i < n; i += blockDim.x) {
            S[i + n * j].re /= djj;
            S[i + n * j].im /= djj;
        }
        __syncthreads();
        // trailing lower triangle: A(i, k) -= L(i, j) conj(L(k, j)), i >= k > j
        for (int k = j + 1 + (tid >> 5); k < n; k += blockDim.x >> 5) {
            const cd lk = {S[k + n * j].re, -S[k + n * j].im};
            for (int i = k + (tid & 31); i < n; i += 32) {
                const cd t = cmul(S[i + n * j], lk);
                S[i + n * k].re -= t.re;
                S[i + n * k].im -= t.im;
            }
        }
        __syncthreads();
    }
    // inverse in place, columns from the right: X_jj = 1 / L_jj (real),
    // X(j+1:, j) = -X_jj X(j+1:, j+1:) L(j+1:, j)
    for (int j = n - 1; j >= 0; --j) {
        const double xjj = 1.0 / S[j + n * j].re;
        for (int i = j + 1 + tid; i < n; i += blockDim.x) {
            cd acc = {0.0, 0.0};
            for (int k = j + 1; k <= i; ++k) acc = cfma(S[i + n * k], S[k + n * j], acc);
            y[i] = acc;
        }
        __syncthreads();
        for (int i = j + 1 + tid; i < n; i += blockDim.x) S[i + n * j] = {-xjj * y[i].re, -xjj * y[i].im};
        if (tid == 0) S[j + n * j] = {xjj, 0.0};
        __syncthreads();
    }
    for (int e = tid; e < n * n; e += blockDim.x) {
        const int i = e % n, j = e / n;
        Linv[e] = (i >= j) ? S[e] : cd{0.0, 0.0};
    }
}

int grid_for(const Plan &P, long total) { return int(std::max(1L, std::min(long(8 * P.num_sms), (total + 255) / 256))); }

int c_gemm(Plan &P, const CGemm &g, cudaStream_t s)
{
    dim3 grid(unsigned((g.Nc + 15) / 16), unsigned((g.M + 15) / 16));
    c_gemm_kernel<<<grid, 256, 0, s>>>(g);
    EXX_LAUNCH("c_gemm_kernel");
    P.launches++;
    return EXX_OK;
}

int invalid_c(const char *msg)
{
    set_error(msg);
    return EXX_ERR_INVALID_ARG;
}

}  // namespace

// Host setup of a Bloch plan: complex eigenbases, the eigenvalue sums and f on them, uploaded
// as the forward (conj(U)^T) and inverse (U) contraction matrices C[k nd + o] per axis.
int bloch_setup(Plan &P, const double theta[3])
{
    P.cplx = 1;
    std::vector<double> lam[3];
    std::vector<std::complex<double>> U[3];
    const int p = P.fd_order / 2;
    std::vector<double> w(size_t(p) + 1);
    fd_weights(p, w.data());
    for (int d = 0; d < 3; ++d) {
        const int nd = P.n[d];
        P.theta[d] = theta[d];
        U[d].assign(size_t(nd) * nd, 0.0);
        lam[d].assign(nd, 0.0);
        if (P.bc[d] == EXX_BC_PERIODIC) {
            const double inv = 1.0 / std::sqrt(double(nd));
            for (int q = 0; q < nd; ++q) {
                const double phi = (2.0 * kPi * q + theta[d]) / nd;
                double l = w[0];
                for (int k = 1; k <= p; ++k) l += 2.0 * w[k] * std::cos(k * phi);
                lam[d][q] = l / (P.h * P.h);
                for (int j = 0; j < nd; ++j) U[d][size_t(j) + size_t(nd) * q] = std::polar(inv, phi * j);
            }
        } else {
            for (size_t e = 0; e < size_t(nd) * nd; ++e) U[d][e] = P.V[d][e];
            lam[d] = P.lam[d];
        }
    }
    const bool zero_mode = P.kernel == EXX_KERNEL_COULOMB && P.bc[0] == EXX_BC_PERIODIC &&
                           P.bc[1] == EXX_BC_PERIODIC && P.bc[2] == EXX_BC_PERIODIC &&
                           std::fabs(std::remainder(theta[0], 2 * kPi)) < 1e-12 &&
                           std::fabs(std::remainder(theta[1], 2 * kPi)) < 1e-12 &&
                           std::fabs(std::remainder(theta[2], 2 * kPi)) < 1e-12;
    if (zero_mode) {
        set_error("exx_plan_create_bloch: the unscreened kernel has a zero eigenvalue at theta = 0 on an all-periodic grid");
        return EXX_ERR_UNSUPPORTED;
    }
    std::vector<double> F(size_t(P.N));
    for (int c = 0; c < P.n[2]; ++c)
        for (int b = 0; b < P.n[1]; ++b)
            for (int a = 0; a < P.n[0]; ++a)
                F[a + size_t(P.n[0]) * (b + size_t(P.n[1]) * c)] =
                    kernel_f(lam[0][a] + lam[1][b] + lam[2][c], P.kernel, P.omega);
    for (int d = 0; d < 3; ++d) P.clam[d] = lam[d];
    P.cF = F;
    size_t total = 0;
    for (int d = 0; d < 3; ++d) total += 2 * size_t(P.n[d]) * P.n[d];
    std::vector<std::complex<double>> mats(total);
    size_t off = 0;
    for (int d = 0; d < 3; ++d) {
        const int nd = P.n[d];
        for (int k = 0; k < nd; ++k)
            for (int o = 0; o < nd; ++o) {
                mats[off + size_t(k) * nd + o] = std::conj(U[d][size_t(k) + size_t(nd) * o]);   // forward
                mats[off + size_t(nd) * nd + size_t(k) * nd + o] = U[d][size_t(o) + size_t(nd) * k];   // inverse
            }
        off += 2 * size_t(nd) * nd;
    }
    if (int rc = dev_reserve(P.cmats, mats.size() * sizeof(std::complex<double>))) return rc;
    EXX_CUDA(cudaMemcpy(P.cmats.p, mats.data(), mats.size() * sizeof(std::complex<double>), cudaMemcpyHostToDevice));
    if (int rc = dev_reserve(P.cFd, F.size() * sizeof(double))) return rc;
    EXX_CUDA(cudaMemcpy(P.cFd.p, F.data(), F.size() * sizeof(double), cudaMemcpyHostToDevice));
    if (int rc = dev_reserve(P.err_d, 16)) return rc;
    EXX_CUDA(cudaMemset(P.err_d.p, 0, 16));
    return EXX_OK;
}

// The complex exchange: fields batched per output column (all occupied partners of one n,
// in chunks that fit the workspace).
int complex_apply(Plan &P, const double *psi_occ_d, int n_occ, long ld_occ, const double *f, const double *psi_in_d,
                  int n_in, long ld_in, double *out_d, long ld_out, int accumulate, cudaStream_t s)
{
    const cd *po = reinterpret_cast<const cd *>(psi_occ_d), *pi = reinterpret_cast<const cd *>(psi_in_d);
    cd *out = reinterpret_cast<cd *>(out_d);
    const long N = P.N;
    const size_t field = size_t(N) * sizeof(cd);
    const int chunk = int(std::max<size_t>(1, std::min<size_t>(size_t(n_occ), (size_t(1) << 30) / field)));
    if (int rc = dev_reserve(P.cwork, 2 * size_t(chunk) * field)) return rc;
    if (int rc = dev_reserve(P.cpairs, size_t(n_occ) * size_t(n_in) * sizeof(int2))) return rc;
    std::vector<int2> pairs(size_t(n_occ) * n_in);
    for (int n = 0; n < n_in; ++n)
        for (int m = 0; m < n_occ; ++m) pairs[size_t(n) * n_occ + m] = make_int2(m, n);
    EXX_CUDA(cudaMemcpyAsync(P.cpairs.p, pairs.data(), pairs.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    EXX_CUDA(cudaStreamSynchronize(s));   // the host vector goes out of scope
    const int2 *pairs_d = static_cast<const int2 *>(P.cpairs.p);
    cd *A = static_cast<cd *>(P.cwork.p), *B = A + size_t(chunk) * N;
    const cd *mats = static_cast<const cd *>(P.cmats.p);
    const cd *Cf[3], *Ci[3];
    size_t off = 0;
    for (int d = 0; d < 3; ++d) {
        Cf[d] = mats + off;
        Ci[d] = mats + off + size_t(P.n[d]) * P.n[d];
        off += 2 * size_t(P.n[d]) * P.n[d];
    }
    const long sd[3] = {1, long(P.n[0]), long(P.n[0]) * P.n[1]};
    const double *F = static_cast<const double *>(P.cFd.p);
    for (int n = 0; n < n_in; ++n) {
        for (int m0 = 0; m0 < n_occ; m0 += chunk) {
            const int cnt = std::min(chunk, n_occ - m0);
            const int2 *pp = pairs_d + size_t(n) * n_occ + m0;
            const long tot = long(cnt) * N;
            const int g = grid_for(P, tot);
            c_pair_kernel<<<g, 256, 0, s>>>(N, cnt, po, ld_occ, pi, ld_in, pp, A);
            EXX_LAUNCH("c_pair_kernel");
            // forward x, y, z (z scaled by f(Lambda)), inverse z, y, x: A -> B -> A -> ...
            cd *src = A, *dst = B;
            const int order[6] = {0, 1, 2, 2, 1, 0};
            for (int st = 0; st < 6; ++st) {
                const int d = order[st];
                c_mode_kernel<<<g, 256, 0, s>>>(N, cnt, P.n[d], sd[d], st < 3 ? Cf[d] : Ci[d], src, dst,
                                                st == 2 ? F : nullptr);
                EXX_LAUNCH("c_mode_kernel");
                std::swap(src, dst);
            }
            c_accum_kernel<<<grid_for(P, N), 256, 0, s>>>(N, cnt, pp, po, ld_occ, f, src, out + size_t(n) * ld_out,
                                                          (accumulate || m0 > 0) ? 1 : 0);
            EXX_LAUNCH("c_accum_kernel");
            P.launches += 8;
        }
    }
    return EXX_OK;
}

int complex_energy(Plan &P, const double *psi_d, int n, long ld, const double *f_d, const double *vx_d, long ld_v,
                   double *E_h, cudaStream_t s)
{
    const int gx = std::min(256, int((P.N + 255) / 256));
    if (int rc = dev_reserve(P.cred, size_t(n) * gx * sizeof(double))) return rc;
    c_dot_kernel<<<dim3(gx, n), 256, 0, s>>>(P.N, reinterpret_cast<const cd *>(psi_d), ld,
                                             reinterpret_cast<const cd *>(vx_d), ld_v, static_cast<double *>(P.cred.p));
    EXX_LAUNCH("c_dot_kernel");
    P.launches++;
    std::vector<double> part(size_t(n) * gx), fh(n);
    EXX_CUDA(cudaMemcpyAsync(part.data(), P.cred.p, part.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    EXX_CUDA(cudaMemcpyAsync(fh.data(), f_d, size_t(n) * sizeof(double), cudaMemcpyDeviceToHost, s));
    EXX_CUDA(cudaStreamSynchronize(s));
    // Neumaier sums in a fixed order
    double sum = 0.0, comp = 0.0;
    auto add = [&](double x) {
        const double t = sum + x;
        comp += std::fabs(sum) >= std::fabs(x) ? (sum - t) + x : (x - t) + sum;
        sum = t;
    };
    for (int j = 0; j < n; ++j) {
        double d = 0.0, dc = 0.0;
        for (int b = 0; b < gx; ++b) {
            const double x = part[size_t(j) * gx + b], t = d + x;
            dc += std::fabs(d) >= std::fabs(x) ? (d - t) + x : (x - t) + d;
            d = t;
        }
        add(0.25 * fh[j] * P.dV * (d + dc));
    }
    *E_h = sum + comp;
    return EXX_OK;
}

int complex_ace_build(Plan &P, const double *psi_d, int n, long ld, const double *W_d, long ld_w, double *xi_d,
                      long ld_xi, int *info_h, cudaStream_t s)
{
    const size_t nn = size_t(n) * n;
    if (int rc = dev_reserve(P.cace, 2 * nn * sizeof(cd) + 64)) return rc;
    cd *M = static_cast<cd *>(P.cace.p), *Linv = M + nn;
    int *info_d = reinterpret_cast<int *>(Linv + nn);
    const cd *psi = reinterpret_cast<const cd *>(psi_d), *W = reinterpret_cast<const cd *>(W_d);
    // M(i, j) = dV sum_r conj(psi_i(r)) W_j(r)
    if (int rc = c_gemm(P, {n, n, P.N, psi, ld, 1, 1, W, 1, ld_w, 0, P.dV, M, 1, long(n)}, s)) return rc;
    const size_t smem = (nn + n) * sizeof(cd);
    EXX_CUDA(cudaFuncSetAttribute(c_chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    c_chol_kernel<<<1, 1024, smem, s>>>(n, M, Linv, info_d);
    EXX_LAUNCH("c_chol_kernel");
    P.launches++;
    int info = 0;
    EXX_CUDA(cudaMemcpyAsync(&info, info_d, sizeof(int), cudaMemcpyDeviceToHost, s));
    EXX_CUDA(cudaStreamSynchronize(s));
    if (info) {
        *info_h = info;
        set_error("ace_build_complex: -herm(M) is not positive definite");
        return EXX_ERR_NOT_POSDEF;
    }
    // xi(r, j) = sum_k W(r, k) conj(Linv(j, k))
    return c_gemm(P, {P.N, n, n, W, 1, ld_w, 0, Linv, long(n), 1, 1, 1.0, reinterpret_cast<cd *>(xi_d), 1, ld_xi}, s);
}

int complex_ace_apply(Plan &P, const double *xi_d, int n, long ld_xi, const double *phi_d, int nphi, long ld_phi,
                      double *out_d, long ld_out, cudaStream_t s)
{
    if (int rc = dev_reserve(P.cace, size_t(n) * nphi * sizeof(cd) + 64)) return rc;
    cd *chi = static_cast<cd *>(P.cace.p);
    const cd *xi = reinterpret_cast<const cd *>(xi_d), *phi = reinterpret_cast<const cd *>(phi_d);
    // chi = xi^H Phi (n x nphi); out = -dV xi chi
    if (int rc = c_gemm(P, {n, nphi, P.N, xi, ld_xi, 1, 1, phi, 1, ld_phi, 0, 1.0, chi, 1, long(n)}, s)) return rc;
    return c_gemm(P, {P.N, nphi, n, xi, 1, ld_xi, 0, chi, 1, long(n), 0, -P.dV, reinterpret_cast<cd *>(out_d), 1,
                      ld_out}, s);
}

}  // namespace exx

using namespace exx;

extern "C" {

int exx_plan_create_bloch(exx_plan *out, int Nx, int Ny, int Nz, double h, const int bc[3], int fd_order,
                          int kernel, double omega, const double theta[3])
{
    if (!out || !bc || !theta) return invalid_c("exx_plan_create_bloch: NULL argument");
    if (long(Nx) * Ny * Nz > (1L << 20)) {
        set_error("exx_plan_create_bloch: the complex path supports grids of at most 2^20 points");
        return EXX_ERR_UNSUPPORTED;
    }
    for (int d = 0; d < 3; ++d)
        if (!std::isfinite(theta[d])) return invalid_c("exx_plan_create_bloch: theta must be finite");
    // the real plan's validation and setup (its periodic unscreened zero mode is checked here
    // against the Bloch phases instead)
    const bool allper = bc[0] == EXX_BC_PERIODIC && bc[1] == EXX_BC_PERIODIC && bc[2] == EXX_BC_PERIODIC;
    const bool dummy = kernel == EXX_KERNEL_COULOMB && allper;
    int rc = exx_plan_create(out, Nx, Ny, Nz, h, bc, fd_order, dummy ? EXX_KERNEL_ERFC : kernel, dummy ? 1.0 : omega);
    if (rc) return rc;
    Plan *P = reinterpret_cast<Plan *>(*out);
    P->kernel = kernel;
    P->omega = omega;
    if ((rc = bloch_setup(*P, theta)) != EXX_OK) {
        exx_plan_destroy(*out);
        *out = nullptr;
        return rc;
    }
    return EXX_OK;
}

static Plan *cplan(exx_plan plan, const char *what)
{
    Plan *P = reinterpret_cast<Plan *>(plan);
    if (!P) {
        invalid_c(what);
        return nullptr;
    }
    if (!P->cplx) {
        set_error(std::string(what) + ": the plan was not created with exx_plan_create_bloch");
        return nullptr;
    }
    return P;
}

int exx_apply_complex(exx_plan plan, const double *Psi_occ, int n_occ, long ld_occ, const double *f,
                      const double *Psi_in, int n_in, long ld_in, double *out, long ld_out, int accumulate,
                      exx_stream_t stream)
{
    Plan *P = cplan(plan, "exx_apply_complex");
    if (!P) return EXX_ERR_INVALID_ARG;
    if (!Psi_occ || !f || !Psi_in || !out) return invalid_c("exx_apply_complex: NULL array");
    if (n_occ < 1 || n_in < 1 || n_occ > 65536 || n_in > 65536) return invalid_c("exx_apply_complex: bad orbital counts");
    if (ld_occ < P->N || ld_in < P->N || ld_out < P->N) return invalid_c("exx_apply_complex: leading dimensions must be >= N");
    const char *o0 = reinterpret_cast<const char *>(out);
    const char *o1 = o0 + (size_t(n_in - 1) * ld_out + P->N) * 16;
    auto overlaps = [&](const double *a, int n, long ld) {
        const char *a0 = reinterpret_cast<const char *>(a);
        const char *a1 = a0 + (size_t(n - 1) * ld + P->N) * 16;
        return a0 < o1 && o0 < a1;
    };
    if (overlaps(Psi_occ, n_occ, ld_occ) || overlaps(Psi_in, n_in, ld_in)) return invalid_c("exx_apply_complex: out overlaps an input");
    P->launches = 0;
    return complex_apply(*P, Psi_occ, n_occ, ld_occ, f, Psi_in, n_in, ld_in, out, ld_out, accumulate,
                         reinterpret_cast<cudaStream_t>(stream));
}

int exx_energy_complex(exx_plan plan, const double *Psi, int n, long ld, const double *f, const double *VxPsi,
                       long ld_v, double *E_x_h, exx_stream_t stream)
{
    Plan *P = cplan(plan, "exx_energy_complex");
    if (!P) return EXX_ERR_INVALID_ARG;
    if (!Psi || !f || !VxPsi || !E_x_h || n < 1 || ld < P->N || ld_v < P->N) return invalid_c("exx_energy_complex: bad arguments");
    P->launches = 0;
    return complex_energy(*P, Psi, n, ld, f, VxPsi, ld_v, E_x_h, reinterpret_cast<cudaStream_t>(stream));
}

int ace_build_complex(exx_plan plan, const double *Psi, int n, long ld, const double *W, long ld_w, double *xi,
                      long ld_xi, int *info_h, exx_stream_t stream)
{
    Plan *P = cplan(plan, "ace_build_complex");
    if (!P) return EXX_ERR_INVALID_ARG;
    if (!Psi || !W || !xi || !info_h) return invalid_c("ace_build_complex: NULL argument");
    if (n < 1 || n > kCCholMax || ld < P->N || ld_w < P->N || ld_xi < P->N)
        return invalid_c("ace_build_complex: n must be in [1, 96] and leading dimensions >= N");
    *info_h = 0;
    P->launches = 0;
    return complex_ace_build(*P, Psi, n, ld, W, ld_w, xi, ld_xi, info_h, reinterpret_cast<cudaStream_t>(stream));
}

int ace_apply_complex(exx_plan plan, const double *xi, int n, long ld_xi, const double *Phi, int nphi, long ld_phi,
                      double *out, long ld_out, exx_stream_t stream)
{
    Plan *P = cplan(plan, "ace_apply_complex");
    if (!P) return EXX_ERR_INVALID_ARG;
    if (!xi || !Phi || !out || n < 1 || nphi < 1 || ld_xi < P->N || ld_phi < P->N || ld_out < P->N)
        return invalid_c("ace_apply_complex: bad arguments");
    P->launches = 0;
    return complex_ace_apply(*P, xi, n, ld_xi, Phi, nphi, ld_phi, out, ld_out, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
