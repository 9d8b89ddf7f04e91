// Fixed-point split GEMM on the tcgen05 tensor cores for the ACE products of Sec. III
// (M = dV Psi^T W and xi = W L^{-T} in the construction, chi = xi^T Phi and -dV xi chi in
// the application), used by plans in a split-precision mode:
//
//     D(i, j) = alpha * sum_k A(i, k) B(j, k)
//
// with FP64 operands addressed through element strides, A(i, k) = A[i as_i + k as_k].
//
// Every 320-long chunk of k is exact up to the operand digits: within the chunk each row
// of A and each row of B gets a power-of-two scale from its largest entry, the scaled
// row is rounded to a 31-bit integer X and cut into four balanced base-256 digits,
//     X = d0 2^24 + d1 2^16 + d2 2^8 + d3,   |d0| <= 64, |d1|, |d2|, |d3| <= 128,
// each stored exactly as a bf16.  Digit products of one level (i + j = l, l <= 4) are
// summed in their own TMEM accumulator (5 levels x 96 output columns per tile); a level
// gains at most 3 * 2^14 per k, so the 320-term sums stay integers below 2^24 and the
// tensor core never rounds.  The levels are combined in FP64 and the chunks are summed in
// FP64.  Dropped digit products (i + j >= 5) weigh below 2^-37 of the row maxima; the
// rounding of X, 2^-31 of the row maxima, is the leading error.
#include "exx_internal.h"
#include "tc_ptx.cuh"

#include <algorithm>

namespace exx {

namespace {

constexpr int kT = 128;              // rows of A per tile (TMEM lanes)
constexpr int kThreads = 4 * kT;     // 4 threads per row (slicing, drain by column groups)
constexpr int kTN = 96;              // rows of B per tile (output columns)
constexpr int kLev = 5;              // level accumulators: digit products with i + j <= 4
constexpr int kSub = 64;             // k per operand image
constexpr int kSubs = 5;             // images per exact chunk
constexpr int kChunk = kSub * kSubs; // 320: 4 levels x 320 x 3 * 2^14 < 2^24
constexpr uint32_t kGemmWait = 1u << 22;

struct GemmArgs {
    int m, n;
    long K;
    const double *A;
    long as_i, as_k;
    const double *B;
    long bs_j, bs_k;
    double *D;                 // this CTA's output slot: D + blockIdx.z * dz
    long ds_i, ds_j, dz;
    long kper;                 // k handled by one CTA (a multiple of kChunk)
    double alpha;
    int *err;
};

__device__ __forceinline__ int exp_field(double x) { return int((__double_as_longlong(x) >> 52) & 0x7ff); }

// Digits of x 2^sh, sh = 1052 - E for the row's largest biased exponent E: |x| < 2^(E-1022)
// gives |X| < 2^30.  The scaling adds sh to the exponent field (x = 0 and values that
// would leave the normal range give X = 0: they are below 2^-1000 of the row maximum).
__device__ __forceinline__ void digits4(double x, int sh, float (&d)[4])
{
    const int ex = exp_field(x);
    int X = 0;
    if (ex != 0 && ex + sh > 0)
        X = __double2int_rn(__longlong_as_double(__double_as_longlong(x) + (static_cast<long long>(sh) << 52)));
    const int d0 = (X + (1 << 23)) >> 24;
    int r = X - (d0 << 24);
    const int d1 = (r + (1 << 15)) >> 16;
    r -= d1 << 16;
    const int d2 = (r + (1 << 7)) >> 8;
    const int d3 = r - (d2 << 8);
    // small integers to FP32 through the 1.5 * 2^23 offset (exact for |d| < 2^22)
    d[0] = __int_as_float(0x4B400000 + d0) - 12582912.f;
    d[1] = __int_as_float(0x4B400000 + d1) - 12582912.f;
    d[2] = __int_as_float(0x4B400000 + d2) - 12582912.f;
    d[3] = __int_as_float(0x4B400000 + d3) - 12582912.f;
}

// canonical K-major no-swizzle image: byte offset of (row, 16-byte chunk c), 64 k per row
__device__ __forceinline__ uint32_t gimg_off(int row, int c) { return uint32_t(row >> 3) * 1024u + uint32_t(c) * 128u + uint32_t(row & 7) * 16u; }

// 4 digits x 4 consecutive k of one row -> the four digit images (8 bytes each)
__device__ __forceinline__ void store_digits(uint8_t *img, int row, int u, const float (&q)[4][4], uint32_t piece)
{
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        const uint32_t w0 = __byte_perm(__float_as_uint(q[l][0]), __float_as_uint(q[l][1]), 0x7632);
        const uint32_t w1 = __byte_perm(__float_as_uint(q[l][2]), __float_as_uint(q[l][3]), 0x7632);
        *reinterpret_cast<uint2 *>(img + l * piece + gimg_off(row, u >> 1) + (u & 1) * 8) = make_uint2(w0, w1);
    }
}

__global__ void __launch_bounds__(kThreads, 1) tc_gemm_kernel(GemmArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    constexpr uint32_t piece = kT * kSub * 2;       // one A digit image: 128 rows x 64 k bf16
    constexpr uint32_t bpiece = kTN * kSub * 2;     // one B digit image: 96 rows
    constexpr uint32_t sbo = kSub * 2 * 8;          // bytes per 8-row group
    uint8_t *sA = smem, *sB = smem + 4 * piece;
    int *sh_a = reinterpret_cast<int *>(sB + 4 * bpiece);   // per A row: its scale shift
    int *sh_b = sh_a + kT;                                   // per B row
    uint64_t *bar = reinterpret_cast<uint64_t *>(sh_b + kTN);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    int *sflag = reinterpret_cast<int *>(tslot + 1);
    const int t = threadIdx.x, warp = t >> 5, row = t & (kT - 1), q = t / kT;
    constexpr int kWarps = kThreads / 32;
    if (t == 0) {
        tc::mbar_init(bar, 1);
        *sflag = 0;
    }
    if (warp == 0) tc::tmem_alloc(tslot, 512);   // 5 levels x 96 columns
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t lane = uint32_t((warp & 3) * 32) << 16;   // this warp's TMEM lane quarter
    const uint32_t idesc = tc::instr_desc(false, kTN);
    const uint32_t a_addr = tc::smem_addr(sA), b_addr = tc::smem_addr(sB);

    const int i0 = blockIdx.x * kT, j0 = blockIdx.y * kTN;
    const int i = i0 + row;              // this thread's output row (TMEM lane)
    const bool arow = i < a.m;
    const long kbeg = long(blockIdx.z) * a.kper, kend = min(a.K, kbeg + a.kper);
    double *D = a.D + long(blockIdx.z) * a.dz;
    uint32_t phase = 0;
    bool first = true;
    // Per-row shifts of a chunk [c0, c1) and digit images of a sub-step [k0, k0 + 64) for an
    // operand X of R tile rows (global rows base + r < valid, element (row, k) at
    // X[row sr + k sk]).  k-contiguous operands (sk = 1) are read a warp per row,
    // consecutive lanes on consecutive k; the others by threads per row, consecutive lanes
    // on consecutive rows: both coalesced.
    auto shifts = [&](const double *X, long sr, long sk, int base, int valid, int R, int *sh, long c0, long c1) {
        if (sk == 1) {
            for (int r = warp; r < R; r += kWarps) {
                int E = 0;
                if (base + r < valid) {
                    const double *xr = X + long(base + r) * sr;
                    for (long k = c0 + (t & 31); k < c1; k += 32) E = max(E, exp_field(xr[k]));
                }
                for (int o = 16; o > 0; o >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));
                if ((t & 31) == 0) sh[r] = 1052 - max(E, 100);   // rows below 2^-922 are zero rows
            }
        } else if (t < R) {
            int E = 0;
            if (base + t < valid) {
                const double *xr = X + long(base + t) * sr;
                for (long k = c0; k < c1; ++k) E = max(E, exp_field(xr[k * sk]));
            }
            sh[t] = 1052 - max(E, 100);
        }
    };
    auto digits_sub = [&](const double *X, long sr, long sk, int base, int valid, int R, const int *sh,
                          uint8_t *img, uint32_t pc, long k0, long c1) {
        if (sk == 1) {
            const int l2 = 2 * (t & 31);   // this lane's k: k0 + l2, k0 + l2 + 1
            for (int r = warp; r < R; r += kWarps) {
                const bool ok = base + r < valid;
                const double *xr = ok ? X + long(base + r) * sr : X;
                const long k = k0 + l2;
                float d0[4], d1[4];
                digits4(ok && k < c1 ? xr[k] : 0.0, sh[r], d0);
                digits4(ok && k + 1 < c1 ? xr[k + 1] : 0.0, sh[r], d1);
#pragma unroll
                for (int lv = 0; lv < 4; ++lv)
                    *reinterpret_cast<uint32_t *>(img + lv * pc + gimg_off(r, l2 >> 3) + (l2 & 7) * 2) =
                        __byte_perm(__float_as_uint(d0[lv]), __float_as_uint(d1[lv]), 0x7632);
            }
        } else if (row < R) {   // 4 threads per row, 4-k units u = q, q + 4, ...
            const bool ok = base + row < valid;
            const double *xr = ok ? X + long(base + row) * sr : X;
            for (int u = q; u < kSub / 4; u += kThreads / kT) {
                float dq[4][4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const long k = k0 + 4 * u + e;
                    float d[4];
                    digits4(ok && k < c1 ? xr[k * sk] : 0.0, sh[row], d);
#pragma unroll
                    for (int lv = 0; lv < 4; ++lv) dq[lv][e] = d[lv];
                }
                store_digits(img, row, u, dq, pc);
            }
        }
    };
    for (long c0 = kbeg; c0 < kend; c0 += kChunk) {
        const long c1 = min(kend, c0 + kChunk);
        shifts(a.A, a.as_i, a.as_k, i0, a.m, kT, sh_a, c0, c1);
        shifts(a.B, a.bs_j, a.bs_k, j0, a.n, kTN, sh_b, c0, c1);
        __syncthreads();   // every row's shift is visible
        for (int sub = 0; sub < kSubs; ++sub) {
            const long k0 = c0 + long(sub) * kSub;
            if (k0 >= c1) break;   // uniform
            digits_sub(a.A, a.as_i, a.as_k, i0, a.m, kT, sh_a, sA, piece, k0, c1);
            digits_sub(a.B, a.bs_j, a.bs_k, j0, a.n, kTN, sh_b, sB, bpiece, k0, c1);
            tc::fence_proxy_async_smem();
            tc::tc_fence_before();
            __syncthreads();
            tc::tc_fence_after();
            if (t == 0) {
                // level l of the chunk accumulates the digit products (p, l - p)
                for (int ks = 0; ks < kSub / 16; ++ks)
                    for (int l = 0; l < kLev; ++l)
                        for (int p = max(0, l - 3); p <= min(l, 3); ++p) {
                            const uint64_t ad = tc::smem_desc(a_addr + p * piece + ks * 256u, 128u, sbo);
                            const uint64_t bd = tc::smem_desc(b_addr + (l - p) * bpiece + ks * 256u, 128u, sbo);
                            const bool acc = sub > 0 || ks > 0 || p > max(0, l - 3);
                            tc::mma_bf16(tmem + uint32_t(l * kTN), ad, bd, idesc, acc ? 1u : 0u);
                        }
                tc::mma_commit(bar);
            }
            // images are rewritten by the next sub-step, TMEM read by the drain: wait
            if (!tc::mbar_wait_bounded(bar, phase, kGemmWait)) atomicExch(sflag, 1);
            phase ^= 1u;
            tc::tc_fence_after();
            __syncthreads();   // the images may be rewritten
        }
        if (*sflag) break;   // uniform: set before the last barrier
        // drain: D(i, j) (+)= alpha 2^(48 - shA - shB) sum_l L_l 2^(-8 l).  The levels are
        // combined in FP32 down to level 1 (rounding ~2^-32 of level 0's scale), level 0 is
        // added with TwoSum, and the pair is scaled and accumulated in FP64.
        const int shA = sh_a[row];
        for (int cg = q; cg < kTN / 8; cg += kThreads / kT) {   // this thread's column groups
            uint32_t r[kLev][8];
#pragma unroll
            for (int l = 0; l < kLev; ++l) tc::tmem_ld8_issue(tmem + lane + uint32_t(l * kTN + cg * 8), r[l]);
            tc::tmem_wait_ld();
#pragma unroll
            for (int l = 0; l < kLev; ++l)
#pragma unroll
                for (int e = 0; e < 8; ++e) tc::order_after_wait(r[l][e]);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int col = j0 + cg * 8 + e;
                if (!arow || col >= a.n) continue;
                float tl = __uint_as_float(r[4][e]);
                tl = tl * (1.f / 256.f) + __uint_as_float(r[3][e]);
                tl = tl * (1.f / 256.f) + __uint_as_float(r[2][e]);
                tl = tl * (1.f / 256.f) + __uint_as_float(r[1][e]);
                tl *= 1.f / 256.f;
                const float l0 = __uint_as_float(r[0][e]);
                const float h = l0 + tl, bp = h - l0;
                const float lo = (l0 - (h - bp)) + (tl - bp);
                // v 2^48 2^-shA 2^-shB alpha, the powers of two as one exponent (a product
                // below the normal range is zero: both rows were below 2^-900)
                const int sc = min(48 - shA - sh_b[cg * 8 + e], 1023);
                double v = double(h) + double(lo);
                v = sc < -1022 ? 0.0 : a.alpha * (v * __longlong_as_double(static_cast<long long>(sc + 1023) << 52));
                double *dp = D + long(i) * a.ds_i + long(col) * a.ds_j;
                *dp = first ? v : *dp + v;
            }
        }
        tc::tc_fence_before();   // TMEM reads before the next chunk's MMAs overwrite it
        __syncthreads();
        first = false;
    }
    if (first && *sflag == 0 && arow && q == 0) {   // empty k range: the slot holds a zero sum
        for (int c = 0; c < kTN; ++c) {
            const int col = j0 + c;
            if (col < a.n) D[long(i) * a.ds_i + long(col) * a.ds_j] = 0.0;
        }
    }
    if (t == 0 && *sflag) atomicExch(a.err, 1);
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
}

// D(i, j) = sum_z W[z][i + m j] with the output strides.
__global__ void tc_gemm_reduce_kernel(const double *W, int Z, int m, int n, double *D, long ds_i, long ds_j)
{
    const long tot = long(m) * n;
    for (long e = long(blockIdx.x) * blockDim.x + threadIdx.x; e < tot; e += long(gridDim.x) * blockDim.x) {
        double s = 0.0;
        for (int z = 0; z < Z; ++z) s += W[long(z) * tot + e];
        const long i = e % m, jj = e / m;
        D[i * ds_i + jj * ds_j] = s;
    }
}

}  // namespace

int tc_gemm(Plan &P, int m, int n, long K, const double *A, long as_i, long as_k, const double *B, long bs_j,
            long bs_k, double alpha, double *D, long ds_i, long ds_j, cudaStream_t s)
{
    if (m < 1 || n < 1 || K < 1) return EXX_ERR_INVALID_ARG;
    if (!P.err_d.p) {
        if (int rc = dev_reserve(P.err_d, 16)) return rc;
        EXX_CUDA(cudaMemsetAsync(P.err_d.p, 0, 16, s));
    }
    const long mt = (m + kT - 1) / kT, nt = (n + kTN - 1) / kTN;
    const long nchunks = (K + kChunk - 1) / kChunk;
    // split k over Z CTAs per output tile when the tiles alone do not fill the GPU twice,
    // each summing its chunks into its own FP64 slot (at most 1 GiB of slots)
    long Z = 1;
    if (nchunks > 1 && mt * nt < 2L * P.num_sms) {
        Z = std::min(nchunks, (2L * P.num_sms + mt * nt - 1) / (mt * nt));
        Z = std::min(Z, std::max(1L, (1L << 30) / (long(m) * n * 8)));
    }
    const long kper = ((nchunks + Z - 1) / Z) * kChunk;
    Z = (K + kper - 1) / kper;
    GemmArgs a{};
    a.m = m;
    a.n = n;
    a.K = K;
    a.A = A;
    a.as_i = as_i;
    a.as_k = as_k;
    a.B = B;
    a.bs_j = bs_j;
    a.bs_k = bs_k;
    a.kper = kper;
    a.alpha = alpha;
    a.err = static_cast<int *>(P.err_d.p);
    if (Z > 1) {
        if (int rc = dev_reserve(P.gemm_ws, size_t(Z) * m * n * sizeof(double))) return rc;
        a.D = static_cast<double *>(P.gemm_ws.p);
        a.ds_i = 1;
        a.ds_j = m;
        a.dz = long(m) * n;
    } else {
        a.D = D;
        a.ds_i = ds_i;
        a.ds_j = ds_j;
        a.dz = 0;
    }
    const size_t smem = 4 * size_t(kT + kTN) * kSub * 2 + (kT + kTN) * sizeof(int) + 64;
    EXX_CUDA(cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    int tb = timing_begin(P, EXX_TIMING_GEMM, s);
    tc_gemm_kernel<<<dim3(unsigned(mt), unsigned(nt), unsigned(Z)), kThreads, smem, s>>>(a);
    timing_end(P, tb, s);
    EXX_LAUNCH("tc_gemm_kernel");
    P.launches++;
    if (Z > 1) {
        const long tot = long(m) * n;
        tb = timing_begin(P, EXX_TIMING_GEMM, s);
        tc_gemm_reduce_kernel<<<unsigned(std::min<long>((tot + 255) / 256, 4L * P.num_sms)), 256, 0, s>>>(
            a.D, int(Z), m, n, D, ds_i, ds_j);
        timing_end(P, tb, s);
        EXX_LAUNCH("tc_gemm_reduce_kernel");
        P.launches++;
    }
    return EXX_OK;
}

}  // namespace exx
