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

constexpr int kT = 128;              // rows of A per tile (TMEM lanes, threads)
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

__global__ void __launch_bounds__(kT, 1) tc_gemm_kernel(GemmArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    constexpr uint32_t piece = kT * kSub * 2;       // one A digit image: 128 rows x 64 k bf16
    constexpr uint32_t bpiece = kTN * kSub * 2;     // one B digit image: 96 rows
    constexpr uint32_t sbo = kSub * 2 * 8;          // bytes per 8-row group
    uint8_t *sA = smem, *sB = smem + 4 * piece;
    int *sh_b = reinterpret_cast<int *>(sB + 4 * bpiece);   // per B row: its scale shift
    uint64_t *bar = reinterpret_cast<uint64_t *>(sh_b + kTN);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    int *sflag = reinterpret_cast<int *>(tslot + 1);
    const int t = threadIdx.x, warp = t >> 5;
    if (t == 0) {
        tc::mbar_init(bar, 1);
        *sflag = 0;
    }
    if (warp == 0) tc::tmem_alloc(tslot, 512);   // 5 levels x 96 columns
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t lane = uint32_t(warp * 32) << 16;
    const uint32_t idesc = tc::instr_desc(false, kTN);
    const uint32_t a_addr = tc::smem_addr(sA), b_addr = tc::smem_addr(sB);

    const int i = blockIdx.x * kT + t, j = blockIdx.y * kTN + t;   // this thread's A row, B row
    const bool arow = i < a.m, brow = t < kTN && j < a.n;
    const double *Ar = a.A + (arow ? long(i) * a.as_i : 0);
    const double *Br = a.B + (brow ? long(j) * a.bs_j : 0);
    const long kbeg = long(blockIdx.z) * a.kper, kend = min(a.K, kbeg + a.kper);
    double *D = a.D + long(blockIdx.z) * a.dz;
    uint32_t phase = 0;
    bool first = true;
    for (long c0 = kbeg; c0 < kend; c0 += kChunk) {
        const long c1 = min(kend, c0 + kChunk);
        // scales of this chunk: largest exponent field of the own A row and B row
        int EA = 0, EB = 0;
        for (long k = c0; k < c1; ++k) {
            if (arow) EA = max(EA, exp_field(Ar[k * a.as_k]));
            if (brow) EB = max(EB, exp_field(Br[k * a.bs_k]));
        }
        EA = max(EA, 100);   // rows below 2^-922 are zero rows
        EB = max(EB, 100);
        const int shA = 1052 - EA, shB = 1052 - EB;
        if (t < kTN) sh_b[t] = shB;
        for (int sub = 0; sub < kSubs; ++sub) {
            const long k0 = c0 + long(sub) * kSub;
            if (k0 >= c1) break;   // uniform
            for (int u = 0; u < kSub / 4; ++u) {
                float qa[4][4], qb[4][4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const long k = k0 + 4 * u + e;
                    const bool in = k < c1;
                    float da[4], db[4];
                    digits4(arow && in ? Ar[k * a.as_k] : 0.0, shA, da);
                    digits4(brow && in ? Br[k * a.bs_k] : 0.0, shB, db);
#pragma unroll
                    for (int l = 0; l < 4; ++l) {
                        qa[l][e] = da[l];
                        qb[l][e] = db[l];
                    }
                }
                store_digits(sA, t, u, qa, piece);
                if (t < kTN) store_digits(sB, t, u, qb, bpiece);
            }
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
        }
        __syncthreads();   // the shift of every B row is visible
        if (*sflag) break;
        // drain: D(i, j) (+)= alpha 2^(-shA - shB) sum_l L_l 2^(48 - 8 l)
        for (int cg = 0; cg < kTN / 8; ++cg) {
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
                const int col = blockIdx.y * kTN + cg * 8 + e;
                if (!arow || col >= a.n) continue;
                double v = double(__uint_as_float(r[4][e]));
                v = v * (1.0 / 256.0) + double(__uint_as_float(r[3][e]));
                v = v * (1.0 / 256.0) + double(__uint_as_float(r[2][e]));
                v = v * (1.0 / 256.0) + double(__uint_as_float(r[1][e]));
                v = v * (1.0 / 256.0) + double(__uint_as_float(r[0][e]));
                // v 2^48 2^-shA 2^-shB alpha, the powers of two as one exponent (a product
                // below the normal range is zero: both rows were below 2^-900)
                const int sc = min(48 - shA - sh_b[cg * 8 + e], 1023);
                v = sc < -1022 ? 0.0 : a.alpha * (v * __longlong_as_double(static_cast<long long>(sc + 1023) << 52));
                double *dp = D + long(i) * a.ds_i + long(col) * a.ds_j;
                *dp = first ? v : *dp + v;
            }
        }
        tc::tc_fence_before();   // TMEM reads before the next chunk's MMAs overwrite it
        __syncthreads();
        first = false;
    }
    if (first && *sflag == 0 && arow) {   // empty k range: the slot still holds a sum (zero)
        for (int c = 0; c < kTN; ++c) {
            const int col = blockIdx.y * kTN + c;
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
    const size_t smem = 4 * size_t(kT + kTN) * kSub * 2 + kTN * sizeof(int) + 64;
    EXX_CUDA(cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    int tb = timing_begin(P, EXX_TIMING_GEMM, s);
    tc_gemm_kernel<<<dim3(unsigned(mt), unsigned(nt), unsigned(Z)), kT, smem, s>>>(a);
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
