// Split-precision path of the batched Kronecker solve on the tcgen05 tensor cores.
//
// Each mode product of Sec. II.B is a GEMM  D[row][n] = sum_k A[row][k] B[n][k]  where a
// row is a pencil of the grid function along the contracted axis (128 rows per tile,
// one row per thread, one TMEM lane per row) and B is the 1D eigenvector matrix (or its
// transpose).  Operands are split into bf16 or tf32 pieces, x = x0 + x1 (+ x2), and the
// cross products that matter are accumulated in one FP32 TMEM accumulator:
//   BF16X3: x1*y0 + x0*y1 + x0*y0          (2 bf16 pieces, ~16 significant bits)
//   BF16X6: x2*y0 + x1*y1 + x0*y2 + x1*y0 + x0*y1 + x0*y0   (3 pieces, ~24 bits)
//   TF32X3: x1*y0 + x0*y1 + x0*y0          (2 tf32 pieces, ~22 bits)
// smallest terms first.  The pair density psi_m psi_n is formed in the prologue from
// compensated FP32 copies of the orbitals (hi + lo), the Hadamard scaling by f(Lambda)
// sits between the forward and the inverse y products of pass 3 (both on-chip), and the
// accumulation over pairs is a separate compensated FP32 kernel.
#include "exx_internal.h"
#include "tc_ptx.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

namespace exx {

namespace {

constexpr int kRows = 128;          // tile rows = TMEM lanes = threads
constexpr uint32_t kWaitLimit = 1u << 22;

struct PrecInfo {
    bool tf32;
    int np;          // pieces per operand
    int es;          // bytes per element
    int nprod;       // products
};
__host__ __device__ inline PrecInfo prec_info(int prec)
{
    switch (prec) {
    case EXX_PREC_BF16X3: return {false, 2, 2, 3};
    case EXX_PREC_BF16X6: return {false, 3, 2, 6};
    default: return {true, 2, 4, 3};   // TF32X3
    }
}
// products (a piece, b piece), smallest first
__host__ __device__ inline void product(int prec, int i, int &pa, int &pb)
{
    if (prec == EXX_PREC_BF16X6) {
        const int A[6] = {2, 1, 0, 1, 0, 0}, B[6] = {0, 1, 2, 0, 1, 0};
        pa = A[i];
        pb = B[i];
    } else {
        const int A[3] = {1, 0, 0}, B[3] = {0, 1, 0};
        pa = A[i];
        pb = B[i];
    }
}

inline int pad16(int n) { return (n + 15) & ~15; }

// canonical K-major no-swizzle image: byte offset of (row, 16-byte chunk c)
__host__ __device__ inline uint32_t img_off(int row, int c, uint32_t sbo)
{
    return uint32_t(row >> 3) * sbo + uint32_t(c) * 128u + uint32_t(row & 7) * 16u;
}

// ---- host rounding (round to nearest even) ----
inline float host_bf16(double v)
{
    float f = float(v);
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    u &= 0xFFFF0000u;
    std::memcpy(&f, &u, 4);
    return f;
}
inline float host_tf32(double v)
{
    float f = float(v);
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0xFFFu + ((u >> 13) & 1u);
    u &= 0xFFFFE000u;
    std::memcpy(&f, &u, 4);
    return f;
}

// ---- device: split a value (hi + lo) into pieces ----
template <bool TF32, int NP>
__device__ __forceinline__ void split(float hi, float lo, float (&p)[3])
{
    if (TF32) {
        p[0] = tc::to_tf32(hi);
        p[1] = tc::to_tf32((hi - p[0]) + lo);
        p[2] = 0.f;
    } else {
        p[0] = __bfloat162float(__float2bfloat16_rn(hi));
        float r = (hi - p[0]) + lo;
        p[1] = __bfloat162float(__float2bfloat16_rn(r));
        p[2] = (NP == 3) ? __bfloat162float(__float2bfloat16_rn(r - p[1])) : 0.f;
    }
}

// Write one 16-byte chunk per piece (8 bf16 or 4 tf32 values of row `row`).
template <bool TF32, int NP>
__device__ __forceinline__ void put_chunk(uint8_t *img, uint32_t piece_bytes, int row, int c, uint32_t sbo,
                                          const float *hi, const float *lo)
{
    constexpr int EPC = TF32 ? 4 : 8;   // elements per 16-byte chunk
    float pc[3][EPC];
#pragma unroll
    for (int e = 0; e < EPC; ++e) {
        float p[3];
        split<TF32, NP>(hi[e], lo ? lo[e] : 0.f, p);
#pragma unroll
        for (int q = 0; q < 3; ++q) pc[q][e] = p[q];
    }
    const uint32_t off = img_off(row, c, sbo);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        uint4 v;
        if (TF32) {
            v.x = __float_as_uint(pc[q][0]);
            v.y = __float_as_uint(pc[q][1]);
            v.z = __float_as_uint(pc[q][2]);
            v.w = __float_as_uint(pc[q][3]);
        } else {
            uint32_t w[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                uint32_t lo16 = __float_as_uint(pc[q][2 * t]) >> 16;
                uint32_t hi16 = __float_as_uint(pc[q][2 * t + 1]) & 0xFFFF0000u;
                w[t] = lo16 | hi16;
            }
            v = make_uint4(w[0], w[1], w[2], w[3]);
        }
        *reinterpret_cast<uint4 *>(img + q * piece_bytes + off) = v;
    }
}

// Issue the split products of one GEMM (A pieces x B pieces) into TMEM column d_col.
template <bool TF32>
__device__ __forceinline__ void issue_gemm(int prec, uint32_t d_tmem, uint32_t a_base, uint32_t a_piece,
                                           uint32_t a_sbo, uint32_t b_base, uint32_t b_piece, uint32_t b_sbo,
                                           int ksteps, uint32_t idesc)
{
    const PrecInfo pi = prec_info(prec);
    uint32_t acc = 0;
    for (int t = 0; t < pi.nprod; ++t) {
        int pa, pb;
        product(prec, t, pa, pb);
        for (int ks = 0; ks < ksteps; ++ks) {
            uint64_t ad = tc::smem_desc(a_base + pa * a_piece + ks * 256u, 128u, a_sbo);
            uint64_t bd = tc::smem_desc(b_base + pb * b_piece + ks * 256u, 128u, b_sbo);
            if (TF32) tc::mma_tf32(d_tmem, ad, bd, idesc, acc);
            else tc::mma_bf16(d_tmem, ad, bd, idesc, acc);
            acc = 1;
        }
    }
}

// ---------------------------------------------------------------------------------------
// Pass kernel.  Rows of the batch are cut into tiles of 128; CTAs loop over tiles.
struct TcPassArgs {
    int nfields, R, K, Np;          // K = n_d (contracted length), Np = K padded to 16
    long N;
    const float *in;
    float *out;
    const uint8_t *B1, *B2;         // operand images (pieces concatenated)
    const float *F;                 // [col][row] scaling for the double pass
    const float *psi_hi, *psi_lo;   // fp32 orbital planes (pair prologue)
    int occ_off;                    // column offset of the occupied set in the planes
    const int2 *pairs;
    int *err;
};

template <bool TF32, int NP, int LOAD, int STORE, bool DOUBLE>
__global__ void __launch_bounds__(kRows, 1) tc_pass_kernel(TcPassArgs a, int prec)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    constexpr int ES = TF32 ? 4 : 2;
    constexpr int EPC = 16 / ES;
    const int Kp = a.Np;
    const uint32_t a_sbo = uint32_t(Kp) * ES * 8;     // bytes per 8-row group
    const uint32_t b_sbo = a_sbo;
    const uint32_t a_piece = uint32_t(kRows) * Kp * ES;
    const uint32_t b_piece = uint32_t(a.Np) * Kp * ES;
    const uint32_t b_bytes = b_piece * NP;
    uint8_t *sB1 = smem;
    uint8_t *sB2 = smem + b_bytes;
    uint8_t *sA = smem + (DOUBLE ? 2 : 1) * b_bytes;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sA + a_piece * NP);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    int *sflag = reinterpret_cast<int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int ncols_tmem = DOUBLE ? (2 * a.Np <= 32 ? 32 : 2 * a.Np <= 64 ? 64 : 2 * a.Np <= 128 ? 128 : 256)
                                  : (a.Np <= 32 ? 32 : a.Np <= 64 ? 64 : a.Np <= 128 ? 128 : 256);

    // operand images of the contraction matrices, copied once per CTA
    for (uint32_t i = tid * 16; i < b_bytes; i += kRows * 16) {
        *reinterpret_cast<uint4 *>(sB1 + i) = *reinterpret_cast<const uint4 *>(a.B1 + i);
        if (DOUBLE) *reinterpret_cast<uint4 *>(sB2 + i) = *reinterpret_cast<const uint4 *>(a.B2 + i);
    }
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        *sflag = 0;
    }
    if (warp == 0) tc::tmem_alloc(tslot, ncols_tmem);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t d1 = tmem, d2 = tmem + (DOUBLE ? uint32_t(a.Np) : 0u);
    const uint32_t lane_off = uint32_t(warp * 32) << 16;
    const uint32_t idesc = tc::instr_desc(TF32, a.Np);
    const int ksteps = Kp * ES / 32;
    const uint32_t sA_addr = tc::smem_addr(sA), sB1_addr = tc::smem_addr(sB1), sB2_addr = tc::smem_addr(sB2);
    uint32_t phase = 0;

    const long rows = long(a.nfields) * a.R;
    const long ntiles = (rows + kRows - 1) / kRows;
    for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long g = tile * kRows + tid;
        const bool active = g < rows;
        const int p = active ? int(g / a.R) : 0;
        const int r = active ? int(g - long(p) * a.R) : 0;
        // ---- prologue: this thread's row (K values) -> split pieces in SMEM ----
        {
            const float *in = a.in + size_t(p) * a.N;
            const float *mh = nullptr, *ml = nullptr, *nh = nullptr, *nl = nullptr;
            if (LOAD == LOAD_PAIR && active) {
                const int2 mn = a.pairs[p];
                mh = a.psi_hi + size_t(a.occ_off + mn.x) * a.N;
                ml = a.psi_lo + size_t(a.occ_off + mn.x) * a.N;
                nh = a.psi_hi + size_t(mn.y) * a.N;
                nl = a.psi_lo + size_t(mn.y) * a.N;
            }
            for (int c = 0; c < Kp / EPC; ++c) {
                float hi[EPC], lo[EPC];
#pragma unroll
                for (int e = 0; e < EPC; ++e) {
                    const int k = c * EPC + e;
                    hi[e] = 0.f;
                    lo[e] = 0.f;
                    if (active && k < a.K) {
                        if (LOAD == LOAD_PAIR) {
                            const size_t idx = size_t(k) * a.R + r;
                            const float ah = mh[idx], al = ml[idx], bh = nh[idx], bl = nl[idx];
                            const float ph = ah * bh;
                            hi[e] = ph;
                            lo[e] = fmaf(ah, bh, -ph) + fmaf(ah, bl, al * bh);
                        } else if (LOAD == LOAD_KSLOW) {
                            hi[e] = in[size_t(k) * a.R + r];
                        } else {
                            hi[e] = in[size_t(r) * a.K + k];
                        }
                    }
                }
                put_chunk<TF32, NP>(sA, a_piece, tid, c, a_sbo, hi, LOAD == LOAD_PAIR ? lo : nullptr);
            }
        }
        tc::fence_proxy_async_smem();
        tc::tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc::tc_fence_after();
            issue_gemm<TF32>(prec, d1, sA_addr, a_piece, a_sbo, sB1_addr, b_piece, b_sbo, ksteps, idesc);
            tc::mma_commit(bar);
        }
        if (!tc::mbar_wait_bounded(bar, phase, kWaitLimit)) atomicExch(sflag, 1);
        phase ^= 1u;
        tc::tc_fence_after();
        __syncthreads();
        if (*sflag) break;
        if (DOUBLE) {
            // D1 -> scale by f(Lambda) -> split -> A (same rows, K = modes) -> second GEMM
            for (int c0 = 0; c0 < a.Np; c0 += 16) {
                float v[16];
                tc::tmem_ld16(d1 + lane_off + uint32_t(c0), v);
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int col = c0 + e;
                    v[e] = (active && col < a.K) ? v[e] * a.F[size_t(col) * a.R + r] : 0.f;
                }
#pragma unroll
                for (int h = 0; h < 16 / EPC; ++h)
                    put_chunk<TF32, NP>(sA, a_piece, tid, c0 / EPC + h, a_sbo, v + h * EPC, nullptr);
            }
            tc::fence_proxy_async_smem();
            tc::tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc::tc_fence_after();
                issue_gemm<TF32>(prec, d2, sA_addr, a_piece, a_sbo, sB2_addr, b_piece, b_sbo, ksteps, idesc);
                tc::mma_commit(bar);
            }
            if (!tc::mbar_wait_bounded(bar, phase, kWaitLimit)) atomicExch(sflag, 1);
            phase ^= 1u;
            tc::tc_fence_after();
            __syncthreads();
            if (*sflag) break;
        }
        // ---- epilogue: TMEM -> registers -> global ----
        float *out = a.out + size_t(p) * a.N;
        const uint32_t dres = DOUBLE ? d2 : d1;
        for (int c0 = 0; c0 < a.Np; c0 += 16) {
            float v[16];
            tc::tmem_ld16(dres + lane_off + uint32_t(c0), v);
            if (active) {
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int col = c0 + e;
                    if (col < a.K) {
                        if (STORE == STORE_NSLOW) out[size_t(col) * a.R + r] = v[e];
                        else out[size_t(r) * a.K + col] = v[e];
                    }
                }
            }
        }
        tc::tc_fence_before();
        __syncthreads();   // TMEM reads done before the next tile's MMA overwrites it
    }
    if (tid == 0 && *sflag) atomicExch(a.err, 1);
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, ncols_tmem);
    }
}

// ---------------------------------------------------------------------------------------
// Single-tile GEMM used by the unit test of the operand layout: D (128 x n) =
// A (128 x k) B (n x k)^T with A, B given in FP32 and rounded to one bf16 / tf32 piece.
template <bool TF32>
__global__ void __launch_bounds__(kRows, 1) tc_unit_gemm_kernel(int n, int k, const float *A, const float *B,
                                                             float *D, int *err)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    constexpr int ES = TF32 ? 4 : 2, EPC = 16 / ES;
    const int Np = n, Kp = k;
    const uint32_t sbo = uint32_t(Kp) * ES * 8;
    const uint32_t a_bytes = uint32_t(kRows) * Kp * ES, b_bytes = uint32_t(Np) * Kp * ES;
    uint8_t *sA = smem, *sB = smem + a_bytes + 4096;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sB + b_bytes + 4096);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int c = 0; c < Kp / EPC; ++c) {
        float v[EPC];
        for (int e = 0; e < EPC; ++e) v[e] = A[size_t(tid) * k + c * EPC + e];
        put_chunk<TF32, 1>(sA, a_bytes, tid, c, sbo, v, nullptr);
        for (int row = tid; row < Np; row += kRows) {
            for (int e = 0; e < EPC; ++e) v[e] = B[size_t(row) * k + c * EPC + e];
            put_chunk<TF32, 1>(sB, b_bytes, row, c, sbo, v, nullptr);
        }
    }
    const int ncols = Np <= 32 ? 32 : Np <= 64 ? 64 : Np <= 128 ? 128 : 256;
    if (tid == 0) tc::mbar_init(bar, 1);
    if (warp == 0) tc::tmem_alloc(tslot, ncols);
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;
    if (tid == 0) {
        const uint32_t idesc = tc::instr_desc(TF32, Np);
        const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB);
        for (int ks = 0; ks < Kp * ES / 32; ++ks) {
            uint64_t ad = tc::smem_desc(a0 + ks * 256u, 128u, sbo);
            uint64_t bd = tc::smem_desc(b0 + ks * 256u, 128u, sbo);
            if (TF32) tc::mma_tf32(tmem, ad, bd, idesc, ks > 0);
            else tc::mma_bf16(tmem, ad, bd, idesc, ks > 0);
        }
        tc::mma_commit(bar);
    }
    const bool ok = tc::mbar_wait_bounded(bar, 0, kWaitLimit);
    tc::tc_fence_after();
    if (!ok && tid == 0) atomicExch(err, 1);
    for (int c0 = 0; c0 < Np; c0 += 16) {
        float v[16];
        tc::tmem_ld16(tmem + (uint32_t(warp * 32) << 16) + uint32_t(c0), v);
        for (int e = 0; e < 16; ++e) D[size_t(tid) * n + c0 + e] = v[e];
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, ncols);
    }
}

// ---------------------------------------------------------------------------------------
// Orbital preparation: fp32 (hi, lo) planes of Psi_in (and Psi_occ when separate), and
// g = f_m psi_m in fp32 for the accumulation; zero the compensated accumulators.
__global__ void tc_prepare_kernel(long N, int n_in, const double *psi_in, long ld_in, int n_occ,
                                  const double *psi_occ, long ld_occ, int copy_occ, const double *f,
                                  float *hi, float *lo, float *g, float *acc_hi, float *acc_lo)
{
    const long total_in = long(n_in) * N;
    const long total = total_in + (copy_occ ? long(n_occ) * N : 0);
    for (long e = long(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += long(gridDim.x) * blockDim.x) {
        double v;
        if (e < total_in) {
            long c = e / N, r = e - c * N;
            v = psi_in[c * ld_in + r];
            acc_hi[e] = 0.f;
            acc_lo[e] = 0.f;
        } else {
            long c = (e - total_in) / N, r = (e - total_in) - c * N;
            v = psi_occ[c * ld_occ + r];
        }
        float h = float(v);
        hi[e] = h;
        lo[e] = float(v - double(h));
    }
    const long tg = long(n_occ) * N;
    for (long e = long(blockIdx.x) * blockDim.x + threadIdx.x; e < tg; e += long(gridDim.x) * blockDim.x) {
        long c = e / N, r = e - c * N;
        g[e] = float(f[c] * psi_occ[c * ld_occ + r]);
    }
}

// Compensated accumulation: acc_t(r) += - sum g_s(r) V_field(r) in FP32 with TwoSum.
__device__ __forceinline__ void two_sum_add(float &s, float &c, float x)
{
    const float t = s + x;
    const float bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
}

__device__ __forceinline__ int diag_idx(int i, int j, int nI) { return i * nI - (i * (i - 1)) / 2 + (j - i); }

__global__ void __launch_bounds__(256) tc_accum_kernel(long N, const Block *blocks, const float *V,
                                                       const float *g, float *acc_hi, float *acc_lo)
{
    const Block b = blocks[blockIdx.y];
    const long r = long(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= N) return;
    const float *Vb = V + size_t(b.field0) * N + r;
    auto finish = [&](int t, float s, float c) {
        float hs = s + c;
        acc_lo[size_t(t) * N + r] = c - (hs - s);
        acc_hi[size_t(t) * N + r] = hs;
    };
    if (b.kind == BLK_SYM_DIAG) {
        for (int t = 0; t < b.nI; ++t) {
            const int o = b.I0 + t;
            float s = acc_hi[size_t(o) * N + r], c = acc_lo[size_t(o) * N + r];
            for (int q = 0; q < b.nI; ++q) {
                const int fi = q <= t ? diag_idx(q, t, b.nI) : diag_idx(t, q, b.nI);
                two_sum_add(s, c, -g[size_t(b.I0 + q) * N + r] * Vb[size_t(fi) * N]);
            }
            finish(o, s, c);
        }
        return;
    }
    for (int j = 0; j < b.nJ; ++j) {
        const int o = b.J0 + j;
        float s = acc_hi[size_t(o) * N + r], c = acc_lo[size_t(o) * N + r];
        for (int i = 0; i < b.nI; ++i) two_sum_add(s, c, -g[size_t(b.I0 + i) * N + r] * Vb[size_t(i * b.nJ + j) * N]);
        finish(o, s, c);
    }
    if (b.kind == BLK_SYM_OFF) {
        for (int i = 0; i < b.nI; ++i) {
            const int o = b.I0 + i;
            float s = acc_hi[size_t(o) * N + r], c = acc_lo[size_t(o) * N + r];
            for (int j = 0; j < b.nJ; ++j)
                two_sum_add(s, c, -g[size_t(b.J0 + j) * N + r] * Vb[size_t(i * b.nJ + j) * N]);
            finish(o, s, c);
        }
    }
}

__global__ void tc_finalize_kernel(long N, int n_in, const float *acc_hi, const float *acc_lo, double *out,
                                   long ld_out)
{
    const long total = long(n_in) * N;
    for (long e = long(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += long(gridDim.x) * blockDim.x) {
        long c = e / N, r = e - c * N;
        out[c * ld_out + r] = double(acc_hi[e]) + double(acc_lo[e]);
    }
}

// ---- launch helpers -------------------------------------------------------------------
size_t pass_smem(int prec, int Np, bool dbl)
{
    const PrecInfo pi = prec_info(prec);
    size_t b = size_t(pi.np) * Np * Np * pi.es;
    size_t a = size_t(pi.np) * kRows * Np * pi.es;
    return (dbl ? 2 : 1) * b + a + 64;
}

int tmem_cols(int Np, bool dbl)
{
    int c = dbl ? 2 * Np : Np;
    return c <= 32 ? 32 : c <= 64 ? 64 : c <= 128 ? 128 : 256;
}

template <bool TF32, int NP, int LOAD, int STORE, bool DOUBLE>
int launch_tc_pass(Plan &P, int kind, int prec, const TcPassArgs &a, cudaStream_t s)
{
    auto kern = tc_pass_kernel<TF32, NP, LOAD, STORE, DOUBLE>;
    size_t smem = pass_smem(prec, a.Np, DOUBLE);
    // TMEM: co-resident CTAs must not ask for more than 512 columns in total, so the
    // shared-memory request is raised until at most 512 / cols CTAs fit on one SM.
    const int cols = tmem_cols(a.Np, DOUBLE);
    const int max_ctas = std::max(1, 512 / cols);
    const size_t sm_total = 233472;   // 228 KB of shared memory per SM
    size_t floor_req = sm_total / size_t(max_ctas + 1) - 1024 + 64;
    smem = std::max(smem, floor_req);
    if (smem > 232448) {
        set_error("split-precision pass: operand images exceed shared memory for this grid size");
        return EXX_ERR_UNSUPPORTED;
    }
    EXX_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    int per_sm = 0;
    EXX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRows, smem));
    per_sm = std::max(1, std::min(per_sm, max_ctas));
    const long rows = long(a.nfields) * a.R;
    const long ntiles = (rows + kRows - 1) / kRows;
    const int grid = int(std::min<long>(ntiles, long(P.num_sms) * per_sm));
    int tb = timing_begin(P, kind, s);
    kern<<<grid, kRows, smem, s>>>(a, prec);
    timing_end(P, tb, s);
    EXX_LAUNCH("tc_pass_kernel");
    P.launches++;
    return EXX_OK;
}

template <bool TF32, int NP>
int solve_batch_t(Plan &P, int prec, const int2 *pairs_d, int nfields, float *bufA, float *bufB, cudaStream_t s)
{
    float *src = nullptr, *dst = bufA;
    for (int pass = 0; pass < 5; ++pass) {
        PassGeom g = pass_geom(P.n, pass);
        TcPassArgs a{};
        a.nfields = nfields;
        a.R = g.R;
        a.K = g.K;
        a.Np = pad16(g.K);
        a.N = P.N;
        a.in = src;
        a.out = dst;
        const int slot = pass < 2 ? pass : pass + 1;   // P3 uses slots 2 (fwd) and 3 (inv)
        a.B1 = static_cast<const uint8_t *>(P.Btc[prec][slot].p);
        a.B2 = pass == 2 ? static_cast<const uint8_t *>(P.Btc[prec][3].p) : nullptr;
        a.F = static_cast<const float *>(P.F32.p);
        a.psi_hi = static_cast<const float *>(P.psi32.p);
        a.psi_lo = a.psi_hi + P.psi32.bytes / 8;
        a.occ_off = P.tc_occ_off;
        a.pairs = pairs_d;
        a.err = static_cast<int *>(P.err_d.p);
        int rc;
        switch (pass) {
        case 0: rc = launch_tc_pass<TF32, NP, LOAD_PAIR, STORE_NSLOW, false>(P, EXX_TIMING_PASS1, prec, a, s); break;
        case 1: rc = launch_tc_pass<TF32, NP, LOAD_KFAST, STORE_NSLOW, false>(P, EXX_TIMING_PASS2, prec, a, s); break;
        case 2: rc = launch_tc_pass<TF32, NP, LOAD_KFAST, STORE_NFAST, true>(P, EXX_TIMING_PASS3, prec, a, s); break;
        case 3: rc = launch_tc_pass<TF32, NP, LOAD_KSLOW, STORE_NFAST, false>(P, EXX_TIMING_PASS4, prec, a, s); break;
        default: rc = launch_tc_pass<TF32, NP, LOAD_KSLOW, STORE_NSLOW, false>(P, EXX_TIMING_PASS5, prec, a, s); break;
        }
        if (rc) return rc;
        src = dst;
        dst = (dst == bufA) ? bufB : bufA;
    }
    P.tc_result = src;
    return EXX_OK;
}

}  // namespace

int tc_upload(Plan &P, int prec)
{
    const PrecInfo pi = prec_info(prec);
    const int axis_of[6] = {2, 0, 1, 1, 0, 2};
    const int inv_of[6] = {0, 0, 0, 1, 1, 1};
    for (int d = 0; d < 3; ++d) {
        const int Np = pad16(P.n[d]);
        if (pass_smem(prec, Np, d == 1) > 232448) {
            set_error("split precision: grid axis too long for the on-chip operand images of this build");
            return EXX_ERR_UNSUPPORTED;
        }
    }
    for (int slot = 0; slot < 6; ++slot) {
        const int d = axis_of[slot], nd = P.n[d], Np = pad16(nd);
        const uint32_t sbo = uint32_t(Np) * pi.es * 8;
        const size_t piece = size_t(Np) * Np * pi.es;
        std::vector<uint8_t> img(piece * pi.np, 0);
        for (int n = 0; n < nd; ++n)
            for (int k = 0; k < nd; ++k) {
                // output mode n from input k: forward V(k, n), inverse V(n, k)
                double v = inv_of[slot] ? P.V[d][n + size_t(nd) * k] : P.V[d][k + size_t(nd) * n];
                double rem = v;
                for (int q = 0; q < pi.np; ++q) {
                    float pv = pi.tf32 ? host_tf32(rem) : host_bf16(rem);
                    rem -= double(pv);
                    const int epc = 16 / pi.es;
                    size_t off = piece * q + img_off(n, k / epc, sbo) + size_t(k % epc) * pi.es;
                    if (pi.tf32) {
                        std::memcpy(&img[off], &pv, 4);
                    } else {
                        uint32_t u;
                        std::memcpy(&u, &pv, 4);
                        uint16_t h = uint16_t(u >> 16);
                        std::memcpy(&img[off], &h, 2);
                    }
                }
            }
        if (int rc = dev_reserve(P.Btc[prec][slot], img.size())) return rc;
        EXX_CUDA(cudaMemcpy(P.Btc[prec][slot].p, img.data(), img.size(), cudaMemcpyHostToDevice));
    }
    if (int rc = dev_reserve(P.err_d, 16)) return rc;
    EXX_CUDA(cudaMemset(P.err_d.p, 0, 16));
    return EXX_OK;
}

int tc_prepare_orbitals(Plan &P, const double *psi_occ, int n_occ, long ld_occ, const double *f,
                        const double *psi_in, int n_in, long ld_in, bool aliased, cudaStream_t s)
{
    const int ncols = n_in + (aliased ? 0 : n_occ);
    const size_t plane = size_t(ncols) * P.N;
    if (int rc = dev_reserve(P.psi32, 2 * plane * sizeof(float))) return rc;
    // psi_lo is located right after psi_hi: keep the reservation exact
    if (P.psi32.bytes != 2 * plane * sizeof(float)) {
        dev_free(P.psi32);
        if (int rc = dev_reserve(P.psi32, 2 * plane * sizeof(float))) return rc;
    }
    if (int rc = dev_reserve(P.g32, size_t(n_occ) * P.N * sizeof(float))) return rc;
    if (int rc = dev_reserve(P.acc_hi, size_t(n_in) * P.N * sizeof(float))) return rc;
    if (int rc = dev_reserve(P.acc_lo, size_t(n_in) * P.N * sizeof(float))) return rc;
    P.tc_occ_off = aliased ? 0 : n_in;
    float *hi = static_cast<float *>(P.psi32.p);
    int tb = timing_begin(P, EXX_TIMING_PREP, s);
    tc_prepare_kernel<<<4 * P.num_sms, 256, 0, s>>>(P.N, n_in, psi_in, ld_in, n_occ, psi_occ, ld_occ, aliased ? 0 : 1,
                                                   f, hi, hi + plane, static_cast<float *>(P.g32.p),
                                                   static_cast<float *>(P.acc_hi.p), static_cast<float *>(P.acc_lo.p));
    timing_end(P, tb, s);
    EXX_LAUNCH("tc_prepare_kernel");
    P.launches++;
    return EXX_OK;
}

int tc_solve_batch(Plan &P, int prec, const int2 *pairs_d, int nfields, float *bufA, float *bufB, cudaStream_t s)
{
    switch (prec) {
    case EXX_PREC_BF16X3: return solve_batch_t<false, 2>(P, prec, pairs_d, nfields, bufA, bufB, s);
    case EXX_PREC_BF16X6: return solve_batch_t<false, 3>(P, prec, pairs_d, nfields, bufA, bufB, s);
    case EXX_PREC_TF32X3: return solve_batch_t<true, 2>(P, prec, pairs_d, nfields, bufA, bufB, s);
    default: return EXX_ERR_INVALID_ARG;
    }
}

int tc_accumulate(Plan &P, const Block *blocks_d, int nblocks, const float *V, cudaStream_t s)
{
    dim3 grid(unsigned((P.N + 255) / 256), unsigned(nblocks));
    int tb = timing_begin(P, EXX_TIMING_ACCUM, s);
    tc_accum_kernel<<<grid, 256, 0, s>>>(P.N, blocks_d, V, static_cast<const float *>(P.g32.p),
                                         static_cast<float *>(P.acc_hi.p), static_cast<float *>(P.acc_lo.p));
    timing_end(P, tb, s);
    EXX_LAUNCH("tc_accum_kernel");
    P.launches++;
    return EXX_OK;
}

int tc_finalize(Plan &P, int n_in, double *out, long ld_out, cudaStream_t s)
{
    int tb = timing_begin(P, EXX_TIMING_PREP, s);
    tc_finalize_kernel<<<4 * P.num_sms, 256, 0, s>>>(P.N, n_in, static_cast<const float *>(P.acc_hi.p),
                                                    static_cast<const float *>(P.acc_lo.p), out, ld_out);
    timing_end(P, tb, s);
    EXX_LAUNCH("tc_finalize_kernel");
    P.launches++;
    return EXX_OK;
}

int tc_check_error(Plan &P, cudaStream_t s)
{
    if (!P.err_d.p) return EXX_OK;
    int h = 0;
    EXX_CUDA(cudaMemcpyAsync(&h, P.err_d.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    EXX_CUDA(cudaStreamSynchronize(s));
    if (h) {
        cudaMemsetAsync(P.err_d.p, 0, sizeof(int), s);
        set_error("a tensor-core pass gave up waiting for its MMA completion barrier");
        return EXX_ERR_TIMEOUT;
    }
    return EXX_OK;
}

int tc_unit_gemm(int tf32, int n, int k, const float *A, const float *B, float *D, int *err)
{
    const int es = tf32 ? 4 : 2;
    if (n < 16 || n > 256 || n % 16 || k < 16 || k % 16 || k > 256) return EXX_ERR_INVALID_ARG;
    size_t smem = size_t(kRows) * k * es + 4096 + size_t(n) * k * es + 4096 + 64;
    if (smem > 232448) return EXX_ERR_INVALID_ARG;
    if (tf32) {
        EXX_CUDA(cudaFuncSetAttribute(tc_unit_gemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        tc_unit_gemm_kernel<true><<<1, kRows, smem>>>(n, k, A, B, D, err);
    } else {
        EXX_CUDA(cudaFuncSetAttribute(tc_unit_gemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        tc_unit_gemm_kernel<false><<<1, kRows, smem>>>(n, k, A, B, D, err);
    }
    EXX_LAUNCH("tc_unit_gemm_kernel");
    EXX_CUDA(cudaDeviceSynchronize());
    return EXX_OK;
}

}  // namespace exx
