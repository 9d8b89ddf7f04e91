// Three-pass split-precision solve (EXX_PREC_BF16X7) on the tcgen05 tensor cores.
//
// The six mode products of the batched Kronecker solve (Sec. II.B, Eqs. 9-13) run as
// three passes over HBM, each grid function kept in its natural layout (x fastest):
//
//   pass A  per z-slice: rho = psi_m psi_n, forward x, forward y       psi -> T1 (a, b, z)
//   pass B  per (a, b) pencil: forward z, x f(Lambda), inverse z       T1 -> T2 (a, b, z)
//   pass C  per z-slice: inverse x, inverse y                          T2 -> V  (x, y, z)
//
// followed by the f-weighted accumulation of Eq. 1 (tc_accum_kernel, shared with the
// five-pass modes).  Passes A and C do two GEMMs per tile of whole z-slices: the first
// contracts x over rows (slice, y), the tile is transposed through shared memory, the
// second contracts y over rows (slice, a).  Pass B does the forward GEMM, the f(Lambda)
// scaling and the inverse GEMM on chip.  Only FP32 values cross HBM between passes.  The 1D
// matrix images stay in shared memory when they fit; otherwise (long z axes, slices wider
// than about 108 points) a producer warp streams them through two buffers as K-chunks, every
// chunk holding all outputs of its contraction indices.
//
// Arithmetic of one mode product D[row][n] = sum_k A[row][k] C[n][k]:
//  * every data row gets a power-of-two scale from its largest entry and is cut into three
//    balanced base-512 digits d0 + d1 + d2 (d0 an integer of magnitude <= 256, d1 a
//    multiple of 2^-9, d2 of 2^-18, each of at most 8 significant bits: exact in bf16);
//  * every row of the 1D matrix C (host, once) into four such digits p0..p3;
//  * the product d0 p0 is summed alone in one FP32 TMEM accumulator: its terms are
//    integers and |sum| <= K 2^16 < 2^24 for K <= 256, so the tensor core never rounds it;
//    the six products d0p1, d1p0, d0p2, d1p1, d2p0 and d0p3 (weights 2^-9 .. 2^-27) share a
//    second accumulator, whose rounding is ~2^-33 of the result;
//  * the epilogue adds the two accumulators and applies the row and column scales.
// The result carries ~27 bits of the data rows and ~36 bits of the matrices; the middle of
// pass B (the fully modal values, the only place where a rounding is common to all terms
// of the exchange energy) is kept as an FP32 hi + lo pair.
#include "exx_internal.h"
#include "tc_ptx.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <vector>

namespace exx {

namespace {

constexpr int kRows = 128;              // tile rows = TMEM lanes
constexpr uint64_t kWaitNs = 1000000000ull;   // every barrier wait gives up after 1 s
constexpr int kMatDig = 4;              // digits of the 1D matrices
constexpr size_t kSmemLimit = 232448;   // dynamic shared memory per CTA (227 KB)

inline int pad16i(int n) { return (n + 15) & ~15; }
inline int pad8i(int n) { return (n + 7) & ~7; }
inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
inline int tmem_pow2(int c) { return c <= 32 ? 32 : c <= 64 ? 64 : c <= 128 ? 128 : c <= 256 ? 256 : 512; }

// canonical K-major no-swizzle bf16 image: byte offset of (row, 16-byte chunk c)
__host__ __device__ inline uint32_t img_at(int row, int c, uint32_t sbo)
{
    return uint32_t(row >> 3) * sbo + uint32_t(c) * 128u + uint32_t(row & 7) * 16u;
}

// bytes of one matrix image: 4 digit planes of Np x Kp bf16, then Np column scales
inline size_t mat_image_bytes(int Np, int Kp)
{
    return align_up(size_t(kMatDig) * Np * Kp * 2 + size_t(Np) * 4, 128);
}

// ---- device arithmetic ---------------------------------------------------------------
// Round x to the nearest multiple of 2^-G (ties to even) for |x| < 2^(22-G).
template <int G>
__device__ __forceinline__ float rnd_grid(float x)
{
    constexpr float kMagic = 12582912.f / float(1u << G);   // 1.5 * 2^(23 - G)
    return __fadd_rn(__fadd_rn(x, kMagic), -kMagic);
}

// Three base-512 digits of (hi + lo) * s, |hi s| < 256, for two elements at once: every
// residual is exact and lo enters once (one FMA rounding, far below the last digit).  The
// packed FP32x2 instructions of sm_100+ take one issue slot for both lanes (the issue rate,
// not the FP32 pipe, bounds these kernels); each rounds as its scalar form, and a - b is
// written fma(b, -1, a), which rounds once like the subtraction.
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f), a); }
template <int G>
__device__ __forceinline__ float2 rnd_grid2(float2 x)
{
    constexpr float kMagic = 12582912.f / float(1u << G);
    return __fadd2_rn(__fadd2_rn(x, f2(kMagic)), f2(-kMagic));
}
template <bool LO>
__device__ __forceinline__ void digits3x2(float2 hi, float2 lo, float2 s, float2 &d0, float2 &d1, float2 &d2)
{
    const float2 t = __fmul2_rn(hi, s);
    d0 = rnd_grid2<0>(t);
    const float2 r0 = sub2(t, d0);
    const float2 r1 = LO ? __ffma2_rn(lo, s, r0) : r0;
    d1 = rnd_grid2<9>(r1);
    d2 = rnd_grid2<18>(sub2(r1, d1));
}

// Row scale s = 2^(8 - e) and its inverse, with m = f 2^e, f in [0.5, 1): |x s| < 256.
__device__ __forceinline__ void row_scales(float m, float &s, float &inv)
{
    int e = int((__float_as_uint(m) >> 23) & 0xffu) - 126;
    e = max(e, -100);   // zero rows (and rows below 2^-100) slice to zero digits
    s = __uint_as_float(uint32_t(127 + 8 - e) << 23);
    inv = __uint_as_float(uint32_t(127 - 8 + e) << 23);
}

// Pack two bf16-exact floats (at most 8 significant bits) into one word: their bf16 forms
// are the upper halves of their FP32 bit patterns.
__device__ __forceinline__ uint32_t pack2(float a, float b)
{
    return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);
}

// Issue the 7 digit products of one GEMM (or of one K-chunk of it): d0 p0 into TMEM column
// d_lead, the rest into d_rest.  A digits i at a_base + i a_piece (SBO a_sbo), C digits j at
// b_base + j b_piece (SBO b_sbo), K-major, LBO 128 bytes, ksteps steps of 16 along K.  The
// first step overwrites both accumulators unless `accumulate` (a later K-chunk).
__device__ __forceinline__ void issue_x7g(uint32_t d_lead, uint32_t d_rest, uint32_t a_base, uint32_t a_piece,
                                          uint32_t a_sbo, uint32_t b_base, uint32_t b_piece, uint32_t b_sbo,
                                          int ksteps, uint32_t idesc, bool accumulate)
{
    const int PA[7] = {0, 0, 1, 0, 1, 2, 0};
    const int PB[7] = {0, 1, 0, 2, 1, 0, 3};
    for (int ks = 0; ks < ksteps; ++ks) {
#pragma unroll
        for (int t = 0; t < 7; ++t) {
            const uint64_t ad = tc::smem_desc(a_base + uint32_t(PA[t]) * a_piece + uint32_t(ks) * 256u, 128u, a_sbo);
            const uint64_t bd = tc::smem_desc(b_base + uint32_t(PB[t]) * b_piece + uint32_t(ks) * 256u, 128u, b_sbo);
            const bool acc = accumulate || ks > 0 || (t > 1);
            tc::mma_bf16(t == 0 ? d_lead : d_rest, ad, bd, idesc, (t == 0 ? (accumulate || ks > 0) : acc) ? 1u : 0u);
        }
    }
}
__device__ __forceinline__ void issue_x7(uint32_t d_lead, uint32_t d_rest, uint32_t a_base, uint32_t a_piece,
                                         uint32_t b_base, uint32_t b_piece, uint32_t sbo, int ksteps,
                                         uint32_t idesc)
{
    issue_x7g(d_lead, d_rest, a_base, a_piece, sbo, b_base, b_piece, sbo, ksteps, idesc, false);
}

// Digits of four consecutive elements (hi + lo) * s of one row: 8 bytes in each of the three
// digit planes (plane stride `piece`) at byte offset o.
// LO = false: l is zero and skipped.
template <bool LO = true>
__device__ __forceinline__ void store_digits4(uint8_t *img, uint32_t piece, uint32_t o, const float (&h)[4],
                                              const float (&l)[4], float s)
{
    float2 d[3][2];
#pragma unroll
    for (int e = 0; e < 2; ++e)
        digits3x2<LO>(make_float2(h[2 * e], h[2 * e + 1]), make_float2(l[2 * e], l[2 * e + 1]), f2(s), d[0][e],
                      d[1][e], d[2][e]);
#pragma unroll
    for (int q = 0; q < 3; ++q)
        *reinterpret_cast<uint2 *>(img + q * piece + o) =
            make_uint2(pack2(d[q][0].x, d[q][0].y), pack2(d[q][1].x, d[q][1].y));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_addr(bar)) : "memory");
}

// Untiled bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16),
// completing as transaction bytes on `bar`.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            tc::smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(tc::smem_addr(bar))
        : "memory");
}

// Four consecutive TMEM columns of this warp's lanes, both accumulators, one wait.
__device__ __forceinline__ void tmem_pair4(uint32_t lead, uint32_t rest, float (&a)[4], float (&b)[4])
{
    uint32_t r0[4], r1[4];
    tc::tmem_ld4_issue(lead, r0);
    tc::tmem_ld4_issue(rest, r1);
    tc::tmem_wait_ld();
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        tc::order_after_wait(r0[e]);
        tc::order_after_wait(r1[e]);
        a[e] = __uint_as_float(r0[e]);
        b[e] = __uint_as_float(r1[e]);
    }
}

// One drained unit: (lead + rest) * (rs * cs[e]) for four consecutive columns.
__device__ __forceinline__ void tmem_unit(uint32_t lead, uint32_t rest, float rs, const float *cs, float (&v)[4])
{
    float v0[4], v1[4];
    tmem_pair4(lead, rest, v0, v1);
    const float4 c4 = *reinterpret_cast<const float4 *>(cs);
    const float2 w01 = __fmul2_rn(__fadd2_rn(make_float2(v0[0], v0[1]), make_float2(v1[0], v1[1])),
                                  __fmul2_rn(f2(rs), make_float2(c4.x, c4.y)));
    const float2 w23 = __fmul2_rn(__fadd2_rn(make_float2(v0[2], v0[3]), make_float2(v1[2], v1[3])),
                                  __fmul2_rn(f2(rs), make_float2(c4.z, c4.w)));
    v[0] = w01.x; v[1] = w01.y; v[2] = w23.x; v[3] = w23.y;
}

// ---------------------------------------------------------------------------------------
// Slice pass (A and C).  A tile is ns <= G consecutive z-slices of one field.
//   GEMM 1: rows (s, j) j < n2, K = i < n1 (contiguous in memory), outputs i' < n1
//   GEMM 2: rows (s, i'), K = j, outputs j' < n2, stored at (z, j', i') of the field
// Pass A reads the field as the pair product psi_m psi_n; pass C reads a stored field.
struct SliceArgs {
    int n1, n2, n3, G, tpf;
    long ntiles;
    long N;
    const float *psi;       // pass A: FP32 orbital planes (column c at c N)
    int occ_off;
    const int2 *pairs;
    const float *in;        // pass C: input fields
    float *out;
    const uint8_t *img1, *img2;
    uint32_t img1_bytes, img2_bytes;
    int Kp1, Kp2;           // pad16(n1), pad16(n2): K and N of GEMM 1 and GEMM 2
    uint32_t offB2, offA, offY, offRs, offBar;   // shared-memory layout (offB2 = 0: shares image 1)
    uint32_t a_piece1, a_piece2;                 // digit plane strides of the two A layouts
    int Pj;                 // row pitch (floats) of the transposed tile
    int tmem_cols;
    int vec;                // rows of n1 floats start 16-byte aligned (n1 % 4 == 0, N % 4 == 0)
    int stage;              // the tile's input arrives in shared memory by bulk copies (R % 4 == 0)
    uint32_t offS, stg_plane;   // staging buffer and its plane stride (bytes)
    int pipe;               // software pipeline over tiles: GEMM 2 has its own A image (offA2) and
    uint32_t offA2;         // TMEM columns (t2col), so each GEMM overlaps the other phase's work
    int t2col;
    int bstream;            // the x/y matrices stream as K-chunks of KC (nkc1, nkc2 per GEMM) through
    int KC, nkc1, nkc2;     // two buffers of buf_bytes at offset 0, their column scales at offCS
    uint32_t offCS, buf_bytes, chunk1_bytes, chunk2_bytes;
    const uint8_t *img1c, *img2c;
    int *err;
};

template <bool PAIR, int TPR>
__global__ void __launch_bounds__(kRows * TPR + 64, 2) slice_pass_kernel(const __grid_constant__ SliceArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    constexpr int NT = kRows * TPR;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t *sB1 = smem;
    uint8_t *sB2 = a.offB2 ? smem + a.offB2 : smem;
    uint8_t *sA1 = smem + a.offA, *sA2 = smem + a.offA2;
    float *Ysm = reinterpret_cast<float *>(smem + a.offY);
    float *rsb1 = reinterpret_cast<float *>(smem + a.offRs);
    float *rsb2 = rsb1 + kRows;
    float *stg = reinterpret_cast<float *>(smem + a.offS);
    uint64_t *bar_a = reinterpret_cast<uint64_t *>(smem + a.offBar);
    uint64_t *bar_d1 = bar_a + 1, *bar_d2 = bar_a + 2;
    uint64_t *stg_full = bar_a + 3, *stg_empty = bar_a + 4;
    uint64_t *bfull = bar_a + 5, *bempty = bar_a + 7;   // matrix-chunk buffers (bstream)
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar_a + 9);
    int *sflag = reinterpret_cast<int *>(tslot + 1);
    float *csS = reinterpret_cast<float *>(smem + a.offCS);   // column scales (bstream)

    if (!a.bstream) {
        for (uint32_t i = tid * 16; i < a.img1_bytes; i += blockDim.x * 16)
            *reinterpret_cast<uint4 *>(sB1 + i) = *reinterpret_cast<const uint4 *>(a.img1 + i);
        if (a.offB2)
            for (uint32_t i = tid * 16; i < a.img2_bytes; i += blockDim.x * 16)
                *reinterpret_cast<uint4 *>(sB2 + i) = *reinterpret_cast<const uint4 *>(a.img2 + i);
    } else {   // every chunk of an image carries the same column scales: take chunk 0's
        const float *c1 = reinterpret_cast<const float *>(a.img1c + size_t(kMatDig) * a.Kp1 * a.KC * 2);
        const float *c2 = reinterpret_cast<const float *>(a.img2c + size_t(kMatDig) * a.Kp2 * a.KC * 2);
        for (int i = tid; i < a.Kp1; i += blockDim.x) csS[i] = c1[i];
        for (int i = tid; i < a.Kp2; i += blockDim.x) csS[a.Kp1 + i] = c2[i];
    }
    for (uint32_t i = a.offA + tid * 16; i < a.offY; i += blockDim.x * 16)   // A images start as zeros
        *reinterpret_cast<uint4 *>(smem + i) = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        for (int i = 0; i < 9; ++i) tc::mbar_init(bar_a + i, 1);
        *sflag = 0;
    }
    if (warp == 0) tc::tmem_alloc(tslot, uint32_t(a.tmem_cols));
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;
    const int n1 = a.n1, n2 = a.n2;
    const long R = long(n1) * n2;
    const int Kp1 = a.Kp1, Kp2 = a.Kp2;
    const uint32_t sbo1 = uint32_t(Kp1) * 16u, sbo2 = uint32_t(Kp2) * 16u;

    if (warp == NT / 32 + 1) {
        // ---- producer warp: the next tile's input slices, once the compute threads have
        //      cut the current tile's first operand (one staging buffer, one tile ahead) ----
        if (a.stage && lane == 0) {
            long it = 0;
            for (long tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++it) {
                if (it > 0 && !tc::mbar_wait_timed(stg_empty, uint32_t((it - 1) & 1), kWaitNs)) {
                    atomicExch(sflag, 1);
                    break;
                }
                const long p = tile / a.tpf;
                const int z0 = int(tile - p * a.tpf) * a.G;
                const int ns = min(a.G, a.n3 - z0);
                const uint32_t bytes = uint32_t(ns) * uint32_t(R) * 4u;
                tc::mbar_arrive_expect_tx(stg_full, (PAIR ? 2u : 1u) * bytes);
                if (PAIR) {
                    const int2 mn = a.pairs[p];
                    bulk_load(stg, a.psi + size_t(a.occ_off + mn.x) * a.N + size_t(z0) * R, bytes, stg_full);
                    bulk_load(reinterpret_cast<uint8_t *>(stg) + a.stg_plane,
                              a.psi + size_t(mn.y) * a.N + size_t(z0) * R, bytes, stg_full);
                } else {
                    bulk_load(stg, a.in + size_t(p) * a.N + size_t(z0) * R, bytes, stg_full);
                }
            }
            // no copy may still target shared memory at exit: the last fill has landed
            if (it > 0 && !tc::mbar_wait_timed(stg_full, uint32_t((it - 1) & 1), kWaitNs)) atomicExch(sflag, 1);
        }
        if (a.bstream && lane == 0) {
            // matrix K-chunks in the MMA warp's order: per tile GEMM 1's chunks, then GEMM 2's
            long seq = 0;
            bool bad = false;
            for (long tile = blockIdx.x; tile < a.ntiles && !bad; tile += gridDim.x)
                for (int g = 0; g < 2 && !bad; ++g) {
                    const int nkc = g ? a.nkc2 : a.nkc1;
                    const uint32_t cb = g ? a.chunk2_bytes : a.chunk1_bytes;
                    const uint8_t *img = g ? a.img2c : a.img1c;
                    for (int kc = 0; kc < nkc; ++kc, ++seq) {
                        const int slot = int(seq & 1);
                        const long use = seq >> 1;
                        if (use > 0 && !tc::mbar_wait_timed(bempty + slot, uint32_t((use - 1) & 1), kWaitNs)) {
                            atomicExch(sflag, 1);
                            bad = true;
                            break;
                        }
                        tc::mbar_arrive_expect_tx(bfull + slot, cb);
                        bulk_load(smem + size_t(slot) * a.buf_bytes, img + size_t(kc) * cb, cb, bfull + slot);
                    }
                }
            for (int slot = 0; slot < 2; ++slot) {   // every issued copy has landed before exit
                const long nf = seq > slot ? (seq - 1 - slot) / 2 + 1 : 0;
                if (nf > 0 && !tc::mbar_wait_timed(bfull + slot, uint32_t((nf - 1) & 1), kWaitNs)) atomicExch(sflag, 1);
            }
        }
    } else if (warp == NT / 32) {
        // ---- MMA warp: two GEMMs per tile, each after the compute threads' hand-off ----
        uint32_t ph = 0;
        const uint32_t idesc1 = tc::instr_desc(false, Kp1), idesc2 = tc::instr_desc(false, Kp2);
        const uint32_t a1 = tc::smem_addr(sA1), a2 = tc::smem_addr(sA2), b1 = tc::smem_addr(sB1),
                       b2 = tc::smem_addr(sB2);
        const uint32_t t2 = tmem + uint32_t(a.t2col);
        bool bad = false;
        long seq = 0;   // matrix chunks consumed (bstream)
        for (long tile = blockIdx.x; tile < a.ntiles && !bad; tile += gridDim.x) {
            for (int g = 0; g < 2 && !bad; ++g) {
                if (!tc::mbar_wait_timed(bar_a, ph, kWaitNs)) {
                    atomicExch(sflag, 1);
                    bad = true;
                }
                ph ^= 1u;
                tc::tc_fence_after();
                if (a.bstream && !bad) {
                    // K-chunk kc of the contraction: A columns kc KC .., all outputs of the chunk
                    const int Kp = g ? Kp2 : Kp1, nkc = g ? a.nkc2 : a.nkc1;
                    const uint32_t ab = g ? a2 : a1, apiece = g ? a.a_piece2 : a.a_piece1, asbo = g ? sbo2 : sbo1;
                    const uint32_t d0 = g ? t2 : tmem;
                    for (int kc = 0; kc < nkc && !bad; ++kc, ++seq) {
                        const int slot = int(seq & 1);
                        if (!tc::mbar_wait_timed(bfull + slot, uint32_t((seq >> 1) & 1), kWaitNs)) {
                            atomicExch(sflag, 1);
                            bad = true;
                            break;
                        }
                        tc::tc_fence_after();
                        if (lane == 0) {
                            issue_x7g(d0, d0 + uint32_t(Kp), ab + uint32_t(kc * a.KC) * 16u, apiece, asbo,
                                      tc::smem_addr(smem) + uint32_t(slot) * a.buf_bytes, uint32_t(Kp) * a.KC * 2u,
                                      uint32_t(a.KC) * 16u, (min(Kp, (kc + 1) * a.KC) - kc * a.KC) / 16,
                                      g ? idesc2 : idesc1, kc > 0);
                            tc::mma_commit(bempty + slot);
                        }
                        __syncwarp();
                    }
                    if (!bad && lane == 0) tc::mma_commit(g ? bar_d2 : bar_d1);
                    __syncwarp();
                    continue;
                }
                if (!bad && lane == 0) {
                    if (g == 0) {
                        issue_x7(tmem, tmem + uint32_t(Kp1), a1, a.a_piece1, b1, uint32_t(Kp1) * Kp1 * 2u, sbo1,
                                 Kp1 / 16, idesc1);
                        tc::mma_commit(bar_d1);
                    } else {
                        issue_x7(t2, t2 + uint32_t(Kp2), a2, a.a_piece2, b2, uint32_t(Kp2) * Kp2 * 2u, sbo2,
                                 Kp2 / 16, idesc2);
                        tc::mma_commit(bar_d2);
                    }
                }
                __syncwarp();
            }
        }
    } else {
        // ---- compute threads ----
        // slicing: row srow, part sq (TPR consecutive lanes share a row: shuffles give the
        // row maximum); drain: TMEM lane drow of this warp's quarter, column part dq
        const int srow = tid / TPR, sq = tid % TPR;
        const int quarter = warp & 3, dq = warp >> 2;
        const int drow = quarter * 32 + lane;
        const uint32_t lane_q = uint32_t(quarter * 32) << 16;
        const float *cs1 = a.bstream ? csS : reinterpret_cast<const float *>(sB1 + size_t(kMatDig) * Kp1 * Kp1 * 2);
        const float *cs2 = a.bstream ? csS + Kp1 : reinterpret_cast<const float *>(sB2 + size_t(kMatDig) * Kp2 * Kp2 * 2);
        uint32_t ph1 = 0, ph2 = 0;
        // publish the A image to the MMA warp (and, after the first operand, hand the staging
        // buffer back to the producer); true = stop (error)
        auto handoff = [&](bool release) {
            tc::fence_proxy_async_smem();
            const bool stop = tc::bar_red_or(1, NT, *sflag != 0);
            if (tid == 0 && !stop) {
                mbar_arrive(bar_a);
                if (release && a.stage) mbar_arrive(stg_empty);
            }
            return stop;
        };
        auto wait_d = [&](uint64_t *bar, uint32_t &ph) {
            if (!tc::mbar_wait_timed(bar, ph, kWaitNs)) atomicExch(sflag, 1);
            ph ^= 1u;
            tc::tc_fence_after();
        };
        struct TileInfo {
            long p;
            int z0, R1, R2;
        };
        auto info = [&](long tile) {
            TileInfo t;
            t.p = tile / a.tpf;
            t.z0 = int(tile - t.p * a.tpf) * a.G;
            const int ns = min(a.G, a.n3 - t.z0);
            t.R1 = ns * n2;
            t.R2 = ns * n1;
            return t;
        };
        // the four phases of a tile
        auto slice1 = [&](const TileInfo &ti, long it) {
            const long p = ti.p;
            const int z0 = ti.z0, R1 = ti.R1;
                // ---- GEMM 1 operand: row (s, j), K = i; sweep 1 finds the row maximum, sweep 2
                //      (the same loads, mostly from L1) cuts the digits ----
                {
                    const bool act = srow < R1;
                    const int s = act ? srow / n2 : 0, j = act ? srow - s * n2 : 0;
                    const size_t off = size_t(z0 + s) * R + size_t(j) * n1;
                    const float *x0, *x1 = nullptr;
                    if (a.stage) {   // rows of this tile's slices in the staging buffer
                        if (!tc::mbar_wait_timed(stg_full, uint32_t(it & 1), kWaitNs)) atomicExch(sflag, 1);
                        const size_t so = size_t(s) * R + size_t(j) * n1;
                        x0 = stg + so;
                        x1 = reinterpret_cast<const float *>(reinterpret_cast<const uint8_t *>(stg) + a.stg_plane) + so;
                    } else if (PAIR) {
                        const int2 mn = a.pairs[p];
                        x0 = a.psi + size_t(a.occ_off + mn.x) * a.N + off;
                        x1 = a.psi + size_t(mn.y) * a.N + off;
                    } else {
                        x0 = a.in + size_t(p) * a.N + off;
                    }
                    // unit u: elements 4u..4u+3 of the row (hi, and with LO the product's rounding error)
                    auto unit = [&](int k0, float (&h)[4], float (&l)[4], auto LO) {
                        float u0[4], u1[4];
                        if (a.vec && k0 + 4 <= n1) {
                            const float4 v = *reinterpret_cast<const float4 *>(x0 + k0);
                            u0[0] = v.x; u0[1] = v.y; u0[2] = v.z; u0[3] = v.w;
                            if (PAIR) {
                                const float4 w = *reinterpret_cast<const float4 *>(x1 + k0);
                                u1[0] = w.x; u1[1] = w.y; u1[2] = w.z; u1[3] = w.w;
                            }
                        } else {
    #pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const bool ok = k0 + e < n1;
                                u0[e] = ok ? x0[k0 + e] : 0.f;
                                if (PAIR) u1[e] = ok ? x1[k0 + e] : 0.f;
                            }
                        }
    #pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            if (PAIR) {
                                const float2 x = make_float2(u0[2 * e], u0[2 * e + 1]);
                                const float2 y = make_float2(u1[2 * e], u1[2 * e + 1]);
                                const float2 hh = __fmul2_rn(x, y);
                                const float2 ll = decltype(LO)::value ? __ffma2_rn(x, y, __fmul2_rn(hh, f2(-1.f)))
                                                                      : f2(0.f);
                                h[2 * e] = hh.x; h[2 * e + 1] = hh.y;
                                l[2 * e] = ll.x; l[2 * e + 1] = ll.y;
                            } else {
                                h[2 * e] = u0[2 * e]; h[2 * e + 1] = u0[2 * e + 1];
                                l[2 * e] = 0.f; l[2 * e + 1] = 0.f;
                            }
                        }
                    };
                    float mx = 0.f;
                    if (act)
                        for (int k0 = 4 * sq; k0 < n1; k0 += 4 * TPR) {
                            float h[4], l[4];
                            unit(k0, h, l, std::false_type{});
    #pragma unroll
                            for (int e = 0; e < 4; ++e) mx = fmaxf(mx, fabsf(h[e]));
                        }
    #pragma unroll
                    for (int o = 1; o < TPR; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                    float sc, inv;
                    row_scales(mx, sc, inv);
                    if (act) {
                        if (sq == 0) rsb1[srow] = inv;
                        for (int k0 = 4 * sq; k0 < n1; k0 += 4 * TPR) {
                            float h[4], l[4];
                            unit(k0, h, l, std::true_type{});
                            store_digits4<PAIR>(sA1, a.a_piece1, img_at(srow, k0 >> 3, sbo1) + uint32_t(k0 & 7) * 2u, h, l, sc);
                        }
                    }
                }
        };
        auto drain1 = [&](const TileInfo &ti) {
            const int R1 = ti.R1;
            wait_d(bar_d1, ph1);
                // ---- GEMM 1 result -> transposed tile Y[(s, i')][j] ----
                {
                    const bool act = drow < R1;
                    const int s = act ? drow / n2 : 0, j = act ? drow - s * n2 : 0;
                    const float rs = act ? rsb1[drow] : 0.f;
                    float *yb = Ysm + size_t(s) * n1 * a.Pj + j;
                    const int nu = quarter * 32 < R1 ? Kp1 / 4 : 0;   // uniform: quarters without rows skip
                    for (int u4 = dq; u4 < nu; u4 += TPR) {
                        float v[4];
                        tmem_unit(tmem + lane_q + uint32_t(4 * u4), tmem + lane_q + uint32_t(Kp1 + 4 * u4), rs,
                                  cs1 + 4 * u4, v);
                        if (act) {
    #pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int col = 4 * u4 + e;
                                if (col < n1) yb[size_t(col) * a.Pj] = v[e];
                            }
                        }
                    }
                    tc::tc_fence_before();
                }
        };
        auto slice2 = [&](const TileInfo &ti) {
            const int R2 = ti.R2;
                // ---- GEMM 2 operand: row (s, i'), K = j, from the transposed tile ----
                {
                    const bool act = srow < R2;
                    const float *yr = Ysm + size_t(act ? srow : 0) * a.Pj;
                    auto unit = [&](int k0, float (&h)[4]) {
                        const float4 v = *reinterpret_cast<const float4 *>(yr + k0);
                        h[0] = v.x; h[1] = v.y; h[2] = v.z; h[3] = v.w;
    #pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (k0 + e >= n2) h[e] = 0.f;   // pitch padding
                    };
                    float mx = 0.f;
                    if (act)
                        for (int k0 = 4 * sq; k0 < n2; k0 += 4 * TPR) {
                            float h[4];
                            unit(k0, h);
    #pragma unroll
                            for (int e = 0; e < 4; ++e) mx = fmaxf(mx, fabsf(h[e]));
                        }
    #pragma unroll
                    for (int o = 1; o < TPR; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                    float sc, inv;
                    row_scales(mx, sc, inv);
                    if (act) {
                        if (sq == 0) rsb2[srow] = inv;
                        for (int k0 = 4 * sq; k0 < n2; k0 += 4 * TPR) {
                            float h[4];
                            const float l[4] = {0.f, 0.f, 0.f, 0.f};
                            unit(k0, h);
                            store_digits4<false>(sA2, a.a_piece2, img_at(srow, k0 >> 3, sbo2) + uint32_t(k0 & 7) * 2u, h, l, sc);
                        }
                    }
                }
        };
        auto drain2 = [&](const TileInfo &ti) {
            const long p = ti.p;
            const int z0 = ti.z0, R2 = ti.R2;
            wait_d(bar_d2, ph2);
                // ---- GEMM 2 result -> the field at (z0 + s, j', i') ----
                {
                    const bool act = drow < R2;
                    const int s = act ? drow / n1 : 0, ip = act ? drow - s * n1 : 0;
                    const float rs = act ? rsb2[drow] : 0.f;
                    float *o = a.out + size_t(p) * a.N + size_t(z0 + s) * R + ip;
                    const int nu = quarter * 32 < R2 ? Kp2 / 4 : 0;
                    for (int u4 = dq; u4 < nu; u4 += TPR) {
                        float v[4];
                        tmem_unit(tmem + lane_q + uint32_t(a.t2col + 4 * u4),
                                  tmem + lane_q + uint32_t(a.t2col + Kp2 + 4 * u4), rs, cs2 + 4 * u4, v);
                        if (act) {
    #pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int col = 4 * u4 + e;
                                if (col < n2) o[size_t(col) * n1] = v[e];
                            }
                        }
                    }
                    tc::tc_fence_before();
                }
        };
        if (!a.pipe) {
            long it = 0;
            for (long tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++it) {
                const TileInfo ti = info(tile);
                slice1(ti, it);
                if (handoff(true)) break;
                drain1(ti);
                tc::bar_sync(1, NT);
                slice2(ti);
                if (handoff(false)) break;
                drain2(ti);
            }
        } else {
            // GEMM 1 of tile t runs while the threads drain GEMM 2 of tile t-1; GEMM 2 of t
            // runs while they cut the first operand of tile t+1
            long it = 0;
            long tile = blockIdx.x;
            bool have_prev = false, stop = false;
            TileInfo prev{};
            if (tile < a.ntiles) {
                slice1(info(tile), it);
                stop = handoff(true);
            }
            for (; tile < a.ntiles && !stop; tile += gridDim.x, ++it) {
                const TileInfo ti = info(tile);
                if (have_prev) drain2(prev);
                drain1(ti);
                tc::bar_sync(1, NT);
                slice2(ti);
                if ((stop = handoff(false))) break;
                const long next = tile + gridDim.x;
                if (next < a.ntiles) {
                    slice1(info(next), it + 1);
                    if ((stop = handoff(true))) break;
                }
                prev = ti;
                have_prev = true;
            }
            if (!stop && have_prev) drain2(prev);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (tid == 0 && *sflag) atomicExch(a.err, 1);
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, uint32_t(a.tmem_cols));
    }
}

// ---------------------------------------------------------------------------------------
// Pass B.  A tile is 128 consecutive rows r = a + n1 b of one field (pencils along z).
//   forward GEMM: rows r, K = z, outputs c in NB blocks of WN columns
//   middle: (D * f(Lambda)) as FP32 hi + lo, re-sliced in place of its own digits
//   inverse GEMM: rows r, K = c, outputs z in NB blocks
// The matrix images stream through nbuf shared-memory buffers (bulk copies by the producer
// warp) unless all 2 NB blocks are resident.
struct ZArgs {
    long ntiles;
    int tpfz, R, n3, Kp;
    long N;
    const float *in;
    float *out;
    const float *Fh, *Fl;        // f(Lambda) hi and lo, natural layout (c R + r)
    const uint8_t *imgF, *imgI;  // NB blocks each, blk_bytes apart
    uint32_t blk_bytes;
    int NB, WN, NC;              // NC = NB WN columns per accumulator (output blocks), or
    int kchunk, KC;              // kchunk: NB blocks of all NC outputs x KC contraction indices
    int nbuf, resident;
    uint32_t offB, offCs, offMax, offBar;
    int tmem_cols;
    int *err;
};

// Input of tile t for this thread's units u = dq + g TPR of row `row` (zeros past n3 and for
// rows past the field or tiles past the end).
template <int TPR, int UPT>
__device__ __forceinline__ void z_load_tile(const ZArgs &a, long t, int row, int dq, float (&x)[UPT][4])
{
    const long pp = t / a.tpfz;
    const long rr = (t - pp * a.tpfz) * kRows + row;
    const bool ok_row = t < a.ntiles && rr < a.R;
    const float *src = a.in + size_t(ok_row ? pp : 0) * a.N + (ok_row ? rr : 0);
#pragma unroll
    for (int g = 0; g < UPT; ++g)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int z = 4 * (dq + g * TPR) + e;
            x[g][e] = (ok_row && z < a.n3) ? src[size_t(z) * a.R] : 0.f;
        }
}

template <int TPR, int UPT>
__global__ void __launch_bounds__(kRows * TPR + 64, (UPT <= 4 ? 2 : 1)) zpass_kernel(const __grid_constant__ ZArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    constexpr int NT = kRows * TPR;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t *sA = smem;
    uint8_t *sB = smem + a.offB;
    float *csF = reinterpret_cast<float *>(smem + a.offCs);
    float *csI = csF + a.NC;
    float *maxb = reinterpret_cast<float *>(smem + a.offMax);
    uint64_t *bar_a = reinterpret_cast<uint64_t *>(smem + a.offBar);
    uint64_t *bar_d = bar_a + 1;
    uint64_t *bfull = bar_a + 2;
    uint64_t *bempty = bfull + a.nbuf;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bempty + a.nbuf);
    int *sflag = reinterpret_cast<int *>(tslot + 1);
    const int Kp = a.Kp, WN = a.WN, NB = a.NB;
    const uint32_t sbo = uint32_t(Kp) * 16u;
    const uint32_t a_piece = uint32_t(kRows) * Kp * 2u;
    const uint32_t b_piece = a.kchunk ? uint32_t(a.NC) * a.KC * 2u : uint32_t(WN) * Kp * 2u;
    const uint32_t b_sbo = a.kchunk ? uint32_t(a.KC) * 16u : sbo;
    const uint32_t cs_off = uint32_t(kMatDig) * b_piece;   // column scales inside a block

    for (uint32_t i = tid * 16; i < 3u * a_piece; i += blockDim.x * 16)
        *reinterpret_cast<uint4 *>(sA + i) = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < a.NC; i += blockDim.x) {
        const int nb = a.kchunk ? 0 : i / WN, c = i - nb * WN;
        csF[i] = reinterpret_cast<const float *>(a.imgF + size_t(nb) * a.blk_bytes + cs_off)[c];
        csI[i] = reinterpret_cast<const float *>(a.imgI + size_t(nb) * a.blk_bytes + cs_off)[c];
    }
    if (tid == 0) {
        tc::mbar_init(bar_a, 1);
        tc::mbar_init(bar_d, 1);
        for (int b = 0; b < a.nbuf; ++b) {
            tc::mbar_init(bfull + b, 1);
            tc::mbar_init(bempty + b, 1);
        }
        *sflag = 0;
    }
    if (warp == 0) tc::tmem_alloc(tslot, uint32_t(a.tmem_cols));
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;
    // block sequence per tile: forward blocks 0..NB-1, then inverse blocks 0..NB-1
    auto block_src = [&](int j) {
        return (j < NB ? a.imgF : a.imgI) + size_t(j < NB ? j : j - NB) * a.blk_bytes;
    };

    if (warp == NT / 32 + 1) {
        // ---- producer warp: matrix blocks into the shared-memory buffers ----
        if (lane == 0) {
            if (a.resident) {
                for (int j = 0; j < 2 * NB; ++j) {
                    tc::mbar_arrive_expect_tx(bfull + j, a.blk_bytes);
                    bulk_load(sB + size_t(j) * a.blk_bytes, block_src(j), a.blk_bytes, bfull + j);
                }
                for (int j = 0; j < 2 * NB; ++j)   // no copy may still target shared memory at exit
                    if (!tc::mbar_wait_timed(bfull + j, 0, kWaitNs)) atomicExch(sflag, 1);
            } else {
                long seq = 0;
                bool bad = false;
                for (long tile = blockIdx.x; tile < a.ntiles && !bad; tile += gridDim.x) {
                    for (int j = 0; j < 2 * NB; ++j, ++seq) {
                        const int slot = int(seq % a.nbuf);
                        const long use = seq / a.nbuf;
                        if (use > 0 && !tc::mbar_wait_timed(bempty + slot, uint32_t((use - 1) & 1), kWaitNs)) {
                            atomicExch(sflag, 1);
                            bad = true;
                            break;
                        }
                        tc::mbar_arrive_expect_tx(bfull + slot, a.blk_bytes);
                        bulk_load(sB + size_t(slot) * a.blk_bytes, block_src(j), a.blk_bytes, bfull + slot);
                    }
                }
                // every issued copy has landed before exit: the last fill of each slot
                for (int slot = 0; slot < a.nbuf; ++slot) {
                    const long nf = seq > slot ? (seq - 1 - slot) / a.nbuf + 1 : 0;   // fills of this slot
                    if (nf > 0 && !tc::mbar_wait_timed(bfull + slot, uint32_t((nf - 1) & 1), kWaitNs))
                        atomicExch(sflag, 1);
                }
            }
        }
    } else if (warp == NT / 32) {
        // ---- MMA warp ----
        uint32_t ph = 0;
        const uint32_t idesc = tc::instr_desc(false, a.kchunk ? a.NC : WN);
        const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB);
        long seq = 0;
        bool bad = false;
        bool first = true;
        for (long tile = blockIdx.x; tile < a.ntiles && !bad; tile += gridDim.x) {
            for (int g = 0; g < 2 && !bad; ++g) {
                if (!tc::mbar_wait_timed(bar_a, ph, kWaitNs)) {
                    atomicExch(sflag, 1);
                    bad = true;
                }
                ph ^= 1u;
                tc::tc_fence_after();
                for (int nb = 0; nb < NB && !bad; ++nb, ++seq) {
                    const int j = g * NB + nb;
                    int slot;
                    uint32_t par;
                    bool need;
                    if (a.resident) {
                        slot = j;
                        par = 0;
                        need = first;
                    } else {
                        slot = int(seq % a.nbuf);
                        par = uint32_t((seq / a.nbuf) & 1);
                        need = true;
                    }
                    if (need && !tc::mbar_wait_timed(bfull + slot, par, kWaitNs)) {
                        atomicExch(sflag, 1);
                        bad = true;
                        break;
                    }
                    tc::tc_fence_after();
                    if (lane == 0) {
                        if (a.kchunk)   // K-chunk nb: all outputs, contraction indices nb KC ..
                            issue_x7g(tmem, tmem + uint32_t(a.NC), a0 + uint32_t(nb * a.KC) * 16u, a_piece, sbo,
                                      b0 + uint32_t(slot) * a.blk_bytes, b_piece, b_sbo,
                                      (min(Kp, (nb + 1) * a.KC) - nb * a.KC) / 16, idesc, nb > 0);
                        else
                            issue_x7(tmem + uint32_t(nb * WN), tmem + uint32_t(a.NC + nb * WN), a0, a_piece,
                                     b0 + uint32_t(slot) * a.blk_bytes, b_piece, sbo, Kp / 16, idesc);
                        if (!a.resident) tc::mma_commit(bempty + slot);
                    }
                    __syncwarp();
                }
                if (!bad && lane == 0) tc::mma_commit(bar_d);
                __syncwarp();
            }
            first = false;
        }
    } else {
        // ---- compute threads: row `row` of this warp's TMEM quarter, part dq.  Each thread
        //      keeps its units u = dq + g TPR (g < UPT) of the row in registers: the tile's
        //      input, then f(Lambda) (loaded while the forward GEMM runs), and the next tile's
        //      input is loaded while the inverse GEMM runs ----
        const int quarter = warp & 3, dq = warp >> 2;
        const int row = quarter * 32 + lane;
        const uint32_t lane_q = uint32_t(quarter * 32) << 16;
        const int n3 = a.n3;
        const long R = a.R;
        uint32_t ph = 0;
        auto rowmax = [&](float part) {
            maxb[dq * kRows + row] = part;
            tc::bar_sync(1, NT);
            float m = 0.f;
#pragma unroll
            for (int q = 0; q < TPR; ++q) m = fmaxf(m, maxb[q * kRows + row]);
            return m;
        };
        auto handoff = [&]() {
            tc::fence_proxy_async_smem();
            const bool stop = tc::bar_red_or(1, NT, *sflag != 0);
            if (tid == 0 && !stop) mbar_arrive(bar_a);
            return stop;
        };
        auto wait_d = [&]() {
            if (!tc::mbar_wait_timed(bar_d, ph, kWaitNs)) atomicExch(sflag, 1);
            ph ^= 1u;
            tc::tc_fence_after();
        };
        float x[UPT][4];
        z_load_tile<TPR, UPT>(a, blockIdx.x, row, dq, x);
        for (long tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
            const long p = tile / a.tpfz;
            const long r0 = (tile - p * a.tpfz) * kRows;
            const bool act = r0 + row < R;
            const long r = act ? r0 + row : 0;
            // ---- forward operand from the registers: row max, digits ----
            float mx = 0.f;
#pragma unroll
            for (int g = 0; g < UPT; ++g)
#pragma unroll
                for (int e = 0; e < 4; ++e) mx = fmaxf(mx, fabsf(x[g][e]));
            float sc, inv;
            row_scales(rowmax(mx), sc, inv);
            const float rs_f = inv;
            if (act) {
#pragma unroll
                for (int g = 0; g < UPT; ++g) {
                    const int z0 = 4 * (dq + g * TPR);
                    if (z0 < n3) {
                        const float l[4] = {0.f, 0.f, 0.f, 0.f};
                        store_digits4<false>(sA, a_piece, img_at(row, z0 >> 3, sbo) + uint32_t(z0 & 7) * 2u, x[g], l, sc);
                    }
                }
            }
            if (handoff()) break;
            // f(Lambda) of this thread's columns, loaded while the forward GEMM runs
            float fh[UPT][4], fl[UPT][4];
#pragma unroll
            for (int g = 0; g < UPT; ++g)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int c = 4 * (dq + g * TPR) + e;
                    const bool ok = act && c < n3;
                    fh[g][e] = ok ? a.Fh[size_t(c) * R + r] : 0.f;
                    fl[g][e] = ok ? a.Fl[size_t(c) * R + r] : 0.f;
                }
            wait_d();
            // ---- middle: (D f) as hi (plane 0: low halves, plane 1: high halves) + lo
            //      (plane 2, bf16) in the bytes its own digits take, then re-slice ----
            float mx2 = 0.f;
#pragma unroll
            for (int g = 0; g < UPT; ++g) {
                const int u4 = dq + g * TPR;
                if (u4 >= a.NC / 4) break;   // uniform across the warp
                float v0[4], v1[4];
                tmem_pair4(tmem + lane_q + uint32_t(4 * u4), tmem + lane_q + uint32_t(a.NC + 4 * u4), v0, v1);
                const int c0 = 4 * u4;
                if (!act || c0 >= n3) continue;
                uint32_t lo16[4], hi16[4], lb[4];
                const float4 cf4 = *reinterpret_cast<const float4 *>(csF + c0);
#pragma unroll
                for (int e2 = 0; e2 < 2; ++e2) {
                    // TwoSum of the accumulators, times the scales, times f (hi and lo)
                    const float2 a0 = make_float2(v0[2 * e2], v0[2 * e2 + 1]);
                    const float2 a1 = make_float2(v1[2 * e2], v1[2 * e2 + 1]);
                    const float2 fhh = make_float2(fh[g][2 * e2], fh[g][2 * e2 + 1]);
                    const float2 fll = make_float2(fl[g][2 * e2], fl[g][2 * e2 + 1]);
                    const float2 scl = __fmul2_rn(f2(rs_f), e2 ? make_float2(cf4.z, cf4.w) : make_float2(cf4.x, cf4.y));
                    const float2 h0 = __fadd2_rn(a0, a1);
                    const float2 bp = sub2(h0, a0);
                    const float2 l0 = __fmul2_rn(__fadd2_rn(sub2(a0, sub2(h0, bp)), sub2(a1, bp)), scl);
                    const float2 h = __fmul2_rn(h0, scl);
                    const float2 prh = __fmul2_rn(h, fhh);   // zero past n3 (f = 0 there)
                    const float2 prl = __fadd2_rn(__ffma2_rn(h, fhh, __fmul2_rn(prh, f2(-1.f))),
                                                  __ffma2_rn(h, fll, __fmul2_rn(l0, fhh)));
                    const float ph[2] = {prh.x, prh.y}, pl[2] = {prl.x, prl.y};
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const int e = 2 * e2 + q;
                        mx2 = fmaxf(mx2, fabsf(ph[q]));
                        const uint32_t hb = __float_as_uint(ph[q]);
                        lo16[e] = hb & 0xffffu;
                        hi16[e] = hb >> 16;
                        lb[e] = uint32_t(__bfloat16_as_ushort(__float2bfloat16_rn(pl[q])));
                    }
                }
                const uint32_t o = img_at(row, c0 >> 3, sbo) + uint32_t(c0 & 7) * 2u;
                *reinterpret_cast<uint2 *>(sA + o) = make_uint2(lo16[0] | (lo16[1] << 16), lo16[2] | (lo16[3] << 16));
                *reinterpret_cast<uint2 *>(sA + a_piece + o) =
                    make_uint2(hi16[0] | (hi16[1] << 16), hi16[2] | (hi16[3] << 16));
                *reinterpret_cast<uint2 *>(sA + 2 * a_piece + o) =
                    make_uint2(lb[0] | (lb[1] << 16), lb[2] | (lb[3] << 16));
            }
            tc::tc_fence_before();
            row_scales(rowmax(mx2), sc, inv);
            const float rs_i = inv;
            if (act) {
#pragma unroll
                for (int g = 0; g < UPT; ++g) {
                    const int c0 = 4 * (dq + g * TPR);
                    if (c0 >= n3) continue;
                    const uint32_t o = img_at(row, c0 >> 3, sbo) + uint32_t(c0 & 7) * 2u;
                    const uint2 wl = *reinterpret_cast<const uint2 *>(sA + o);
                    const uint2 wh = *reinterpret_cast<const uint2 *>(sA + a_piece + o);
                    const uint2 wb = *reinterpret_cast<const uint2 *>(sA + 2 * a_piece + o);
                    const uint32_t lw[4] = {wl.x & 0xffffu, wl.x >> 16, wl.y & 0xffffu, wl.y >> 16};
                    const uint32_t hw[4] = {wh.x & 0xffffu, wh.x >> 16, wh.y & 0xffffu, wh.y >> 16};
                    const uint32_t bw[4] = {wb.x & 0xffffu, wb.x >> 16, wb.y & 0xffffu, wb.y >> 16};
                    float h[4], l[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        h[e] = __uint_as_float((hw[e] << 16) | lw[e]);
                        l[e] = __uint_as_float(bw[e] << 16);
                    }
                    store_digits4(sA, a_piece, o, h, l, sc);
                }
            }
            if (handoff()) break;
            z_load_tile<TPR, UPT>(a, tile + gridDim.x, row, dq, x);   // the next tile, while the inverse GEMM runs
            wait_d();
            // ---- inverse result -> (r, z) of the output field ----
            float *dst = a.out + size_t(p) * a.N + r;
#pragma unroll
            for (int g = 0; g < UPT; ++g) {
                const int u4 = dq + g * TPR;
                if (u4 >= a.NC / 4) break;
                float v[4];
                tmem_unit(tmem + lane_q + uint32_t(4 * u4), tmem + lane_q + uint32_t(a.NC + 4 * u4), rs_i, csI + 4 * u4, v);
                if (!act) continue;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int z = 4 * u4 + e;
                    if (z < n3) dst[size_t(z) * R] = v[e];
                }
            }
            tc::tc_fence_before();
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (tid == 0 && *sflag) atomicExch(a.err, 1);
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, uint32_t(a.tmem_cols));
    }
}

// ---- host: matrix images -----------------------------------------------------------------
// Image of C(n, k), n < nout rows (outputs), k < nk (contraction), in a WN x Kp block of
// rows n0.. and contraction indices k0..: 4 base-512 digit planes (every row scaled by the
// largest entry of the whole row, so the K-chunks of a row share one scale), then WN column
// scales (the inverse row scales).
template <class Coef>
void build_block(uint8_t *img, int WN, int Kp, int n0, int nout, int nk, Coef coef, int k0 = 0)
{
    const uint32_t sbo = uint32_t(Kp) * 16u;
    const size_t piece = size_t(WN) * Kp * 2;
    std::vector<float> cs(WN, 1.0f);
    for (int n = 0; n < WN; ++n) {
        const int gn = n0 + n;
        if (gn >= nout) continue;
        double mx = 0.0;
        for (int k = 0; k < nk; ++k) mx = std::max(mx, std::fabs(coef(gn, k)));
        int e = 0;
        if (mx > 0.0) std::frexp(mx, &e);
        const double sc = std::ldexp(1.0, 8 - e);
        cs[n] = float(std::ldexp(1.0, e - 8));
        for (int k = k0; k < std::min(nk, k0 + Kp); ++k) {
            double t = coef(gn, k) * sc;
            const int kl = k - k0;
            for (int q = 0; q < kMatDig; ++q) {   // t = p0 + p1 2^-9 + p2 2^-18 + p3 2^-27
                const double dq = std::nearbyint(t);
                const float v = float(std::ldexp(dq, -9 * q));   // |dq| <= 256: exact in bf16
                uint32_t u;
                std::memcpy(&u, &v, 4);
                const uint16_t hb = uint16_t(u >> 16);
                std::memcpy(img + piece * q + img_at(n, kl / 8, sbo) + size_t(kl % 8) * 2, &hb, 2);
                t = (t - dq) * 512.0;
            }
        }
    }
    std::memcpy(img + piece * kMatDig, cs.data(), size_t(WN) * 4);
}

struct SliceLayout {
    size_t smem;
    uint32_t offB2, offA, offA2, offY, offRs, offBar, a_piece1, a_piece2, offS, stg_plane;
    int G, Pj, tmem_cols, stage, pipe, t2col;
    int bstream, KC, nkc1, nkc2;
    uint32_t offCS, buf_bytes, chunk1_bytes, chunk2_bytes;
};

// pair: pass A (two staged planes) or pass C (one).  pipe: separate A images and TMEM
// columns for the two GEMMs (software pipeline over tiles, one CTA per SM with staging).
// bstream: the x/y matrix images stream through two buffers as K-chunks of KC (for slices whose
// resident images do not fit next to the A images and the transposed tile).
SliceLayout slice_layout_for(const Plan &P, bool pair, bool pipe, bool bstream = false, int KC = 0)
{
    SliceLayout L{};
    const int n1 = P.n[0], n2 = P.n[1];
    const int Kp1 = pad16i(n1), Kp2 = pad16i(n2);
    L.G = kRows / std::max(n1, n2);
    L.Pj = (n2 + 3) & ~3;
    if (((L.Pj / 4) & 1) == 0) L.Pj += 4;   // odd number of 16-byte units: conflict-free rows
    const bool share = P.t3_share01 != 0;
    size_t off;
    L.offB2 = 0;
    if (bstream) {
        L.bstream = 1;
        L.KC = KC;
        L.nkc1 = (Kp1 + KC - 1) / KC;
        L.nkc2 = (Kp2 + KC - 1) / KC;
        L.chunk1_bytes = uint32_t(mat_image_bytes(Kp1, KC));
        L.chunk2_bytes = uint32_t(mat_image_bytes(Kp2, KC));
        L.buf_bytes = uint32_t(align_up(std::max(L.chunk1_bytes, L.chunk2_bytes), 1024));
        off = 2 * size_t(L.buf_bytes);
    } else {
        off = mat_image_bytes(Kp1, Kp1);
        if (!share) {
            off = align_up(off, 1024);
            L.offB2 = uint32_t(off);
            off += mat_image_bytes(Kp2, Kp2);
        }
    }
    off = align_up(off, 1024);
    L.offA = uint32_t(off);
    const int R1 = L.G * n2, R2 = L.G * n1;
    L.a_piece1 = uint32_t(pad8i(R1)) * Kp1 * 2u;
    L.a_piece2 = uint32_t(pad8i(R2)) * Kp2 * 2u;
    // the MMA reads 128 rows of every digit plane: the last plane's reach past the image
    // must stay inside this CTA's shared memory (rows past the tile are never read back)
    const size_t reach1 = 2 * size_t(L.a_piece1) + size_t(kRows) * Kp1 * 2;
    const size_t reach2 = 2 * size_t(L.a_piece2) + size_t(kRows) * Kp2 * 2;
    size_t end_reach;
    if (pipe) {
        L.offA2 = uint32_t(align_up(L.offA + 3 * size_t(L.a_piece1), 1024));
        off = L.offA2 + 3 * size_t(L.a_piece2);
        end_reach = std::max(L.offA + reach1, L.offA2 + reach2);
    } else {
        L.offA2 = L.offA;
        off += std::max(3 * size_t(L.a_piece1), 3 * size_t(L.a_piece2));
        end_reach = L.offA + std::max(reach1, reach2);
    }
    L.offY = uint32_t(align_up(off, 16));
    off = L.offY + (size_t(L.G) * n1 * L.Pj + 8) * 4;
    off = std::max(off, end_reach);
    L.offRs = uint32_t(align_up(off, 16));
    off = L.offRs + 2 * kRows * 4;
    L.offCS = uint32_t(align_up(off, 16));   // column scales of streamed images
    off = L.offCS + size_t(Kp1 + Kp2) * 4;
    L.offBar = uint32_t(align_up(off, 16));
    off = L.offBar + 128;                      // 9 mbarriers, the TMEM slot, the error flag
    // staging of the tile's input slices, when rows of slices are 16-byte aligned
    const long R = long(n1) * n2;
    L.stg_plane = uint32_t(align_up(size_t(L.G) * R * 4, 128));
    L.offS = uint32_t(align_up(off, 128));
    const size_t with_stage = L.offS + size_t(pair ? 2 : 1) * L.stg_plane;
    // staging hides the load latency of one CTA per SM; a second CTA per SM hides it too,
    // so the buffer is used only where it does not cost that second CTA (and always when
    // pipelined: one CTA per SM by design)
    const size_t two_per_sm = 233472 / 2 - 1024;
    L.stage = (R % 4 == 0 && with_stage <= kSmemLimit &&
               (pipe || with_stage <= two_per_sm || off > two_per_sm)) ? 1 : 0;
    if (P.t3_stage >= 0) L.stage = (P.t3_stage && R % 4 == 0 && with_stage <= kSmemLimit) ? 1 : 0;   // tuned
    if (bstream) L.stage = 0;   // the producer warp streams the matrices instead
    L.smem = L.stage ? with_stage : off;
    L.pipe = pipe ? 1 : 0;
    L.t2col = pipe ? 2 * Kp1 : 0;
    L.tmem_cols = tmem_pow2(pipe ? 2 * Kp1 + 2 * Kp2 : 2 * std::max(Kp1, Kp2));
    return L;
}

// The plan's choice: pipelined when tuned so, or (automatic) when it fits and the serial form
// cannot run two CTAs per SM.
SliceLayout slice_layout(const Plan &P, bool pair = true)
{
    const SliceLayout ser = slice_layout_for(P, pair, false);
    const SliceLayout pip = slice_layout_for(P, pair, true);
    const bool pip_ok = pip.smem <= kSmemLimit && pip.tmem_cols <= 512;
    if (ser.smem > kSmemLimit && !pip_ok) {
        // the resident images do not fit: stream them, widest chunk first (serial form)
        for (int KC : {64, 48, 32, 16}) {
            const SliceLayout b = slice_layout_for(P, pair, false, true, KC);
            if (b.smem <= kSmemLimit) return b;
        }
        return ser;   // unsupported: tc3_supported reports it
    }
    if (P.t3_pipe == 1 && pip_ok) return pip;
    if (P.t3_pipe == 0 || !pip_ok) return ser;
    const bool ser_two = ser.smem + 1024 <= 233472 / 2 && ser.tmem_cols <= 256;
    return ser_two ? ser : pip;
}

struct ZLayout {
    size_t smem;
    uint32_t offB, offCs, offMax, offBar, blk_bytes;
    int NB, WN, NC, nbuf, resident, tmem_cols, kchunk, KC;
};

constexpr int kTPRz = 4;
constexpr int kTPRs = 4;

// Matrix blocks of pass B.  All 2 NB output blocks resident when they fit; else streamed
// through 2 (or 3) buffers, as K-chunks (every MMA covers all NC outputs, so the A image is
// read once per K-step and digit product) or as output blocks (WN outputs, the full K).
// want_wn > 0 asks for output blocks of want_wn columns, want_wn < 0 for K-chunks of
// -want_wn contraction indices, with want_nbuf buffers; 0 = the first that fits in the order
// resident, K-chunks / 2 buffers, output blocks / 2, K-chunks / 3, output blocks / 3.
bool z_layout(int n3, ZLayout &L, int want_wn = 0, int want_nbuf = 0)
{
    const int Kp = pad16i(n3);
    const size_t abytes = 3 * size_t(kRows) * Kp * 2;
    auto fits = [&](int NB, int WN, int NC, int kchunk, int KC, int nbuf, int resident) {
        const size_t blk = kchunk ? mat_image_bytes(NC, KC) : mat_image_bytes(WN, Kp);
        size_t off = align_up(abytes, 1024);
        const uint32_t offB = uint32_t(off);
        off += size_t(nbuf) * blk;
        const uint32_t offCs = uint32_t(align_up(off, 16));
        off = offCs + 2 * size_t(NC) * 4;
        const uint32_t offMax = uint32_t(align_up(off, 16));
        off = offMax + size_t(kTPRz) * kRows * 4;
        const uint32_t offBar = uint32_t(align_up(off, 16));
        off = offBar + 16 + 16 * size_t(nbuf) + 16;
        if (off > kSmemLimit || 2 * NC > 512) return false;
        L = {off, offB, offCs, offMax, offBar, uint32_t(blk), NB, WN, NC, nbuf, resident, tmem_pow2(2 * NC),
             kchunk, KC};
        return true;
    };
    for (int pass = 0; pass < 5; ++pass) {
        const bool chunk = pass == 1 || pass == 3;
        const int nbuf_s = pass <= 2 ? 2 : 3;
        for (int NB = 1; NB <= 16; ++NB) {
            if (chunk) {
                if (NB < 2) continue;
                const int KC = pad16i((Kp + NB - 1) / NB);
                if (KC * (NB - 1) >= Kp) continue;   // no empty chunk
                if (nbuf_s >= 2 * NB) continue;
                if (want_wn && (want_wn != -KC || want_nbuf != nbuf_s)) continue;
                if (fits(NB, Kp, Kp, 1, KC, nbuf_s, 0)) return true;
            } else {
                const int WN = pad16i((n3 + NB - 1) / NB);
                if (WN * (NB - 1) >= n3) continue;   // no empty block
                const int nbuf = pass == 0 ? 2 * NB : nbuf_s;
                if (pass > 0 && nbuf >= 2 * NB) continue;
                if (want_wn && (WN != want_wn || nbuf != want_nbuf)) continue;   // a tuned choice
                if (fits(NB, WN, NB * WN, 0, 0, nbuf, pass == 0 ? 1 : 0)) return true;
            }
        }
    }
    return false;
}

}  // namespace

// The (block width, buffers) choices of pass B that fit for an axis of n3 points; a
// negative width is a K-chunk of that many contraction indices.
std::vector<std::pair<int, int>> tc3_z_choices(int n3)
{
    std::vector<std::pair<int, int>> out;
    const int Kp = pad16i(n3);
    for (int NB = 1; NB <= 16; ++NB) {
        const int WN = pad16i((n3 + NB - 1) / NB);
        const int KC = pad16i((Kp + NB - 1) / NB);
        for (int nbuf : {2 * NB, 2, 3})
            for (int w : {WN, -KC}) {
                ZLayout L;
                if (z_layout(n3, L, w, nbuf)) {
                    std::pair<int, int> c{L.kchunk ? -L.KC : L.WN, L.nbuf};
                    if (std::find(out.begin(), out.end(), c) == out.end()) out.push_back(c);
                }
            }
    }
    return out;
}

namespace {

// Units of 4 grid points per thread and row in pass B, from a few compiled widths.
int z_upt(int n3)
{
    const int need = ((n3 + 3) / 4 + kTPRz - 1) / kTPRz;
    for (int u : {2, 3, 4, 6, 9, 13})
        if (need <= u) return u;
    return 0;
}

// CTAs per SM from the SM's limits (registers in 256-register warp units, shared memory with
// the driver's 1 KB per CTA, threads) and TMEM columns; the shared-memory request is raised
// so that no more CTAs than TMEM allows become resident (an allocation would otherwise wait).
template <class K>
int launch_setup(K kern, int threads, size_t &smem, int tmem_cols, int &per_sm)
{
    const int max_ctas = std::max(1, 512 / tmem_cols);
    const size_t sm_total = 233472;
    smem = std::max(smem, sm_total / size_t(max_ctas + 1) - 1024 + 64);
    smem = std::min(smem, kSmemLimit);
    EXX_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    // all of the unified L1 / shared memory as shared memory, so that two CTAs of ~100 KB fit
    EXX_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    cudaFuncAttributes fa{};
    EXX_CUDA(cudaFuncGetAttributes(&fa, kern));
    const int warps = (threads + 31) / 32;
    const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;
    const int by_regs = 65536 / std::max(1, regs_warp * warps);
    const int by_smem = int(sm_total / (smem + 1024));
    const int by_threads = 2048 / threads;
    per_sm = std::max(1, std::min({by_regs, by_smem, by_threads, max_ctas}));
    return EXX_OK;
}

}  // namespace

bool tc3_supported(const Plan &P, std::string *why)
{
    if (std::max(P.n[0], P.n[1]) > kRows) {
        if (why) *why = "BF16X7: the x and y axes must have at most 128 points (a z-slice per GEMM tile)";
        return false;
    }
    const SliceLayout L = slice_layout(P, false);
    if (L.smem > kSmemLimit) {
        if (why) *why = "BF16X7: the x/y operand images exceed shared memory for this grid";
        return false;
    }
    ZLayout Z;
    if (!z_layout(P.n[2], Z) || z_upt(P.n[2]) == 0) {
        if (why) *why = "BF16X7: the z axis is too long for the on-chip operand images";
        return false;
    }
    return true;
}

int tc3_upload(Plan &P)
{
    std::string why;
    P.t3_share01 = (P.n[0] == P.n[1] && P.bc[0] == P.bc[1]) ? 1 : 0;
    if (!tc3_supported(P, &why)) {
        set_error(why);
        return EXX_ERR_UNSUPPORTED;
    }
    // x and y: one block each, forward C(n, k) = V(k, n) and inverse C(n, k) = V(n, k)
    for (int d = 0; d < 2; ++d) {
        const int nd = P.n[d], Kp = pad16i(nd);
        const std::vector<double> &V = P.V[d];
        for (int inv = 0; inv < 2; ++inv) {
            std::vector<uint8_t> img(mat_image_bytes(Kp, Kp), 0);
            build_block(img.data(), Kp, Kp, 0, nd, nd, [&](int n, int k) {
                return inv ? V[size_t(n) + size_t(nd) * k] : V[size_t(k) + size_t(nd) * n];
            });
            DevBuf &b = P.t3img[d][inv];
            if (int rc = dev_reserve(b, img.size())) return rc;
            EXX_CUDA(cudaMemcpy(b.p, img.data(), img.size(), cudaMemcpyHostToDevice));
        }
    }
    // x and y as K-chunks when the slice passes stream them (every chunk: all outputs)
    {
        const SliceLayout L = slice_layout(P, true);
        if (L.bstream)
            for (int d = 0; d < 2; ++d) {
                const int nd = P.n[d], Kp = pad16i(nd), nkc = (Kp + L.KC - 1) / L.KC;
                const size_t cb = mat_image_bytes(Kp, L.KC);
                const std::vector<double> &V = P.V[d];
                for (int inv = 0; inv < 2; ++inv) {
                    std::vector<uint8_t> img(size_t(nkc) * cb, 0);
                    auto coef = [&](int n, int k) {
                        return inv ? V[size_t(n) + size_t(nd) * k] : V[size_t(k) + size_t(nd) * n];
                    };
                    for (int kc = 0; kc < nkc; ++kc) build_block(img.data() + size_t(kc) * cb, Kp, L.KC, 0, nd, nd, coef, kc * L.KC);
                    DevBuf &b = P.t3imgc[d][inv];
                    if (int rc = dev_reserve(b, img.size())) return rc;
                    EXX_CUDA(cudaMemcpy(b.p, img.data(), img.size(), cudaMemcpyHostToDevice));
                }
            }
    }
    // z: NB blocks of WN outputs each
    ZLayout Z;
    if (!z_layout(P.n[2], Z, P.t3_zwn, P.t3_znbuf)) z_layout(P.n[2], Z);
    {
        const int nd = P.n[2], Kp = pad16i(nd);
        const std::vector<double> &V = P.V[2];
        for (int inv = 0; inv < 2; ++inv) {
            std::vector<uint8_t> img(size_t(Z.NB) * Z.blk_bytes, 0);
            auto coef = [&](int n, int k) {
                return inv ? V[size_t(n) + size_t(nd) * k] : V[size_t(k) + size_t(nd) * n];
            };
            for (int nb = 0; nb < Z.NB; ++nb) {
                uint8_t *dst = img.data() + size_t(nb) * Z.blk_bytes;
                if (Z.kchunk)   // all outputs, contraction indices nb KC ..
                    build_block(dst, Z.NC, Z.KC, 0, nd, nd, coef, nb * Z.KC);
                else
                    build_block(dst, Z.WN, Kp, nb * Z.WN, nd, nd, coef);
            }
            DevBuf &b = P.t3img[2][inv];
            if (int rc = dev_reserve(b, img.size())) return rc;
            EXX_CUDA(cudaMemcpy(b.p, img.data(), img.size(), cudaMemcpyHostToDevice));
        }
    }
    // f(Lambda) in the natural layout as FP32 hi and lo planes
    {
        std::vector<float> fl(2 * size_t(P.N));
        for (size_t i = 0; i < size_t(P.N); ++i) {
            const float h = float(P.F[i]);
            fl[i] = h;
            fl[size_t(P.N) + i] = float(P.F[i] - double(h));
        }
        if (int rc = dev_reserve(P.F32n, fl.size() * sizeof(float))) return rc;
        EXX_CUDA(cudaMemcpy(P.F32n.p, fl.data(), fl.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    if (int rc = dev_reserve(P.err_d, 16)) return rc;
    EXX_CUDA(cudaMemset(P.err_d.p, 0, 16));
    return EXX_OK;
}

// One batch: pass A (bufA), pass B (bufB), pass C (bufA); the solutions end in bufA.
int tc3_solve_batch(Plan &P, const int2 *pairs_d, int nfields, float *bufA, float *bufB, cudaStream_t s)
{
    const int n1 = P.n[0], n2 = P.n[1], n3 = P.n[2];
    // passes A and C
    auto slice = [&](bool pair, const float *in, float *out, int kind) -> int {
        const SliceLayout L = slice_layout(P, pair);
        SliceArgs a{};
        a.n1 = n1;
        a.n2 = n2;
        a.n3 = n3;
        a.G = L.G;
        a.tpf = (n3 + L.G - 1) / L.G;
        a.ntiles = long(nfields) * a.tpf;
        a.N = P.N;
        a.psi = static_cast<const float *>(P.psi32.p);
        a.occ_off = P.tc_occ_off;
        a.pairs = pairs_d;
        a.in = in;
        a.out = out;
        const int inv = pair ? 0 : 1;
        a.img1 = static_cast<const uint8_t *>(P.t3img[0][inv].p);
        a.img2 = static_cast<const uint8_t *>(P.t3img[1][inv].p);
        a.Kp1 = pad16i(n1);
        a.Kp2 = pad16i(n2);
        a.img1_bytes = uint32_t(mat_image_bytes(a.Kp1, a.Kp1));
        a.img2_bytes = uint32_t(mat_image_bytes(a.Kp2, a.Kp2));
        a.offB2 = L.offB2;
        a.offA = L.offA;
        a.offY = L.offY;
        a.offRs = L.offRs;
        a.offBar = L.offBar;
        a.a_piece1 = L.a_piece1;
        a.a_piece2 = L.a_piece2;
        a.Pj = L.Pj;
        a.tmem_cols = L.tmem_cols;
        a.vec = ((n1 & 3) == 0 && (P.N & 3) == 0) ? 1 : 0;
        a.stage = L.stage;
        a.offS = L.offS;
        a.stg_plane = L.stg_plane;
        a.pipe = L.pipe;
        a.offA2 = L.offA2;
        a.t2col = L.t2col;
        a.bstream = L.bstream;
        a.KC = L.KC;
        a.nkc1 = L.nkc1;
        a.nkc2 = L.nkc2;
        a.offCS = L.offCS;
        a.buf_bytes = L.buf_bytes;
        a.chunk1_bytes = L.chunk1_bytes;
        a.chunk2_bytes = L.chunk2_bytes;
        a.img1c = static_cast<const uint8_t *>(P.t3imgc[0][inv].p);
        a.img2c = static_cast<const uint8_t *>(P.t3imgc[1][inv].p);
        a.err = static_cast<int *>(P.err_d.p);
        size_t smem = L.smem;
        auto kern = pair ? slice_pass_kernel<true, kTPRs> : slice_pass_kernel<false, kTPRs>;
        const int threads = kRows * kTPRs + 64;
        int per_sm = 1;
        if (int rc = launch_setup(kern, threads, smem, L.tmem_cols, per_sm)) return rc;
        const int grid = int(std::min<long>(a.ntiles, long(P.num_sms) * per_sm));
        const int tb = timing_begin(P, kind, s);
        kern<<<grid, threads, smem, s>>>(a);
        timing_end(P, tb, s);
        EXX_LAUNCH("slice_pass_kernel");
        P.launches++;
        return EXX_OK;
    };
    if (int rc = slice(true, nullptr, bufA, EXX_TIMING_PASS1)) return rc;
    // pass B
    {
        ZLayout Z;
        if (!z_layout(n3, Z, P.t3_zwn, P.t3_znbuf)) z_layout(n3, Z);
        ZArgs a{};
        a.R = n1 * n2;
        a.tpfz = (a.R + kRows - 1) / kRows;
        a.ntiles = long(nfields) * a.tpfz;
        a.n3 = n3;
        a.Kp = pad16i(n3);
        a.N = P.N;
        a.in = bufA;
        a.out = bufB;
        a.Fh = static_cast<const float *>(P.F32n.p);
        a.Fl = a.Fh + P.N;
        a.imgF = static_cast<const uint8_t *>(P.t3img[2][0].p);
        a.imgI = static_cast<const uint8_t *>(P.t3img[2][1].p);
        a.blk_bytes = Z.blk_bytes;
        a.NB = Z.NB;
        a.WN = Z.WN;
        a.NC = Z.NC;
        a.kchunk = Z.kchunk;
        a.KC = Z.KC;
        a.nbuf = Z.nbuf;
        a.resident = Z.resident;
        a.offB = Z.offB;
        a.offCs = Z.offCs;
        a.offMax = Z.offMax;
        a.offBar = Z.offBar;
        a.tmem_cols = Z.tmem_cols;
        a.err = static_cast<int *>(P.err_d.p);
        void (*kern)(const ZArgs) = nullptr;
        switch (z_upt(n3)) {
        case 2: kern = zpass_kernel<kTPRz, 2>; break;
        case 3: kern = zpass_kernel<kTPRz, 3>; break;
        case 4: kern = zpass_kernel<kTPRz, 4>; break;
        case 6: kern = zpass_kernel<kTPRz, 6>; break;
        case 9: kern = zpass_kernel<kTPRz, 9>; break;
        default: kern = zpass_kernel<kTPRz, 13>; break;
        }
        const int threads = kRows * kTPRz + 64;
        size_t smem = Z.smem;
        int per_sm = 1;
        if (int rc = launch_setup(kern, threads, smem, Z.tmem_cols, per_sm)) return rc;
        const int grid = int(std::min<long>(a.ntiles, long(P.num_sms) * per_sm));
        const int tb = timing_begin(P, EXX_TIMING_PASS3, s);
        kern<<<grid, threads, smem, s>>>(a);
        timing_end(P, tb, s);
        EXX_LAUNCH("zpass_kernel");
        P.launches++;
    }
    if (int rc = slice(false, bufB, bufA, EXX_TIMING_PASS5)) return rc;
    P.tc_result = bufA;
    return EXX_OK;
}

// Host only: the automatic BF16X7 layouts of an n1 x n2 x n3 grid (no device involved).
// out[0] supported; [1] [2] shared memory of pass A / pass C; [3] [4] pass A streams its x/y
// matrices, chunk width; [5] [6] the same for pass C; [7] pass A pipelined, [8] staged;
// [9] pass B shared memory (0: none fits); [10] pass B K-chunks; [11] chunk or block width;
// [12] buffers; [13] resident; [14] units per thread; [15] the shared-memory limit.
void tc3_debug_layout(int n1, int n2, int n3, int share01, int *out)
{
    Plan P;
    P.n[0] = n1;
    P.n[1] = n2;
    P.n[2] = n3;
    P.t3_share01 = share01;
    std::string why;
    out[0] = tc3_supported(P, &why) ? 1 : 0;
    const SliceLayout A = slice_layout(P, true), C = slice_layout(P, false);
    out[1] = int(A.smem);
    out[2] = int(C.smem);
    out[3] = A.bstream;
    out[4] = A.KC;
    out[5] = C.bstream;
    out[6] = C.KC;
    out[7] = A.pipe;
    out[8] = A.stage;
    ZLayout Z{};
    const bool zok = z_layout(n3, Z);
    out[9] = zok ? int(Z.smem) : 0;
    out[10] = Z.kchunk;
    out[11] = Z.kchunk ? Z.KC : Z.WN;
    out[12] = Z.nbuf;
    out[13] = Z.resident;
    out[14] = z_upt(n3);
    out[15] = int(kSmemLimit);
}

// Host only: the digit image of C(n, k) (row-major nout x nk, HOST) in a WN x Kp block of rows
// n0.. and contraction indices k0.., decoded back to values: digits[q][n][k] (the weighted
// digit q of row n, index k of the block) and the WN column scales.
void tc3_debug_matrix_digits(int nout, int nk, const double *C, int WN, int Kp, int n0, int k0, float *digits,
                             float *scales)
{
    std::vector<uint8_t> img(mat_image_bytes(WN, Kp), 0);
    build_block(img.data(), WN, Kp, n0, nout, nk, [&](int n, int k) { return C[size_t(n) * nk + k]; }, k0);
    const size_t piece = size_t(WN) * Kp * 2;
    const uint32_t sbo = uint32_t(Kp) * 16u;
    for (int q = 0; q < kMatDig; ++q)
        for (int n = 0; n < WN; ++n)
            for (int k = 0; k < Kp; ++k) {
                uint16_t hb;
                std::memcpy(&hb, img.data() + piece * q + img_at(n, k / 8, sbo) + size_t(k % 8) * 2, 2);
                const uint32_t u = uint32_t(hb) << 16;
                std::memcpy(digits + (size_t(q) * WN + n) * Kp + k, &u, 4);
            }
    std::memcpy(scales, img.data() + piece * kMatDig, size_t(WN) * 4);
}

}  // namespace exx
