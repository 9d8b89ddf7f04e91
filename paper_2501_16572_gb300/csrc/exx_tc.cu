// Split-precision path of the batched Kronecker solve on the tcgen05 tensor cores.
//
// Each mode product of Sec. II.B is a GEMM  D[row][n] = sum_k A[row][k] B[n][k]  where a
// row is a pencil of the grid function along the contracted axis (128 rows per tile,
// one row per thread, one TMEM lane per row) and B is the 1D eigenvector matrix (or its
// transpose).  Two ways of splitting the FP32 operands are built:
//
//  * Fixed-point bf16 slices (BF16X3: 2 slices, BF16X6: 3 slices).  Every row of A and
//    every row of B gets a power-of-two scale from its largest entry, and the scaled
//    row is cut into slices x = 2^(e-7) (q0 + q1/2^8 + q2/2^16) with integers q_i of at
//    most 8 bits; slice i is stored as q_i 2^(-8i), exact in bf16.  Slice products of one
//    "level" (i + j = l) share the weight 2^(-8l), so each level is summed in its own TMEM
//    accumulator as 2^(-8l) times an integer below 2^24: the tensor core never rounds.
//    The levels are added and rescaled in FP32 in the epilogue.  The result is the fixed-point product to about 2^-8S of the row maxima,
//    with round-to-nearest slicing and no directed rounding anywhere.
//  * Floating tf32 split (TF32X3): x = x0 + x1 with x0 = tf32(x), x1 = tf32(x - x0), the
//    three leading cross products accumulated in one FP32 accumulator.  The tensor core
//    rounds its FP32 accumulation toward zero, which biases every product slightly
//    toward zero; this form is kept for comparison.
//
// The pair density psi_m psi_n is formed in the prologue from compensated FP32 copies of
// the orbitals (hi + lo), the Hadamard scaling by f(Lambda) sits between the forward and
// inverse y products of pass 3 (both on-chip), and the accumulation over pairs is a
// separate compensated FP32 kernel.
#include "exx_internal.h"
#include "tc_ptx.cuh"

#include <cuda.h>   // CUtensorMap and its enums (the encoder is fetched at run time)
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

namespace exx {

namespace {

constexpr int kRows = 128;          // tile rows = TMEM lanes = threads
constexpr uint32_t kWaitLimit = 1u << 22;

enum { MODE_FLOAT_TF32 = 0, MODE_FIXED_BF16 = 1 };

struct PrecInfo {
    int mode;
    int S;           // pieces (float) or slices (fixed) of the data operand A
    int SB;          // pieces / slices of the matrix operand B
    int es;          // bytes per element
    int nacc;        // TMEM accumulators per GEMM
    int hl;          // intermediates between passes kept as hi + lo FP32 pairs
};
// BF16X6 carries the matrices with a fourth slice, used only against the leading data
// slice: the matrices are shared by every pair, so their representation error does not
// average out over pairs the way the data's does.
__host__ __device__ inline PrecInfo prec_info(int prec)
{
    switch (prec) {
    case EXX_PREC_BF16X3: return {MODE_FIXED_BF16, 2, 2, 2, 2, 0};
    case EXX_PREC_BF16X6: return {MODE_FIXED_BF16, 3, 4, 2, 4, 0};
    case EXX_PREC_BF16X10: return {MODE_FIXED_BF16, 4, 4, 2, 4, 1};
    case EXX_PREC_BF16X7: return {MODE_FIXED_BF16, 3, 4, 2, 2, 0};   // three-pass kernels (exx_tc3.cu)
    default: return {MODE_FLOAT_TF32, 2, 2, 4, 1, 0};   // TF32X3
    }
}

inline int pad16(int n) { return (n + 15) & ~15; }
inline int pow2_cols(int c) { return c <= 32 ? 32 : c <= 64 ? 64 : c <= 128 ? 128 : c <= 256 ? 256 : 512; }

// bytes of one operand image: SB pieces of Np x Np, then (fixed mode) Np column scales
inline size_t image_bytes(int prec, int Np)
{
    const PrecInfo pi = prec_info(prec);
    size_t b = size_t(pi.SB) * Np * Np * pi.es;
    if (pi.mode == MODE_FIXED_BF16) b += size_t(Np) * 4;
    return (b + 127) & ~size_t(127);   // keeps the staging buffers behind the images 128-byte aligned
}

// canonical K-major no-swizzle image: byte offset of (row, 16-byte chunk c)
__host__ __device__ inline uint32_t img_off(int row, int c, uint32_t sbo)
{
    return uint32_t(row >> 3) * sbo + uint32_t(c) * 128u + uint32_t(row & 7) * 16u;
}

// ---- host rounding (round to nearest even) ----
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

// ---- device: operand pieces -------------------------------------------------------------
// Floating tf32 split of (hi + lo).
__device__ __forceinline__ void split_tf32(float hi, float lo, float (&p)[4])
{
    p[0] = tc::to_tf32(hi);
    p[1] = tc::to_tf32((hi - p[0]) + lo);
    p[2] = 0.f;
    p[3] = 0.f;
}

// Round x to the nearest multiple of 2^-G (ties to even) for |x| < 2^(22-G): adding
// 1.5 * 2^(23-G) leaves no bits below 2^-G, so the FP32 addition itself rounds; both
// additions stay on the FMA pipe.
template <int G>
__device__ __forceinline__ float round_grid(float x)
{
    constexpr float kMagic = 12582912.f / float(1u << G);
    return __fadd_rn(__fadd_rn(x, kMagic), -kMagic);
}

// Fixed-point slices of (hi + lo) * s, s = 2^(7 - e): q[i] = q_i 2^(-8i) with q_i an integer
// of at most 8 bits (balanced digits, each rounded to nearest).  Each residual r_i - q[i]
// is exact; only the first one absorbs lo.
template <int S>
__device__ __forceinline__ void slice_fixed(float hi, float lo, float s, float (&q)[4])
{
    const float t = hi * s;
    q[0] = round_grid<0>(t);
    const float r1 = fmaf(lo, s, t - q[0]);
    q[1] = (S >= 2) ? round_grid<8>(r1) : 0.f;
    const float r2 = r1 - q[1];
    q[2] = (S >= 3) ? round_grid<16>(r2) : 0.f;
    q[3] = (S >= 4) ? round_grid<24>(r2 - q[2]) : 0.f;
}

// Store one 16-byte chunk per piece: vals[q][e] for e < 16/ES elements of row `row`.
template <int ES, int S>
__device__ __forceinline__ void store_chunk(uint8_t *img, uint32_t piece_bytes, int row, int c, uint32_t sbo,
                                            const float (&vals)[4][8])
{
    const uint32_t off = img_off(row, c, sbo);
#pragma unroll
    for (int q = 0; q < S; ++q) {
        uint4 v;
        if (ES == 4) {
            v = make_uint4(__float_as_uint(vals[q][0]), __float_as_uint(vals[q][1]), __float_as_uint(vals[q][2]),
                           __float_as_uint(vals[q][3]));
        } else {
            uint32_t w[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                // values are bf16-exact (small integers or bf16-rounded): one packing cvt
                __nv_bfloat162 b2 = __floats2bfloat162_rn(vals[q][2 * t], vals[q][2 * t + 1]);
                w[t] = *reinterpret_cast<uint32_t *>(&b2);
            }
            v = make_uint4(w[0], w[1], w[2], w[3]);
        }
        *reinterpret_cast<uint4 *>(img + q * piece_bytes + off) = v;
    }
}

// Store one 4-element unit per piece: vals[q][e], elements 4u..4u+3 of row `row` (half a
// 16-byte core-matrix row for bf16, a whole one for tf32).
template <int ES, int S>
__device__ __forceinline__ void store_unit(uint8_t *img, uint32_t piece_bytes, int row, int u, uint32_t sbo,
                                           const float (&vals)[4][4])
{
#pragma unroll
    for (int q = 0; q < S; ++q) {
        if (ES == 4) {
            *reinterpret_cast<uint4 *>(img + q * piece_bytes + img_off(row, u, sbo)) =
                make_uint4(__float_as_uint(vals[q][0]), __float_as_uint(vals[q][1]), __float_as_uint(vals[q][2]),
                           __float_as_uint(vals[q][3]));
        } else {
            // the values have at most 8 significant bits (q_i 2^(-8i)), so their bf16 form is
            // the upper half of their FP32 bits: pack two with one byte permute
            const uint32_t w0 = __byte_perm(__float_as_uint(vals[q][0]), __float_as_uint(vals[q][1]), 0x7632);
            const uint32_t w1 = __byte_perm(__float_as_uint(vals[q][2]), __float_as_uint(vals[q][3]), 0x7632);
            *reinterpret_cast<uint2 *>(img + q * piece_bytes + img_off(row, u >> 1, sbo) + (u & 1) * 8) =
                make_uint2(w0, w1);
        }
    }
}

// Issue one GEMM into the accumulator(s) starting at TMEM column `d`.  Fixed mode:
// level l < S holds the products (i, l - i); level S (when SB > S) the product (0, S).
template <int MODE, int S, int SB>
__device__ __forceinline__ void issue_gemm(uint32_t d, int Np, uint32_t a_base, uint32_t a_piece, uint32_t b_base,
                                           uint32_t b_piece, uint32_t sbo, int ksteps, uint32_t idesc)
{
    if (MODE == MODE_FLOAT_TF32) {
        const int PA[3] = {1, 0, 0}, PB[3] = {0, 1, 0};   // small terms first
        uint32_t acc = 0;
        for (int t = 0; t < 3; ++t)
            for (int ks = 0; ks < ksteps; ++ks) {
                uint64_t ad = tc::smem_desc(a_base + PA[t] * a_piece + ks * 256u, 128u, sbo);
                uint64_t bd = tc::smem_desc(b_base + PB[t] * b_piece + ks * 256u, 128u, sbo);
                tc::mma_tf32(d, ad, bd, idesc, acc);
                acc = 1;
            }
    } else {
        // k-step outermost, then level: consecutive MMAs accumulate into different TMEM
        // accumulators instead of forming one dependent chain
        for (int ks = 0; ks < ksteps; ++ks) {
            for (int l = 0; l < S; ++l) {
                for (int i = 0; i <= l; ++i) {
                    const int j = l - i;
                    uint64_t ad = tc::smem_desc(a_base + i * a_piece + ks * 256u, 128u, sbo);
                    uint64_t bd = tc::smem_desc(b_base + j * b_piece + ks * 256u, 128u, sbo);
                    tc::mma_bf16(d + uint32_t(l * Np), ad, bd, idesc, (ks > 0 || i > 0) ? 1u : 0u);
                }
            }
            if (SB > S) {
                uint64_t ad = tc::smem_desc(a_base + ks * 256u, 128u, sbo);
                uint64_t bd = tc::smem_desc(b_base + S * b_piece + ks * 256u, 128u, sbo);
                tc::mma_bf16(d + uint32_t(S * Np), ad, bd, idesc, ks > 0 ? 1u : 0u);
            }
        }
    }
}

// Read 4 result columns [c0, c0+4) of this thread's row: add the NACC levels (level l holds
// its weight 2^(-8 l) already) and apply the row and column scales.  All level loads are
// issued before one tcgen05.wait::ld.  With HL the value is returned as an unevaluated
// sum vh + vl: level 0 is an exact integer, the lower levels are folded into t, and
// TwoSum keeps the rounding error of l0 + t (the scales are powers of two, exact).
template <int MODE, int NACC, bool HL>
__device__ __forceinline__ void read4(uint32_t d, int Np, int c0, float rs, const float *cs, float (&vh)[4],
                                      float (&vl)[4])
{
    uint32_t r[NACC][4];
#pragma unroll
    for (int l = 0; l < NACC; ++l) tc::tmem_ld4_issue(d + uint32_t(l * Np + c0), r[l]);
    tc::tmem_wait_ld();
#pragma unroll
    for (int l = 0; l < NACC; ++l)
#pragma unroll
        for (int e = 0; e < 4; ++e) tc::order_after_wait(r[l][e]);
    if constexpr (MODE == MODE_FLOAT_TF32) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            vh[e] = __uint_as_float(r[0][e]);
            vl[e] = 0.f;
        }
    } else {
        // t = sum_{l>=1} level l, added from the lowest level up, one rounding per level
        float t[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float acc = NACC >= 2 ? __uint_as_float(r[NACC - 1][e]) : 0.f;
#pragma unroll
            for (int l = NACC - 2; l >= 1; --l) acc = __uint_as_float(r[l][e]) + acc;
            t[e] = acc;
        }
        const float4 c4 = *reinterpret_cast<const float4 *>(cs + c0);   // 16-byte aligned
        const float csv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float l0 = __uint_as_float(r[0][e]);
            const float sc = rs * csv[e];
            if (HL) {
                const float h = l0 + t[e];
                const float bp = h - l0;
                vl[e] = ((l0 - (h - bp)) + (t[e] - bp)) * sc;
                vh[e] = h * sc;
            } else {
                vh[e] = (l0 + t[e]) * sc;
                vl[e] = 0.f;
            }
        }
    }
}

// ---------------------------------------------------------------------------------------
// Pass kernel.  Rows of the batch are cut into tiles of 128 (= TMEM lanes); TPR threads
// share a row, thread (q, row) = threadIdx.x = q*128 + row owning the 4-element units
// u = q, q+TPR, ... of the row (slicing) and the 4-column units of the result (TMEM read,
// stores).  The 32 threads of a warp share q, so they run the same number of units and the
// warp-collective TMEM loads stay uniform (threads with different q may differ by one unit).
// Warps w, w+4, ... see TMEM lane quarter w%4.  CTAs loop over tiles; the next tile's rows
// arrive (TMA boxes or cp.async copies) while the current tile's MMAs and epilogue run.
struct TcPassArgs {
    // Tiles by TMA (use_tma): tm[0] hi plane, tm[1] lo plane of the input (pair pass: of the
    // orbitals).  [k][row] loads: 3D tensors (R rows, n_d lines, fields or orbitals), a
    // 128 x K x 1 box; koff = first line of this K-block.  K-fast loads: 2D tensors (K, rows
    // of the batch) read in 16 x 128 boxes with the 64-byte swizzle, one per 16 columns.
    CUtensorMap tm[2];
    int use_tma, koff;
    int nfields, R, K, Np;          // K = contracted length of this block, Np = padded block size
    int Kout;                       // outputs of this block (K = Kout = n_d when not blocked)
    int in_pitch, out_pitch;        // KFAST / NFAST row pitch (= n_d)
    long in_off, out_off;           // block offsets: k0 (KFAST) or k0 * R (KSLOW, PAIR); same for n0
    int acc;                        // add to out instead of overwriting it (K-blocks after the first)
    const float *Fs, *Fs_lo;        // if set: scale the finished sums by f(Lambda) before storing
    int f_noff;                     // first output mode of this block (index into Fs)
    long N;
    FastDiv divR;                   // division by R (row of the batch -> field, row in field)
    FastDiv divK4;                  // division by K / 4 (contiguous KFAST tiles: chunk -> row)
    FastDiv divKo4;                 // division by Kout / 4 (contiguous NFAST output tiles)
    const float *in;
    float *out;
    long lo_off;                    // hi + lo intermediates: offset of the lo plane (floats)
    const uint8_t *B1, *B2;         // operand images
    uint32_t img_bytes;             // bytes of one image
    const float *F, *Flo;           // [col][row] scaling for the double pass, hi + lo
    const float *psi_hi, *psi_lo;   // fp32 orbital planes (pair prologue)
    int occ_off;                    // column offset of the occupied set in the planes
    const int2 *pairs;
    int *err;
};

template <int MODE, int S, int SB, bool HL, int LOAD, int STORE, bool DOUBLE, int TPR, int NBUF, int NSETS>
__global__ void __launch_bounds__(kRows * TPR + 64, 1) tc_pass_kernel(const __grid_constant__ TcPassArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    constexpr int ES = MODE == MODE_FLOAT_TF32 ? 4 : 2;
    constexpr int NACC = MODE == MODE_FLOAT_TF32 ? 1 : (SB > S ? S + 1 : S);
    // compute threads, then one warp that issues the MMAs and one that issues the input
    // copies of the coalesced layouts (the producer)
    constexpr int NT = kRows * TPR;
    constexpr int kBarHandoff = 1, kBarCompute = 2;
    const int Np = a.Np, Kp = a.Np;
    const int nunit = Np / 4;                // 4-element units per row
    const uint32_t sbo = uint32_t(Kp) * ES * 8;          // bytes per 8-row group
    const uint32_t a_piece = uint32_t(kRows) * Kp * ES;
    const uint32_t b_piece = uint32_t(Np) * Kp * ES;
    uint8_t *sB1 = smem;
    uint8_t *sB2 = smem + a.img_bytes;
    // NSETS = 2: two A buffers (slices of tile t and t+1) and two TMEM accumulator sets,
    // so the GEMMs of tile t overlap the epilogue of t-1 and the slicing of t+1.
    // NSETS = 1 (long axes): one of each, the epilogue of t-1 comes before slicing t.
    uint8_t *sA0 = smem + (DOUBLE ? 2 : 1) * a.img_bytes;
    // Input staging.  KSLOW / PAIR: [k][row] (a warp touches 32 consecutive words; rows
    // k >= K are zero from the start and never written); KFAST: [row][Kp + 4] (16-byte
    // copies, read back conflict-free because (Kp + 4)/4 is odd; columns k >= K are
    // masked when read).  PAIR stages psi_m hi, psi_m lo, psi_n hi, psi_n lo; the others
    // hi (and lo).  NBUF staging buffers = tiles whose copies are in flight.
    constexpr int NSTG = LOAD == LOAD_PAIR ? 4 : (HL ? 2 : 1);
    const int stg_len = kRows * (LOAD == LOAD_KFAST ? Kp + 4 : Kp);
    // The last tile's NFAST output is also staged here ([row][Kp + 4], hi then lo) to leave
    // as contiguous runs; earlier tiles' outputs go through the previous A image (see the
    // epilogue)
    const int buf_len = max(NSTG * stg_len, STORE == STORE_NFAST ? (HL ? 2 : 1) * kRows * (Kp + 4) : 0);
    // K-fast staging starts 1024-byte aligned (the 64-byte TMA swizzle repeats every 512)
    uint8_t *stg_b = sA0 + NSETS * a_piece * S;
    if (LOAD == LOAD_KFAST) stg_b += (1024u - (tc::smem_addr(stg_b) & 1023u)) & 1023u;
    float *stg0 = reinterpret_cast<float *>(stg_b);
    float *maxbuf = stg0 + NBUF * buf_len;
    uint64_t *bar1 = reinterpret_cast<uint64_t *>(maxbuf + NT);   // [2]: first GEMM of each set
    uint64_t *bar2 = bar1 + 2;                                      // [2]: second GEMM (pass 3)
    uint64_t *full = bar2 + 2;                                      // [2]: staging buffer filled
    uint32_t *tslot = reinterpret_cast<uint32_t *>(full + 2);
    int *sflag = reinterpret_cast<int *>(tslot + 1);
    const float *cs1 = reinterpret_cast<const float *>(sB1 + SB * b_piece);
    const float *cs2 = reinterpret_cast<const float *>(sB2 + SB * b_piece);
    const int tid = threadIdx.x, warp = tid >> 5, row = tid & (kRows - 1), q = tid / kRows;
    const int set_cols = NACC * Np;
    const int ncols = NSETS * set_cols <= 32 ? 32 : NSETS * set_cols <= 64 ? 64 : NSETS * set_cols <= 128 ? 128 : NSETS * set_cols <= 256 ? 256 : 512;

    for (uint32_t i = tid * 16; i < a.img_bytes; i += (NT + 64) * 16) {
        *reinterpret_cast<uint4 *>(sB1 + i) = *reinterpret_cast<const uint4 *>(a.B1 + i);
        if (DOUBLE) *reinterpret_cast<uint4 *>(sB2 + i) = *reinterpret_cast<const uint4 *>(a.B2 + i);
    }
    for (int i = tid; i < NBUF * buf_len; i += NT + 64) stg0[i] = 0.f;   // padding k >= K stays zero
    tc::fence_proxy_async_smem();
    if (tid == 0) {
        for (int i = 0; i < 4; ++i) tc::mbar_init(bar1 + i, 1);
        // the producer's 32 cp.async arrivals, or its one expect_tx arrival (TMA)
        for (int i = 0; i < 2; ++i) tc::mbar_init(full + i, a.use_tma ? 1 : 32);
        *sflag = 0;
    }
    if (warp == 0) tc::tmem_alloc(tslot, ncols);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t lane_q = uint32_t((warp & 3) * 32) << 16;   // this warp's TMEM lane quarter
    const uint32_t idesc = tc::instr_desc(MODE == MODE_FLOAT_TF32, Np);
    const int ksteps = Kp * ES / 32;
    const uint32_t sB1_addr = tc::smem_addr(sB1), sB2_addr = tc::smem_addr(sB2);
    uint32_t ph1 = 0u, ph2 = 0u;   // bit st = phase parity of bar1[st] / bar2[st]
    auto set_tmem = [&](int st) { return tmem + uint32_t(st * set_cols); };
    auto set_A = [&](int st) { return sA0 + st * S * a_piece; };

    const long rows = long(a.nfields) * a.R;   // < 2^31 (checked on the host)
    const long ntiles = (rows + kRows - 1) / kRows;
    const bool vec16 = ((a.K & 3) == 0) && ((a.in_pitch & 3) == 0) && ((a.in_off & 3) == 0) &&
                       ((a.N & 3) == 0) && ((a.lo_off & 3) == 0);
    const bool vec_out = ((a.out_pitch & 3) == 0) && ((a.out_off & 3) == 0) && ((a.N & 3) == 0) &&
                         ((a.lo_off & 3) == 0);
    // KSLOW / PAIR rows come 4 at a time (16-byte copies) when a field's rows are a
    // multiple of 4: a group of 4 consecutive rows then never straddles two fields
    const bool rvec = ((a.R & 3) == 0) && ((a.lo_off & 3) == 0);
    // KFAST rows of a whole (unblocked) axis are back to back across fields (N = R K), so a
    // tile is one contiguous run of 128 K values: copied by consecutive lanes (coalesced)
    const bool kcont = LOAD == LOAD_KFAST && vec16 && a.in_pitch == a.K && a.in_off == 0;
    // the same holds for NFAST outputs of a whole axis: the epilogue stages the tile in
    // shared memory and writes it back with consecutive lanes on consecutive 16 bytes
    const bool ostage = STORE == STORE_NFAST && (NSETS == 2 || DOUBLE) && vec_out && a.out_pitch == a.Kout &&
                        a.out_off == 0 && !a.acc && (a.Kout & 3) == 0;
    // row `rl` of tile t -> (field pp, row rr of the field); false past the last row
    auto locate = [&](long t, int rl, int &pp, int &rr) {
        const long gg = t * kRows + rl;
        if (t >= ntiles || gg >= rows) return false;
        const uint32_t g = uint32_t(gg);
        const uint32_t f = fast_div(g, a.divR);
        pp = int(f);
        rr = int(g - f * uint32_t(a.R));
        return true;
    };
    // The coalesced layouts (contiguous KFAST tiles, 4-row groups of [k][row] tiles) put
    // a thread's copies into other threads' staging rows.  KSLOW tiles (two staging
    // buffers) are copied by the producer warp, whose `full` mbarrier tells the compute
    // threads when a tile is in; KFAST and pair tiles (measured faster that way: pass 3
    // and the pair pass have one buffer, and the next tile must be requested at once
    // by many threads) are copied by the compute threads, with a barrier after the wait.
    const bool use_tma = a.use_tma != 0;   // set by the host where the layout allows it
    const bool use_prod = use_tma || (LOAD == LOAD_KSLOW && rvec);
    const bool coal = !use_prod && (kcont || (LOAD == LOAD_PAIR && rvec));
    // Producer, TMA: one box per plane (128 rows x K lines), the tile being one field's
    // rows; expect_tx announces the bytes, the boxes complete them.
    auto fill_tma = [&](long t, float *stg, uint64_t *fb) {
        const uint32_t g0 = uint32_t(t * kRows);
        const uint32_t f = fast_div(g0, a.divR);
        const int rr = int(g0 - f * uint32_t(a.R));
        constexpr int NPL = LOAD == LOAD_PAIR ? 4 : (HL ? 2 : 1);
        if (LOAD == LOAD_KFAST) {   // ceil(K / 16) swizzled 16 x 128 boxes per plane, rows g0..g0+127
            const int nsl = (a.K + 15) >> 4;
            tc::mbar_arrive_expect_tx(fb, uint32_t(NPL) * uint32_t(nsl) * uint32_t(kRows) * 64u);
            for (int sl = 0; sl < nsl; ++sl) {
                tc::tma_load_2d(stg + sl * (kRows * 16), &a.tm[0], 16 * sl, int(g0), fb);
                if (HL) tc::tma_load_2d(stg + stg_len + sl * (kRows * 16), &a.tm[1], 16 * sl, int(g0), fb);
            }
            return;
        }
        tc::mbar_arrive_expect_tx(fb, uint32_t(NPL) * uint32_t(kRows) * uint32_t(a.K) * 4u);
        if (LOAD == LOAD_PAIR) {
            const int2 mn = a.pairs[f];
            tc::tma_load_3d(stg, &a.tm[0], rr, a.koff, a.occ_off + mn.x, fb);
            tc::tma_load_3d(stg + stg_len, &a.tm[1], rr, a.koff, a.occ_off + mn.x, fb);
            tc::tma_load_3d(stg + 2 * stg_len, &a.tm[0], rr, a.koff, mn.y, fb);
            tc::tma_load_3d(stg + 3 * stg_len, &a.tm[1], rr, a.koff, mn.y, fb);
        } else {
            tc::tma_load_3d(stg, &a.tm[0], rr, a.koff, int(f), fb);
            if (HL) tc::tma_load_3d(stg + stg_len, &a.tm[1], rr, a.koff, int(f), fb);
        }
    };
    // Copies of tile t into `stg` by issuer x of nx (nx a multiple of 32).
    auto copy_coalesced = [&](long t, float *stg, int x, int nx) {
        int pp, rr;
        if (LOAD == LOAD_KFAST) {
            const long g0 = t * kRows;
            const int nrow = int(min(long(kRows), rows - g0));
            const int nchk = nrow * (a.K >> 2);   // 16-byte chunks of the tile
            const float *src = a.in + size_t(g0) * a.K;
            for (int c = x; c < nchk; c += nx) {
                const int rw = int(fast_div(uint32_t(c), a.divK4));
                float *dh = stg + rw * (Kp + 4) + 4 * (c - rw * (a.K >> 2));
                tc::cp_async16(dh, src + 4 * c);
                if (HL) tc::cp_async16(dh + stg_len, src + a.lo_off + 4 * c);
            }
        } else {
            // issuer -> rows 4g..4g+3 (g = x mod 32) and lines k = x / 32, + nx / 32, ...:
            // 32 consecutive issuers copy 512 contiguous bytes per line
            const int g4 = 4 * (x & 31);
            if (locate(t, g4, pp, rr)) {
                if (LOAD == LOAD_PAIR) {
                    const int2 mn = a.pairs[pp];
                    const size_t o = size_t(rr) + a.in_off;
                    const float *src[4] = {a.psi_hi + size_t(a.occ_off + mn.x) * a.N + o,
                                           a.psi_lo + size_t(a.occ_off + mn.x) * a.N + o,
                                           a.psi_hi + size_t(mn.y) * a.N + o, a.psi_lo + size_t(mn.y) * a.N + o};
                    for (int k = x >> 5; k < a.K; k += nx >> 5)
#pragma unroll
                        for (int w = 0; w < 4; ++w)
                            tc::cp_async16(stg + w * stg_len + k * kRows + g4, src[w] + size_t(k) * a.R);
                } else {
                    const float *src = a.in + size_t(pp) * a.N + a.in_off + rr;
                    for (int k = x >> 5; k < a.K; k += nx >> 5) {
                        tc::cp_async16(stg + k * kRows + g4, src + size_t(k) * a.R);
                        if (HL) tc::cp_async16(stg + stg_len + k * kRows + g4, src + a.lo_off + size_t(k) * a.R);
                    }
                }
            }
        }
    };
    // Copies of tile t by the compute threads: coalesced (see above), or for ragged
    // layouts each thread the elements of its own units of its own row (rows past the end
    // are skipped; the slicing treats them as zero).  Exactly one copy group is committed
    // per call, empty or not, so that wait_group counts tiles.
    auto prefetch = [&](long t, float *stg) {
        int pp, rr;
        if (coal) {
            if (t < ntiles) copy_coalesced(t, stg, tid, NT);
        } else if (!use_prod && locate(t, row, pp, rr)) {
            if (LOAD == LOAD_KFAST) {
                const float *src = a.in + size_t(pp) * a.N + size_t(rr) * a.in_pitch + a.in_off;
                float *dh = stg + row * (Kp + 4);
                if (vec16) {
                    for (int k = 4 * q; k < a.K; k += 4 * TPR) {
                        tc::cp_async16(dh + k, src + k);
                        if (HL) tc::cp_async16(dh + stg_len + k, src + a.lo_off + k);
                    }
                } else {
                    for (int u = q; 4 * u < a.K; u += TPR)
                        for (int k = 4 * u; k < min(a.K, 4 * u + 4); ++k) {
                            tc::cp_async4(dh + k, src + k);
                            if (HL) tc::cp_async4(dh + stg_len + k, src + a.lo_off + k);
                        }
                }
            } else if (LOAD == LOAD_PAIR) {
                const int2 mn = a.pairs[pp];
                const size_t o = size_t(rr) + a.in_off;
                const float *src[4] = {a.psi_hi + size_t(a.occ_off + mn.x) * a.N + o,
                                       a.psi_lo + size_t(a.occ_off + mn.x) * a.N + o,
                                       a.psi_hi + size_t(mn.y) * a.N + o, a.psi_lo + size_t(mn.y) * a.N + o};
                for (int u = q; 4 * u < a.K; u += TPR)
                    for (int k = 4 * u; k < min(a.K, 4 * u + 4); ++k)
#pragma unroll
                        for (int w = 0; w < 4; ++w)
                            tc::cp_async4(stg + w * stg_len + k * kRows + row, src[w] + size_t(k) * a.R);
            } else {
                const float *src = a.in + size_t(pp) * a.N + a.in_off + rr;
                for (int u = q; 4 * u < a.K; u += TPR)
                    for (int k = 4 * u; k < min(a.K, 4 * u + 4); ++k) {
                        tc::cp_async4(stg + k * kRows + row, src + size_t(k) * a.R);
                        if (HL) tc::cp_async4(stg + stg_len + k * kRows + row, src + a.lo_off + size_t(k) * a.R);
                    }
            }
        }
        tc::cp_async_commit();
    };
    // Offset (floats) of unit u (elements 4u..4u+3) of this thread's row in a K-fast staging
    // plane: padded rows [row][Kp + 4] for cp.async copies; for TMA, 16-column slabs of 128
    // rows x 64 bytes whose 16-byte chunk c sits at c ^ ((row >> 1) & 3) (the 64-byte swizzle)
    auto kfast_off = [&](int u) {
        if (use_tma) return (u >> 2) * (kRows * 16) + row * 16 + 4 * ((u & 3) ^ ((row >> 1) & 3));
        return row * (Kp + 4) + 4 * u;
    };
    // Staged values (hi, lo) of unit u (elements 4u..4u+3) of this thread's row.
    auto staged_unit = [&](const float *stg, int u, float (&hi)[4], float (&lo)[4]) {
        const int k0 = 4 * u;
        if constexpr (LOAD == LOAD_KFAST) {
            const int so = kfast_off(u);
            const float4 h = *reinterpret_cast<const float4 *>(stg + so);
            hi[0] = h.x; hi[1] = h.y; hi[2] = h.z; hi[3] = h.w;
            if (HL) {
                const float4 l = *reinterpret_cast<const float4 *>(stg + stg_len + so);
                lo[0] = l.x; lo[1] = l.y; lo[2] = l.z; lo[3] = l.w;
            } else {
                lo[0] = lo[1] = lo[2] = lo[3] = 0.f;
            }
            // columns k >= K of a KFAST row are not copied (and may hold stale values): zero them
            if (k0 + 4 > a.K) {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (k0 + e >= a.K) hi[e] = lo[e] = 0.f;
            }
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = k0 + e;
                if (LOAD == LOAD_PAIR) {
                    const float ah = stg[k * kRows + row], al = stg[stg_len + k * kRows + row];
                    const float bh = stg[2 * stg_len + k * kRows + row], bl = stg[3 * stg_len + k * kRows + row];
                    hi[e] = ah * bh;
                    lo[e] = fmaf(ah, bh, -hi[e]) + fmaf(ah, bl, al * bh);
                } else {
                    hi[e] = stg[k * kRows + row];
                    lo[e] = HL ? stg[stg_len + k * kRows + row] : 0.f;
                }
            }
        }
    };
    // Largest |hi| over this thread's units (the row scale needs only the leading parts).
    auto staged_max = [&](const float *stg) {
        float mx = 0.f;
        for (int u = q; u < nunit; u += TPR) {
            const int k0 = 4 * u;
            if constexpr (LOAD == LOAD_KFAST) {
                const float4 h = *reinterpret_cast<const float4 *>(stg + kfast_off(u));
                const float v[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (k0 + e < a.K) mx = fmaxf(mx, fabsf(v[e]));
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int k = k0 + e;
                    const float v = LOAD == LOAD_PAIR ? stg[k * kRows + row] * stg[2 * stg_len + k * kRows + row]
                                                      : stg[k * kRows + row];
                    mx = fmaxf(mx, fabsf(v));
                }
            }
        }
        return mx;
    };
    // Row maximum from the per-thread partial maxima of the TPR threads of a row.
    auto row_max = [&](float part) {
        maxbuf[q * kRows + row] = part;
        tc::bar_sync(kBarCompute, NT);
        float m = 0.f;
#pragma unroll
        for (int qq = 0; qq < TPR; ++qq) m = fmaxf(m, maxbuf[qq * kRows + row]);
        return m;
    };
    auto scales = [&](float mx, float &sc, float &rs) {
        sc = 1.f;
        rs = 1.f;
        if (MODE == MODE_FIXED_BF16) {
            // e with mx = f 2^e, f in [0.5, 1) (as frexp), from the biased exponent field
            int e = int((__float_as_uint(mx) >> 23) & 0xffu) - 126;
            e = max(e, -100);   // rows below 2^-100 (and zero rows) are flushed to zero slices
            sc = __uint_as_float(uint32_t(127 + 7 - e) << 23);   // 2^(7 - e), a normal number
            rs = __uint_as_float(uint32_t(127 - 7 + e) << 23);   // 2^(e - 7)
        }
    };
    // Compute threads: publish the A slices written so far to the tensor core and hand
    // them to the MMA warp (which issues A[st] x B into TMEM set st).  Returns true when
    // any thread has recorded an error, uniformly on both sides of the hand-off.
    auto handoff = [&]() {
        tc::fence_proxy_async_smem();
        tc::tc_fence_before();
        return tc::bar_red_or(kBarHandoff, NT + 64, *sflag != 0);
    };

    if (tid >= NT + 32) {
        // ---- producer warp: the copies of tile t + NBUF go out once every compute thread
        //      is done with its buffer, i.e. after the first hand-off of tile t (the slices
        //      of tile t are its last use: epilogues stage their output in A images, and
        //      pass 3 keeps its middle values in the A image) ----
        const int lane = tid - NT - 32;
        int fills0 = 0, fills1 = 0;   // fills issued per staging buffer
        auto fill = [&](long tt, int b) {
            if (use_tma) {
                if (lane == 0) fill_tma(tt, stg0 + b * buf_len, full + b);
            } else {
                copy_coalesced(tt, stg0 + b * buf_len, lane, 32);
                tc::cp_async_mbar_arrive_noinc(full + b);
            }
            if (b == 0) ++fills0;
            else ++fills1;
        };
        if (use_prod)
            for (int jb = 0; jb < NBUF; ++jb) {
                const long t0 = blockIdx.x + long(jb) * gridDim.x;
                if (t0 < ntiles) fill(t0, jb);
            }
        long it = 0;
        for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            if (tc::bar_red_or(kBarHandoff, NT + 64, false)) break;
            const long tn = tile + long(NBUF) * gridDim.x;
            if (use_prod && tn < ntiles) fill(tn, int(it % NBUF));
            if (DOUBLE && tc::bar_red_or(kBarHandoff, NT + 64, false)) break;
        }
        tc::cp_async_wait_all();   // no copy may still target shared memory at exit
        if (use_tma) {   // nor a box: only the last fill of a buffer can be unconsumed (after a stop)
            if (fills0 > 0 && !tc::mbar_wait_bounded(full, uint32_t((fills0 - 1) & 1), kWaitLimit)) atomicExch(sflag, 1);
            if (fills1 > 0 && !tc::mbar_wait_bounded(full + 1, uint32_t((fills1 - 1) & 1), kWaitLimit))
                atomicExch(sflag, 1);
        }
    } else if (tid >= NT) {
        // ---- MMA warp: one hand-off per GEMM, in the compute threads' order ----
        long it = 0;
        for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const int st = int(it % NSETS);
            if (tc::bar_red_or(kBarHandoff, NT + 64, *sflag != 0)) break;
            if (tid == NT) {
                tc::tc_fence_after();
                issue_gemm<MODE, S, SB>(set_tmem(st), Np, tc::smem_addr(set_A(st)), a_piece, sB1_addr, b_piece, sbo,
                                        ksteps, idesc);
                tc::mma_commit(bar1 + st);
            }
            if (DOUBLE) {
                if (tc::bar_red_or(kBarHandoff, NT + 64, *sflag != 0)) break;
                if (tid == NT) {
                    tc::tc_fence_after();
                    issue_gemm<MODE, S, SB>(set_tmem(st), Np, tc::smem_addr(set_A(st)), a_piece, sB2_addr, b_piece, sbo,
                                            ksteps, idesc);
                    tc::mma_commit(bar2 + st);
                }
            }
        }
    } else {
    auto wait_bar = [&](uint64_t *bar, uint32_t &ph, int st) {
        if (!tc::mbar_wait_bounded(bar, (ph >> st) & 1u, kWaitLimit)) atomicExch(sflag, 1);
        ph ^= 1u << st;
        tc::tc_fence_after();
    };
    // Epilogue of tile t from TMEM set st: own 4-column units -> global (added to the
    // stored partial sums for K-blocks after the first; scaled by f(Lambda) when Fs is set).
    // With obuf (free shared memory) and ostage, through shared memory: every compute thread
    // must call it then, as it contains compute-thread barriers.  obuf: [row][Kp + 4]
    // rows (an idle staging buffer), or with swz a [row][Kp] layout whose 16-byte chunk u of
    // row r sits at u ^ sw(r) (the previous tile's A image, whose GEMMs have completed).
    auto epilogue = [&](long t, int st, float rs_out, const float *cs_out, float *obuf, bool swz) {
        if (ostage && obuf != nullptr) {
            const int opitch = swz ? Kp : Kp + 4;
            // rows Kp floats apart meet the banks at 16 r mod 32 (Kp = 16 mod 32) or at 0:
            // XOR the chunk with 2 or 3 row bits so that 8 rows cover all 32 banks
            auto chunk = [&](int r, int u) { return !swz ? u : ((Kp & 16) ? u ^ ((r >> 1) & 3) : u ^ (r & 7)); };
            float *oh = obuf, *ol = obuf + kRows * opitch;
            int fp = 0, fr = 0;
            const bool fact = a.Fs != nullptr && locate(t, row, fp, fr);
            for (int u = q; u < nunit; u += TPR) {
                float v[4], vlo[4];
                read4<MODE, NACC, HL>(set_tmem(st) + lane_q, Np, 4 * u, rs_out, cs_out, v, vlo);
                if (fact) {   // f(Lambda) scaling of a finished forward product
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int col = 4 * u + e;
                        const size_t fi = size_t(a.f_noff + min(col, a.Kout - 1)) * a.R + fr;
                        const float fh = a.Fs[fi], fl = a.Fs_lo[fi];
                        if (HL) {
                            const float x = v[e] * fh;
                            vlo[e] = fmaf(v[e], fh, -x) + fmaf(v[e], fl, vlo[e] * fh);
                            v[e] = x;
                        } else {
                            v[e] = fmaf(v[e], fh, v[e] * fl);
                        }
                    }
                }
                const int cu = row * opitch + 4 * chunk(row, u);
                *reinterpret_cast<float4 *>(oh + cu) = make_float4(v[0], v[1], v[2], v[3]);
                if (HL) *reinterpret_cast<float4 *>(ol + cu) = make_float4(vlo[0], vlo[1], vlo[2], vlo[3]);
            }
            tc::tc_fence_before();
            tc::bar_sync(kBarCompute, NT);
            const long g0 = t * kRows;
            const int nrow = int(min(long(kRows), rows - g0));
            const int kq = a.Kout >> 2;
            float *dst = a.out + size_t(g0) * a.Kout;
            for (int c = tid; c < nrow * kq; c += NT) {
                const int rw = int(fast_div(uint32_t(c), a.divKo4));
                const int k = rw * opitch + 4 * chunk(rw, c - rw * kq);
                *reinterpret_cast<float4 *>(dst + 4 * c) = *reinterpret_cast<const float4 *>(oh + k);
                if (HL) *reinterpret_cast<float4 *>(dst + a.lo_off + 4 * c) = *reinterpret_cast<const float4 *>(ol + k);
            }
            // obuf is free again once every thread is past here.  An A image (swz) needs no
            // barrier for that: its next writer is the slicing of the next tile, which every
            // thread reaches only through that tile's row-maximum barrier.
            if (!swz) tc::bar_sync(kBarCompute, NT);
            return;
        }
        int pp = 0, rr = 0;
        const bool act = locate(t, row, pp, rr);
        float *out = a.out + size_t(pp) * a.N + a.out_off;
        for (int u = q; u < nunit; u += TPR) {
            float v[4], vlo[4];
            read4<MODE, NACC, HL>(set_tmem(st) + lane_q, Np, 4 * u, rs_out, cs_out, v, vlo);
            if (!act) continue;
            const int c0 = 4 * u;
            if (!a.acc && !a.Fs) {   // plain store of the unit
                if (STORE == STORE_NFAST && vec_out && c0 + 4 <= a.Kout) {
                    float *o = out + size_t(rr) * a.out_pitch + c0;
                    *reinterpret_cast<float4 *>(o) = make_float4(v[0], v[1], v[2], v[3]);
                    if (HL) *reinterpret_cast<float4 *>(o + a.lo_off) = make_float4(vlo[0], vlo[1], vlo[2], vlo[3]);
                } else {
                    const size_t step = STORE == STORE_NSLOW ? size_t(a.R) : 1;
                    float *o = out + (STORE == STORE_NSLOW ? size_t(c0) * a.R + rr : size_t(rr) * a.out_pitch + c0);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (c0 + e < a.Kout) {
                            o[0] = v[e];
                            if (HL) o[a.lo_off] = vlo[e];
                        }
                        o += step;
                    }
                }
                continue;
            }
            // element e of this unit: out[idx(e)] (hi) and out[lo_off + idx(e)] (lo)
            auto idx = [&](int e) {
                return STORE == STORE_NSLOW ? size_t(c0 + e) * a.R + rr : size_t(rr) * a.out_pitch + c0 + e;
            };
            if (a.acc) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (c0 + e >= a.Kout) continue;
                    const float oh = out[idx(e)];
                    if (HL) {   // (oh + ol) + (v + vlo), renormalised
                        const float ol = out[a.lo_off + idx(e)];
                        const float sh = oh + v[e], bp = sh - oh;
                        const float err = (oh - (sh - bp)) + (v[e] - bp);
                        const float sl = (ol + vlo[e]) + err;
                        v[e] = sh + sl;
                        vlo[e] = sl - (v[e] - sh);
                    } else {
                        v[e] += oh;
                    }
                }
            }
            if (a.Fs) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (c0 + e >= a.Kout) continue;
                    const size_t fi = size_t(a.f_noff + c0 + e) * a.R + rr;
                    const float fh = a.Fs[fi], fl = a.Fs_lo[fi];
                    if (HL) {
                        const float x = v[e] * fh;
                        vlo[e] = fmaf(v[e], fh, -x) + fmaf(v[e], fl, vlo[e] * fh);
                        v[e] = x;
                    } else {
                        v[e] = fmaf(v[e], fh, v[e] * fl);
                    }
                }
            }
            if (STORE == STORE_NFAST && vec_out && c0 + 4 <= a.Kout) {
                *reinterpret_cast<float4 *>(out + idx(0)) = make_float4(v[0], v[1], v[2], v[3]);
                if (HL)
                    *reinterpret_cast<float4 *>(out + a.lo_off + idx(0)) = make_float4(vlo[0], vlo[1], vlo[2], vlo[3]);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (c0 + e < a.Kout) {
                        out[idx(e)] = v[e];
                        if (HL) out[a.lo_off + idx(e)] = vlo[e];
                    }
                }
            }
        }
        tc::tc_fence_before();   // these TMEM reads precede the next thread sync
    };

    // Software pipeline over this CTA's tiles: the GEMM(s) of tile t run on the tensor
    // core while the threads finish tile t-1 (epilogue) and slice tile t+1.
#pragma unroll
    for (int j = 0; j < NBUF; ++j) prefetch(blockIdx.x + long(j) * gridDim.x, stg0 + j * buf_len);
    long prev_tile = -1;
    int prev_set = 0;
    float prev_rs = 1.f;
    const float *prev_cs = cs1;
    long it = 0;
    for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int st = int(it % NSETS);
        if (NSETS == 1 && prev_tile >= 0) {   // one A buffer / TMEM set: finish t-1 first
            if (DOUBLE) wait_bar(bar2 + prev_set, ph2, prev_set);
            else wait_bar(bar1 + prev_set, ph1, prev_set);
            epilogue(prev_tile, prev_set, prev_rs, prev_cs, nullptr, false);
            prev_tile = -1;
        }
        int p = 0, r = 0;
        const bool active = locate(tile, row, p, r);
        float *stg = stg0 + (it % NBUF) * buf_len;
        uint8_t *sA = set_A(st);
        // ---- slice tile -> A[st] (A[st] was last read by the GEMMs of tile it-2,
        //      which completed before that tile's epilogue) ----
        if (use_prod) {   // the producer's copies of this tile landed
            if (!tc::mbar_wait_bounded(full + it % NBUF, uint32_t((it / NBUF) & 1), kWaitLimit)) atomicExch(sflag, 1);
        } else {
            tc::cp_async_wait_group<NBUF - 1>();   // own copies (one group per tile) landed
            if (coal) tc::bar_sync(kBarCompute, NT);   // and every other thread's
        }
        const float mx = row_max(active ? staged_max(stg) : 0.f);
        float s_in, rs1;
        scales(mx, s_in, rs1);
        // rows past the end slice to zeros: fixed mode through a zero scale (the staging
        // buffers hold only finite values: zeros, loaded inputs or earlier tiles' inputs)
        if (!active) s_in = 0.f;
        for (int u = q; u < nunit; u += TPR) {
            float vals[4][4], hi[4], lo[4];
            staged_unit(stg, u, hi, lo);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                float qv[4];
                if (MODE == MODE_FLOAT_TF32 && !active) hi[e] = lo[e] = 0.f;
                if (MODE == MODE_FLOAT_TF32) split_tf32(hi[e], lo[e], qv);
                else slice_fixed<S>(hi[e], lo[e], s_in, qv);
#pragma unroll
                for (int t2 = 0; t2 < 4; ++t2) vals[t2][e] = qv[t2];
            }
            store_unit<ES, S>(sA, a_piece, row, u, sbo, vals);
        }
        // ---- first GEMM of this tile; TMEM set st was last read by the epilogue of
        //      tile it-2, which every thread finished before this hand-off ----
        if (handoff()) break;
        // every thread has consumed this staging buffer: fetch the tile NBUF steps ahead
        prefetch(tile + long(NBUF) * gridDim.x, stg);
        // pass 3: f(Lambda) of the next unit of the middle step is loaded while the current
        // one is processed, the first one while the previous tile's epilogue runs
        float fh_n[4], fl_n[4];
        auto load_f = [&](int u) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int col = 4 * u + e;
                const bool ok = active && u < nunit && col < a.Kout;
                const size_t fi = size_t(col) * a.R + r;
                fh_n[e] = ok ? a.F[fi] : 0.f;
                fl_n[e] = ok ? a.Flo[fi] : 0.f;
            }
        };
        if (DOUBLE) load_f(q);
        // ---- epilogue of the previous tile, overlapping this tile's (first) GEMM; the
        //      output (N-fast) is staged in the previous tile's A image, whose GEMMs are
        //      complete ----
        if (prev_tile >= 0) {
            if (DOUBLE) wait_bar(bar2 + prev_set, ph2, prev_set);
            else wait_bar(bar1 + prev_set, ph1, prev_set);
            epilogue(prev_tile, prev_set, prev_rs, prev_cs, reinterpret_cast<float *>(set_A(prev_set)), true);
        }
        float rs_out = rs1;
        const float *cs_out = cs1;
        if (DOUBLE) {
            // D1 * f(Lambda) -> A[st] (its first GEMM is complete), each thread's values of
            // unit u in the very bytes its slices of unit u take (two 8-byte slots for the
            // hi parts, two for the lo parts; one 16-byte slot for tf32), so no other
            // thread writes there before it has read them back -> row maximum -> slices in
            // place -> second GEMM into the same TMEM set.
            static_assert(!HL || S >= 4, "hi + lo middle values need four slots per unit");
            auto mid_slot = [&](int u) {
                return ES == 4 ? sA + img_off(row, u, sbo) : sA + img_off(row, u >> 1, sbo) + (u & 1) * 8;
            };
            wait_bar(bar1 + st, ph1, st);
            float mx2 = 0.f;
            for (int u = q; u < nunit; u += TPR) {
                float v[4], vlo[4], fh[4], fl[4], x[4], xl[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    fh[e] = fh_n[e];
                    fl[e] = fl_n[e];
                }
                load_f(u + TPR);
                read4<MODE, NACC, HL>(set_tmem(st) + lane_q, Np, 4 * u, rs1, cs1, v, vlo);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (HL) {   // (v + vlo)(fh + fl) as x + xl
                        x[e] = v[e] * fh[e];
                        xl[e] = fmaf(v[e], fh[e], -x[e]) + fmaf(v[e], fl[e], vlo[e] * fh[e]);
                    } else {
                        x[e] = fmaf(v[e], fh[e], v[e] * fl[e]);
                        xl[e] = 0.f;
                    }
                    mx2 = fmaxf(mx2, fabsf(x[e]));
                }
                uint8_t *p = mid_slot(u);
                if (ES == 4) {
                    *reinterpret_cast<float4 *>(p) = make_float4(x[0], x[1], x[2], x[3]);
                } else {
                    *reinterpret_cast<float2 *>(p) = make_float2(x[0], x[1]);
                    *reinterpret_cast<float2 *>(p + a_piece) = make_float2(x[2], x[3]);
                    if (HL) {
                        *reinterpret_cast<float2 *>(p + 2 * a_piece) = make_float2(xl[0], xl[1]);
                        *reinterpret_cast<float2 *>(p + 3 * a_piece) = make_float2(xl[2], xl[3]);
                    }
                }
            }
            tc::tc_fence_before();
            mx2 = row_max(mx2);   // (its sync also orders these TMEM reads before GEMM 2)
            float s2, rs2;
            scales(mx2, s2, rs2);
            for (int u = q; u < nunit; u += TPR) {   // the same units: own values only
                float hi[4], lo[4] = {0.f, 0.f, 0.f, 0.f}, vals[4][4];
                const uint8_t *p = mid_slot(u);
                if (ES == 4) {
                    const float4 h = *reinterpret_cast<const float4 *>(p);
                    hi[0] = h.x; hi[1] = h.y; hi[2] = h.z; hi[3] = h.w;
                } else {
                    const float2 h0 = *reinterpret_cast<const float2 *>(p);
                    const float2 h1 = *reinterpret_cast<const float2 *>(p + a_piece);
                    hi[0] = h0.x; hi[1] = h0.y; hi[2] = h1.x; hi[3] = h1.y;
                    if (HL) {
                        const float2 l0 = *reinterpret_cast<const float2 *>(p + 2 * a_piece);
                        const float2 l1 = *reinterpret_cast<const float2 *>(p + 3 * a_piece);
                        lo[0] = l0.x; lo[1] = l0.y; lo[2] = l1.x; lo[3] = l1.y;
                    }
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    float qv[4];
                    if (MODE == MODE_FLOAT_TF32) split_tf32(hi[e], 0.f, qv);
                    else slice_fixed<S>(hi[e], lo[e], s2, qv);
#pragma unroll
                    for (int t2 = 0; t2 < 4; ++t2) vals[t2][e] = qv[t2];
                }
                store_unit<ES, S>(sA, a_piece, row, u, sbo, vals);
            }
            if (handoff()) break;
            rs_out = rs2;
            cs_out = cs2;
        }
        prev_tile = tile;
        prev_set = st;
        prev_rs = rs_out;
        prev_cs = cs_out;
    }
    // last tile (every staging buffer is idle now); the decision is made uniform first,
    // since the staged epilogue synchronizes the compute threads
    if (prev_tile >= 0 && !tc::bar_red_or(kBarCompute, NT, *sflag != 0)) {
        if (DOUBLE) wait_bar(bar2 + prev_set, ph2, prev_set);
        else wait_bar(bar1 + prev_set, ph1, prev_set);
        epilogue(prev_tile, prev_set, prev_rs, prev_cs, stg0, false);
    }
    tc::cp_async_wait_all();   // no copy may still target shared memory at exit
    }   // compute threads
    if (tid == 0 && *sflag) atomicExch(a.err, 1);
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, ncols);
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
    auto round1 = [](float x) {
        return TF32 ? tc::to_tf32(x) : __bfloat162float(__float2bfloat16_rn(x));
    };
    for (int c = 0; c < Kp / EPC; ++c) {
        float v[4][8] = {};
        for (int e = 0; e < EPC; ++e) v[0][e] = round1(A[size_t(tid) * k + c * EPC + e]);
        store_chunk<ES, 1>(sA, a_bytes, tid, c, sbo, v);
        for (int row = tid; row < Np; row += kRows) {
            for (int e = 0; e < EPC; ++e) v[0][e] = round1(B[size_t(row) * k + c * EPC + e]);
            store_chunk<ES, 1>(sB, b_bytes, row, c, sbo, v);
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
                                  float *hi, float *lo, float *g, float *g_lo, float *acc_hi, float *acc_lo)
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
        const double gv = f[c] * psi_occ[c * ld_occ + r];   // f_s psi_s as an FP32 pair
        const float gh = float(gv);
        g[e] = gh;
        g_lo[e] = float(gv - double(gh));
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

// (s, c) -= (gh + gl)(vh + vl): the leading product exactly (its rounding error from an
// FMA), the second-order products rounded into the compensation word.
__device__ __forceinline__ void sub_product(float &s, float &c, float gh, float gl, float vh, float vl)
{
    const float p = __fmul_rn(gh, vh);
    const float e = fmaf(gh, vh, -p);
    two_sum_add(s, c, -p);
    c -= e + fmaf(gh, vl, gl * vh);
}

__device__ __forceinline__ int diag_idx(int i, int j, int nI) { return i * nI - (i * (i - 1)) / 2 + (j - i); }

constexpr int kAccBlock = 8;    // widest block edge whose one-sweep J sums live in registers
constexpr int kAccWide = 16;   // widest edge of the one-sweep form with the J sums in shared memory

// One launch per batch: CUDA block (x, y) = 256 grid points of the outputs of Block y.
// Blocks of one batch have disjoint outputs, so no atomics are needed.  WIDE: plans with
// 16-orbital blocks keep the J-side sums of a block in shared memory ([j][thread], 32 KB
// per CTA), so each pair field is still read once without spending registers on them.
template <bool HL, bool WIDE>
__global__ void __launch_bounds__(256, 6) tc_accum_kernel(long N, const Block *blocks, const float *__restrict__ V,
                                                       long lo_off, const float *__restrict__ g,
                                                       const float *__restrict__ g_lo, float *__restrict__ acc_hi,
                                                       float *__restrict__ acc_lo)
{
    const Block b = blocks[blockIdx.y];
    const long r = long(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= N) return;
    const float *Vb = V + size_t(b.field0) * N + r;
    auto vh_at = [&](size_t fo) { return Vb[fo]; };
    auto vl_at = [&](size_t fo) { return HL ? Vb[lo_off + fo] : 0.f; };
    auto add = [&](float &s, float &c, int src, size_t fo) {
        sub_product(s, c, g[size_t(src) * N + r], g_lo[size_t(src) * N + r], vh_at(fo), vl_at(fo));
    };
    auto finish = [&](int t, float s, float c) {
        float hs = s + c;
        acc_lo[size_t(t) * N + r] = c - (hs - s);
        acc_hi[size_t(t) * N + r] = hs;
    };
    if constexpr (WIDE) {
        if (b.kind == BLK_SYM_OFF && b.nJ > kAccBlock && b.nJ <= kAccWide) {
            __shared__ float shs[kAccWide][256], shc[kAccWide][256];
            const int t = threadIdx.x;
            for (int j = 0; j < b.nJ; ++j) {
                shs[j][t] = acc_hi[size_t(b.J0 + j) * N + r];
                shc[j][t] = acc_lo[size_t(b.J0 + j) * N + r];
            }
#pragma unroll 1
            for (int i = 0; i < b.nI; ++i) {
                const int oi = b.I0 + i;
                const float gih = g[size_t(oi) * N + r], gil = g_lo[size_t(oi) * N + r];
                float si = acc_hi[size_t(oi) * N + r], ci = acc_lo[size_t(oi) * N + r];
#pragma unroll 4
                for (int j = 0; j < b.nJ; ++j) {
                    const size_t fo = size_t(i * b.nJ + j) * N;
                    const float vh = vh_at(fo), vl = vl_at(fo);
                    float sj = shs[j][t], cj = shc[j][t];
                    sub_product(sj, cj, gih, gil, vh, vl);
                    shs[j][t] = sj;
                    shc[j][t] = cj;
                    const size_t src = size_t(b.J0 + j) * N + r;
                    sub_product(si, ci, g[src], g_lo[src], vh, vl);
                }
                finish(oi, si, ci);
            }
            for (int j = 0; j < b.nJ; ++j) finish(b.J0 + j, shs[j][t], shc[j][t]);
            return;
        }
    }
    if (b.kind == BLK_SYM_OFF && b.nJ <= kAccBlock) {
        // Both sides in one sweep over the block's fields: field (i, j) adds to output J0+j
        // (source I0+i) and to output I0+i (source J0+j), so each field is read from memory
        // once. Per output the terms still come in the order of the other index, as below.
        float sj[kAccBlock], cj[kAccBlock];
#pragma unroll
        for (int j = 0; j < kAccBlock; ++j)
            if (j < b.nJ) {
                sj[j] = acc_hi[size_t(b.J0 + j) * N + r];
                cj[j] = acc_lo[size_t(b.J0 + j) * N + r];
            }
#pragma unroll 1
        for (int i = 0; i < b.nI; ++i) {
            const int oi = b.I0 + i;
            const float gih = g[size_t(oi) * N + r], gil = g_lo[size_t(oi) * N + r];
            float si = acc_hi[size_t(oi) * N + r], ci = acc_lo[size_t(oi) * N + r];
#pragma unroll
            for (int j = 0; j < kAccBlock; ++j)
                if (j < b.nJ) {
                    const size_t fo = size_t(i * b.nJ + j) * N;
                    const float vh = vh_at(fo), vl = vl_at(fo);
                    sub_product(sj[j], cj[j], gih, gil, vh, vl);
                    const size_t src = size_t(b.J0 + j) * N + r;
                    sub_product(si, ci, g[src], g_lo[src], vh, vl);
                }
            finish(oi, si, ci);
        }
#pragma unroll
        for (int j = 0; j < kAccBlock; ++j)
            if (j < b.nJ) finish(b.J0 + j, sj[j], cj[j]);
        return;
    }
    if (b.kind == BLK_SYM_DIAG) {
        for (int t = 0; t < b.nI; ++t) {
            const int o = b.I0 + t;
            float s = acc_hi[size_t(o) * N + r], c = acc_lo[size_t(o) * N + r];
            for (int q = 0; q < b.nI; ++q) {
                const int fi = q <= t ? diag_idx(q, t, b.nI) : diag_idx(t, q, b.nI);
                add(s, c, b.I0 + q, size_t(fi) * N);
            }
            finish(o, s, c);
        }
        return;
    }
    for (int j = 0; j < b.nJ; ++j) {
        const int o = b.J0 + j;
        float s = acc_hi[size_t(o) * N + r], c = acc_lo[size_t(o) * N + r];
        for (int i = 0; i < b.nI; ++i) add(s, c, b.I0 + i, size_t(i * b.nJ + j) * N);
        finish(o, s, c);
    }
    if (b.kind == BLK_SYM_OFF) {
        for (int i = 0; i < b.nI; ++i) {
            const int o = b.I0 + i;
            float s = acc_hi[size_t(o) * N + r], c = acc_lo[size_t(o) * N + r];
            for (int j = 0; j < b.nJ; ++j) add(s, c, b.J0 + j, size_t(i * b.nJ + j) * N);
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
// Threads per tile row.  The pass kernels are bound by instruction issue: 6 or 7 threads
// per row (more warps, less work each) measured slower than 4.
constexpr int kTPR = 4;
size_t pass_smem(int prec, int Np, bool dbl, int load, int nbuf = 1, int nsets = 1, int store = STORE_NSLOW)
{
    const PrecInfo pi = prec_info(prec);
    size_t a = size_t(nsets) * pi.S * kRows * Np * pi.es;   // A buffers
    const int pitch = load == LOAD_KFAST ? Np + 4 : Np;   // KFAST rows are padded, [k][row] layouts not
    size_t staging = size_t(load == LOAD_PAIR ? 4 : (pi.hl ? 2 : 1)) * kRows * pitch * sizeof(float);
    if (store == STORE_NFAST) staging = std::max(staging, size_t(pi.hl ? 2 : 1) * kRows * (Np + 4) * sizeof(float));
    staging *= size_t(nbuf);                                   // staging buffers in flight
    const size_t maxbuf = size_t(kRows) * kTPR * sizeof(float);   // one partial maximum per thread
    const size_t align = load == LOAD_KFAST ? 1024 : 0;          // K-fast staging alignment slack
    return (dbl ? 2 : 1) * image_bytes(prec, Np) + a + staging + maxbuf + 64 + align;
}

int tmem_cols(int prec, int Np, int nsets = 1) { return pow2_cols(nsets * prec_info(prec).nacc * Np); }

template <int MODE, int S, int SB, bool HL, int LOAD, int STORE, bool DOUBLE, int NBUF, int NSETS>
int launch_tc_pass_nb(Plan &P, int kind, int prec, const TcPassArgs &a, cudaStream_t s)
{
    auto kern = tc_pass_kernel<MODE, S, SB, HL, LOAD, STORE, DOUBLE, kTPR, NBUF, NSETS>;
    size_t smem = pass_smem(prec, a.Np, DOUBLE, LOAD, NBUF, NSETS, STORE);
    // TMEM: co-resident CTAs must not ask for more than 512 columns in total, so the
    // shared-memory request is raised until at most 512 / cols CTAs fit on one SM.
    const int cols = tmem_cols(prec, a.Np, NSETS);
    const int max_ctas = std::max(1, 512 / cols);
    const size_t sm_total = 233472;   // 228 KB of shared memory per SM
    size_t floor_req = sm_total / size_t(max_ctas + 1) - 1024 + 64;
    smem = std::max(smem, floor_req);
    if (smem > 232448 || cols > 512) {
        set_error("split-precision pass: operand images exceed on-chip memory for this grid size");
        return EXX_ERR_UNSUPPORTED;
    }
    EXX_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    int per_sm = 0;
    EXX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRows * kTPR + 64, smem));
    per_sm = std::max(1, std::min(per_sm, max_ctas));
    const long rows = long(a.nfields) * a.R;
    const long ntiles = (rows + kRows - 1) / kRows;
    const int grid = int(std::min<long>(ntiles, long(P.num_sms) * per_sm));
    int tb = timing_begin(P, kind, s);
    kern<<<grid, kRows * kTPR + 64, smem, s>>>(a);
    timing_end(P, tb, s);
    EXX_LAUNCH("tc_pass_kernel");
    P.launches++;
    return EXX_OK;
}

// Largest configuration that fits: pipelined with two staging buffers, pipelined with one,
// or (long axes) one A buffer and one TMEM set.
template <int MODE, int S, int SB, bool HL, int LOAD, int STORE, bool DOUBLE>
int launch_tc_pass(Plan &P, int kind, int prec, const TcPassArgs &a, cudaStream_t s)
{
    const size_t lim = 232448;
    const bool tm2 = tmem_cols(prec, a.Np, 2) <= 512;
    if (LOAD != LOAD_PAIR && tm2 && pass_smem(prec, a.Np, DOUBLE, LOAD, 2, 2, STORE) <= lim)
        return launch_tc_pass_nb<MODE, S, SB, HL, LOAD, STORE, DOUBLE, 2, 2>(P, kind, prec, a, s);
    if (tm2 && pass_smem(prec, a.Np, DOUBLE, LOAD, 1, 2, STORE) <= lim)
        return launch_tc_pass_nb<MODE, S, SB, HL, LOAD, STORE, DOUBLE, 1, 2>(P, kind, prec, a, s);
    return launch_tc_pass_nb<MODE, S, SB, HL, LOAD, STORE, DOUBLE, 1, 1>(P, kind, prec, a, s);
}

// cuTensorMapEncodeTiled, fetched from the driver through the runtime once (no link
// dependency on the driver library; without a driver the TMA path is simply not taken).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// 3D FP32 tensor (R rows fastest, L lines, F fields) at `base`, lines R apart, fields N
// apart, read in 128 x K x 1 boxes.  Requires 16-byte aligned base and R, N multiples of 4.
bool make_tile_map(CUtensorMap *m, const float *base, long R, long L, long F, long N, int K)
{
    EncodeTiledFn fn = encode_tiled();
    if (!fn || (reinterpret_cast<uintptr_t>(base) & 15) || (R & 3) || (N & 3) || K < 1 || K > 256) return false;
    const cuuint64_t dims[3] = {cuuint64_t(R), cuuint64_t(L), cuuint64_t(F)};
    const cuuint64_t strides[2] = {cuuint64_t(R) * 4, cuuint64_t(N) * 4};
    const cuuint32_t box[3] = {cuuint32_t(kRows), cuuint32_t(K), 1};
    const cuuint32_t es[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2D FP32 tensor (K columns fastest, `rows` rows, rows K apart) read in 16 x 128 boxes with
// the 64-byte swizzle; columns >= K of the last box come back as zeros.
bool make_kfast_map(CUtensorMap *m, const float *base, int K, long rows)
{
    EncodeTiledFn fn = encode_tiled();
    if (!fn || (reinterpret_cast<uintptr_t>(base) & 15) || (K & 3) || K < 16 || rows < kRows) return false;
    const cuuint64_t dims[2] = {cuuint64_t(K), cuuint64_t(rows)};
    const cuuint64_t strides[1] = {cuuint64_t(K) * 4};
    const cuuint32_t box[2] = {16, cuuint32_t(kRows)};
    const cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// One launch of pass kernel `kind` (0..4 = P1..P5; 5 = P3's forward half alone, 6 = its
// inverse half alone, used when the y axis is cut into blocks).
template <int MODE, int S, int SB, bool HL>
int launch_kind(Plan &P, int kind, int prec, const TcPassArgs &a, cudaStream_t s)
{
    switch (kind) {
    case 0: return launch_tc_pass<MODE, S, SB, HL, LOAD_PAIR, STORE_NSLOW, false>(P, EXX_TIMING_PASS1, prec, a, s);
    case 1: return launch_tc_pass<MODE, S, SB, HL, LOAD_KFAST, STORE_NSLOW, false>(P, EXX_TIMING_PASS2, prec, a, s);
    case 2: return launch_tc_pass<MODE, S, SB, HL, LOAD_KFAST, STORE_NFAST, true>(P, EXX_TIMING_PASS3, prec, a, s);
    case 3: return launch_tc_pass<MODE, S, SB, HL, LOAD_KSLOW, STORE_NFAST, false>(P, EXX_TIMING_PASS4, prec, a, s);
    case 4: return launch_tc_pass<MODE, S, SB, HL, LOAD_KSLOW, STORE_NSLOW, false>(P, EXX_TIMING_PASS5, prec, a, s);
    default: return launch_tc_pass<MODE, S, SB, HL, LOAD_KFAST, STORE_NFAST, false>(P, EXX_TIMING_PASS3, prec, a, s);
    }
}

template <int MODE, int S, int SB, bool HL>
int solve_batch_t(Plan &P, int prec, const int2 *pairs_d, int nfields, float *bufA, float *bufB, cudaStream_t s)
{
    float *src = nullptr, *dst = bufA;
    // passes as (kind, B slot): P3 is one kernel (two GEMMs) unless y is cut into blocks
    const bool ycut = P.tc_ysplit[prec] != 0;
    int kinds[6], slots[6], np = 0;
    for (int pass = 0; pass < 5; ++pass) {
        if (pass == 2 && ycut) {
            kinds[np] = 5; slots[np++] = 2;
            kinds[np] = 6; slots[np++] = 3;
        } else {
            kinds[np] = pass;
            slots[np++] = pass <= 2 ? pass : pass + 1;   // fused P3 uses slots 2 (fwd) and 3 (inv)
        }
    }
    const int axis_of[6] = {2, 0, 1, 1, 0, 2};
    for (int i = 0; i < np; ++i) {
        const int kind = kinds[i], slot = slots[i];
        const PassGeom g = pass_geom(P.n, kind >= 5 ? 2 : kind);
        const int d = axis_of[slot], nd = P.n[d], nb = P.tc_nblk[prec][d], bs = P.tc_bsz[prec][d];
        TcPassArgs a{};
        a.nfields = nfields;
        a.R = g.R;
        a.divR = make_fastdiv(uint32_t(g.R));
        if (long(nfields) * g.R >= (1L << 31)) {
            set_error("split-precision pass: more than 2^31 rows in one batch");
            return EXX_ERR_UNSUPPORTED;
        }
        a.Np = pad16(bs);
        a.N = P.N;
        a.in = src;
        a.out = dst;
        a.in_pitch = a.out_pitch = nd;
        a.lo_off = HL ? P.tc_lo_off : 0;
        a.img_bytes = uint32_t(image_bytes(prec, a.Np));
        a.F = static_cast<const float *>(P.F32.p);
        a.Flo = a.F + P.N;
        a.psi_hi = static_cast<const float *>(P.psi32.p);
        a.psi_lo = a.psi_hi + P.psi32.bytes / 8;
        a.occ_off = P.tc_occ_off;
        a.pairs = pairs_d;
        a.err = static_cast<int *>(P.err_d.p);
        const uint8_t *img1 = static_cast<const uint8_t *>(P.Btc[prec][slot].p);
        const bool kslow_in = g.load != LOAD_KFAST, nslow_out = g.store == STORE_NSLOW;
        for (int h = 0; h < nb; ++h)
            for (int c = 0; c < nb; ++c) {   // K-blocks in order: the first writes, the others add
                a.K = std::min(bs, nd - c * bs);
                a.Kout = std::min(bs, nd - h * bs);
                a.divK4 = make_fastdiv(uint32_t(std::max(1, a.K / 4)));
                a.divKo4 = make_fastdiv(uint32_t(std::max(1, a.Kout / 4)));
                a.in_off = kslow_in ? long(c) * bs * g.R : long(c) * bs;
                a.out_off = nslow_out ? long(h) * bs * g.R : long(h) * bs;
                a.acc = c > 0;
                a.B1 = img1 + size_t(c * nb + h) * a.img_bytes;
                a.B2 = kind == 2 ? static_cast<const uint8_t *>(P.Btc[prec][3].p) : nullptr;
                // [k][row] inputs of fields of R = 128 m rows: one TMA box per plane per tile
                a.use_tma = 0;
                a.koff = c * bs;
                if (g.load == LOAD_KFAST && nb == 1 && (a.K & 3) == 0 && (a.lo_off & 3) == 0 && (P.N & 3) == 0) {
                    // rows of the batch are back to back: a 2D tensor (K, nfields R)
                    const long nrows = long(nfields) * g.R;
                    a.use_tma = make_kfast_map(&a.tm[0], a.in, a.K, nrows) &&
                                (!HL || make_kfast_map(&a.tm[1], a.in + a.lo_off, a.K, nrows));
                } else if ((g.load == LOAD_PAIR || g.load == LOAD_KSLOW) && g.R % kRows == 0 && (a.lo_off & 3) == 0) {
                    bool ok;
                    if (g.load == LOAD_PAIR) {
                        const long ncols = long(P.psi32.bytes / (8 * size_t(P.N)));
                        ok = make_tile_map(&a.tm[0], a.psi_hi, g.R, nd, ncols, P.N, a.K) &&
                             make_tile_map(&a.tm[1], a.psi_lo, g.R, nd, ncols, P.N, a.K);
                    } else {
                        ok = make_tile_map(&a.tm[0], a.in, g.R, nd, nfields, P.N, a.K) &&
                             (!HL || make_tile_map(&a.tm[1], a.in + a.lo_off, g.R, nd, nfields, P.N, a.K));
                    }
                    a.use_tma = ok ? 1 : 0;
                }
                const bool scale = kind == 5 && c == nb - 1;   // the sums of this block are complete
                a.Fs = scale ? a.F : nullptr;
                a.Fs_lo = scale ? a.Flo : nullptr;
                a.f_noff = h * bs;
                if (int rc = launch_kind<MODE, S, SB, HL>(P, kind, prec, a, s)) return rc;
            }
        src = dst;
        dst = (dst == bufA) ? bufB : bufA;
    }
    P.tc_result = src;
    return EXX_OK;
}

}  // namespace

// Does every pass on axis d fit on chip with blocks of Np (padded) points?  x is read by
// passes 2 (KFAST) and 4 (KSLOW), y by pass 3 (KFAST; two GEMMs in one kernel unless
// split), z by passes 1 (pair products) and 5 (KSLOW).
static bool axis_fits(int prec, int d, int Np, bool split)
{
    size_t need = 0;
    if (d == 0)
        need = std::max(pass_smem(prec, Np, false, LOAD_KFAST),
                        pass_smem(prec, Np, false, LOAD_KSLOW, 1, 1, STORE_NFAST));
    if (d == 1) need = pass_smem(prec, Np, !split, LOAD_KFAST, 1, 1, STORE_NFAST);
    if (d == 2) need = std::max(pass_smem(prec, Np, false, LOAD_PAIR), pass_smem(prec, Np, false, LOAD_KSLOW));
    return need <= 232448 && tmem_cols(prec, Np) <= 512;
}

int tc_upload(Plan &P, int prec)
{
    const PrecInfo pi = prec_info(prec);
    const int axis_of[6] = {2, 0, 1, 1, 0, 2};
    const int inv_of[6] = {0, 0, 0, 1, 1, 1};
    // Long axes are cut into nb blocks of b = ceil(n / nb) points: a mode product then
    // becomes nb x nb block products, out_h = sum_c in_c V_ch, summed in hi/lo FP32.
    // Pass 3 runs its two GEMMs in one kernel when y fits whole with both images on chip,
    // else as two kernels (forward with the f(Lambda) scaling, inverse).
    int nblk[3], bsz[3];
    const bool ysplit = !axis_fits(prec, 1, pad16(P.n[1]), false);
    for (int d = 0; d < 3; ++d) {
        int nb = 1;
        while (nb <= 16 && !axis_fits(prec, d, pad16((P.n[d] + nb - 1) / nb), d == 1 && ysplit)) ++nb;
        if (nb > 16) {
            set_error("split precision: grid axis too long for the on-chip operand images of this build");
            return EXX_ERR_UNSUPPORTED;
        }
        nblk[d] = nb;
        bsz[d] = (P.n[d] + nb - 1) / nb;
    }
    for (int slot = 0; slot < 6; ++slot) {
        const int d = axis_of[slot], nd = P.n[d], nb = nblk[d], bs = bsz[d], Np = pad16(bs);
        const uint32_t sbo = uint32_t(Np) * pi.es * 8;
        const size_t piece = size_t(Np) * Np * pi.es;
        const size_t ib = image_bytes(prec, Np);
        const int epc = 16 / pi.es;
        std::vector<uint8_t> all(ib * nb * nb, 0);
        for (int c = 0; c < nb; ++c)
            for (int h = 0; h < nb; ++h) {
                uint8_t *img = all.data() + ib * size_t(c * nb + h);
                // coefficient of output mode n0+n from input k0+k: forward V(k, n), inverse V(n, k)
                const int k0 = c * bs, n0 = h * bs;
                const int kl = std::min(bs, nd - k0), nl = std::min(bs, nd - n0);
                auto coef = [&](int n, int k) {
                    if (n >= nl || k >= kl) return 0.0;
                    const size_t gn = size_t(n0 + n), gk = size_t(k0 + k);
                    return inv_of[slot] ? P.V[d][gn + size_t(nd) * gk] : P.V[d][gk + size_t(nd) * gn];
                };
                auto put = [&](int q, int n, int k, float v) {
                    size_t off = piece * q + img_off(n, k / epc, sbo) + size_t(k % epc) * pi.es;
                    if (pi.es == 4) {
                        std::memcpy(&img[off], &v, 4);
                    } else {
                        uint32_t u;
                        std::memcpy(&u, &v, 4);
                        uint16_t hb = uint16_t(u >> 16);   // v is bf16-exact (at most 8 significant bits)
                        std::memcpy(&img[off], &hb, 2);
                    }
                };
                std::vector<float> cs(Np, 1.0f);
                for (int n = 0; n < Np; ++n) {
                    if (pi.mode == MODE_FIXED_BF16) {
                        double mx = 0.0;
                        for (int k = 0; k < Np; ++k) mx = std::max(mx, std::fabs(coef(n, k)));
                        int e = 0;
                        if (mx > 0.0) std::frexp(mx, &e);
                        const double sc = std::ldexp(1.0, 7 - e);
                        cs[n] = float(std::ldexp(1.0, e - 7));
                        for (int k = 0; k < Np; ++k) {
                            double t = coef(n, k) * sc;
                            for (int q = 0; q < pi.SB; ++q) {   // t = q0 + q1/2^8 + q2/2^16 + ...
                                const double qq = std::nearbyint(t);
                                put(q, n, k, float(std::ldexp(qq, -8 * q)));   // slice q carries 2^(-8q)
                                t = (t - qq) * 256.0;
                            }
                        }
                    } else {
                        for (int k = 0; k < Np; ++k) {
                            double rem = coef(n, k);
                            for (int q = 0; q < pi.SB; ++q) {
                                float pv = host_tf32(rem);
                                rem -= double(pv);
                                put(q, n, k, pv);
                            }
                        }
                    }
                }
                if (pi.mode == MODE_FIXED_BF16) std::memcpy(&img[piece * pi.SB], cs.data(), size_t(Np) * 4);
            }
        if (int rc = dev_reserve(P.Btc[prec][slot], all.size())) return rc;
        EXX_CUDA(cudaMemcpy(P.Btc[prec][slot].p, all.data(), all.size(), cudaMemcpyHostToDevice));
    }
    for (int d = 0; d < 3; ++d) {
        P.tc_nblk[prec][d] = nblk[d];
        P.tc_bsz[prec][d] = bsz[d];
    }
    P.tc_ysplit[prec] = ysplit;
    if (int rc = dev_reserve(P.err_d, 16)) return rc;
    EXX_CUDA(cudaMemset(P.err_d.p, 0, 16));
    return EXX_OK;
}

int tc_reserve_orbitals(Plan &P, int n_occ, int n_in, bool aliased)
{
    const int ncols = n_in + (aliased ? 0 : n_occ);
    const size_t plane = size_t(ncols) * P.N;
    if (P.psi32.bytes != 2 * plane * sizeof(float)) dev_free(P.psi32);   // psi_lo follows psi_hi exactly
    if (int rc = dev_reserve(P.psi32, 2 * plane * sizeof(float))) return rc;
    if (int rc = dev_reserve(P.g32, 2 * size_t(n_occ) * P.N * sizeof(float))) return rc;   // hi, lo planes
    if (int rc = dev_reserve(P.acc_hi, size_t(n_in) * P.N * sizeof(float))) return rc;
    if (int rc = dev_reserve(P.acc_lo, size_t(n_in) * P.N * sizeof(float))) return rc;
    P.tc_occ_off = aliased ? 0 : n_in;
    P.tc_n_occ = n_occ;
    return EXX_OK;
}

int tc_prepare_orbitals(Plan &P, const double *psi_occ, int n_occ, long ld_occ, const double *f,
                        const double *psi_in, int n_in, long ld_in, bool aliased, cudaStream_t s)
{
    const int ncols = n_in + (aliased ? 0 : n_occ);
    const size_t plane = size_t(ncols) * P.N;
    float *hi = static_cast<float *>(P.psi32.p);
    int tb = timing_begin(P, EXX_TIMING_PREP, s);
    tc_prepare_kernel<<<4 * P.num_sms, 256, 0, s>>>(P.N, n_in, psi_in, ld_in, n_occ, psi_occ, ld_occ, aliased ? 0 : 1,
                                                   f, hi, hi + plane, static_cast<float *>(P.g32.p),
                                                   static_cast<float *>(P.g32.p) + size_t(n_occ) * P.N,
                                                   static_cast<float *>(P.acc_hi.p), static_cast<float *>(P.acc_lo.p));
    timing_end(P, tb, s);
    EXX_LAUNCH("tc_prepare_kernel");
    P.launches++;
    return EXX_OK;
}

int tc_solve_batch(Plan &P, int prec, const int2 *pairs_d, int nfields, float *bufA, float *bufB, cudaStream_t s)
{
    switch (prec) {
    case EXX_PREC_BF16X3: return solve_batch_t<MODE_FIXED_BF16, 2, 2, false>(P, prec, pairs_d, nfields, bufA, bufB, s);
    case EXX_PREC_BF16X6: return solve_batch_t<MODE_FIXED_BF16, 3, 4, false>(P, prec, pairs_d, nfields, bufA, bufB, s);
    case EXX_PREC_BF16X10: return solve_batch_t<MODE_FIXED_BF16, 4, 4, true>(P, prec, pairs_d, nfields, bufA, bufB, s);
    case EXX_PREC_TF32X3: return solve_batch_t<MODE_FLOAT_TF32, 2, 2, false>(P, prec, pairs_d, nfields, bufA, bufB, s);
    case EXX_PREC_BF16X7: return tc3_solve_batch(P, pairs_d, nfields, bufA, bufB, s);
    default: return EXX_ERR_INVALID_ARG;
    }
}

int tc_accumulate(Plan &P, const Block *blocks_d, int nblocks, const float *V, cudaStream_t s)
{
    dim3 grid(unsigned((P.N + 255) / 256), unsigned(nblocks));
    int tb = timing_begin(P, EXX_TIMING_ACCUM, s);
    const float *g = static_cast<const float *>(P.g32.p), *g_lo = g + size_t(P.tc_n_occ) * P.N;
    float *ah = static_cast<float *>(P.acc_hi.p), *al = static_cast<float *>(P.acc_lo.p);
    const bool wide = P.block_orbitals > kAccBlock;
    if (prec_info(P.prec).hl) {
        if (wide)
            tc_accum_kernel<true, true><<<grid, 256, 0, s>>>(P.N, blocks_d, V, P.tc_lo_off, g, g_lo, ah, al);
        else
            tc_accum_kernel<true, false><<<grid, 256, 0, s>>>(P.N, blocks_d, V, P.tc_lo_off, g, g_lo, ah, al);
    } else {
        if (wide)
            tc_accum_kernel<false, true><<<grid, 256, 0, s>>>(P.N, blocks_d, V, 0, g, g_lo, ah, al);
        else
            tc_accum_kernel<false, false><<<grid, 256, 0, s>>>(P.N, blocks_d, V, 0, g, g_lo, ah, al);
    }
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

bool tc_is_hilo(int prec) { return prec_info(prec).hl != 0; }

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

namespace {
// The bounded waits of the pass kernels on a barrier that nothing completes: the poll limit
// (five-pass kernels) or the wall-time limit (three-pass kernels) runs out, the kernel
// records the timeout in the error word (bit 0: polled wait, bit 1: timed wait) and returns.
__global__ void tc_wait_timeout_kernel(uint32_t limit, uint64_t limit_ns, int *err)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) tc::mbar_init(&bar, 1);
    __syncthreads();
    if (!tc::mbar_wait_bounded(&bar, 0, limit) && threadIdx.x == 0) atomicOr(err, 1);
    if (!tc::mbar_wait_timed(&bar, 0, limit_ns) && threadIdx.x == 0) atomicOr(err, 2);
}
}  // namespace

int tc_wait_timeout_probe(int *status_h)
{
    int *err = nullptr;
    EXX_CUDA(cudaMalloc(&err, sizeof(int)));
    cudaError_t e = cudaMemset(err, 0, sizeof(int));
    if (e == cudaSuccess) {
        tc_wait_timeout_kernel<<<1, 32>>>(1u << 12, 2000000ull, err);
        e = cudaGetLastError();
    }
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(err);
    if (e != cudaSuccess) return cuda_fail(e, "tc_wait_timeout_probe");
    // both waits must give up: status EXX_ERR_TIMEOUT only when both did
    *status_h = h == 3 ? EXX_ERR_TIMEOUT : EXX_OK;
    if (h == 3) set_error("both bounded mbarrier waits ran out (wait-timeout probe)");
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
