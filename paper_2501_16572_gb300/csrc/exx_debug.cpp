// Host-only inspection hooks (include/exx_debug.h).
#include "exx_internal.h"
#include "../../include/exx_debug.h"

#include <algorithm>

extern "C" {

int exx_debug_tc3_layout(int n1, int n2, int n3, int share01, int *out)
{
    if (n1 < 2 || n2 < 2 || n3 < 2 || n1 > 256 || n2 > 256 || n3 > 256 || !out) return EXX_ERR_INVALID_ARG;
    exx::tc3_debug_layout(n1, n2, n3, share01 != 0, out);
    return EXX_OK;
}

int exx_debug_matrix_digits(int nout, int nk, const double *C, int WN, int Kp, int n0, int k0, float *digits,
                            float *scales)
{
    if (nout < 1 || nk < 1 || WN < 1 || Kp < 8 || Kp % 8 || WN % 8 || n0 < 0 || k0 < 0 || !C || !digits || !scales)
        return EXX_ERR_INVALID_ARG;
    exx::tc3_debug_matrix_digits(nout, nk, C, WN, Kp, n0, k0, digits, scales);
    return EXX_OK;
}

int exx_debug_fd_weights(int p, double *w)
{
    if (p < 1 || p > 12 || !w) return EXX_ERR_INVALID_ARG;
    exx::fd_weights(p, w);
    return EXX_OK;
}

int exx_debug_second_derivative(int n, double h, int bc, int p, double *D)
{
    if (n < 1 || p < 1 || p > 12 || !D || !(h > 0)) return EXX_ERR_INVALID_ARG;
    exx::second_derivative(n, h, bc, p, D);
    return EXX_OK;
}

int exx_debug_sym_eig(int n, const double *A, double *V, double *lam)
{
    if (n < 1 || !A || !V || !lam) return EXX_ERR_INVALID_ARG;
    return exx::sym_eig(n, A, V, lam) ? EXX_ERR_UNSUPPORTED : EXX_OK;
}

int exx_debug_schedule(int n_occ, int n_in, int aliased, int block, int max_pairs, long *npairs,
                       long *nbatches, long *nblocks, int *pairs, int *batches, int *blocks)
{
    if (n_occ < 1 || n_in < 1 || block < 1 || block > 32 || max_pairs < 1 || !npairs || !nbatches || !nblocks)
        return EXX_ERR_INVALID_ARG;
    exx::Schedule S = exx::build_schedule(n_occ, n_in, aliased != 0, block, max_pairs);
    *npairs = long(S.pairs.size());
    *nbatches = long(S.batches.size());
    *nblocks = long(S.blocks.size());
    if (pairs)
        for (size_t i = 0; i < S.pairs.size(); ++i) {
            pairs[2 * i] = S.pairs[i].x;
            pairs[2 * i + 1] = S.pairs[i].y;
        }
    if (batches)
        for (size_t i = 0; i < S.batches.size(); ++i) {
            batches[3 * i] = S.batches[i].nfields;
            batches[3 * i + 1] = S.batches[i].block0;
            batches[3 * i + 2] = S.batches[i].nblocks;
        }
    if (blocks)
        for (size_t i = 0; i < S.blocks.size(); ++i) {
            const exx::Block &b = S.blocks[i];
            int v[6] = {b.I0, b.nI, b.J0, b.nJ, b.kind, b.field0};
            std::copy(v, v + 6, blocks + 6 * i);
        }
    return EXX_OK;
}

int exx_debug_tc_gemm(int tf32, int n, int k, const float *A, const float *B, float *D, int *err)
{
    if (!A || !B || !D || !err) return EXX_ERR_INVALID_ARG;
    return exx::tc_unit_gemm(tf32, n, k, A, B, D, err);
}

int exx_debug_fastdiv(unsigned d, int count, const unsigned *n, unsigned *q)
{
    if (d < 1 || count < 0 || (count > 0 && (!n || !q))) return EXX_ERR_INVALID_ARG;
    const exx::FastDiv f = exx::make_fastdiv(d);
    for (int i = 0; i < count; ++i) q[i] = exx::fast_div(n[i], f);
    return EXX_OK;
}

int exx_debug_wait_timeout(int *status_h)
{
    if (!status_h) return EXX_ERR_INVALID_ARG;
    return exx::tc_wait_timeout_probe(status_h);
}

}  // extern "C"
