// Host-side FP64 setup of a plan and the pair scheduler.
//
//  * FD weights of the central second difference of order 2p (closed form).
//  * 1D second-derivative operators with Dirichlet (zero outside) or periodic ends.
//  * Symmetric eigen-decomposition: Householder reduction to tridiagonal form, then
//    implicit QL sweeps with a Wilkinson-type shift (Sec. II.A, Eqs. 6-7 need
//    D_d = V_d diag(lambda_d) V_d^T for each axis).
//  * f of Eq. 5 on the eigenvalue sums.
//  * Pair blocks grouped into rounds whose blocks write disjoint outputs, the rounds
//    cut into batches of at most n_c pairs (Sec. II.B's batch of right-hand sides).
#include "exx_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace exx {

void fd_weights(int p, double *w)
{
    double sum = 0.0;
    for (int k = 1; k <= p; ++k) {
        // 2 (-1)^(k+1) (p!)^2 / (k^2 (p-k)! (p+k)!), ratio of factorials as a product
        double ratio = 1.0;
        for (int i = 0; i < k; ++i) ratio *= double(p - i) / double(p + 1 + i);
        double v = 2.0 * ratio / (double(k) * double(k));
        w[k] = (k & 1) ? v : -v;
        sum += w[k];
    }
    w[0] = -2.0 * sum;
}

void second_derivative(int n, double h, int bc, int p, double *D)
{
    std::vector<double> w(p + 1);
    fd_weights(p, w.data());
    const double s = 1.0 / (h * h);
    std::fill(D, D + size_t(n) * n, 0.0);
    for (int row = 0; row < n; ++row) {
        for (int k = -p; k <= p; ++k) {
            int col = row + k;
            if (bc == EXX_BC_PERIODIC) {
                col %= n;
                if (col < 0) col += n;
            } else if (col < 0 || col >= n) {
                continue;
            }
            D[row + size_t(n) * col] += w[k < 0 ? -k : k] * s;
        }
    }
}

// Householder tridiagonalisation: on return Q (n x n, column-major) is orthogonal and
// Q^T A Q is tridiagonal with diagonal d and sub-diagonal e[0..n-2].
static void householder_tridiag(int n, std::vector<double> &A, std::vector<double> &Q,
                                std::vector<double> &d, std::vector<double> &e)
{
    auto a = [&](int i, int j) -> double & { return A[i + size_t(n) * j]; };
    Q.assign(size_t(n) * n, 0.0);
    for (int i = 0; i < n; ++i) Q[i + size_t(n) * i] = 1.0;
    std::vector<double> v(n), pvec(n);
    for (int k = 0; k + 2 < n; ++k) {
        double norm2 = 0.0;
        for (int i = k + 1; i < n; ++i) norm2 += a(i, k) * a(i, k);
        double xnorm = std::sqrt(norm2);
        if (xnorm == 0.0) continue;
        double x0 = a(k + 1, k);
        double alpha = x0 >= 0.0 ? -xnorm : xnorm;
        // v = x - alpha e_1, normalised
        for (int i = 0; i < n; ++i) v[i] = 0.0;
        v[k + 1] = x0 - alpha;
        for (int i = k + 2; i < n; ++i) v[i] = a(i, k);
        double vn = 0.0;
        for (int i = k + 1; i < n; ++i) vn += v[i] * v[i];
        vn = std::sqrt(vn);
        if (vn == 0.0) continue;
        for (int i = k + 1; i < n; ++i) v[i] /= vn;
        // trailing block update A <- H A H with H = I - 2 v v^T (rows/cols k..n-1)
        for (int i = k; i < n; ++i) {
            double s = 0.0;
            for (int j = k + 1; j < n; ++j) s += a(i, j) * v[j];
            pvec[i] = s;
        }
        double K = 0.0;
        for (int i = k + 1; i < n; ++i) K += v[i] * pvec[i];
        for (int i = k; i < n; ++i) pvec[i] -= K * v[i];   // q = p - K v  (v[k] = 0)
        for (int j = k; j < n; ++j)
            for (int i = k; i < n; ++i) a(i, j) -= 2.0 * (v[i] * pvec[j] + pvec[i] * v[j]);
        // accumulate Q <- Q H
        for (int r = 0; r < n; ++r) {
            double s = 0.0;
            for (int j = k + 1; j < n; ++j) s += Q[r + size_t(n) * j] * v[j];
            for (int j = k + 1; j < n; ++j) Q[r + size_t(n) * j] -= 2.0 * s * v[j];
        }
    }
    d.resize(n);
    e.assign(n, 0.0);
    for (int i = 0; i < n; ++i) d[i] = a(i, i);
    for (int i = 0; i + 1 < n; ++i) e[i] = a(i + 1, i);
}

// Implicit QL iteration on the symmetric tridiagonal (d, e); rotations are applied to
// the columns of Q.  Returns 0 on convergence.
static int tridiag_ql(int n, std::vector<double> &d, std::vector<double> &e, std::vector<double> &Q)
{
    const double eps = 2.220446049250313e-16;
    for (int l = 0; l < n; ++l) {
        for (int sweep = 0;; ++sweep) {
            int m = l;
            for (; m + 1 < n; ++m) {
                double scale = std::fabs(d[m]) + std::fabs(d[m + 1]);
                if (std::fabs(e[m]) <= eps * scale) break;
            }
            if (m == l) break;
            if (sweep > 60) return -1;
            // shift: eigenvalue of the leading 2x2 block closest to d[l]
            double theta = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double rad = std::hypot(theta, 1.0);
            double shift = d[l] - e[l] / (theta + (theta >= 0 ? rad : -rad));
            // chase the bulge from the bottom (m) up to l
            double g = d[m] - shift;
            double s = 1.0, c = 1.0, pdel = 0.0;
            bool early = false;
            for (int i = m - 1; i >= l; --i) {
                double f = s * e[i], b = c * e[i];
                double r = std::hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) {       // split: the matrix decoupled at i+1
                    d[i + 1] -= pdel;
                    e[m] = 0.0;
                    early = true;
                    break;
                }
                s = f / r;
                c = g / r;
                double gg = d[i + 1] - pdel;
                double t = (d[i] - gg) * s + 2.0 * c * b;
                pdel = s * t;
                d[i + 1] = gg + pdel;
                g = c * t - b;
                for (int k = 0; k < n; ++k) {
                    double qi = Q[k + size_t(n) * i], qi1 = Q[k + size_t(n) * (i + 1)];
                    Q[k + size_t(n) * (i + 1)] = s * qi + c * qi1;
                    Q[k + size_t(n) * i] = c * qi - s * qi1;
                }
            }
            if (early) continue;
            d[l] -= pdel;
            e[l] = g;
            e[m] = 0.0;
        }
    }
    return 0;
}

int sym_eig(int n, const double *A_in, double *V, double *lam)
{
    std::vector<double> A(A_in, A_in + size_t(n) * n), Q, d, e;
    if (n == 1) {
        V[0] = 1.0;
        lam[0] = A[0];
        return 0;
    }
    householder_tridiag(n, A, Q, d, e);
    if (tridiag_ql(n, d, e, Q)) return -1;
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return d[x] < d[y]; });
    for (int j = 0; j < n; ++j) {
        lam[j] = d[order[j]];
        for (int i = 0; i < n; ++i) V[i + size_t(n) * j] = Q[i + size_t(n) * order[j]];
    }
    return 0;
}

double kernel_f(double lam, int kernel, double omega)
{
    const double four_pi = 12.566370614359172;
    if (kernel == EXX_KERNEL_COULOMB) return -four_pi / lam;
    const double a = (kernel == EXX_KERNEL_ERFC_PAPER16PI) ? 4.0 * four_pi * omega * omega
                                                           : 4.0 * omega * omega;
    const double x = -lam;
    if (x == 0.0) return four_pi / a;
    return four_pi * (-std::expm1(-x / a)) / x;
}

PassGeom pass_geom(const int n[3], int pass)
{
    const int n1 = n[0], n2 = n[1], n3 = n[2];
    switch (pass) {
    case 0: return {LOAD_PAIR, STORE_NSLOW, 2, 0, 0, n1 * n2, n3};
    case 1: return {LOAD_KFAST, STORE_NSLOW, 0, 0, 0, n2 * n3, n1};
    case 2: return {LOAD_KFAST, STORE_NFAST, 1, 0, 1, n1 * n3, n2};
    case 3: return {LOAD_KSLOW, STORE_NFAST, 0, 1, 0, n2 * n3, n1};
    default: return {LOAD_KSLOW, STORE_NSLOW, 2, 1, 0, n1 * n2, n3};
    }
}

// Circle-method round robin over G groups: each round is a list of disjoint group pairs.
static std::vector<std::vector<std::pair<int, int>>> round_robin(int G)
{
    std::vector<std::vector<std::pair<int, int>>> rounds;
    if (G < 2) return rounds;
    const int Gp = (G % 2) ? G + 1 : G;   // Gp-1 is a dummy (bye) when G is odd
    const int ring = Gp - 1;
    for (int r = 0; r < ring; ++r) {
        std::vector<std::pair<int, int>> rd;
        int a = Gp - 1, b = r;
        if (a < G && b < G) rd.push_back({std::min(a, b), std::max(a, b)});
        for (int k = 1; k < Gp / 2; ++k) {
            int x = (r + k) % ring, y = (r - k + ring) % ring;
            if (x < G && y < G) rd.push_back({std::min(x, y), std::max(x, y)});
        }
        rounds.push_back(rd);
    }
    return rounds;
}

static int block_pairs(const Block &b)
{
    return b.kind == BLK_SYM_DIAG ? b.nI * (b.nI + 1) / 2 : b.nI * b.nJ;
}

Schedule build_schedule(int n_occ, int n_in, bool aliased, int B, int max_pairs)
{
    Schedule S;
    if (max_pairs < B * B) max_pairs = B * B;
    const int Go = (n_occ + B - 1) / B;
    auto gsize = [&](int g0, int nmax) { return std::min(B, nmax - g0); };
    std::vector<std::vector<Block>> rounds;
    int t_begin = 0;
    if (aliased) {
        for (auto &rd : round_robin(Go)) {
            std::vector<Block> blks;
            for (auto &pr : rd) {
                int I0 = pr.first * B, J0 = pr.second * B;
                blks.push_back({I0, gsize(I0, n_occ), J0, gsize(J0, n_occ), BLK_SYM_OFF, 0});
            }
            rounds.push_back(blks);
        }
        std::vector<Block> diag;
        for (int g = 0; g < Go; ++g) {
            int I0 = g * B;
            diag.push_back({I0, gsize(I0, n_occ), I0, gsize(I0, n_occ), BLK_SYM_DIAG, 0});
        }
        rounds.push_back(diag);
        t_begin = n_occ;
    }
    const int nt = n_in - t_begin;
    if (nt > 0) {
        const int Gt = (nt + B - 1) / B;
        for (int r = 0; r < Go; ++r) {
            std::vector<Block> blks;
            for (int t = 0; t < Gt; ++t) {
                int g = (t + r) % Go;
                int I0 = g * B, J0 = t_begin + t * B;
                blks.push_back({I0, gsize(I0, n_occ), J0, std::min(B, n_in - J0), BLK_ONE_SIDE, 0});
            }
            rounds.push_back(blks);
        }
    }
    // cut rounds into batches; a batch never mixes rounds (outputs stay disjoint)
    for (auto &rd : rounds) {
        size_t i = 0;
        while (i < rd.size()) {
            Batch bt{0, int(S.blocks.size()), 0};
            S.pair0.push_back(int(S.pairs.size()));
            while (i < rd.size() && (bt.nblocks == 0 || bt.nfields + block_pairs(rd[i]) <= max_pairs)) {
                Block b = rd[i++];
                b.field0 = bt.nfields;
                if (b.kind == BLK_SYM_DIAG) {
                    for (int x = 0; x < b.nI; ++x)
                        for (int y = x; y < b.nI; ++y) S.pairs.push_back(make_int2(b.I0 + x, b.I0 + y));
                } else {
                    for (int x = 0; x < b.nI; ++x)
                        for (int y = 0; y < b.nJ; ++y) S.pairs.push_back(make_int2(b.I0 + x, b.J0 + y));
                }
                bt.nfields += block_pairs(b);
                S.blocks.push_back(b);
                bt.nblocks++;
            }
            S.max_fields = std::max(S.max_fields, bt.nfields);
            S.max_blocks = std::max(S.max_blocks, bt.nblocks);
            S.batches.push_back(bt);
        }
    }
    S.unique_pairs = long(S.pairs.size());
    return S;
}

}  // namespace exx
