"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: exact rational FD
weights, closed-form eigenvalues of the 1D operators (Eqs. 6-7), the direct stencil
Laplacian applied to a solution (Eq. 2), a dense brute-force solve and a dense
eigen-decomposition on a 6^3 grid (Eqs. 4-5), the two forms of the exchange energy
(Eq. 1), invariance under rotations of equally occupied orbitals, and the ACE
identities (Sec. III.A).  A planted mistake in the oracle must fail a pin.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from tests import pinmath as pm

P6_EXACT = [Fraction(-5369, 1800), Fraction(12, 7), Fraction(-15, 56), Fraction(10, 189),
            Fraction(-1, 112), Fraction(2, 1925), Fraction(-1, 16632)]


def test_fd_weights_order12_rational():
    w = oracle.fd_weights(6)
    for k in range(7):
        assert abs(w[k] - float(P6_EXACT[k])) <= 2e-16 * max(1.0, abs(float(P6_EXACT[k])))
    assert pm.fd_weights_taylor(6) == P6_EXACT


def _published_fd_table():
    """tests/golden/fd_second_derivative_central.txt: {p: [w_0, ..., w_p]} as Fractions."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "fd_second_derivative_central.txt")
    table = {}
    for line in open(path):
        line = line.split("#", 1)[0].split()
        if line:
            table[int(line[0])] = [Fraction(v) for v in line[1:]]
    return table


def test_fd_weights_match_published_table():
    # Fornberg (1988), Table 1: the oracle's closed form and the exact Taylor solve of the
    # pins both reproduce the published centred second-derivative weights, orders 2..12
    table = _published_fd_table()
    assert sorted(table) == [1, 2, 3, 4, 5, 6]
    for p, w_pub in table.items():
        assert len(w_pub) == p + 1
        assert pm.fd_weights_taylor(p) == w_pub
        np.testing.assert_allclose(oracle.fd_weights(p), [float(x) for x in w_pub], rtol=2e-16, atol=0)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7, 8])
def test_fd_weights_match_taylor_conditions(p):
    w = oracle.fd_weights(p)
    exact = pm.fd_weights_taylor(p)
    np.testing.assert_allclose(w, [float(x) for x in exact], rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("p", [1, 3, 6])
def test_operator_exact_on_polynomials(p):
    n, h = 40, 0.37
    D = oracle.second_derivative_1d(n, h, 0, p)
    x = (np.arange(n) - n / 2) * h
    inner = slice(p, n - p)
    for q in range(0, 2 * p + 2):
        f = x ** q
        d2 = q * (q - 1) * x ** (q - 2) if q >= 2 else np.zeros_like(x)
        got = (D @ f)[inner]
        scale = max(1.0, np.max(np.abs(f)) / h ** 2)
        assert np.max(np.abs(got - d2[inner])) <= 1e-9 * scale, q


@pytest.mark.parametrize("n,p", [(20, 6), (48, 6), (7, 6), (6, 6), (9, 1), (13, 3)])
def test_periodic_eigenvalues_closed_form(n, p):
    h = 0.25
    pl = oracle.Plan((n, 4, 4), h, (1, 1, 1), 2 * p, kernel=1, omega=0.106)
    lam = pl.eigvals(0)
    w = [float(v) for v in pm.fd_weights_taylor(p)]
    q = np.arange(n)
    closed = np.full(n, w[0])
    for k in range(1, p + 1):
        closed = closed + 2 * w[k] * np.cos(2 * np.pi * q * k / n)
    closed = np.sort(closed / h ** 2)
    np.testing.assert_allclose(lam, closed, rtol=0, atol=1e-12 * np.max(np.abs(closed)))


@pytest.mark.parametrize("n", [5, 24, 31])
def test_dirichlet_second_order_sine_closed_form(n):
    h = 0.3
    pl = oracle.Plan((n, 3, 3), h, (0, 0, 0), 2, kernel=0)
    lam = pl.eigvals(0)
    q = np.arange(1, n + 1)
    closed = np.sort(-(4.0 / h ** 2) * np.sin(q * np.pi / (2 * (n + 1))) ** 2)
    np.testing.assert_allclose(lam, closed, rtol=0, atol=1e-12 * np.max(np.abs(closed)))
    V = pl.eigvecs(0)
    # eigenvector of the q-th sine mode, up to sign: sin(i q pi/(n+1)); lam ascending means q descending
    i = np.arange(1, n + 1)
    for col in range(n):
        qq = n - col
        s = np.sin(i * qq * np.pi / (n + 1))
        s /= np.linalg.norm(s)
        assert abs(abs(s @ V[:, col]) - 1.0) < 1e-12


@pytest.mark.parametrize("n,bc", [(24, 0), (37, 0), (30, 1), (6, 0)])
def test_jacobi_residual_orthogonality_and_eigvalsh(n, bc):
    h = 0.2
    D = pm.op1d_dense(n, h, bc, 6)
    lam, V = oracle.jacobi_eigh(D)
    nrm = np.linalg.norm(D, 2)
    assert np.linalg.norm(D @ V - V * lam[None, :]) <= 1e-13 * nrm * n
    assert np.linalg.norm(V.T @ V - np.eye(n)) <= 1e-13 * n
    np.testing.assert_allclose(lam, np.linalg.eigvalsh(D), rtol=0, atol=1e-12 * nrm)
    # the oracle's own operator assembly equals the independent dense one
    np.testing.assert_allclose(oracle.second_derivative_1d(n, h, bc, 6), D, rtol=1e-15, atol=1e-12)


def _rho(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    N = n[0] * n[1] * n[2]
    return rng.normal(size=N)


@pytest.mark.parametrize("n,bc", [((12, 10, 9), (0, 0, 0)), ((11, 8, 14), (1, 1, 0)),
                                  ((9, 16, 7), (0, 1, 1)), ((20, 20, 20), (0, 0, 0))])
def test_unscreened_solution_recovers_minus_4pi_rho(n, bc):
    """Eq. 2: -(1/4 pi) L phi = rho, checked by applying the direct stencil to phi."""
    h = 0.3
    pl = oracle.Plan(n, h, bc, 12, kernel=0)
    rho = _rho(n, 3)
    phi = pl.solve(rho)
    lap = pm.apply_stencil(phi, n, h, bc, 6)
    assert pm.rel(lap, -4 * np.pi * rho) < 1e-11


@pytest.mark.parametrize("p", [1, 2, 6])
@pytest.mark.parametrize("bc,kernel", [((0, 0, 0), 0), ((1, 1, 1), 1), ((1, 1, 0), 1),
                                       ((0, 1, 0), 0), ((1, 1, 1), 2)])
def test_dense_bruteforce_6cube(p, bc, kernel):
    """6^3 grid, dense N=216 operator: LU solve (unscreened) or dense eigh (screened).
    With order 12 the stencil radius equals n: periodic rows fold, Dirichlet truncates."""
    n, h, omega = (6, 6, 6), 0.45, 0.106
    pl = oracle.Plan(n, h, bc, 2 * p, kernel=kernel, omega=omega)
    rho = _rho(n, 11)
    got = pl.solve(rho)
    L = pm.laplacian_dense(n, h, bc, p)
    if kernel == 0:
        ref = np.linalg.solve(L, -4 * np.pi * rho)
    else:
        lam, U = np.linalg.eigh(L)
        ref = U @ (pm.erfc_kernel(-lam, omega, a_is_16pi=(kernel == 2)) * (U.T @ rho))
    assert pm.rel(got, ref) < 1e-12


def test_screened_limits():
    n, h = (10, 9, 8), 0.3
    rho = _rho(n, 5)
    ref = oracle.Plan(n, h, (0, 0, 0), 12, kernel=0).solve(rho)
    small_w = oracle.Plan(n, h, (0, 0, 0), 12, kernel=1, omega=1e-6).solve(rho)
    assert pm.rel(small_w, ref) < 1e-12
    w = 0.106
    assert oracle.kernel_value(0.0, 1, w) == pytest.approx(np.pi / w ** 2, rel=1e-15)
    assert oracle.kernel_value(-1e-12, 1, w) == pytest.approx(np.pi / w ** 2, rel=1e-9)
    # large omega: f -> pi/omega^2 -> 0 for every eigenvalue
    big = 1e4
    assert oracle.kernel_value(-50.0, 1, big) == pytest.approx(np.pi / big ** 2, rel=1e-5)
    # literal 16 pi reading
    assert oracle.kernel_value(0.0, 2, w) == pytest.approx(1.0 / (4 * w ** 2), rel=1e-15)


def _small(n=(9, 8, 10), bc=(0, 0, 0), n_orb=5, kernel=0, omega=0.0, occ="fd", seed=1):
    return synth.small_system(n=n, h=0.45, bc=bc, n_orb=n_orb, kernel=kernel, omega=omega,
                              seed=seed, occ=occ)


@pytest.mark.parametrize("bc,kernel", [((0, 0, 0), 0), ((1, 1, 1), 1), ((1, 1, 0), 1)])
def test_energy_two_forms_and_signs(bc, kernel):
    s = _small(bc=bc, kernel=kernel, omega=0.106 if kernel else 0.0)
    pl = oracle.Plan(s.n, s.h, s.bc, 12, kernel=s.kernel, omega=s.omega)
    occ = s.psi[:s.n_occ]
    vx = pl.exx_apply(occ, s.f, s.psi)
    e1 = pl.energy(occ, s.f, vx)
    e2 = pl.energy_pairs(occ, s.f)
    assert e1 < 0
    assert abs(e1 - e2) <= 1e-13 * abs(e2)
    # M = dV Psi^T Vx Psi is symmetric and negative definite
    M = s.dV * (s.psi @ vx.T)
    assert np.linalg.norm(M - M.T) <= 1e-12 * np.linalg.norm(M)
    assert np.max(np.linalg.eigvalsh(0.5 * (M + M.T))) < 0


def test_exchange_matches_dense_definition():
    """Eq. 1 on a 6^3 grid with the dense inverse Laplacian in place of the Kronecker solve."""
    n, h = (6, 6, 6), 0.5
    s = synth.small_system(n=n, h=h, bc=(0, 0, 0), n_orb=4, kernel=0, seed=4, occ="const2")
    pl = oracle.Plan(n, h, (0, 0, 0), 12, kernel=0)
    got = pl.exx_apply(s.psi, s.f, s.psi)
    Linv = np.linalg.inv(pm.laplacian_dense(n, h, (0, 0, 0), 6))
    ref = np.zeros_like(got)
    for nn in range(4):
        for m in range(4):
            phi = Linv @ (-4 * np.pi * s.psi[m] * s.psi[nn])
            ref[nn] -= s.f[m] * s.psi[m] * phi
    assert pm.rel(got, ref) < 1e-12


def test_rotation_invariance_equal_occupations():
    s = _small(occ="const2", n_orb=4, seed=2)
    pl = oracle.Plan(s.n, s.h, s.bc, 12, kernel=0)
    vx = pl.exx_apply(s.psi, s.f, s.psi)
    e = pl.energy(s.psi, s.f, vx)
    rng = np.random.Generator(np.random.PCG64(99))
    Q, _ = np.linalg.qr(rng.normal(size=(4, 4)))
    psi_r = Q.T @ s.psi                        # rows: rotated orbitals (Psi Q as columns)
    vx_r = pl.exx_apply(psi_r, s.f, psi_r)
    e_r = pl.energy(psi_r, s.f, vx_r)
    assert abs(e_r - e) <= 1e-12 * abs(e)
    assert pm.rel(vx_r, Q.T @ vx) < 1e-12


def test_cols_subset_matches_full():
    s = _small(n_orb=5, seed=3)
    pl = oracle.Plan(s.n, s.h, s.bc, 12, kernel=0)
    full = pl.exx_apply(s.psi[:3], s.f[:3], s.psi)
    sub = pl.exx_apply(s.psi[:3], s.f[:3], s.psi, cols=[4, 1])
    np.testing.assert_array_equal(sub[0], full[4])
    np.testing.assert_array_equal(sub[1], full[1])


@pytest.mark.parametrize("bc,kernel", [((0, 0, 0), 0), ((1, 1, 1), 1)])
def test_ace_identities(bc, kernel):
    s = _small(bc=bc, kernel=kernel, omega=0.106 if kernel else 0.0, n_orb=6, seed=5)
    pl = oracle.Plan(s.n, s.h, s.bc, 12, kernel=s.kernel, omega=s.omega)
    W = pl.exx_apply(s.psi[:s.n_occ], s.f, s.psi)
    M, L, xi = oracle.ace(s.psi, W, s.dV)
    assert np.allclose(np.triu(L, 1), 0)
    assert np.all(np.diag(L) > 0)
    np.testing.assert_allclose(L @ L.T, -0.5 * (M + M.T), rtol=0, atol=1e-12 * np.abs(M).max())
    # xi L^T = W
    assert pm.rel(xi.T @ L.T, W.T) < 1e-12
    # compressed operator reproduces W on the orbitals and M in the orbital basis
    VW = oracle.ace_apply(xi, s.psi, s.dV)
    assert pm.rel(VW, W) < 1e-11
    assert pm.rel(s.dV * (s.psi @ VW.T), M) < 1e-11


def test_ace_not_positive_definite_reports_pivot():
    s = _small(n_orb=4, seed=6)
    W = np.zeros_like(s.psi)
    W[:2] = -s.psi[:2]           # only two columns non-zero: M has a zero diagonal at 2
    with pytest.raises(ValueError, match="pivot 2"):
        oracle.ace(s.psi, W, s.dV)


@pytest.mark.parametrize("mutation", [1, 2, 3])
def test_planted_mistakes_fail_the_stencil_pin(mutation):
    """A transposed V3, a dropped eigen-kernel, or a flipped sign in f must break Eq. 2."""
    n, h, bc = (8, 7, 9), 0.3, (0, 0, 0)
    rho = _rho(n, 21)
    oracle.set_mutation(mutation)
    try:
        pl = oracle.Plan(n, h, bc, 12, kernel=0)
        phi = pl.solve(rho)
    finally:
        oracle.set_mutation(0)
    lap = pm.apply_stencil(phi, n, h, bc, 6)
    assert pm.rel(lap, -4 * np.pi * rho) > 1e-3


def test_synthetic_inputs_are_orthonormal_and_seeded():
    s1 = _small(n_orb=6, seed=8)
    s2 = _small(n_orb=6, seed=8)
    np.testing.assert_array_equal(s1.psi, s2.psi)
    G = s1.dV * (s1.psi @ s1.psi.T)
    assert np.max(np.abs(G - np.eye(6))) < 1e-13
    assert np.all(s1.f > 0) and np.all(s1.f <= 2)
