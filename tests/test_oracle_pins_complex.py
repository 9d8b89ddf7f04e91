"""Pins of the oracle's complex (Bloch) path: Eq. 1 with Brillouin-zone wavevectors, the pair
problems of Eqs. 2-3 under Bloch boundary conditions at k - q (Sec. II).  Each pin checks the
oracle against something other than itself:
  * the 1D Bloch operator's eigenvalues against the closed form w0 + 2 sum_k w_k cos(k phi_p),
    phi_p = (2 pi p + theta) / n (folding stencils included), and its assembly on Bloch plane
    waves directly;
  * the Hermitian Jacobi eigensolver: residual and unitarity; theta = 0 equals the real
    periodic operator;
  * a solve against the 3D Bloch stencil applied in the test (unscreened: L X = -4 pi B) and
    against a dense 6^3 brute force built here from the FD weights;
  * theta = 0 with real orbitals reproduces the real oracle's exchange;
  * with k != q the exchange matrix <psi_a, Vx psi_b> dV is Hermitian and negative
    semidefinite (a misplaced conjugate breaks it: planted mistake 4);
  * complex ACE identities.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.filterwarnings("ignore")


def closed_form(n, h, p, theta):
    w = oracle.fd_weights(p)
    phi = (2 * np.pi * np.arange(n) + theta) / n
    lam = w[0] + 2 * sum(w[k] * np.cos(k * phi) for k in range(1, p + 1))
    return np.sort(lam / h ** 2)


def bloch_apply_1d(u, h, p, theta, axis, periodic):
    """Second derivative along `axis` of u, neighbours past the ends taken with the Bloch
    phase (periodic) or as zero (Dirichlet): written here independently of the oracle."""
    w = oracle.fd_weights(p)
    n = u.shape[axis]
    out = w[0] * u.astype(np.complex128)
    idx = np.arange(n)
    for k in range(1, p + 1):
        for sgn in (1, -1):
            j = idx + sgn * k
            wraps = np.floor_divide(j, n)
            jj = j - wraps * n
            if periodic:
                ph = np.exp(1j * theta * wraps)
                shape = [1] * u.ndim
                shape[axis] = n
                out = out + w[k] * np.take(u, jj, axis=axis) * ph.reshape(shape)
            else:
                ok = (j >= 0) & (j < n)
                shape = [1] * u.ndim
                shape[axis] = n
                out = out + w[k] * np.take(u, np.clip(j, 0, n - 1), axis=axis) * ok.reshape(shape)
    return out / h ** 2


@pytest.mark.parametrize("n,p,theta", [(12, 6, 0.7), (30, 6, -2.1), (7, 6, np.pi), (5, 6, 1.3), (9, 1, 0.4),
                                       (16, 3, 0.0)])
def test_bloch_eigenvalues_closed_form_and_vectors(n, p, theta):
    h = 0.3
    D = oracle.bloch_operator_1d(n, h, 1, p, theta)
    assert np.max(np.abs(D - D.conj().T)) <= 1e-13 * np.max(np.abs(D))
    lam, V = oracle.hermitian_eigh(D)
    ref = closed_form(n, h, p, theta)
    assert np.max(np.abs(lam - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.linalg.norm(D @ V - V * lam) <= 1e-12 * np.linalg.norm(D)
    assert np.linalg.norm(V.conj().T @ V - np.eye(n)) <= 1e-13 * n
    # the assembly itself on a Bloch plane wave: D u = lambda u, u(j) = exp(i phi j)
    for q in (0, 1, n // 2):
        phi = (2 * np.pi * q + theta) / n
        u = np.exp(1j * phi * np.arange(n))
        lam_q = (oracle.fd_weights(p)[0] + 2 * sum(oracle.fd_weights(p)[k] * np.cos(k * phi)
                                                   for k in range(1, p + 1))) / h ** 2
        assert np.linalg.norm(D @ u - lam_q * u) <= 1e-12 * np.linalg.norm(D) * np.sqrt(n)


def test_theta_zero_matches_real_periodic_operator():
    for n in (6, 11, 24):
        D = oracle.bloch_operator_1d(n, 0.25, 1, 6, 0.0)
        Dr = oracle.second_derivative_1d(n, 0.25, 1, 6)
        assert np.max(np.abs(D - Dr)) <= 1e-14 * np.max(np.abs(Dr))
    P = oracle.CPlan((10, 9, 8), 0.4, (1, 0, 1), 12, 1, 0.106, theta=(0.0, 0.0, 0.0))
    Pr = oracle.Plan((10, 9, 8), 0.4, (1, 0, 1), 12, 1, 0.106)
    for d in range(3):
        assert np.max(np.abs(P.eigvals(d) - Pr.eigvals(d))) <= 1e-11 * np.max(np.abs(Pr.eigvals(d)))


@pytest.mark.parametrize("bc", [(1, 1, 1), (1, 0, 1), (0, 1, 0)])
def test_bloch_solve_stencil_residual(bc):
    n, h, theta = (11, 9, 10), 0.35, (0.9, -0.4, 2.2)
    rng = np.random.Generator(np.random.PCG64(3))
    B = rng.normal(size=n[::-1]) + 1j * rng.normal(size=n[::-1])       # array (z, y, x)
    P = oracle.CPlan(n, h, bc, 12, 0, 0.0, theta=theta)
    X = P.solve(B.reshape(-1)).reshape(n[::-1])
    LX = sum(bloch_apply_1d(X, h, 6, theta[d], 2 - d, bc[d] == 1) for d in range(3))
    assert np.linalg.norm(LX + 4 * np.pi * B) <= 1e-11 * np.linalg.norm(4 * np.pi * B)


@pytest.mark.parametrize("kernel,omega", [(0, 0.0), (1, 0.106)])
def test_bloch_solve_dense_brute_force_6cube(kernel, omega):
    n, h, bc, theta = (6, 6, 6), 0.4, (1, 1, 0), (1.1, -0.3, 0.0)
    N = 216
    # dense Laplacian: columns are the stencil applied to unit vectors (assembled in this test)
    L = np.zeros((N, N), dtype=np.complex128)
    for c in range(N):
        e = np.zeros(N, dtype=np.complex128)
        e[c] = 1.0
        u = e.reshape(n[::-1])
        L[:, c] = sum(bloch_apply_1d(u, h, 6, theta[d], 2 - d, bc[d] == 1) for d in range(3)).reshape(-1)
    rng = np.random.Generator(np.random.PCG64(4))
    B = rng.normal(size=N) + 1j * rng.normal(size=N)
    P = oracle.CPlan(n, h, bc, 12, kernel, omega, theta=theta)
    X = P.solve(B)
    if kernel == 0:
        ref = np.linalg.solve(L, -4 * np.pi * B)
    else:
        lam, U = np.linalg.eigh((L + L.conj().T) / 2)
        x = -lam
        f = 4 * np.pi / x * (1 - np.exp(-x / (4 * omega ** 2)))
        ref = U @ (f * (U.conj().T @ B))
    assert np.linalg.norm(X - ref) <= 1e-12 * np.linalg.norm(ref)


def test_theta_zero_real_orbitals_match_real_exchange():
    s = synth.small_system(n=(10, 9, 8), h=0.4, bc=(1, 0, 1), n_orb=5, kernel=1, omega=0.106, seed=3)
    P = oracle.CPlan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega, theta=(0.0, 0.0, 0.0))
    Pr = oracle.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    out = P.exx_apply(s.psi[:s.n_occ].astype(np.complex128), s.f, s.psi.astype(np.complex128))
    ref = Pr.exx_apply(s.psi[:s.n_occ], s.f, s.psi)
    assert np.linalg.norm(out - ref) <= 1e-12 * np.linalg.norm(ref)
    e = P.energy(s.psi[:s.n_occ].astype(np.complex128), s.f, out[:s.n_occ])
    assert abs(e - Pr.energy(s.psi[:s.n_occ], s.f, ref)) <= 1e-12 * abs(e)


def bloch_orbitals(n, h, bc, n_orb, theta, seed):
    """Seeded complex orbitals with Bloch character: real synthetic orbitals times the plane
    wave exp(i theta_d x_d / L_d) along periodic axes, orthonormalised (dV metric)."""
    s = synth.small_system(n=n, h=h, bc=bc, n_orb=n_orb, kernel=1, omega=0.106, seed=seed)
    ph = np.ones(n[::-1], dtype=np.complex128)
    for d in range(3):
        if bc[d] == 1:
            x = np.arange(n[d]) / n[d]
            shape = [1, 1, 1]
            shape[2 - d] = n[d]
            ph = ph * np.exp(1j * theta[d] * x).reshape(shape)
    raw = s.psi * ph.reshape(1, -1)
    q, _ = np.linalg.qr(raw.T)
    return s, np.ascontiguousarray((q / np.sqrt(s.dV)).T)


def test_exchange_matrix_hermitian_negative_semidefinite_and_planted_conj():
    n, h, bc = (9, 8, 7), 0.4, (1, 1, 0)
    tq, tk = (0.3, -0.5, 0.0), (1.2, 0.4, 0.0)
    _, psi_q = bloch_orbitals(n, h, bc, 4, tq, 5)      # occupied orbitals at q
    s, psi_k = bloch_orbitals(n, h, bc, 5, tk, 6)      # functions at k
    f = np.array([2.0, 1.5, 1.0, 0.4])
    theta = tuple(a - b for a, b in zip(tk, tq))
    P = oracle.CPlan(n, h, bc, 12, 1, 0.106, theta=theta)

    def gram():
        vx = P.exx_apply(psi_q, f, psi_k)
        return s.dV * psi_k.conj() @ vx.T          # G_ab = dV <psi_a, Vx psi_b>

    G = gram()
    assert np.max(np.abs(G - G.conj().T)) <= 1e-12 * np.max(np.abs(G))
    assert np.max(np.linalg.eigvalsh((G + G.conj().T) / 2)) <= 1e-12 * np.max(np.abs(G))
    oracle.set_mutation(4)                           # planted: rho without the conjugate
    try:
        Gm = gram()
    finally:
        oracle.set_mutation(0)
    assert np.max(np.abs(Gm - Gm.conj().T)) > 1e-6 * np.max(np.abs(Gm))


def test_complex_ace_identities():
    n, h, bc = (9, 8, 7), 0.4, (1, 1, 0)
    s, psi = bloch_orbitals(n, h, bc, 6, (0.7, 0.2, 0.0), 8)
    P = oracle.CPlan(n, h, bc, 12, 1, 0.106, theta=(0.0, 0.0, 0.0))   # same k: q = k
    f = np.array([2.0, 2.0, 1.6, 1.0, 0.5, 0.1])
    W = P.exx_apply(psi, f, psi)
    M, L, xi = oracle.cace(psi, W, s.dV)
    assert np.max(np.abs(M - M.conj().T)) <= 1e-12 * np.max(np.abs(M))
    assert np.allclose(np.triu(L, 1), 0) and np.all(np.diag(L).real > 0) and np.allclose(np.diag(L).imag, 0)
    Mh = (M + M.conj().T) / 2
    assert np.linalg.norm(L @ L.conj().T + Mh) <= 1e-12 * np.linalg.norm(Mh)
    back = -s.dV * xi.T @ (xi.conj() @ psi.T)        # -dV xi xi^H Psi
    assert np.linalg.norm(back.T - W) <= 1e-11 * np.linalg.norm(W)
