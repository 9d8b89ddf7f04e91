"""ACE construction (Sec. III.A) for many orbitals: the blocked multi-CTA Cholesky factor
of -sym(M) and its triangular inverse (64-column blocks: diagonal block on one CTA, panel
solve, trailing update; then the inverse block row by block row), FP64 in every mode.
Against the oracle's plain column-by-column Cholesky and row-by-row substitution for n = 300
(a ragged last block) and n = 1024 (the slab workload's orbital count), for FP64 and split
plans; and a failing pivot past the first block."""
import numpy as np
import pytest

import oracle
import synth
from tests import pinmath as pm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def exx():
    import paper_2501_16572_gb300 as m
    m.load()
    assert torch.cuda.is_available()
    return m


def _system(n_orb):
    # orthonormal orbitals and a symmetric negative-definite exchange-like W = -Psi K,
    # K symmetric positive definite with a spread of eigenvalues (seeded), so that the
    # Gram matrix M = dV Psi^T W = -K is known and well conditioned
    s = synth.small_system(n=(16, 16, 16), h=0.4, bc=(1, 1, 1), n_orb=n_orb, kernel=1, omega=0.106, seed=71)
    rng = np.random.Generator(np.random.PCG64(n_orb))
    Q, _ = np.linalg.qr(rng.normal(size=(n_orb, n_orb)))
    K = (Q * rng.uniform(0.5, 2.0, n_orb)) @ Q.T
    W = -(K @ s.psi)          # rows are orbitals: W_n = -sum_m K_nm psi_m
    return s, np.ascontiguousarray(W)


@pytest.mark.parametrize("n_orb", [300, 1024])
@pytest.mark.parametrize("prec", ["fp64", "bf16x7"])
def test_blocked_ace_matches_oracle(exx, n_orb, prec):
    s, Wh = _system(n_orb)
    M_ref, L_ref, xi_ref = oracle.ace(s.psi, Wh, s.dV)
    plan = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    plan.set_precision({"fp64": exx.EXX_PREC_FP64, "bf16x7": exx.EXX_PREC_BF16X7}[prec])
    psi = torch.from_numpy(s.psi).cuda()
    W = torch.from_numpy(Wh).cuda()
    M = torch.zeros((n_orb, n_orb), dtype=torch.float64, device="cuda")
    xi = plan.ace_build(psi, W, M=M)
    tol = 1e-11 if prec == "fp64" else 1e-8
    assert pm.rel(M.cpu().numpy().T, M_ref) < tol
    assert pm.rel(xi.cpu().numpy(), xi_ref) < tol
    back = plan.ace_apply(xi, psi)          # the compressed operator reproduces W on Psi
    assert pm.rel(back.cpu().numpy(), Wh) < tol


def test_blocked_cholesky_reports_pivot_past_first_block(exx):
    s, Wh = _system(300)
    Wf = Wh.copy()
    Wf[200] = -Wf[200]        # row 200 of -M flips sign: the pivot at 200 fails
    plan = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    psi = torch.from_numpy(s.psi).cuda()
    with pytest.raises(exx.ExxError) as ei:
        plan.ace_build(psi, torch.from_numpy(Wf).cuda())
    assert ei.value.status == exx.EXX_ERR_NOT_POSDEF
    assert ei.value.pivot == 200          # 0-based index of the failing pivot
