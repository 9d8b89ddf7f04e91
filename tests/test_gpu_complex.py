"""GPU complex (Bloch) path against the CPU oracle's complex path: Eq. 1 with k-point pairs,
the pair problems under Bloch conditions at k - q (Sec. II), FP64.  VxPsi to 1e-10 relative
on mixed boundaries with different phases, the sum over two q-terms through the accumulate
flag, the energy, theta = 0 against the real GPU path, complex ACE (Sec. III.A) against the
oracle, and the refusals (a Bloch plan takes no real call; Coulomb at theta = 0 on an
all-periodic grid)."""
import numpy as np
import pytest

import oracle
from tests import pinmath as pm
from tests.test_oracle_pins_complex import bloch_orbitals

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def exx():
    import paper_2501_16572_gb300 as m
    m.load()
    assert torch.cuda.is_available()
    return m


def _c(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


CASES = [dict(n=(9, 8, 7), bc=(1, 1, 0), tq=(0.3, -0.5, 0.0), tk=(1.2, 0.4, 0.0), kernel=1),
         dict(n=(10, 6, 8), bc=(1, 0, 1), tq=(0.0, 0.0, 0.7), tk=(2.5, 0.0, -1.1), kernel=0),
         dict(n=(5, 7, 6), bc=(1, 1, 1), tq=(0.2, 0.1, 0.0), tk=(0.9, -1.3, 0.4), kernel=0)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c["n"])))
def test_complex_exchange_matches_oracle(exx, case):
    n, bc, h = case["n"], case["bc"], 0.4
    _, psi_q = bloch_orbitals(n, h, bc, 4, case["tq"], 5)
    s, psi_k = bloch_orbitals(n, h, bc, 5, case["tk"], 6)
    f = np.array([2.0, 1.5, 1.0, 0.4])
    theta = tuple(a - b for a, b in zip(case["tk"], case["tq"]))
    om = 0.106 if case["kernel"] == 1 else 0.0
    orc = oracle.CPlan(n, h, bc, 12, case["kernel"], om, theta=theta)
    ref = orc.exx_apply(psi_q, f, psi_k)
    p = exx.Plan.bloch(n, h, bc, theta, 12, case["kernel"], om)
    fd = torch.from_numpy(f).cuda()
    vx = p.apply_complex(_c(psi_q), fd, _c(psi_k))
    assert pm.rel(vx.cpu().numpy(), ref) < 1e-10
    e = p.energy_complex(_c(psi_k), torch.from_numpy(np.full(5, 1.0)).cuda(), vx)
    e_ref = orc.energy(psi_k, np.full(5, 1.0), ref)
    assert abs(e - e_ref) <= 1e-10 * abs(e_ref)
    # a second q-term added through `accumulate` (another occupied set, its own k - q)
    tq2 = tuple(t + 0.8 for t in case["tq"])
    _, psi_q2 = bloch_orbitals(n, h, bc, 3, tq2, 9)
    theta2 = tuple(a - b for a, b in zip(case["tk"], tq2))
    p2 = exx.Plan.bloch(n, h, bc, theta2, 12, case["kernel"], om)
    f2 = np.array([1.0, 0.7, 0.2])
    p2.apply_complex(_c(psi_q2), torch.from_numpy(f2).cuda(), _c(psi_k), out=vx, accumulate=True)
    ref2 = ref + oracle.CPlan(n, h, bc, 12, case["kernel"], om, theta=theta2).exx_apply(psi_q2, f2, psi_k)
    assert pm.rel(vx.cpu().numpy(), ref2) < 1e-10


def test_theta_zero_matches_real_gpu_path(exx):
    import synth
    s = synth.small_system(n=(12, 10, 9), h=0.4, bc=(1, 0, 1), n_orb=6, kernel=1, omega=0.106, seed=4)
    p = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    psi = torch.from_numpy(s.psi).cuda()
    f = torch.from_numpy(s.f).cuda()
    real = p.apply(psi[:s.n_occ], f, psi)
    pc = exx.Plan.bloch(s.n, s.h, s.bc, (0.0, 0.0, 0.0), s.fd_order, s.kernel, s.omega)
    cz = psi.to(torch.complex128)
    vc = pc.apply_complex(cz[:s.n_occ].contiguous(), f, cz)
    assert pm.rel(vc.cpu().numpy(), real.cpu().numpy()) < 1e-11
    assert float(vc.imag.abs().max()) <= 1e-12 * float(real.abs().max())


def test_complex_ace_matches_oracle(exx):
    n, bc, h = (9, 8, 7), (1, 1, 0), 0.4
    s, psi = bloch_orbitals(n, h, bc, 6, (0.7, 0.2, 0.0), 8)
    f = np.array([2.0, 2.0, 1.6, 1.0, 0.5, 0.1])
    orc = oracle.CPlan(n, h, bc, 12, 1, 0.106, theta=(0.0, 0.0, 0.0))
    W = orc.exx_apply(psi, f, psi)
    M_ref, L_ref, xi_ref = oracle.cace(psi, W, s.dV)
    p = exx.Plan.bloch(n, h, bc, (0.0, 0.0, 0.0), 12, 1, 0.106)
    xi = p.ace_build_complex(_c(psi), _c(W))
    assert pm.rel(xi.cpu().numpy(), xi_ref) < 1e-11
    back = p.ace_apply_complex(xi, _c(psi))
    assert pm.rel(back.cpu().numpy(), W) < 1e-11


def test_bloch_plan_refusals(exx):
    p = exx.Plan.bloch((6, 6, 6), 0.4, (1, 1, 1), (0.5, 0.0, 0.0), 12, 0, 0.0)   # Coulomb, theta != 0: fine
    psi = torch.zeros((2, 216), dtype=torch.float64, device="cuda")
    with pytest.raises(exx.ExxError) as ei:
        p.apply(psi, torch.ones(2, dtype=torch.float64, device="cuda"), psi)
    assert ei.value.status == exx.EXX_ERR_UNSUPPORTED
    with pytest.raises(exx.ExxError) as ei:
        exx.Plan.bloch((6, 6, 6), 0.4, (1, 1, 1), (0.0, 0.0, 2 * np.pi), 12, 0, 0.0)
    assert ei.value.status == exx.EXX_ERR_UNSUPPORTED
