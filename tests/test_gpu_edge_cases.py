"""Degenerate inputs of exx_apply on the GPU against the CPU oracle, through the C interface.

Cases the method admits at any size:
- an orbital that is identically zero: every pair density with it vanishes, so its own output
  is exactly zero, and it adds nothing to the others (the split modes give its rows a zero scale);
- a single occupied orbital (one pair block, partly empty);
- all occupations zero: VxPsi is exactly zero;
- an empty occupied set, which is rejected with EXX_ERR_INVALID_ARG.
Bars: FP64 <= 1e-10 relative Frobenius error on VxPsi, energy <= 1e-11; BF16X10 <= 1e-6 and
1e-8 (the split-precision targets).
"""
import numpy as np
import pytest

import oracle
import synth
from tests import pinmath as pm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = {"fp64": (0, 1e-10, 1e-11), "bf16x10": (4, 1e-6, 1e-8)}


@pytest.fixture(scope="module")
def exx():
    import paper_2501_16572_gb300 as m
    m.load()
    assert torch.cuda.is_available()
    return m


def _system():
    return synth.small_system(n=(16, 13, 11), h=0.4, bc=(1, 0, 1), n_orb=7, kernel=synth.KERNEL_ERFC,
                              omega=0.106, seed=41)


def _gpu_apply(exx, s, prec, psi, f, n_occ):
    plan = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    plan.set_precision(prec)
    dpsi = torch.from_numpy(np.ascontiguousarray(psi)).cuda()
    df = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    vx = plan.apply(dpsi[:n_occ], df, dpsi)
    e = plan.energy(dpsi[:n_occ], df, vx)
    out = vx.cpu().numpy()
    plan.close()
    return out, e


def _oracle_apply(s, psi, f, n_occ):
    orc = oracle.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    ref = orc.exx_apply(psi[:n_occ], f[:n_occ], psi)
    return ref, orc.energy(psi[:n_occ], f[:n_occ], ref)


@pytest.mark.parametrize("name", list(PRECS))
def test_zero_orbital(exx, name):
    prec, tol_v, tol_e = PRECS[name]
    s = _system()
    psi = s.psi.copy()
    psi[3] = 0.0                      # occupied (f_3 > 0) and identically zero
    out, e = _gpu_apply(exx, s, prec, psi, s.f, s.n_occ)
    ref, e_ref = _oracle_apply(s, psi, s.f, s.n_occ)
    assert np.all(out[3] == 0.0)
    assert pm.rel(out, ref) < tol_v
    assert abs(e - e_ref) <= tol_e * abs(e_ref)


@pytest.mark.parametrize("name", list(PRECS))
def test_single_occupied_orbital(exx, name):
    prec, tol_v, tol_e = PRECS[name]
    s = _system()
    out, e = _gpu_apply(exx, s, prec, s.psi, s.f[:1], 1)
    ref, e_ref = _oracle_apply(s, s.psi, s.f, 1)
    assert pm.rel(out, ref) < tol_v
    assert abs(e - e_ref) <= tol_e * abs(e_ref)


@pytest.mark.parametrize("name", list(PRECS))
def test_zero_occupations_give_zero(exx, name):
    prec = PRECS[name][0]
    s = _system()
    out, e = _gpu_apply(exx, s, prec, s.psi, np.zeros_like(s.f), s.n_occ)
    assert np.all(out == 0.0)
    assert e == 0.0


def test_empty_occupied_set_rejected(exx):
    s = _system()
    plan = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    psi = torch.from_numpy(s.psi).cuda()
    f = torch.from_numpy(s.f).cuda()
    with pytest.raises(exx.ExxError) as err:
        plan.apply(psi[:0], f, psi)
    assert err.value.status == exx.EXX_ERR_INVALID_ARG
    plan.close()
