"""exx_plan_autotune: tile and schedule settings measured on the grid with the caller's data,
kept in the plan and in a process-wide cache (Sec. II.B's batch size n_c, the orbital block,
and the three-pass kernels' pass-B matrix blocks / buffers and slice staging).  The chosen
setting must be one of the candidates, a second plan with the same key must take it from the
cache without measuring, and exx_apply after tuning must still match the oracle."""
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


@pytest.mark.parametrize("prec", ["bf16x7", "fp64"])
def test_autotune_choice_cache_and_results(exx, prec):
    code = {"bf16x7": exx.EXX_PREC_BF16X7, "fp64": exx.EXX_PREC_FP64}[prec]
    # long z (streamed pass-B blocks: several block / buffer choices), 40 orbitals
    s = synth.small_system(n=(12, 10, 150) if prec == "bf16x7" else (12, 10, 14), h=0.3, bc=(1, 1, 0),
                           n_orb=40, kernel=1, omega=0.106, seed=61)
    psi = torch.from_numpy(s.psi).cuda()
    f = torch.from_numpy(s.f).cuda()
    p = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    p.set_precision(code)
    t = p.autotune(psi[:s.n_occ], f, psi, remeasure=True)
    assert t["tuned"] == 1 and t["ms_per_pair"] > 0
    assert t["pairs_per_batch"] in (0, 256, 512, 1024) and t["block_orbitals"] in (8, 16)
    if prec == "bf16x7":
        assert t["staging"] in (-1, 0, 1)
    vx = p.apply(psi[:s.n_occ], f, psi)
    orc = oracle.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    ref = orc.exx_apply(s.psi[:s.n_occ], s.f, s.psi)
    assert pm.rel(vx.cpu().numpy(), ref) < (1e-6 if prec == "bf16x7" else 1e-10)
    # a second plan with the same grid, precision and orbital counts: from the cache
    q = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    q.set_precision(code)
    t2 = q.autotune(psi[:s.n_occ], f, psi)
    assert t2["tuned"] == 2
    assert {k: t2[k] for k in t2 if k != "tuned"} == {k: t[k] for k in t if k != "tuned"}
    vx2 = q.apply(psi[:s.n_occ], f, psi)
    assert pm.rel(vx2.cpu().numpy(), vx.cpu().numpy()) < 1e-9
    p.close()
    q.close()
