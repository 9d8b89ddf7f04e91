"""The original (non-batched) Kronecker formalism on the GPU (exx_apply_original): Eq. 8's
per-pair solve with 4 n_z + 2 dense GEMM launches (per frontal slice Vx^T B_k Vy, the z
axis, the f(Lambda) product, the inverse), FP64, against the CPU oracle to 1e-10, with
aliased (symmetric pairs) and separate orbital blocks, and its launch count."""
import numpy as np
import pytest

import oracle
import synth
from tests import pinmath as pm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [dict(n=(14, 12, 10), bc=(0, 1, 0), n_orb=5, kernel=0),
         dict(n=(16, 16, 16), bc=(1, 1, 1), n_orb=4, kernel=1, omega=0.106),
         dict(n=(17, 19, 23), bc=(0, 0, 0), n_orb=4, kernel=0, n_occ=3)]


@pytest.fixture(scope="module")
def exx():
    import paper_2501_16572_gb300 as m
    m.load()
    assert torch.cuda.is_available()
    return m


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c["n"])))
def test_original_formalism_matches_oracle(exx, case):
    s = synth.small_system(h=0.4, seed=51, **case)
    plan = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    psi = torch.from_numpy(s.psi).cuda()
    f = torch.from_numpy(s.f).cuda()
    vx = plan.apply_original(psi[:s.n_occ], f, psi)
    orc = oracle.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    ref = orc.exx_apply(s.psi[:s.n_occ], s.f, s.psi)
    assert pm.rel(vx.cpu().numpy(), ref) < 1e-10
    # one pair per solve: 4 n_z + 2 GEMMs + the pair density and accumulation launches
    n3, no, ni = s.n[2], s.n_occ, s.n_orb
    pairs = no * (no + 1) // 2 + no * (ni - no)
    assert plan.launch_count() == pairs * (4 * n3 + 2 + 2)
    # separate (not aliased) output block: every ordered pair solved
    other = psi.clone()
    vx2 = plan.apply_original(psi[:s.n_occ], f, other)
    assert pm.rel(vx2.cpu().numpy(), ref) < 1e-10
    assert plan.launch_count() == no * ni * (4 * n3 + 4)
