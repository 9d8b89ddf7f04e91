"""Parity at the full workload sizes, in the launch configuration bench.py times, on
sampled outputs that the CPU oracle recomputes one by one (Sec. II.B solves + Eq. 1):

* 48^3 periodic, 256 orbitals (the precision study): BF16X10 <= 1e-6 on sampled output
  orbitals (FP64 and BF16X7 are compared on every column in test_gpu_oracle_full.py);
* the 48-system batch, through one exx_apply_batched call: sampled outputs of systems with
  every boundary mix against the oracle;
* the 72x72x144 slab with 1024 orbitals (800 occupied): BF16X10 on sampled outputs, one of
  them unoccupied, against the oracle.
"""
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_periodic48_256_orbitals_sampled(exx):
    s = synth.config3()
    psi, f = _dev(s.psi), _dev(s.f)
    orc = oracle.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    cols = [3, 200]
    ref = orc.exx_apply(s.psi[:s.n_occ], s.f, s.psi, cols=cols)
    p = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    p.set_precision(exx.EXX_PREC_BF16X10)
    vx = p.apply(psi[:s.n_occ], f, psi)
    assert pm.rel(vx.cpu().numpy()[cols], ref) < 1e-6
    p.close()


def test_batch_of_48_systems_sampled(exx):
    specs = synth.config4_specs()
    systems = [synth.config4_system(i, specs) for i in range(len(specs))]
    plans, bufs = [], []
    for s in systems:
        p = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
        p.set_precision(exx.EXX_PREC_BF16X10)
        plans.append(p)
        psi = _dev(s.psi)
        bufs.append((psi, _dev(s.f), torch.empty_like(psi)))
    args = [(psi[:s.n_occ], f, psi, out) for (psi, f, out), s in zip(bufs, systems)]
    exx.exx_apply_batched(plans, args, stream=torch.cuda.Stream())
    torch.cuda.synchronize()
    # all-Dirichlet (0), all-periodic (1) and mixed systems; one sampled output each
    for k in (0, 1, 2, 4):
        s = systems[k]
        orc = oracle.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
        col = [s.n_orb // 2]
        ref = orc.exx_apply(s.psi[:s.n_occ], s.f, s.psi, cols=col)
        assert pm.rel(bufs[k][2].cpu().numpy()[col], ref) < 1e-6, (k, s.n, s.bc)
    for p in plans:
        p.close()


def test_slab_1024_orbitals_sampled(exx):
    s = synth.config5()
    psi, f = _dev(s.psi), _dev(s.f)
    p = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    p.set_precision(exx.EXX_PREC_BF16X10)
    vx = p.apply(psi[:s.n_occ], f, psi)
    cols = [17, 901]                       # an occupied and an unoccupied output orbital
    orc = oracle.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    ref = orc.exx_apply(s.psi[:s.n_occ], s.f, s.psi, cols=cols)
    assert pm.rel(vx.cpu().numpy()[cols], ref) < 1e-6
    p.close()
