"""exx_apply_batched: many independent systems in one call (Sec. II.B's batching of
pair solves carried across systems), through the C interface.

1. On a side stream the launches of all systems are captured once into a CUDA graph (the
   systems on concurrent branches); every output must equal, bit for bit, what exx_apply
   writes for that system alone,
   on the first call (capture + replay) and on a second call after the inputs were
   refilled in place (replay of the cached graph).
2. On the legacy default stream the same launches are issued one by one; same outputs.
3. Systems with 64-point axes in BF16X10 (the variants with one accumulator set and
   unpadded pair staging) against the CPU oracle.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import pinmath as pm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SYSTEMS = [
    dict(n=(14, 12, 10), bc=(0, 1, 0), n_orb=6, kernel=0),
    dict(n=(9, 16, 7), bc=(1, 1, 1), n_orb=5, kernel=1, omega=0.106),
    dict(n=(20, 11, 13), bc=(1, 1, 0), n_orb=9, kernel=1, omega=0.106, n_occ=6),
    dict(n=(17, 19, 23), bc=(0, 0, 0), n_orb=11, kernel=0),
]


@pytest.fixture(scope="module")
def exx():
    import paper_2501_16572_gb300 as m
    m.load()
    assert torch.cuda.is_available()
    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _setup(exx, prec, seed):
    systems, plans, bufs = [], [], []
    for i, c in enumerate(SYSTEMS):
        s = synth.small_system(h=0.4, seed=seed + i, **c)
        p = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
        p.set_precision(prec)
        psi = _dev(s.psi)
        f = _dev(s.f)
        out = torch.full_like(psi, float("nan"))
        systems.append(s)
        plans.append(p)
        bufs.append((psi, f, out))
    return systems, plans, bufs


def _individual(plans, bufs, systems):
    res = []
    for p, (psi, f, _), s in zip(plans, bufs, systems):
        res.append(p.apply(psi[:s.n_occ], f, psi).clone())
        res[-1] = (res[-1], p.launch_count())
    torch.cuda.synchronize()
    return res


def _batched(exx, plans, bufs, systems, stream):
    args = [(psi[:s.n_occ], f, psi, out) for (psi, f, out), s in zip(bufs, systems)]
    exx.exx_apply_batched(plans, args, stream=stream)
    stream.synchronize()
    return [out.clone() for (_, _, out) in bufs]


@pytest.mark.parametrize("prec", [0, 4, 5], ids=["fp64", "bf16x10", "bf16x7"])
def test_graph_equals_individual_applies_twice(exx, prec):
    systems, plans, bufs = _setup(exx, prec, seed=60)
    ref = _individual(plans, bufs, systems)
    side = torch.cuda.Stream()
    got = _batched(exx, plans, bufs, systems, side)
    for (r, nl), g, p in zip(ref, got, plans):
        assert torch.equal(r, g)
        assert p.launch_count() == nl
    # refill the same buffers with other orbitals: the second call replays the graph
    others = [synth.small_system(h=0.4, seed=80 + i, **c) for i, c in enumerate(SYSTEMS)]
    for (psi, f, out), o in zip(bufs, others):
        psi.copy_(_dev(o.psi))
        f.copy_(_dev(o.f))
        out.fill_(float("nan"))
    ref2 = _individual(plans, bufs, others)
    got2 = _batched(exx, plans, bufs, others, side)
    for (r, nl), g, p in zip(ref2, got2, plans):
        assert torch.equal(r, g)
        assert p.launch_count() == nl
    # and the graph's results are the method's: oracle on one system
    o = others[2]
    orc = oracle.Plan(o.n, o.h, o.bc, o.fd_order, o.kernel, o.omega)
    e = orc.exx_apply(o.psi[:o.n_occ], o.f, o.psi)
    assert pm.rel(got2[2].cpu().numpy(), e) < (1e-10 if prec == 0 else 1e-6)


def test_default_stream_issues_launches_directly(exx):
    systems, plans, bufs = _setup(exx, 4, seed=70)
    ref = _individual(plans, bufs, systems)
    args = [(psi[:s.n_occ], f, psi, out) for (psi, f, out), s in zip(bufs, systems)]
    exx.exx_apply_batched(plans, args, stream=torch.cuda.default_stream())
    torch.cuda.synchronize()
    for (r, _), (_, _, out) in zip(ref, bufs):
        assert torch.equal(r, out)


def test_mixed_precisions_rejected(exx):
    systems, plans, bufs = _setup(exx, 0, seed=75)
    plans[1].set_precision(4)
    args = [(psi[:s.n_occ], f, psi, out) for (psi, f, out), s in zip(bufs, systems)]
    with pytest.raises(exx.ExxError) as ei:
        exx.exx_apply_batched(plans, args, stream=torch.cuda.Stream())
    assert ei.value.status == exx.EXX_ERR_INVALID_ARG


@pytest.mark.parametrize("n,bc", [((64, 20, 64), (1, 0, 1)), ((33, 64, 49), (0, 1, 0))],
                         ids=["64x20x64", "33x64x49"])
def test_long_axes_bf16x10_match_oracle(exx, n, bc):
    s = synth.small_system(n=n, h=0.3, bc=bc, n_orb=4, kernel=1, omega=0.106, seed=90)
    p = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    p.set_precision(4)
    psi, f = _dev(s.psi), _dev(s.f)
    out = torch.empty_like(psi)
    exx.exx_apply_batched([p], [(psi[:s.n_occ], f, psi, out)], stream=torch.cuda.Stream())
    torch.cuda.synchronize()
    orc = oracle.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    ref = orc.exx_apply(s.psi[:s.n_occ], s.f, s.psi)
    assert pm.rel(out.cpu().numpy(), ref) < 1e-6
    e = p.energy(psi[:s.n_occ], f, out)
    e_ref = orc.energy(s.psi[:s.n_occ], s.f, ref)
    assert abs(e - e_ref) <= 1e-8 * abs(e_ref)


def test_repeated_plan_is_rejected(exx):
    """A plan holds one schedule: the same plan twice in one call is refused before any
    launch, and the outputs are left untouched."""
    systems, plans, bufs = _setup(exx, exx.EXX_PREC_FP64, 70)
    psi, f, out = bufs[0]
    s = systems[0]
    other = torch.full_like(psi, float("nan"))
    args = [(psi[:s.n_occ], f, psi, out), (psi[:2], f, psi, other)]
    with pytest.raises(exx.ExxError) as ei:
        exx.exx_apply_batched([plans[0], plans[0]], args, stream=torch.cuda.Stream())
    assert ei.value.status == exx.EXX_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert bool(torch.isnan(out).all()) and bool(torch.isnan(other).all())
    for p in plans:
        p.close()
