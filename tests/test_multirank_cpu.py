"""Sharded exact exchange across ranks, on CPU with gloo (world size 2).

The library shards exx_apply by batch (batch b belongs to rank b mod world, see
exx_plan_set_shard); every rank writes partial outputs and one sum-reduction completes
them.  Here two gloo ranks take the library's own schedule (host code, no GPU), solve
their batches' pairs with the oracle, accumulate partial outputs, and all-reduce; the
result must equal the single-process oracle, and every unique pair must be solved by
exactly one rank.
"""
import ctypes
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _schedule(n_occ, n_in, block, maxp):
    from paper_2501_16572_gb300 import _build
    _build.build()
    import paper_2501_16572_gb300 as exx
    L = exx.load()
    Lp, Ip = ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_int)
    L.exx_debug_schedule.argtypes = [ctypes.c_int] * 5 + [Lp, Lp, Lp, Ip, Ip, Ip]
    a, b, c = ctypes.c_long(), ctypes.c_long(), ctypes.c_long()
    L.exx_debug_schedule(n_occ, n_in, 1, block, maxp, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                         None, None, None)
    pairs = np.zeros(2 * a.value, np.int32)
    batches = np.zeros(3 * b.value, np.int32)
    L.exx_debug_schedule(n_occ, n_in, 1, block, maxp, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                         pairs.ctypes.data_as(Ip), batches.ctypes.data_as(Ip), None)
    return pairs.reshape(-1, 2), batches.reshape(-1, 3)


def _rank_main(rank, world, port, result_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import synth
    s = synth.small_system(n=(9, 8, 7), h=0.45, bc=(0, 1, 0), n_orb=7, kernel=0, seed=41, n_occ=5)
    pairs, batches = _schedule(s.n_occ, s.n_orb, 2, 4)
    orc = oracle.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    out = np.zeros((s.n_orb, s.N))
    solved = []
    start = 0
    for b, (nf, _, _) in enumerate(batches):
        mine = (b % world) == rank
        for m, n in pairs[start:start + nf]:
            if not mine:
                continue
            phi = orc.solve(s.psi[m] * s.psi[n])
            out[n] -= s.f[m] * s.psi[m] * phi
            if n != m and n < s.n_occ:
                out[m] -= s.f[n] * s.psi[n] * phi
            solved.append((int(m), int(n)))
        start += nf
    t = torch.from_numpy(out)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    counts = [None] * world
    dist.all_gather_object(counts, solved)
    if rank == 0:
        np.save(result_path, t.numpy())
        np.save(result_path + ".pairs.npy", np.array([p for c in counts for p in c]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_full_exchange(tmp_path):
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    path = str(tmp_path / "vx.npy")
    mp.spawn(_rank_main, args=(2, port, path), nprocs=2, join=True)
    got = np.load(path)
    import oracle
    import synth
    s = synth.small_system(n=(9, 8, 7), h=0.45, bc=(0, 1, 0), n_orb=7, kernel=0, seed=41, n_occ=5)
    ref = oracle.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega).exx_apply(s.psi[:5], s.f, s.psi)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    solved = [tuple(p) for p in np.load(path + ".pairs.npy")]
    assert len(solved) == len(set(solved))
    expect = {(m, n) for m in range(5) for n in range(m, 7)}
    assert set(solved) == expect
