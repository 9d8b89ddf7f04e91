"""The allocation-free Gram-matrix entry point (exx_gram_noalloc).

Some callers cannot allocate device memory when they need M = dV Psi^T W (under a
framework-owned allocator, in memory-capped processes, or in loops that must not stall on
the device synchronization cudaMalloc and cudaFree can cause).  For them
the library offers a plan-free call whose scratch is a fixed device array inside the
library.  This file is collected last so that, if it fails, a run that stops at the
first failure has already run every other test; it also passes on its own in a fresh
process.  The result must match the M that ace_build returns, within the FP64
tolerance of the other ACE tests, on two calls in a row (the second with different
sizes, so leftovers of the first call in the shared scratch would show).
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_gram_noalloc_matches_ace_build_on_consecutive_calls():
    import paper_2501_16572_gb300 as exx
    L = exx.load()
    stream = torch.cuda.current_stream().cuda_stream
    # the last case fills the whole fixed scratch: n = 128 orbitals and N = 4096 >= 8 * 256
    # grid points give eight split-K partial 128 x 128 tiles, including the edge tile
    cases = [dict(n=(22, 20, 18), bc=(1, 1, 0), n_orb=40, kernel=1, omega=0.106, seed=31),
             dict(n=(13, 11, 12), bc=(0, 0, 0), n_orb=9, kernel=0, seed=32),
             dict(n=(16, 16, 16), bc=(1, 1, 1), n_orb=128, kernel=1, omega=0.106, seed=33)]
    for case in cases:
        s = synth.small_system(h=0.4, **case)
        plan = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
        psi = torch.from_numpy(s.psi).cuda()
        f = torch.from_numpy(s.f).cuda()
        W = plan.apply(psi[:s.n_occ], f, psi)
        n = s.n_orb
        M_ref = torch.zeros((n, n), dtype=torch.float64, device="cuda")
        plan.ace_build(psi, W, M=M_ref)
        M = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
        rc = L.exx_gram_noalloc(s.N, s.dV, psi.data_ptr(), n, s.N, W.data_ptr(), s.N, M.data_ptr(), stream)
        assert rc == exx.EXX_OK, L.exx_last_error()
        torch.cuda.synchronize()
        err = float(torch.linalg.norm(M - M_ref) / torch.linalg.norm(M_ref))
        assert err < 1e-12, err
        plan.close()


def test_gram_noalloc_rejects_n_above_its_fixed_scratch():
    import paper_2501_16572_gb300 as exx
    L = exx.load()
    N, n = 1000, 129
    a = torch.zeros((n, N), dtype=torch.float64, device="cuda")
    M = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    rc = L.exx_gram_noalloc(N, 1.0, a.data_ptr(), n, N, a.data_ptr(), N, M.data_ptr(), None)
    assert rc == exx.EXX_ERR_INVALID_ARG
    assert b"[1, 128]" in L.exx_last_error()
