"""CPU checks of libexx_gb300: it loads, exports every symbol its headers declare,
rejects bad arguments before touching a GPU, and its host-side plan setup and pair
scheduler are right (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from tests import pinmath as pm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2501_16572_gb300 import _build
    _build.build()
    import paper_2501_16572_gb300 as exx
    L = exx.load()
    D = ctypes.POINTER(ctypes.c_double)
    L.exx_debug_fd_weights.argtypes = [ctypes.c_int, D]
    L.exx_debug_second_derivative.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, D]
    L.exx_debug_sym_eig.argtypes = [ctypes.c_int, D, D, D]
    Lp = ctypes.POINTER(ctypes.c_long)
    Ip = ctypes.POINTER(ctypes.c_int)
    L.exx_debug_schedule.argtypes = [ctypes.c_int] * 5 + [Lp, Lp, Lp, Ip, Ip, Ip]
    return L


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|long|void|char|double)\s*\*?\s*(\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    import paper_2501_16572_gb300 as exx
    decl = _declared("exx.h") + _declared("exx_debug.h")
    assert "exx_apply" in decl and "ace_build" in decl and "exx_debug_schedule" in decl
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(exx.EXPORTED) == sorted(_declared("exx.h"))


def test_status_strings(lib):
    lib.exx_status_string.restype = ctypes.c_char_p
    for st in range(7):
        s = lib.exx_status_string(st)
        assert s and s.startswith(b"EXX_")
    assert lib.exx_status_string(99) == b"unknown exx status"


def test_invalid_arguments_rejected_on_host(lib):
    import paper_2501_16572_gb300 as exx
    h = ctypes.c_void_p()
    bc = (ctypes.c_int * 3)(0, 0, 0)
    create = lib.exx_plan_create
    assert create(ctypes.byref(h), 1, 8, 8, 0.3, bc, 12, 0, 0.0) == exx.EXX_ERR_INVALID_ARG
    assert create(ctypes.byref(h), 8, 8, 8, -0.3, bc, 12, 0, 0.0) == exx.EXX_ERR_INVALID_ARG
    assert create(ctypes.byref(h), 8, 8, 8, 0.3, bc, 11, 0, 0.0) == exx.EXX_ERR_INVALID_ARG
    assert create(ctypes.byref(h), 8, 8, 8, 0.3, bc, 12, 1, 0.0) == exx.EXX_ERR_INVALID_ARG
    assert create(ctypes.byref(h), 8, 8, 8, 0.3, bc, 12, 7, 0.1) == exx.EXX_ERR_INVALID_ARG
    per = (ctypes.c_int * 3)(1, 1, 1)
    assert create(ctypes.byref(h), 8, 8, 8, 0.3, per, 12, 0, 0.0) == exx.EXX_ERR_UNSUPPORTED
    bad = (ctypes.c_int * 3)(0, 2, 0)
    assert create(ctypes.byref(h), 8, 8, 8, 0.3, bad, 12, 0, 0.0) == exx.EXX_ERR_INVALID_ARG
    assert h.value is None
    null = ctypes.c_void_p()
    assert lib.exx_apply(null, null, 1, 8, null, null, 1, 8, null, 8, null) == exx.EXX_ERR_INVALID_ARG
    lib.exx_last_error.restype = ctypes.c_char_p
    assert b"plan is NULL" in lib.exx_last_error()


@pytest.mark.parametrize("p", [1, 2, 6, 9])
def test_fd_weights_match_exact(lib, p):
    w = np.zeros(p + 1)
    assert lib.exx_debug_fd_weights(p, w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == 0
    np.testing.assert_allclose(w, [float(x) for x in pm.fd_weights_taylor(p)], rtol=1e-14, atol=1e-16)


@pytest.mark.parametrize("n,bc,p", [(24, 0, 6), (48, 1, 6), (6, 1, 6), (6, 0, 6), (37, 0, 2), (144, 0, 6),
                                    (72, 1, 6), (2, 0, 6), (3, 1, 1)])
def test_plan_eigensolver(lib, n, bc, p):
    """Library eigensolver (Householder + QL) vs the closed form / an independent solver."""
    h = 0.25
    D = np.zeros(n * n)
    Dp = D.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.exx_debug_second_derivative(n, h, bc, p, Dp) == 0
    Dm = D.reshape(n, n, order="F")
    np.testing.assert_allclose(Dm, pm.op1d_dense(n, h, bc, p), rtol=1e-15, atol=1e-12)
    V = np.zeros(n * n)
    lam = np.zeros(n)
    assert lib.exx_debug_sym_eig(n, Dp, V.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == 0
    V = V.reshape(n, n, order="F")
    nrm = max(1.0, np.linalg.norm(Dm, 2))
    assert np.linalg.norm(Dm @ V - V * lam[None, :]) <= 1e-13 * nrm * n
    assert np.linalg.norm(V.T @ V - np.eye(n)) <= 1e-13 * n
    assert np.all(np.diff(lam) >= 0)
    np.testing.assert_allclose(lam, oracle.jacobi_eigh(Dm)[0], rtol=0, atol=1e-12 * nrm)


def schedule(lib, n_occ, n_in, aliased, block, maxp):
    Lp = ctypes.c_long
    npairs, nb, nbl = Lp(), Lp(), Lp()
    assert lib.exx_debug_schedule(n_occ, n_in, aliased, block, maxp, ctypes.byref(npairs), ctypes.byref(nb),
                                  ctypes.byref(nbl), None, None, None) == 0
    pairs = np.zeros(2 * npairs.value, dtype=np.int32)
    batches = np.zeros(3 * nb.value, dtype=np.int32)
    blocks = np.zeros(6 * nbl.value, dtype=np.int32)
    Ip = ctypes.POINTER(ctypes.c_int)
    assert lib.exx_debug_schedule(n_occ, n_in, aliased, block, maxp, ctypes.byref(npairs), ctypes.byref(nb),
                                  ctypes.byref(nbl), pairs.ctypes.data_as(Ip), batches.ctypes.data_as(Ip),
                                  blocks.ctypes.data_as(Ip)) == 0
    return pairs.reshape(-1, 2), batches.reshape(-1, 3), blocks.reshape(-1, 6)


@pytest.mark.parametrize("n_occ,n_in,aliased,block,maxp", [
    (16, 16, 1, 8, 128), (128, 128, 1, 8, 128), (100, 128, 1, 8, 64), (13, 29, 1, 4, 16),
    (7, 7, 1, 8, 64), (1, 5, 1, 8, 64), (10, 12, 0, 4, 48), (800, 1024, 1, 8, 512), (5, 3, 0, 2, 4)])
def test_schedule_covers_each_pair_once_with_disjoint_outputs(lib, n_occ, n_in, aliased, block, maxp):
    pairs, batches, blocks = schedule(lib, n_occ, n_in, aliased, block, maxp)
    seen = {}
    for m, n in pairs:
        key = (min(m, n), max(m, n)) if (aliased and n < n_occ) else (m, n)
        seen[key] = seen.get(key, 0) + 1
    if aliased:
        expect = {(m, n) for m in range(n_occ) for n in range(m, n_occ)}
        expect |= {(m, n) for m in range(n_occ) for n in range(n_occ, n_in)}
    else:
        expect = {(m, n) for m in range(n_occ) for n in range(n_in)}
    assert set(seen) == expect
    assert all(v == 1 for v in seen.values())
    p0 = 0
    for nf, b0, nbk in batches:
        assert nf <= max(maxp, block * block)
        outs = set()
        field = 0
        for I0, nI, J0, nJ, kind, f0 in blocks[b0:b0 + nbk]:
            assert f0 == field
            w = set(range(J0, J0 + nJ)) if kind == 2 else set(range(I0, I0 + nI))
            if kind == 0:
                w |= set(range(J0, J0 + nJ))
            assert not (outs & w), "two blocks of one batch write the same output"
            outs |= w
            cnt = nI * (nI + 1) // 2 if kind == 1 else nI * nJ
            # the block's fields hold exactly its pairs, in order
            blk_pairs = pairs[p0 + f0:p0 + f0 + cnt]
            if kind == 1:
                ref = [(I0 + x, I0 + y) for x in range(nI) for y in range(x, nI)]
            else:
                ref = [(I0 + x, J0 + y) for x in range(nI) for y in range(nJ)]
            assert [tuple(v) for v in blk_pairs] == ref
            field += cnt
        assert field == nf
        p0 += nf
    assert p0 == len(pairs)


def test_fast_division_matches_integer_division(lib):
    """Row -> (field, row in field) in the pass kernels divides by multiply and shift;
    every quotient must equal the integer one, at the divisor and quotient edges too."""
    U = ctypes.POINTER(ctypes.c_uint)
    lib.exx_debug_fastdiv.argtypes = [ctypes.c_uint, ctypes.c_int, U, U]
    rng = np.random.Generator(np.random.PCG64(1994))
    divisors = [1, 2, 3, 5, 7, 143, 2304, 4096, 5184, 746496, 2**31 - 1, 2**31, 2**31 + 1, 2**32 - 1]
    divisors += [int(x) for x in rng.integers(1, 2**32, size=40)] + [int(x) for x in rng.integers(1, 5000, size=40)]
    for d in divisors:
        n = np.concatenate([rng.integers(0, 2**32, size=2000, dtype=np.uint64),
                            np.array([0, 1, d - 1, d, d + 1, 2 * d - 1, 2 * d, 2**31 - 1, 2**31, 2**32 - 1],
                                     dtype=np.uint64)])
        n = (n % 2**32).astype(np.uint32)
        q = np.zeros_like(n)
        assert lib.exx_debug_fastdiv(d, len(n), n.ctypes.data_as(U), q.ctypes.data_as(U)) == 0
        assert np.array_equal(q.astype(np.uint64), n.astype(np.uint64) // d), d
    assert lib.exx_debug_fastdiv(0, 0, None, None) != 0


def test_stored_slab_energy_matches_the_input_recipe():
    """The stored full-oracle energy of the slab workload belongs to the current synthetic-input
    recipe (workload, sizes, seed and a hash of synth/), and is a plausible exchange energy."""
    import json
    import os
    import sys
    here = os.path.join(os.path.dirname(__file__), "golden")
    path = os.path.join(here, "slab72x72x144_energy.json")
    if not os.path.exists(path):
        pytest.skip("the stored slab energy has not been written yet")
    sys.path.insert(0, here)
    import make_slab_energy as mk
    import synth

    class Recipe:   # the fields recipe_key reads, without generating 6 GB of orbitals
        name, n, h, bc, fd_order = "slab72x72x144_erfc_1024", (72, 72, 144), 0.2, (1, 1, 0), 12
        kernel, omega, n_orb, n_occ = synth.KERNEL_ERFC, synth.HSE_OMEGA, 1024, 800
    g = json.load(open(path))
    assert mk.stored_matches(g, Recipe())
    assert g["unique_pair_solves"] == 800 * 801 // 2
    assert g["E_x"] < 0 and len(g["fingerprint"]["sum_sq"]) == 1024


def _tc3_layout(lib, n1, n2, n3, share):
    out = (ctypes.c_int * 16)()
    lib.exx_debug_tc3_layout.argtypes = [ctypes.c_int] * 4 + [ctypes.c_void_p]
    assert lib.exx_debug_tc3_layout(n1, n2, n3, share, out) == 0
    keys = ["supported", "smem_a", "smem_c", "stream_a", "kc_a", "stream_c", "kc_c", "pipe_a", "stage_a",
            "smem_b", "kchunk_b", "width_b", "nbuf_b", "resident_b", "upt", "limit"]
    return dict(zip(keys, list(out)))


def test_three_pass_layouts_fit_shared_memory(lib):
    """Every grid the three-pass mode accepts (x, y <= 128, z <= 208) gets layouts within the
    shared-memory limit; the two slice passes agree on streaming the x/y matrices; the bench
    slab keeps its x/y images resident and streams z as K-chunks; the 117-point capacity
    slices stream their x/y images; wider slices and longer z axes are refused."""
    sizes = [2, 5, 16, 17, 31, 48, 64, 72, 90, 100, 108, 112, 117, 120, 128]
    for n1 in sizes:
        for n2 in sizes:
            for n3 in (2, 9, 48, 119, 144, 150, 200, 208):
                for share in ((0, 1) if n1 == n2 else (0,)):
                    L = _tc3_layout(lib, n1, n2, n3, share)
                    assert L["supported"] == 1, (n1, n2, n3, L)
                    assert max(L["smem_a"], L["smem_c"], L["smem_b"]) <= L["limit"], (n1, n2, n3, L)
                    assert (L["stream_a"], L["kc_a"]) == (L["stream_c"], L["kc_c"]), (n1, n2, n3)
                    if L["stream_a"]:
                        assert L["kc_a"] in (16, 32, 48, 64) and L["stage_a"] == 0
                    assert L["upt"] * 4 * 4 >= n3
    slab = _tc3_layout(lib, 72, 72, 144, 1)
    assert slab["stream_a"] == 0 and slab["kchunk_b"] == 1 and slab["width_b"] == 48 and slab["nbuf_b"] == 2
    cap = _tc3_layout(lib, 117, 117, 119, 1)
    assert cap["stream_a"] == 1 and cap["kc_a"] == 32
    assert _tc3_layout(lib, 130, 8, 8, 0)["supported"] == 0
    assert _tc3_layout(lib, 16, 16, 240, 1)["supported"] == 0


def test_matrix_digit_images_reproduce_the_matrix(lib):
    """The four base-512 digits of a matrix row (row scaled by the largest entry of the whole row
    into [128, 256)) reproduce every entry to 2^-35 of the row maximum (the last digit rounds
    at 2^-27 of a first digit below 256); each weighted digit q is an integer of magnitude
    <= 256 times 2^-9q (exact in bf16); padding is zero; a K-chunk is the same digits as the
    matching columns of the whole image, with the same row scales."""
    rng = np.random.default_rng(7)
    nout, nk = 40, 37
    C = rng.standard_normal((nout, nk)) * 10.0 ** rng.uniform(-3, 3, size=(nout, 1))
    C[5] = 0.0
    Cc = np.ascontiguousarray(C)
    dp = ctypes.POINTER(ctypes.c_double)
    fp = ctypes.POINTER(ctypes.c_float)
    lib.exx_debug_matrix_digits.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, fp, fp]

    def image(WN, Kp, n0, k0):
        d = np.zeros((4, WN, Kp), np.float32)
        sc = np.zeros(WN, np.float32)
        assert lib.exx_debug_matrix_digits(nout, nk, Cc.ctypes.data_as(dp), WN, Kp, n0, k0,
                                           d.ctypes.data_as(fp), sc.ctypes.data_as(fp)) == 0
        return d.astype(np.float64), sc.astype(np.float64)

    d, sc = image(48, 48, 0, 0)
    recon = d.sum(axis=0) * sc[:, None]
    for n in range(nout):
        rmax = np.max(np.abs(C[n]))
        assert np.max(np.abs(recon[n, :nk] - C[n])) <= 2.0 ** -35 * rmax + 1e-300, n
    for q in range(4):
        w = d[q] * 2.0 ** (9 * q)
        assert np.all(w == np.round(w)) and np.max(np.abs(w)) <= 256
    assert np.all(d[:, nout:, :] == 0) and np.all(d[:, :, nk:] == 0)
    assert np.all(d[:, 5, :] == 0)
    dc, scc = image(48, 16, 0, 16)        # the K-chunk of contraction indices 16..31
    assert np.array_equal(dc, d[:, :, 16:32]) and np.array_equal(scc, sc)
    dl, _ = image(48, 16, 0, 32)          # the last chunk: indices 32..36, zeros after
    assert np.array_equal(dl[:, :, :nk - 32], d[:, :, 32:nk]) and np.all(dl[:, :, nk - 32:] == 0)
    db, scb = image(16, 48, 16, 0)        # an output block: rows 16..31
    assert np.array_equal(db, d[:, 16:32, :]) and np.array_equal(scb, sc[16:32])
