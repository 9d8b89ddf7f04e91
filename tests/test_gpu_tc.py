"""GPU checks of the split-precision tensor-core path (tcgen05), through the C interface.

1. One 128 x n x k tcgen05 tile with bf16 / tf32 operands against an FP64 matmul of the
   same rounded operands (checks descriptors, operand layout, TMEM read-back).
2. exx_apply against the CPU oracle.  The modes that meet the split-precision targets
   (<= 1e-6 relative Frobenius on VxPsi, <= 1e-8 relative on E_x) are held to them:
   BF16X7 (three-pass, base-512 digits) and BF16X10 (four base-256 slices, hi+lo
   intermediates).  The other split forms DO NOT MEET the target and are kept only as
   comparison modes; their tests record the error band they stay in (measured at 48^3 x
   256 orbitals: BF16X6 E_x 1.45e-8, TF32X3 VxPsi 5.6e-7 / E_x 5.7e-7, BF16X3 5.6e-5 /
   5.4e-5) and fail only if a mode leaves its band:
     BF16X6  VxPsi 1e-6, E_x 1e-7   (three base-256 slices, FP32 intermediates, ~24 bits)
     TF32X3  VxPsi 1e-6, E_x 1e-6   (floating split; the tensor core's FP32 accumulation
                                     rounds toward zero, a bias shared by every pair)
     BF16X3  VxPsi 2e-4, E_x 1e-4   (two slices, ~16 bits)
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from tests import pinmath as pm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# modes that meet the split-precision targets: (code, VxPsi, E_x)
TARGET = {"bf16x7": (5, 1e-6, 1e-8), "bf16x10": (4, 1e-6, 1e-8)}
# comparison modes that do not meet the target: the error bands they are recorded in
BANDS = {"bf16x6": (3, 1e-6, 1e-7), "tf32x3": (2, 1e-6, 1e-6), "bf16x3": (1, 2e-4, 1e-4)}
SPLIT = {**TARGET, **BANDS}


@pytest.fixture(scope="module")
def exx():
    import paper_2501_16572_gb300 as m
    L = m.load()
    vp = ctypes.c_void_p
    L.exx_debug_tc_gemm.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp]
    return m


def _round_tf32(x):
    u = x.astype(np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0xFFF + ((u >> 13) & 1)) & 0xFFFFE000
    return u.astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("tf32", [0, 1], ids=["bf16", "tf32"])
@pytest.mark.parametrize("n,k", [(16, 16), (48, 48), (64, 32), (128, 96), (256, 64), (32, 144)])
def test_single_tile_tcgen05_gemm(exx, tf32, n, k):
    rng = np.random.Generator(np.random.PCG64(n * 1000 + k + tf32))
    A = rng.normal(size=(128, k)).astype(np.float32)
    B = rng.normal(size=(n, k)).astype(np.float32)
    if tf32:
        A, B = _round_tf32(A), _round_tf32(B)
    else:
        A = torch.from_numpy(A).to(torch.bfloat16).float().numpy()
        B = torch.from_numpy(B).to(torch.bfloat16).float().numpy()
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dD = torch.zeros((128, n), dtype=torch.float32, device="cuda")
    err = torch.zeros(4, dtype=torch.int32, device="cuda")
    rc = exx.load().exx_debug_tc_gemm(tf32, n, k, dA.data_ptr(), dB.data_ptr(), dD.data_ptr(), err.data_ptr())
    assert rc == 0
    assert int(err[0]) == 0
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    got = dD.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))


def _apply(exx, s, prec, batch=None):
    plan = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    plan.set_precision(prec)
    if batch:
        plan.set_batch(*batch)
    psi = torch.from_numpy(s.psi).cuda()
    f = torch.from_numpy(s.f).cuda()
    vx = plan.apply(psi[:s.n_occ], f, psi)
    e = plan.energy(psi[:s.n_occ], f, vx)
    return plan, psi, f, vx, e


CASES = [
    dict(n=(14, 12, 10), bc=(0, 1, 0), n_orb=6, kernel=0),
    dict(n=(16, 16, 16), bc=(1, 1, 1), n_orb=9, kernel=1, omega=0.106),
    dict(n=(20, 11, 13), bc=(1, 1, 0), n_orb=8, kernel=1, omega=0.106),
    dict(n=(17, 19, 23), bc=(0, 0, 0), n_orb=7, kernel=0),
]


@pytest.mark.parametrize("name", list(SPLIT))
@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c["n"])))
def test_split_exx_apply_matches_oracle(exx, name, case):
    code, tol_v, tol_e = SPLIT[name]
    s = synth.small_system(h=0.4, seed=21, **case)
    plan, psi, f, vx, e = _apply(exx, s, code)
    orc = oracle.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    ref = orc.exx_apply(s.psi[:s.n_occ], s.f, s.psi)
    e_ref = orc.energy(s.psi[:s.n_occ], s.f, ref)
    err_v = pm.rel(vx.cpu().numpy(), ref)
    err_e = abs(e - e_ref) / abs(e_ref)
    print(f"{name} {case['n']}: VxPsi {err_v:.2e}  E_x {err_e:.2e}")
    assert err_v < tol_v
    assert err_e < tol_e


@pytest.mark.parametrize("name", ["bf16x7", "bf16x10", "bf16x6", "tf32x3"])
def test_split_config1_all_pairs(exx, name):
    code, tol_v, tol_e = SPLIT[name]
    s = synth.config1()
    plan, psi, f, vx, e = _apply(exx, s, code)
    orc = oracle.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    ref = orc.exx_apply(s.psi, s.f, s.psi)
    e_ref = orc.energy(s.psi, s.f, ref)
    assert pm.rel(vx.cpu().numpy(), ref) < tol_v
    assert abs(e - e_ref) <= tol_e * abs(e_ref)


@pytest.mark.parametrize("name", ["bf16x7", "bf16x10", "bf16x6", "tf32x3"])
def test_split_batch_invariance_and_separate_inputs(exx, name):
    code = SPLIT[name][0]
    s = synth.small_system(n=(13, 11, 12), h=0.4, bc=(0, 0, 1), n_orb=10, kernel=0, seed=5, n_occ=6)
    _, psi, f, ref, _ = _apply(exx, s, code, batch=(0, 0))
    _, _, _, vx, _ = _apply(exx, s, code, batch=(4, 2))
    # the same solves in different batches: identical up to the compensated sum order
    assert pm.rel(vx.cpu().numpy(), ref.cpu().numpy()) < 1e-9
    plan = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    plan.set_precision(code)
    other = psi.clone()
    vx2 = plan.apply(psi[:6], f, other)
    orc = oracle.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    full = orc.exx_apply(s.psi[:6], s.f, s.psi)
    assert pm.rel(vx2.cpu().numpy(), full) < 1e-6


LONG = [dict(n=(72, 20, 24), bc=(1, 0, 1)), dict(n=(20, 72, 16), bc=(0, 1, 1)), dict(n=(16, 20, 144), bc=(1, 1, 0)),
        dict(n=(20, 100, 20), bc=(0, 0, 1)), dict(n=(130, 16, 12), bc=(1, 0, 0)), dict(n=(12, 16, 150), bc=(0, 1, 1))]


@pytest.mark.parametrize("name", ["bf16x10", "bf16x6", "tf32x3"])
@pytest.mark.parametrize("case", LONG, ids=lambda c: "x".join(map(str, c["n"])))
def test_split_long_axes_match_oracle(exx, name, case):
    """Axes longer than one on-chip operand image: cut into blocks whose products are
    summed in hi/lo FP32 (y alone may also just split pass 3 into two kernels)."""
    code, tol_v, tol_e = SPLIT[name]
    s = synth.small_system(h=0.3, seed=33, n_orb=4, kernel=1, omega=0.106, **case)
    plan, psi, f, vx, e = _apply(exx, s, code)
    orc = oracle.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    ref = orc.exx_apply(s.psi[:s.n_occ], s.f, s.psi)
    e_ref = orc.energy(s.psi[:s.n_occ], s.f, ref)
    assert pm.rel(vx.cpu().numpy(), ref) < tol_v
    assert abs(e - e_ref) < tol_e * abs(e_ref)


@pytest.fixture(scope="module")
def slab64():
    # the slab grid (72 x 72 x 144, periodic x, y, vacuum along Dirichlet z) with 64 orbitals
    return synth.make_system("slab72x72x144_erfc_64", (72, 72, 144), 0.2, (1, 1, 0), 64, synth.KERNEL_ERFC,
                             synth.HSE_OMEGA, "fd", synth.SEED_BASE + 5, slab_axis=2, fermi_index=49)


@pytest.mark.parametrize("name", ["bf16x10", "fp64"])
def test_slab_grid_sampled_columns(exx, slab64, name):
    s = slab64
    code = 0 if name == "fp64" else SPLIT[name][0]
    plan, psi, f, vx, e = _apply(exx, s, code)
    cols = [5, 60]
    orc = oracle.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    ref = orc.exx_apply(s.psi[:s.n_occ], s.f, s.psi, cols=cols)
    assert pm.rel(vx.cpu().numpy()[cols], ref) < (1e-10 if name == "fp64" else 1e-6)


ACE_CASES = [dict(n=(13, 11, 12), bc=(0, 0, 1), n_orb=10, kernel=0),      # N = 1716: 6 k chunks, split k
             dict(n=(8, 7, 9), bc=(1, 0, 0), n_orb=150, kernel=0),         # n = 150: 2 x 2 output tiles
             dict(n=(24, 20, 22), bc=(1, 1, 1), n_orb=40, kernel=1, omega=0.106)]


@pytest.mark.parametrize("case", ACE_CASES, ids=lambda c: f"{'x'.join(map(str, c['n']))}_{c['n_orb']}")
def test_split_ace_on_tensor_cores_matches_oracle(exx, case):
    """ACE products in a split plan (fixed-point digits on the tensor cores) against the
    FP64 oracle of Sec. III, for an exact W (taken from the FP64 path)."""
    s = synth.small_system(h=0.4, seed=41, **case)
    n = s.n_orb
    p64 = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    psi = torch.from_numpy(s.psi).cuda()
    f = torch.from_numpy(s.f).cuda()
    W = p64.apply(psi[:s.n_occ], f, psi)
    Wh = W.cpu().numpy()
    M_ref, L_ref, xi_ref = oracle.ace(s.psi, Wh, s.dV)
    p = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    p.set_precision(SPLIT["bf16x10"][0])
    Md = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    # strided operands: rows of Psi and W padded past N
    pad = torch.zeros((n, s.N + 9), dtype=torch.float64, device="cuda")
    pad[:, :s.N] = psi
    wpad = torch.zeros((n, s.N + 5), dtype=torch.float64, device="cuda")
    wpad[:, :s.N] = W
    xi = p.ace_build(pad[:, :s.N], wpad[:, :s.N], M=Md)
    assert pm.rel(Md.cpu().numpy().T, M_ref) < 1e-8
    assert pm.rel(xi.cpu().numpy(), xi_ref) < 1e-8
    back = p.ace_apply(xi, psi)
    assert pm.rel(back.cpu().numpy(), Wh) < 1e-8
    # a block of 3 vectors that are not orbitals: -dV xi (xi^T Phi) against numpy
    rng = np.random.Generator(np.random.PCG64(7))
    phi = rng.normal(size=(3, s.N))
    got = p.ace_apply(xi, torch.from_numpy(phi).cuda()).cpu().numpy()
    X = xi.cpu().numpy()
    want = -s.dV * (X.T @ (X @ phi.T)).T
    assert pm.rel(got, want) < 1e-8


def test_bounded_wait_reports_timeout_and_context_survives(exx):
    """A wait that runs out (a barrier nothing completes) comes back as EXX_ERR_TIMEOUT
    from the device error word, and the GPU keeps working afterwards."""
    L = exx.load()
    L.exx_debug_wait_timeout.argtypes = [ctypes.POINTER(ctypes.c_int)]
    st = ctypes.c_int(-1)
    assert L.exx_debug_wait_timeout(ctypes.byref(st)) == 0
    assert st.value == exx.EXX_ERR_TIMEOUT
    # the context is intact: a small apply still matches the oracle
    s = synth.small_system(n=(10, 9, 8), h=0.4, bc=(0, 0, 0), n_orb=4, kernel=0, seed=2)
    plan, psi, f, vx, e = _apply(exx, s, SPLIT["bf16x10"][0])
    orc = oracle.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    assert pm.rel(vx.cpu().numpy(), orc.exx_apply(s.psi[:s.n_occ], s.f, s.psi)) < 1e-6
