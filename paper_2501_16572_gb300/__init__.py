"""Python binding of libexx_gb300 (exact exchange + ACE on GB300).

Argument marshalling only: every step of the computation runs in the CUDA kernels of
``libexx_gb300.so`` behind the C interface of ``include/exx.h``.  PyTorch supplies
device memory and streams.  There is no CPU fallback: when the library has not been
built (``python -m paper_2501_16572_gb300._build``) or no GPU is usable, the calls
raise.

Orbital blocks are ``torch.float64`` CUDA tensors of shape ``(n_orb, N)`` with rows
contiguous, i.e. the column-major ``N x n_orb`` matrices of the C interface with
leading dimension ``N`` (row stride).  Grid index r = ix + Nx*(iy + Ny*iz).
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libexx_gb300.so")

EXX_OK = 0
EXX_ERR_INVALID_ARG = 1
EXX_ERR_CUDA = 2
EXX_ERR_OOM = 3
EXX_ERR_NOT_POSDEF = 4
EXX_ERR_TIMEOUT = 5
EXX_ERR_UNSUPPORTED = 6

EXX_BC_DIRICHLET = 0
EXX_BC_PERIODIC = 1
EXX_KERNEL_COULOMB = 0
EXX_KERNEL_ERFC = 1
EXX_KERNEL_ERFC_PAPER16PI = 2
EXX_PREC_FP64 = 0
EXX_PREC_BF16X3 = 1
EXX_PREC_TF32X3 = 2
EXX_PREC_BF16X6 = 3
EXX_PREC_BF16X10 = 4
EXX_PREC_BF16X7 = 5
PREC_NAMES = {EXX_PREC_FP64: "fp64", EXX_PREC_BF16X3: "bf16x3", EXX_PREC_TF32X3: "tf32x3",
              EXX_PREC_BF16X6: "bf16x6", EXX_PREC_BF16X10: "bf16x10", EXX_PREC_BF16X7: "bf16x7"}

# symbols declared in include/exx.h (checked by the CPU tests)
EXPORTED = ["exx_plan_create", "exx_plan_set_precision", "exx_plan_set_batch", "exx_plan_destroy",
            "exx_plan_get", "exx_apply", "exx_energy", "ace_build", "ace_apply", "exx_ace_step_host",
            "exx_apply_batched", "exx_plan_launch_count", "exx_status_string", "exx_last_error",
            "exx_plan_set_timing", "exx_plan_get_timing", "exx_gram_noalloc", "exx_plan_set_shard",
            "exx_apply_original", "exx_plan_autotune", "exx_plan_get_tuning", "exx_plan_create_bloch",
            "exx_apply_complex", "exx_energy_complex", "ace_build_complex", "ace_apply_complex",
            "exx_plan_set_tuning"]
TIMING_KINDS = ["pass1", "pass2", "pass3", "pass4", "pass5", "accum", "prep", "gemm", "chol", "energy"]

_lib = None
_vp = ctypes.c_void_p
_d = ctypes.c_double
_i = ctypes.c_int
_l = ctypes.c_long


class ExxError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: {load().exx_status_string(status).decode()} -- "
                         f"{load().exx_last_error().decode()}")


class ExxApplyArgs(ctypes.Structure):
    _fields_ = [("Psi_occ", _vp), ("n_occ", _i), ("ld_occ", _l), ("f", _vp),
                ("Psi_in", _vp), ("n_in", _i), ("ld_in", _l), ("out", _vp), ("ld_out", _l)]


def load():
    """Load libexx_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2501_16572_gb300._build` "
                          "(or __graft_entry__.build()); there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    L.exx_plan_create.argtypes = [ctypes.POINTER(_vp), _i, _i, _i, _d, ctypes.POINTER(_i), _i, _i, _d]
    L.exx_plan_set_precision.argtypes = [_vp, _i]
    L.exx_plan_set_batch.argtypes = [_vp, _i, _i]
    L.exx_plan_destroy.argtypes = [_vp]
    L.exx_plan_get.argtypes = [_vp, _i, ctypes.POINTER(_d), _l]
    L.exx_apply.argtypes = [_vp, _vp, _i, _l, _vp, _vp, _i, _l, _vp, _l, _vp]
    L.exx_energy.argtypes = [_vp, _vp, _i, _l, _vp, _vp, _l, ctypes.POINTER(_d), _vp]
    L.ace_build.argtypes = [_vp, _vp, _i, _l, _vp, _l, _vp, _l, _vp, ctypes.POINTER(_i), _vp]
    L.ace_apply.argtypes = [_vp, _vp, _i, _l, _vp, _i, _l, _vp, _l, _vp]
    L.exx_ace_step_host.argtypes = [_vp, _vp, _i, _l, _i, _vp, _vp, _l, ctypes.POINTER(_d),
                                    ctypes.POINTER(_i), _vp]
    L.exx_apply_batched.argtypes = [ctypes.POINTER(_vp), _i, ctypes.POINTER(ExxApplyArgs), _vp]
    L.exx_apply_original.argtypes = [_vp, _vp, _i, _l, _vp, _vp, _i, _l, _vp, _l, _vp]
    L.exx_plan_autotune.argtypes = [_vp, _vp, _i, _l, _vp, _vp, _i, _l, _vp, _l, _i, _vp]
    L.exx_plan_create_bloch.argtypes = [ctypes.POINTER(_vp), _i, _i, _i, _d, ctypes.POINTER(_i), _i, _i, _d,
                                        ctypes.POINTER(_d)]
    L.exx_apply_complex.argtypes = [_vp, _vp, _i, _l, _vp, _vp, _i, _l, _vp, _l, _i, _vp]
    L.exx_energy_complex.argtypes = [_vp, _vp, _i, _l, _vp, _vp, _l, ctypes.POINTER(_d), _vp]
    L.ace_build_complex.argtypes = [_vp, _vp, _i, _l, _vp, _l, _vp, _l, ctypes.POINTER(_i), _vp]
    L.ace_apply_complex.argtypes = [_vp, _vp, _i, _l, _vp, _i, _l, _vp, _l, _vp]
    L.exx_plan_get_tuning.argtypes = [_vp, ctypes.POINTER(_i), ctypes.POINTER(_d), ctypes.POINTER(_i)]
    L.exx_plan_set_tuning.argtypes = [_vp, ctypes.POINTER(_i)]
    L.exx_plan_launch_count.argtypes = [_vp]
    L.exx_plan_launch_count.restype = _l
    L.exx_plan_set_timing.argtypes = [_vp, _i]
    L.exx_plan_get_timing.argtypes = [_vp, _i, ctypes.POINTER(_d), ctypes.POINTER(_l)]
    L.exx_plan_set_shard.argtypes = [_vp, _i, _i]
    L.exx_gram_noalloc.argtypes = [_i, _d, _vp, _i, _l, _vp, _l, _vp, _vp]
    L.exx_status_string.argtypes = [_i]
    L.exx_status_string.restype = ctypes.c_char_p
    L.exx_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(rc, what):
    if rc != EXX_OK:
        raise ExxError(rc, what)


def _ptr(t):
    return _vp(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return _vp(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return _vp(stream)
    return _vp(stream.cuda_stream)


def _orb(t, N, name):
    """Validate a (n, N) float64 CUDA block with contiguous rows; returns (n, ld)."""
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda:
        raise TypeError(f"{name} must be a float64 CUDA tensor")
    if t.dim() != 2 or t.shape[1] != N or t.stride(1) != 1:
        raise ValueError(f"{name} must have shape (n, {N}) with contiguous rows")
    return t.shape[0], t.stride(0)


def _corb(t, N, name):
    """Validate a (n, N) complex128 CUDA block with contiguous rows; returns (n, ld)."""
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.complex128 or not t.is_cuda:
        raise TypeError(f"{name} must be a complex128 CUDA tensor")
    if t.dim() != 2 or t.shape[1] != N or t.stride(1) != 1:
        raise ValueError(f"{name} must have shape (n, {N}) with contiguous rows")
    return t.shape[0], t.stride(0)


class Plan:
    """A grid plan (exx_plan_create)."""

    def __init__(self, n, h, bc, fd_order=12, kernel=EXX_KERNEL_COULOMB, omega=0.0):
        L = load()
        self.n = tuple(int(v) for v in n)
        self.N = self.n[0] * self.n[1] * self.n[2]
        self.h = float(h)
        self.dV = self.h ** 3
        self.bc = tuple(int(b) for b in bc)
        self.kernel = int(kernel)
        self.omega = float(omega)
        self.precision = EXX_PREC_FP64
        h_ = _vp()
        bca = (_i * 3)(*self.bc)
        _check(L.exx_plan_create(ctypes.byref(h_), self.n[0], self.n[1], self.n[2], self.h, bca,
                                 int(fd_order), self.kernel, self.omega), "exx_plan_create")
        self._h = h_

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().exx_plan_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_precision(self, prec):
        _check(load().exx_plan_set_precision(self._h, int(prec)), "exx_plan_set_precision")
        self.precision = int(prec)

    def set_batch(self, pairs_per_batch=0, block_orbitals=0):
        _check(load().exx_plan_set_batch(self._h, int(pairs_per_batch), int(block_orbitals)),
               "exx_plan_set_batch")

    def set_shard(self, rank, world):
        """Run only batches b with b % world == rank; outputs become partial sums."""
        _check(load().exx_plan_set_shard(self._h, int(rank), int(world)), "exx_plan_set_shard")

    def eigvals(self, d):
        import numpy as np
        out = np.zeros(self.n[d])
        _check(load().exx_plan_get(self._h, d, out.ctypes.data_as(ctypes.POINTER(_d)), out.size), "exx_plan_get")
        return out

    def F(self):
        import numpy as np
        out = np.zeros(self.N)
        _check(load().exx_plan_get(self._h, 3, out.ctypes.data_as(ctypes.POINTER(_d)), out.size), "exx_plan_get")
        return out

    def launch_count(self):
        return int(load().exx_plan_launch_count(self._h))

    def set_timing(self, enable=True):
        _check(load().exx_plan_set_timing(self._h, 1 if enable else 0), "exx_plan_set_timing")

    def timing(self):
        """{kernel class: (total ms, launches)} recorded since set_timing(True)."""
        out = {}
        for k, name in enumerate(TIMING_KINDS):
            ms, n = _d(0.0), _l(0)
            _check(load().exx_plan_get_timing(self._h, k, ctypes.byref(ms), ctypes.byref(n)), "exx_plan_get_timing")
            if n.value:
                out[name] = (ms.value, n.value)
        return out

    # -- the hot path ------------------------------------------------------------------
    def apply(self, psi_occ, f, psi_in, out=None, stream=None):
        """(Vx psi)_n for the rows of psi_in (exx_apply); returns out (n_in, N)."""
        import torch
        n_occ, ld_occ = _orb(psi_occ, self.N, "psi_occ")
        n_in, ld_in = _orb(psi_in, self.N, "psi_in")
        if f.dtype != torch.float64 or not f.is_cuda or f.numel() < n_occ or not f.is_contiguous():
            raise ValueError("f must be a contiguous float64 CUDA tensor with n_occ entries")
        if out is None:
            out = torch.empty((n_in, self.N), dtype=torch.float64, device=psi_in.device)
        n_o, ld_out = _orb(out, self.N, "out")
        if n_o != n_in:
            raise ValueError("out must have n_in rows")
        _check(load().exx_apply(self._h, _ptr(psi_occ), n_occ, ld_occ, _ptr(f), _ptr(psi_in), n_in, ld_in,
                                _ptr(out), ld_out, _stream(stream)), "exx_apply")
        return out

    def autotune(self, psi_occ, f, psi_in, out=None, remeasure=False, stream=None):
        """exx_plan_autotune on these buffers; returns tuning() afterwards."""
        import torch
        n_occ, ld_occ = _orb(psi_occ, self.N, "psi_occ")
        n_in, ld_in = _orb(psi_in, self.N, "psi_in")
        if out is None:
            out = torch.empty((n_in, self.N), dtype=torch.float64, device=psi_in.device)
        _, ld_out = _orb(out, self.N, "out")
        _check(load().exx_plan_autotune(self._h, _ptr(psi_occ), n_occ, ld_occ, _ptr(f), _ptr(psi_in), n_in, ld_in,
                                        _ptr(out), ld_out, 1 if remeasure else 0, _stream(stream)), "exx_plan_autotune")
        return self.tuning()

    def set_tuning(self, pairs_per_batch=0, block_orbitals=0, z_block=0, z_buffers=0, staging=-1, pipeline=-1):
        v = (_i * 6)(pairs_per_batch, block_orbitals, z_block, z_buffers, staging, pipeline)
        _check(load().exx_plan_set_tuning(self._h, v), "exx_plan_set_tuning")

    def tuning(self):
        """{'pairs_per_batch', 'block_orbitals', 'z_block', 'z_buffers', 'staging', 'pipeline', 'ms_per_pair',
        'tuned'}"""
        v = (_i * 6)()
        ms, tuned = _d(0.0), _i(0)
        _check(load().exx_plan_get_tuning(self._h, v, ctypes.byref(ms), ctypes.byref(tuned)), "exx_plan_get_tuning")
        return {"pairs_per_batch": v[0], "block_orbitals": v[1], "z_block": v[2], "z_buffers": v[3],
                "staging": v[4], "pipeline": v[5], "ms_per_pair": ms.value, "tuned": tuned.value}

    # -- complex (Bloch) plans ------------------------------------------------------------
    @classmethod
    def bloch(cls, n, h, bc, theta, fd_order=12, kernel=EXX_KERNEL_COULOMB, omega=0.0):
        """A Bloch plan (exx_plan_create_bloch): theta[d] = phase across one period of axis d."""
        self = cls.__new__(cls)
        self.n = tuple(int(v) for v in n)
        self.N = self.n[0] * self.n[1] * self.n[2]
        self.h = float(h)
        self.dV = self.h ** 3
        self.bc = tuple(int(b) for b in bc)
        self.kernel = int(kernel)
        self.omega = float(omega)
        self.precision = EXX_PREC_FP64
        h_ = _vp()
        bca = (_i * 3)(*self.bc)
        th = (_d * 3)(*[float(t) for t in theta])
        _check(load().exx_plan_create_bloch(ctypes.byref(h_), self.n[0], self.n[1], self.n[2], self.h, bca,
                                            int(fd_order), self.kernel, self.omega, th), "exx_plan_create_bloch")
        self._h = h_
        return self

    def apply_complex(self, psi_occ, f, psi_in, out=None, accumulate=False, stream=None):
        import torch
        n_occ, ld_occ = _corb(psi_occ, self.N, "psi_occ")
        n_in, ld_in = _corb(psi_in, self.N, "psi_in")
        if f.dtype != torch.float64 or not f.is_cuda or f.numel() < n_occ or not f.is_contiguous():
            raise ValueError("f must be a contiguous float64 CUDA tensor with n_occ entries")
        if out is None:
            out = torch.empty((n_in, self.N), dtype=torch.complex128, device=psi_in.device)
        n_o, ld_out = _corb(out, self.N, "out")
        if n_o != n_in:
            raise ValueError("out must have n_in rows")
        _check(load().exx_apply_complex(self._h, _ptr(psi_occ), n_occ, ld_occ, _ptr(f), _ptr(psi_in), n_in, ld_in,
                                        _ptr(out), ld_out, 1 if accumulate else 0, _stream(stream)),
               "exx_apply_complex")
        return out

    def energy_complex(self, psi, f, vx, stream=None):
        n, ld = _corb(psi, self.N, "psi")
        _, ld_v = _corb(vx, self.N, "vx")
        e = _d(0.0)
        _check(load().exx_energy_complex(self._h, _ptr(psi), n, ld, _ptr(f), _ptr(vx), ld_v, ctypes.byref(e),
                                         _stream(stream)), "exx_energy_complex")
        return e.value

    def ace_build_complex(self, psi, W, xi=None, stream=None):
        import torch
        n, ld = _corb(psi, self.N, "psi")
        _, ld_w = _corb(W, self.N, "W")
        if xi is None:
            xi = torch.empty_like(psi)
        _, ld_xi = _corb(xi, self.N, "xi")
        info = _i(0)
        rc = load().ace_build_complex(self._h, _ptr(psi), n, ld, _ptr(W), ld_w, _ptr(xi), ld_xi, ctypes.byref(info),
                                      _stream(stream))
        if rc != EXX_OK:
            err = ExxError(rc, "ace_build_complex")
            err.pivot = info.value - 1
            raise err
        return xi

    def ace_apply_complex(self, xi, phi, out=None, stream=None):
        import torch
        n, ld_xi = _corb(xi, self.N, "xi")
        nphi, ld_phi = _corb(phi, self.N, "phi")
        if out is None:
            out = torch.empty_like(phi)
        _, ld_out = _corb(out, self.N, "out")
        _check(load().ace_apply_complex(self._h, _ptr(xi), n, ld_xi, _ptr(phi), nphi, ld_phi, _ptr(out), ld_out,
                                        _stream(stream)), "ace_apply_complex")
        return out

    def apply_original(self, psi_occ, f, psi_in, out=None, stream=None):
        """exx_apply_original: the same result, one pair at a time with Eq. 8's 4 n_z + 2 GEMMs."""
        import torch
        n_occ, ld_occ = _orb(psi_occ, self.N, "psi_occ")
        n_in, ld_in = _orb(psi_in, self.N, "psi_in")
        if f.dtype != torch.float64 or not f.is_cuda or f.numel() < n_occ or not f.is_contiguous():
            raise ValueError("f must be a contiguous float64 CUDA tensor with n_occ entries")
        if out is None:
            out = torch.empty((n_in, self.N), dtype=torch.float64, device=psi_in.device)
        n_o, ld_out = _orb(out, self.N, "out")
        if n_o != n_in:
            raise ValueError("out must have n_in rows")
        _check(load().exx_apply_original(self._h, _ptr(psi_occ), n_occ, ld_occ, _ptr(f), _ptr(psi_in), n_in,
                                         ld_in, _ptr(out), ld_out, _stream(stream)), "exx_apply_original")
        return out

    def energy(self, psi_occ, f, vx, stream=None):
        n_occ, ld = _orb(psi_occ, self.N, "psi_occ")
        _, ld_v = _orb(vx, self.N, "vx")
        e = _d(0.0)
        _check(load().exx_energy(self._h, _ptr(psi_occ), n_occ, ld, _ptr(f), _ptr(vx), ld_v, ctypes.byref(e),
                                 _stream(stream)), "exx_energy")
        return e.value

    def ace_build(self, psi, W, xi=None, M=None, stream=None):
        """xi (n, N) and, optionally, M (n x n, column-major) of the ACE operator."""
        import torch
        n, ld = _orb(psi, self.N, "psi")
        _, ld_w = _orb(W, self.N, "W")
        if xi is None:
            xi = torch.empty_like(psi)
        _, ld_xi = _orb(xi, self.N, "xi")
        info = _i(0)
        mp = _vp(M.data_ptr()) if M is not None else _vp()
        rc = load().ace_build(self._h, _ptr(psi), n, ld, _ptr(W), ld_w, _ptr(xi), ld_xi, mp, ctypes.byref(info),
                              _stream(stream))
        if rc == EXX_ERR_NOT_POSDEF:
            err = ExxError(rc, "ace_build")
            err.pivot = info.value - 1
            raise err
        _check(rc, "ace_build")
        return xi

    def ace_apply(self, xi, phi, out=None, stream=None):
        import torch
        n, ld_xi = _orb(xi, self.N, "xi")
        nphi, ld_phi = _orb(phi, self.N, "phi")
        if out is None:
            out = torch.empty_like(phi)
        _, ld_out = _orb(out, self.N, "out")
        _check(load().ace_apply(self._h, _ptr(xi), n, ld_xi, _ptr(phi), nphi, ld_phi, _ptr(out), ld_out,
                                _stream(stream)), "ace_apply")
        return out

    def ace_step_host(self, psi_h, n_occ, f_h, xi_h, stream=None):
        """Host-buffer ACE step (exx_ace_step_host): numpy/torch CPU arrays in, xi_h out; returns E_x."""
        import numpy as np
        n = psi_h.shape[0]
        e = _d(0.0)
        info = _i(0)
        def hp(a):
            return _vp(a.data_ptr()) if hasattr(a, "data_ptr") else _vp(a.ctypes.data)
        _check(load().exx_ace_step_host(self._h, hp(psi_h), n, self.N, int(n_occ), hp(f_h), hp(xi_h), self.N,
                                        ctypes.byref(e), ctypes.byref(info), _stream(stream)), "exx_ace_step_host")
        return e.value


# ---- module-level names matching the C interface --------------------------------------
def exx_plan_create(n, h, bc, fd_order=12, kernel=EXX_KERNEL_COULOMB, omega=0.0):
    return Plan(n, h, bc, fd_order, kernel, omega)


def exx_plan_set_precision(plan, prec):
    plan.set_precision(prec)


def exx_plan_set_batch(plan, pairs_per_batch=0, block_orbitals=0):
    plan.set_batch(pairs_per_batch, block_orbitals)


def exx_plan_destroy(plan):
    plan.close()


def exx_apply(plan, psi_occ, f, psi_in, out=None, stream=None):
    return plan.apply(psi_occ, f, psi_in, out, stream)


def exx_energy(plan, psi_occ, f, vx, stream=None):
    return plan.energy(psi_occ, f, vx, stream)


def ace_build(plan, psi, W, xi=None, M=None, stream=None):
    return plan.ace_build(psi, W, xi, M, stream)


def ace_apply(plan, xi, phi, out=None, stream=None):
    return plan.ace_apply(xi, phi, out, stream)


def exx_ace_step_host(plan, psi_h, n_occ, f_h, xi_h, stream=None):
    return plan.ace_step_host(psi_h, n_occ, f_h, xi_h, stream)


def exx_apply_batched(plans, args, stream=None):
    """args: list of (psi_occ, f, psi_in, out) tensor tuples, one per plan."""
    n = len(plans)
    hs = (_vp * n)(*[p.handle.value for p in plans])
    arr = (ExxApplyArgs * n)()
    keep = []
    for i, (p, (po, f, pi, out)) in enumerate(zip(plans, args)):
        n_occ, ld_occ = _orb(po, p.N, "psi_occ")
        n_in, ld_in = _orb(pi, p.N, "psi_in")
        _, ld_out = _orb(out, p.N, "out")
        arr[i] = ExxApplyArgs(po.data_ptr(), n_occ, ld_occ, f.data_ptr(), pi.data_ptr(), n_in, ld_in,
                              out.data_ptr(), ld_out)
        keep.append((po, f, pi, out))
    _check(load().exx_apply_batched(hs, n, arr, _stream(stream)), "exx_apply_batched")
    return [a[3] for a in args]
