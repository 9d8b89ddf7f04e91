"""CPU FP64 oracle of the exact-exchange path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  The CUDA library never does; the two share no code.

Thin ctypes wrapper around ``exx_oracle.c`` (plain C, FP64).  ``build()`` compiles
it with gcc into ``liboracle.so`` beside this file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "exx_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, FP64, OpenMP, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-std=c99",
               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.exo_fd_weights.argtypes = [ctypes.c_int, _D]
        L.exo_second_derivative_1d.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, _D]
        L.exo_jacobi_eigh.argtypes = [ctypes.c_int, _D, _D, _D]
        L.exo_kernel_value.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_double]
        L.exo_kernel_value.restype = ctypes.c_double
        L.exo_plan_new.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _I,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_double]
        L.exo_plan_new.restype = ctypes.c_void_p
        L.exo_plan_free.argtypes = [ctypes.c_void_p]
        L.exo_plan_eigvecs.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.exo_plan_eigvecs.restype = _D
        L.exo_plan_eigvals.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.exo_plan_eigvals.restype = _D
        L.exo_plan_F.argtypes = [ctypes.c_void_p]
        L.exo_plan_F.restype = _D
        L.exo_solve.argtypes = [ctypes.c_void_p, _D, _D]
        L.exo_exx_apply.argtypes = [ctypes.c_void_p, _D, ctypes.c_int, _D, _D, ctypes.c_int, _I,
                                    ctypes.c_int, _D]
        L.exo_energy.argtypes = [ctypes.c_void_p, _D, ctypes.c_int, _D, _D, ctypes.c_long]
        L.exo_energy.restype = ctypes.c_double
        L.exo_bloch_operator_1d.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_double, _D]
        L.exo_hermitian_eigh.argtypes = [ctypes.c_int, _D, _D, _D]
        L.exo_cplan_new.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _I, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_double, _D]
        L.exo_cplan_new.restype = ctypes.c_void_p
        L.exo_cplan_free.argtypes = [ctypes.c_void_p]
        for nm in ("exo_cplan_eigvecs", "exo_cplan_eigvals"):
            getattr(L, nm).argtypes = [ctypes.c_void_p, ctypes.c_int]
            getattr(L, nm).restype = _D
        L.exo_cplan_F.argtypes = [ctypes.c_void_p]
        L.exo_cplan_F.restype = _D
        L.exo_csolve.argtypes = [ctypes.c_void_p, _D, _D]
        L.exo_cexx_apply.argtypes = [ctypes.c_void_p, _D, ctypes.c_int, _D, _D, ctypes.c_int, _I, ctypes.c_int, _D]
        L.exo_cenergy.argtypes = [ctypes.c_void_p, _D, ctypes.c_int, _D, _D]
        L.exo_cenergy.restype = ctypes.c_double
        L.exo_cace.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _D, _D, _D, _D, _D]
        L.exo_energy_pairs.argtypes = [ctypes.c_void_p, _D, ctypes.c_int, _D]
        L.exo_energy_pairs.restype = ctypes.c_double
        L.exo_ace.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _D, _D, _D, _D, _D]
        L.exo_ace_apply.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _D, _D, ctypes.c_int, _D]
        L.exo_set_mutation.argtypes = [ctypes.c_int]
        L.exo_num_threads.restype = ctypes.c_int
        L.exo_set_num_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(_D)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(lib().exo_num_threads())


def set_num_threads(n: int) -> None:
    """Thread count of the oracle's OpenMP loops (for timing on n cores)."""
    lib().exo_set_num_threads(int(n))


def set_mutation(m: int) -> None:
    """Plant a deliberate mistake (tests only): 1 transposed V3, 2 dropped F, 3 sign flip."""
    lib().exo_set_mutation(int(m))


def fd_weights(p: int) -> np.ndarray:
    w = np.zeros(p + 1)
    if lib().exo_fd_weights(p, _p(w)):
        raise ValueError("bad FD order")
    return w


def second_derivative_1d(n, h, bc, p) -> np.ndarray:
    """n x n operator (returned as a numpy array D[i, j])."""
    D = np.zeros(n * n)
    if lib().exo_second_derivative_1d(n, h, bc, p, _p(D)):
        raise ValueError("bad operator arguments")
    return D.reshape(n, n, order="F")


def jacobi_eigh(A):
    A = np.asfortranarray(A, dtype=np.float64)
    n = A.shape[0]
    Af = np.ascontiguousarray(A.reshape(-1, order="F"))
    V = np.zeros(n * n)
    lam = np.zeros(n)
    lib().exo_jacobi_eigh(n, _p(Af), _p(V), _p(lam))
    return lam, V.reshape(n, n, order="F")


def kernel_value(lam, kernel, omega) -> float:
    return float(lib().exo_kernel_value(float(lam), int(kernel), float(omega)))


class Plan:
    """Oracle plan: 1D eigenbases and f(Lambda) for one grid."""

    def __init__(self, n, h, bc, fd_order=12, kernel=0, omega=0.0):
        self.n = tuple(int(v) for v in n)
        self.N = self.n[0] * self.n[1] * self.n[2]
        self.h = float(h)
        self.dV = self.h ** 3
        bca = (ctypes.c_int * 3)(*[int(b) for b in bc])
        self._p = lib().exo_plan_new(self.n[0], self.n[1], self.n[2], self.h, bca, int(fd_order),
                                     int(kernel), float(omega))
        if not self._p:
            raise ValueError("oracle plan creation failed")

    def __del__(self):
        if getattr(self, "_p", None) and _lib is not None:
            _lib.exo_plan_free(self._p)
            self._p = None

    def eigvals(self, d):
        nd = self.n[d]
        ptr = lib().exo_plan_eigvals(self._p, d)
        return np.ctypeslib.as_array(ptr, shape=(nd,)).copy()

    def eigvecs(self, d):
        nd = self.n[d]
        ptr = lib().exo_plan_eigvecs(self._p, d)
        return np.ctypeslib.as_array(ptr, shape=(nd * nd,)).copy().reshape(nd, nd, order="F")

    def F(self):
        ptr = lib().exo_plan_F(self._p)
        return np.ctypeslib.as_array(ptr, shape=(self.N,)).copy()

    def solve(self, rho):
        rho = _c64(rho).reshape(-1)
        assert rho.size == self.N
        out = np.zeros(self.N)
        if lib().exo_solve(self._p, _p(rho), _p(out)):
            raise MemoryError
        return out

    def exx_apply(self, psi_occ, f, psi_in, cols=None):
        """(n_cols, N) array of (Vx psi)_n for n in cols (all columns of psi_in by default)."""
        psi_occ = _c64(psi_occ)
        psi_in = _c64(psi_in)
        f = _c64(f)
        n_occ, n_in = psi_occ.shape[0], psi_in.shape[0]
        assert f.shape[0] == n_occ
        if cols is None:
            out = np.zeros((n_in, self.N))
            rc = lib().exo_exx_apply(self._p, _p(psi_occ), n_occ, _p(f), _p(psi_in), n_in, None, n_in, _p(out))
        else:
            ci = np.ascontiguousarray(cols, dtype=np.int32)
            out = np.zeros((ci.size, self.N))
            rc = lib().exo_exx_apply(self._p, _p(psi_occ), n_occ, _p(f), _p(psi_in), n_in,
                                     ci.ctypes.data_as(_I), ci.size, _p(out))
        if rc:
            raise RuntimeError(f"oracle exx_apply failed ({rc})")
        return out

    def energy(self, psi_occ, f, vx):
        psi_occ = _c64(psi_occ)
        vx = _c64(vx)
        f = _c64(f)
        return float(lib().exo_energy(self._p, _p(psi_occ), psi_occ.shape[0], _p(f), _p(vx), self.N))

    def energy_pairs(self, psi_occ, f):
        psi_occ = _c64(psi_occ)
        f = _c64(f)
        return float(lib().exo_energy_pairs(self._p, _p(psi_occ), psi_occ.shape[0], _p(f)))


def ace(psi, W, dV):
    """Returns (M, L, xi) or raises ValueError(pivot) when -M is not positive definite."""
    psi = _c64(psi)
    W = _c64(W)
    n, N = psi.shape
    M = np.zeros(n * n)
    L = np.zeros(n * n)
    xi = np.zeros((n, N))
    rc = lib().exo_ace(N, n, float(dV), _p(psi), _p(W), _p(M), _p(L), _p(xi))
    if rc:
        raise ValueError(f"not positive definite at pivot {rc - 1}")
    return M.reshape(n, n, order="F"), L.reshape(n, n, order="F"), xi


def ace_apply(xi, phi, dV):
    xi = _c64(xi)
    phi = _c64(phi)
    n, N = xi.shape
    out = np.zeros_like(phi)
    lib().exo_ace_apply(N, n, float(dV), _p(xi), _p(phi), phi.shape[0], _p(out))
    return out


# ---- complex (Bloch) path -----------------------------------------------------------------

def _cz(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _pz(a):
    return a.ctypes.data_as(_D)


def bloch_operator_1d(n, h, bc, p, theta) -> np.ndarray:
    D = np.zeros((n, n), dtype=np.complex128, order="F")
    if lib().exo_bloch_operator_1d(n, float(h), int(bc), int(p), float(theta), _pz(D)):
        raise ValueError("bad operator arguments")
    return D


def hermitian_eigh(A):
    A = np.asfortranarray(A, dtype=np.complex128)
    n = A.shape[0]
    V = np.zeros((n, n), dtype=np.complex128, order="F")
    lam = np.zeros(n)
    if lib().exo_hermitian_eigh(n, _pz(A), _pz(V), _p(lam)):
        raise MemoryError
    return lam, V


class CPlan:
    """Oracle plan of the Bloch problem: theta[d] = phase across one period of axis d."""

    def __init__(self, n, h, bc, fd_order=12, kernel=0, omega=0.0, theta=(0.0, 0.0, 0.0)):
        self.n = tuple(int(v) for v in n)
        self.N = self.n[0] * self.n[1] * self.n[2]
        self.h = float(h)
        self.dV = self.h ** 3
        bca = (ctypes.c_int * 3)(*[int(b) for b in bc])
        th = np.ascontiguousarray(theta, dtype=np.float64)
        self._p = lib().exo_cplan_new(self.n[0], self.n[1], self.n[2], self.h, bca, int(fd_order), int(kernel),
                                      float(omega), _p(th))
        if not self._p:
            raise ValueError("oracle Bloch plan creation failed")

    def __del__(self):
        if getattr(self, "_p", None) and _lib is not None:
            _lib.exo_cplan_free(self._p)
            self._p = None

    def eigvals(self, d):
        return np.ctypeslib.as_array(lib().exo_cplan_eigvals(self._p, d), shape=(self.n[d],)).copy()

    def eigvecs(self, d):
        nd = self.n[d]
        raw = np.ctypeslib.as_array(lib().exo_cplan_eigvecs(self._p, d), shape=(2 * nd * nd,)).copy()
        return raw.view(np.complex128).reshape(nd, nd, order="F")

    def F(self):
        return np.ctypeslib.as_array(lib().exo_cplan_F(self._p), shape=(self.N,)).copy()

    def solve(self, rho):
        rho = _cz(rho).reshape(-1)
        out = np.zeros(self.N, dtype=np.complex128)
        if lib().exo_csolve(self._p, _pz(rho), _pz(out)):
            raise MemoryError
        return out

    def exx_apply(self, psi_occ, f, psi_in, cols=None):
        psi_occ, psi_in, f = _cz(psi_occ), _cz(psi_in), _c64(f)
        n_occ, n_in = psi_occ.shape[0], psi_in.shape[0]
        if cols is None:
            out = np.zeros((n_in, self.N), dtype=np.complex128)
            rc = lib().exo_cexx_apply(self._p, _pz(psi_occ), n_occ, _p(f), _pz(psi_in), n_in, None, n_in, _pz(out))
        else:
            ci = np.ascontiguousarray(cols, dtype=np.int32)
            out = np.zeros((ci.size, self.N), dtype=np.complex128)
            rc = lib().exo_cexx_apply(self._p, _pz(psi_occ), n_occ, _p(f), _pz(psi_in), n_in,
                                      ci.ctypes.data_as(_I), ci.size, _pz(out))
        if rc:
            raise RuntimeError(f"oracle complex exx_apply failed ({rc})")
        return out

    def energy(self, psi, f, vx):
        psi, vx, f = _cz(psi), _cz(vx), _c64(f)
        return float(lib().exo_cenergy(self._p, _pz(psi), psi.shape[0], _p(f), _pz(vx)))


def cace(psi, W, dV):
    """Complex ACE: (M, L, xi) with M = dV Psi^H W, -(M + M^H)/2 = L L^H, xi = W L^{-H}."""
    psi, W = _cz(psi), _cz(W)
    n, N = psi.shape
    M = np.zeros(n * n, dtype=np.complex128)
    L = np.zeros(n * n, dtype=np.complex128)
    xi = np.zeros((n, N), dtype=np.complex128)
    rc = lib().exo_cace(N, n, float(dV), _pz(psi), _pz(W), _pz(M), _pz(L), _pz(xi))
    if rc:
        raise ValueError(f"not positive definite at pivot {rc - 1}")
    return M.reshape(n, n, order="F"), L.reshape(n, n, order="F"), xi
