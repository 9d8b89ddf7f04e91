"""Seeded synthetic inputs for the exact-exchange path (orbitals, occupations, grids).

This module serves both the CPU oracle (``oracle/``) and the CUDA library
(``paper_2501_16572_gb300``); it holds none of the method's arithmetic (no finite
differences, no eigen-decomposition, no Poisson solve, no exchange sums).  It only
draws numbers and orthonormalises them.

The paper's workloads (Mo and TiO2 with ONCV pseudopotentials, Sec. IV) are not
available, so smooth localized orbitals on grids of the paper's size stand in for
them:

* each orbital is a sum of 6 Gaussians a*exp(-|r-c|^2/(2 s^2)), s ~ U(0.6, 1.5) bohr,
  a ~ N(0, 1), centres uniform in the inner 60% of the box along every axis
  (slab systems: centres along z restricted to the lower 70% of the box, the top 30%
  being vacuum);
* periodic axes use periodic images (-1, 0, +1) so every orbital is smooth across the
  cell boundary;
* systems with at least one periodic axis add a mix of 4 plane waves
  b*cos(2*pi*k.r/L + theta), k in {0..3} along periodic axes (0 along Dirichlet axes),
  b ~ N(0, 0.3^2); along Dirichlet axes the plane waves are multiplied by a Gaussian
  envelope (width 0.15 L) centred on the orbital region so they stay localized;
* orbitals are orthonormalised in FP64 with the grid metric: sum_r psi_m psi_n h^3 =
  delta_mn (Householder QR, then a second Gram-Schmidt pass for safety).

Grid index convention: r = ix + nx*(iy + ny*iz) (x fastest); point coordinates are
x_i = i*h, box length L = n*h.  Arrays are returned column-major as numpy arrays of
shape (n_orb, N) (row p is orbital p, contiguous), i.e. the N x n_orb column-major
matrix the C interface takes with leading dimension N.
"""
from __future__ import annotations

import dataclasses
import numpy as np

BC_DIRICHLET = 0
BC_PERIODIC = 1
KERNEL_COULOMB = 0
KERNEL_ERFC = 1
KERNEL_ERFC_PAPER16PI = 2

SEED_BASE = 2501_16572
HSE_OMEGA = 0.106


@dataclasses.dataclass
class System:
    """One exact-exchange problem: grid, boundary conditions, kernel and orbitals."""
    name: str
    n: tuple            # (nx, ny, nz)
    h: float
    bc: tuple           # per axis, BC_DIRICHLET / BC_PERIODIC
    fd_order: int
    kernel: int
    omega: float
    psi: np.ndarray     # (n_orb, N) float64, orthonormal with metric h^3
    f: np.ndarray       # (n_occ,) occupations of the leading n_occ orbitals (all > 0)
    n_occ: int

    @property
    def N(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def dV(self) -> float:
        return float(self.h ** 3)

    @property
    def n_orb(self) -> int:
        return int(self.psi.shape[0])

    def unique_pairs(self) -> int:
        """Poisson solves when V_mn = V_nm is used (outputs = all orbitals, occupied leading)."""
        no, ni = self.n_occ, self.n_orb
        return no * (no + 1) // 2 + no * (ni - no)

    def ordered_pairs(self) -> int:
        return self.n_occ * self.n_orb


def _axis_gauss(x, c, s, L, periodic):
    """1D Gaussian factor exp(-(x-c)^2/(2 s^2)), summed over images -1,0,1 if periodic."""
    if periodic:
        g = np.zeros_like(x)
        for img in (-1.0, 0.0, 1.0):
            d = x - c + img * L
            g += np.exp(-d * d / (2.0 * s * s))
        return g
    d = x - c
    return np.exp(-d * d / (2.0 * s * s))


def make_orbitals(rng, n, h, bc, n_orb, slab_axis=None, n_gauss=6, n_pw=4):
    """Draw n_orb raw orbitals (not orthonormal), shape (n_orb, N)."""
    nx, ny, nz = n
    L = [n[d] * h for d in range(3)]
    coords = [np.arange(n[d], dtype=np.float64) * h for d in range(3)]
    periodic = [bc[d] == BC_PERIODIC for d in range(3)]
    any_periodic = any(periodic)
    out = np.zeros((n_orb, nz, ny, nx), dtype=np.float64)
    for p in range(n_orb):
        acc = out[p]
        for _ in range(n_gauss):
            s = rng.uniform(0.6, 1.5)
            a = rng.normal(0.0, 1.0)
            c = []
            for d in range(3):
                lo, hi = 0.2 * L[d], 0.8 * L[d]
                if slab_axis is not None and d == slab_axis:
                    lo, hi = 0.2 * (0.7 * L[d]), 0.8 * (0.7 * L[d])
                c.append(rng.uniform(lo, hi))
            gx = _axis_gauss(coords[0], c[0], s, L[0], periodic[0])
            gy = _axis_gauss(coords[1], c[1], s, L[1], periodic[1])
            gz = _axis_gauss(coords[2], c[2], s, L[2], periodic[2])
            acc += a * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
        if any_periodic:
            for _ in range(n_pw):
                k = [int(rng.integers(0, 4)) if periodic[d] else 0 for d in range(3)]
                theta = rng.uniform(0.0, 2.0 * np.pi)
                b = rng.normal(0.0, 0.3)
                ph = (2 * np.pi * k[0] / L[0]) * coords[0][None, None, :] \
                    + (2 * np.pi * k[1] / L[1]) * coords[1][None, :, None] \
                    + (2 * np.pi * k[2] / L[2]) * coords[2][:, None, None]
                term = b * np.cos(ph + theta)
                for d in range(3):
                    if not periodic[d]:
                        cen = 0.5 * L[d] if (slab_axis is None or d != slab_axis) else 0.35 * L[d]
                        env = np.exp(-(coords[d] - cen) ** 2 / (2 * (0.15 * L[d]) ** 2))
                        shape = [1, 1, 1]
                        shape[2 - d] = n[d]
                        term = term * env.reshape(shape)
                acc += term
    return out.reshape(n_orb, -1)


def orthonormalize(raw, h):
    """Orthonormalise rows of raw (n_orb, N) with metric h^3 (FP64)."""
    dV = h ** 3
    q, r = np.linalg.qr(raw.T)                       # N x n_orb, orthonormal columns
    # fix the sign so the result does not depend on LAPACK's Householder sign choice
    sgn = np.sign(np.diag(r))
    sgn[sgn == 0] = 1.0
    q = q * sgn[None, :]
    # one more classical Gram-Schmidt pass (re-orthogonalisation)
    q = q - q @ (q.T @ q - np.eye(q.shape[1]))
    nrm = np.sqrt(np.sum(q * q, axis=0))
    q = q / nrm[None, :]
    return np.ascontiguousarray((q / np.sqrt(dV)).T)


def fermi_dirac(n_orb, fermi_index, kT=0.01, e0=-0.5, de=0.002, n_zero_from=None):
    """Occupations f_j = 2/(1+exp((eps_j - mu)/kT)), eps_j = e0 + de*j, mu = eps_{fermi_index}."""
    j = np.arange(n_orb, dtype=np.float64)
    eps = e0 + de * j
    mu = e0 + de * fermi_index
    f = 2.0 / (1.0 + np.exp((eps - mu) / kT))
    if n_zero_from is not None:
        f[n_zero_from:] = 0.0
    return f


def make_system(name, n, h, bc, n_orb, kernel, omega, occ, seed, fd_order=12,
                slab_axis=None, fermi_index=None, n_occ=None):
    rng = np.random.Generator(np.random.PCG64(seed))
    raw = make_orbitals(rng, n, h, bc, n_orb, slab_axis=slab_axis)
    psi = orthonormalize(raw, h)
    if occ == "const2":
        f = np.full(n_orb, 2.0)
    else:
        f = fermi_dirac(n_orb, fermi_index, n_zero_from=n_occ)
    if n_occ is None:
        n_occ = n_orb
    return System(name=name, n=tuple(int(v) for v in n), h=float(h), bc=tuple(int(b) for b in bc),
                  fd_order=fd_order, kernel=kernel, omega=float(omega), psi=psi,
                  f=np.ascontiguousarray(f[:n_occ]), n_occ=int(n_occ))


# ---- the five workloads ---------------------------------------------------------------

def config1():
    """Isolated (Dirichlet) 24^3, h=0.3, unscreened, 16 orbitals, f=2 (all 256 pairs)."""
    return make_system("dirichlet24_coulomb_16", (24, 24, 24), 0.3, (0, 0, 0), 16,
                       KERNEL_COULOMB, 0.0, "const2", SEED_BASE + 1)


def config2(n_orb=128):
    """Periodic 48^3, h=0.25, erfc-screened omega=0.106, 128 orbitals, Fermi level at orbital 100."""
    return make_system("periodic48_erfc_128", (48, 48, 48), 0.25, (1, 1, 1), n_orb,
                       KERNEL_ERFC, HSE_OMEGA, "fd", SEED_BASE + 2, fermi_index=99)


def config3():
    """Same periodic 48^3 screened system with 256 orbitals (precision study)."""
    s = make_system("periodic48_erfc_256", (48, 48, 48), 0.25, (1, 1, 1), 256,
                    KERNEL_ERFC, HSE_OMEGA, "fd", SEED_BASE + 3, fermi_index=99)
    return s


def config4_specs(n_systems=48):
    """Grid/bc/orbital-count draws of the 48-system batch (no orbitals yet)."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 4))
    specs = []
    for i in range(n_systems):
        n = tuple(int(rng.integers(20, 65)) for _ in range(3))
        bc = tuple(int(rng.integers(0, 2)) for _ in range(3))
        if i == 0:
            bc = (0, 0, 0)
        if i == 1:
            bc = (1, 1, 1)
        n_orb = int(rng.integers(8, 161))
        specs.append((n, bc, n_orb))
    return specs


def config4_system(i, specs=None, orb_scale=1.0):
    specs = specs or config4_specs()
    n, bc, n_orb = specs[i]
    n_orb = max(2, int(round(n_orb * orb_scale)))
    kernel = KERNEL_COULOMB if any(b == BC_DIRICHLET for b in bc) else KERNEL_ERFC
    omega = 0.0 if kernel == KERNEL_COULOMB else HSE_OMEGA
    return make_system(f"batch{i}_{n[0]}x{n[1]}x{n[2]}", n, 0.3, bc, n_orb, kernel, omega,
                       "fd", SEED_BASE + 4 + 1000 * (i + 1), fermi_index=int(0.78 * n_orb))


def config5(n_orb=1024, n_occ=800):
    """Slab 72x72x144, periodic x,y, Dirichlet z (top 30% vacuum), h=0.2, screened."""
    return make_system("slab72x72x144_erfc_1024", (72, 72, 144), 0.2, (1, 1, 0), n_orb,
                       KERNEL_ERFC, HSE_OMEGA, "fd", SEED_BASE + 5, slab_axis=2,
                       fermi_index=779, n_occ=n_occ)


def capacity_slab(n_orb=1848, n_occ=1440):
    """Paper-scale mixed-boundary slab 117x117x119 (periodic x,y, Dirichlet z, top 30% of z
    vacuum), h=0.2, screened, 1848 orbitals of which the first 1440 are occupied."""
    return make_system("slab117x117x119_erfc_1848", (117, 117, 119), 0.2, (1, 1, 0), n_orb,
                       KERNEL_ERFC, HSE_OMEGA, "fd", SEED_BASE + 6, slab_axis=2,
                       fermi_index=1400, n_occ=n_occ)


def small_system(n=(10, 9, 8), h=0.4, bc=(0, 1, 0), n_orb=6, kernel=KERNEL_COULOMB,
                 omega=0.0, seed=7, fd_order=12, occ="fd", n_occ=None):
    """Small seeded system for fast tests (ragged, non-cubic grids allowed)."""
    fi = max(0, int(0.7 * n_orb) - 1)
    return make_system(f"small_{n[0]}x{n[1]}x{n[2]}", n, h, bc, n_orb, kernel, omega, occ,
                       SEED_BASE + 100 + seed, fd_order=fd_order, fermi_index=fi, n_occ=n_occ)
