"""Independent mathematics used to pin the oracle (tests only).

Nothing here is shared with ``oracle/`` or with the CUDA library: FD weights come from
an exact rational solve of the Taylor conditions (not the closed form the oracle uses),
operators are assembled as dense Kronecker sums, and the Laplacian is applied as a
direct stencil with shifted arrays.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def fd_weights_taylor(p: int):
    """Exact weights w_0..w_p of the (2p)-th order central second difference, from the
    moment conditions sum_{k=-p..p} w_|k| k^q = 2 delta_{q,2}, q = 0, 2, ..., 2p."""
    n = p + 1
    A = [[Fraction(0)] * n for _ in range(n)]
    b = [Fraction(0)] * n
    for row in range(n):
        q = 2 * row
        A[row][0] = Fraction(1 if q == 0 else 0)
        for k in range(1, p + 1):
            A[row][k] = Fraction(2 * k ** q)
        b[row] = Fraction(2 if q == 2 else 0)
    # Gauss-Jordan elimination in exact arithmetic
    for col in range(n):
        piv = next(r for r in range(col, n) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        b[col], b[piv] = b[piv], b[col]
        for r in range(n):
            if r != col and A[r][col] != 0:
                fac = A[r][col] / A[col][col]
                A[r] = [x - fac * y for x, y in zip(A[r], A[col])]
                b[r] -= fac * b[col]
    return [b[i] / A[i][i] for i in range(n)]


def op1d_dense(n, h, bc, p):
    """Dense 1D second-derivative operator from the Taylor weights."""
    w = [float(x) for x in fd_weights_taylor(p)]
    D = np.zeros((n, n))
    for i in range(n):
        for k in range(-p, p + 1):
            j = i + k
            if bc == 1:
                D[i, j % n] += w[abs(k)]
            elif 0 <= j < n:
                D[i, j] += w[abs(k)]
    return D / (h * h)


def laplacian_dense(n, h, bc, p):
    """Dense 3D Laplacian (N x N) for x-fastest indexing r = ix + nx*(iy + ny*iz)."""
    nx, ny, nz = n
    D1, D2, D3 = (op1d_dense(n[d], h, bc[d], p) for d in range(3))
    I1, I2, I3 = np.eye(nx), np.eye(ny), np.eye(nz)
    return (np.kron(I3, np.kron(I2, D1)) + np.kron(I3, np.kron(D2, I1))
            + np.kron(D3, np.kron(I2, I1)))


def apply_stencil(X, n, h, bc, p):
    """Direct 3D stencil Laplacian of the grid function X (length N, x fastest)."""
    w = [float(x) for x in fd_weights_taylor(p)]
    nx, ny, nz = n
    G = np.asarray(X, dtype=np.float64).reshape(nz, ny, nx)
    out = 3.0 * w[0] * G
    for d, ax in ((0, 2), (1, 1), (2, 0)):
        for k in range(1, p + 1):
            for s in (k, -k):
                if bc[d] == 1:
                    out = out + w[k] * np.roll(G, -s, axis=ax)
                else:
                    sh = np.zeros_like(G)
                    L = G.shape[ax]
                    src = [slice(None)] * 3
                    dst = [slice(None)] * 3
                    if s > 0 and s < L:
                        src[ax] = slice(s, L)
                        dst[ax] = slice(0, L - s)
                        sh[tuple(dst)] = G[tuple(src)]
                    elif s < 0 and -s < L:
                        src[ax] = slice(0, L + s)
                        dst[ax] = slice(-s, L)
                        sh[tuple(dst)] = G[tuple(src)]
                    out = out + w[k] * sh
    return (out / (h * h)).reshape(-1)


def erfc_kernel(x, omega, a_is_16pi=False):
    """Screened kernel on -eigenvalues x >= 0 (reading R1), numpy, for dense checks."""
    a = 16.0 * np.pi * omega ** 2 if a_is_16pi else 4.0 * omega ** 2
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    small = np.abs(x) < 1e-300
    out[small] = 4.0 * np.pi / a
    xs = x[~small]
    out[~small] = (4.0 * np.pi / xs) * (-np.expm1(-xs / a))
    return out


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
