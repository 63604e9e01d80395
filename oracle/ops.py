"""Discrete operators of Section 4.1 and the projection of Appendix B (FP64).

Test infrastructure only (see the package header).

Layout: a scalar field on a grid with R rows (y, index i) and C columns
(x, index j) is a float64 array of shape (R, C).  A 2-vector field is shape
(2, R, C) with component 0 the x-part and component 1 the y-part, so that
``div(u) = D-_x u[0] + D-_y u[1]``.  A 2x2 field p = (p_1, p_2) (one 2-vector
per channel k) is shape (2, 2, R, C), ``p[k]`` being the 2-vector of channel k.

The mesh size is h = 1 as in all of the paper's experiments (Section 5.2).

Pins (tests/test_oracle_ops.py): hand-computed 3x3/3x4 stencils from the
definitions, adjointness div = -grad^*, DCT matrix orthogonality and equality
with the textbook DCT-II, the Laplacian pseudo-inverse against numpy's pinv of
the assembled matrix, and the projection's idempotence, self-adjointness,
zero divergence, annihilation of gradients and identity on K.
"""
from __future__ import annotations

import numpy as np
import scipy.fft

# --------------------------------------------------------------------------
# Forward / backward differences, Section 4.1 (definitions of D^+_x, D^+_y,
# D^-_x, D^-_y on a rectangular grid).
# --------------------------------------------------------------------------


def dxp(u: np.ndarray) -> np.ndarray:
    """D^+_x: u[i, j+1] - u[i, j] for j < C-1, zero in the last column."""
    out = np.zeros_like(u)
    out[..., :, :-1] = u[..., :, 1:] - u[..., :, :-1]
    return out


def dyp(u: np.ndarray) -> np.ndarray:
    """D^+_y: u[i+1, j] - u[i, j] for i < R-1, zero in the last row."""
    out = np.zeros_like(u)
    out[..., :-1, :] = u[..., 1:, :] - u[..., :-1, :]
    return out


def dxm(u: np.ndarray) -> np.ndarray:
    """D^-_x: u[i,0] at j=0; u[i,j]-u[i,j-1] inside; -u[i,C-2] at j=C-1."""
    c = u.shape[-1]
    if c < 2:
        raise ValueError("D^-_x needs at least two columns")
    out = np.empty_like(u)
    out[..., :, 0] = u[..., :, 0]
    out[..., :, 1:c - 1] = u[..., :, 1:c - 1] - u[..., :, 0:c - 2]
    out[..., :, c - 1] = -u[..., :, c - 2]
    return out


def dym(u: np.ndarray) -> np.ndarray:
    """D^-_y: u[0,j] at i=0; u[i,j]-u[i-1,j] inside; -u[R-2,j] at i=R-1."""
    r = u.shape[-2]
    if r < 2:
        raise ValueError("D^-_y needs at least two rows")
    out = np.empty_like(u)
    out[..., 0, :] = u[..., 0, :]
    out[..., 1:r - 1, :] = u[..., 1:r - 1, :] - u[..., 0:r - 2, :]
    out[..., r - 1, :] = -u[..., r - 2, :]
    return out


def grad(u: np.ndarray) -> np.ndarray:
    """Discrete gradient (D^+_x u, D^+_y u), eq. defGradDis; shape (2, R, C)."""
    return np.stack([dxp(u), dyp(u)])


def div(v: np.ndarray) -> np.ndarray:
    """Discrete divergence D^-_x v_1 + D^-_y v_2, eq. defDivDis."""
    return dxm(v[0]) + dym(v[1])


def vecgrad(u: np.ndarray) -> np.ndarray:
    """Multi-gradient (grad u_1, grad u_2) of a 2-channel field; (2, 2, R, C)."""
    return np.stack([grad(u[0]), grad(u[1])])


def vecdiv(p: np.ndarray) -> np.ndarray:
    """Multi-divergence (div p_1, div p_2) of a 2x2 field; shape (2, R, C)."""
    return np.stack([div(p[0]), div(p[1])])


def laplacian(u: np.ndarray) -> np.ndarray:
    """Delta = div grad (homogeneous Neumann), Section 4.1."""
    return div(grad(u))


# --------------------------------------------------------------------------
# Neumann backward differences Omega -> extended grid, eq.
# def:backdiffNeumann, and the tangent field tau_0 of Section 4.2.
# --------------------------------------------------------------------------


def dx_neum(d: np.ndarray) -> np.ndarray:
    """D^{neum-}_x d on the extended grid (N2+1) x (N1+1).

    Zero in the first and last column; d[i,j]-d[i,j-1] inside for the N2 image
    rows; the extra last row repeats the differences of the last image row.
    """
    n2, n1 = d.shape
    out = np.zeros((n2 + 1, n1 + 1))
    out[:n2, 1:n1] = d[:, 1:] - d[:, :-1]
    out[n2, 1:n1] = d[n2 - 1, 1:] - d[n2 - 1, :-1]
    return out


def dy_neum(d: np.ndarray) -> np.ndarray:
    """D^{neum-}_y d on the extended grid (N2+1) x (N1+1).

    Zero in the first and last row; d[i,j]-d[i-1,j] inside for the N1 image
    columns; the extra last column repeats the differences of the last image
    column.
    """
    n2, n1 = d.shape
    out = np.zeros((n2 + 1, n1 + 1))
    out[1:n2, :n1] = d[1:, :] - d[:-1, :]
    out[1:n2, n1] = d[1:, n1 - 1] - d[:-1, n1 - 1]
    return out


def tangent(d0: np.ndarray) -> np.ndarray:
    """tau_0 = (-D^{neum-}_y d0, D^{neum-}_x d0) on the extended grid (Sec. 4.2)."""
    return np.stack([-dy_neum(d0), dx_neum(d0)])


# --------------------------------------------------------------------------
# DCT and the Laplacian pseudo-inverse, eqs. form:DiscInvLapl,
# form:DiscInvLaplTild, eq:DCT2D, form:DCTmat, eq:DCT2Dinv.
# --------------------------------------------------------------------------


def dct_matrix(n: int) -> np.ndarray:
    """Orthonormal DCT matrix C_N of eq. form:DCTmat.

    Row k, column m: sqrt(2/N) * cos(k*pi*(2m+1)/(2N)), with the first row
    sqrt(2/N)/sqrt(2).
    """
    k = np.arange(n)[:, None].astype(np.float64)
    m = np.arange(n)[None, :].astype(np.float64)
    c = np.sqrt(2.0 / n) * np.cos(k * np.pi * (2.0 * m + 1.0) / (2.0 * n))
    c[0, :] = np.sqrt(2.0 / n) / np.sqrt(2.0)
    return c


def sigma(n: int) -> np.ndarray:
    """sigma_{N,j} = (2/h) sin((j-1) pi / (2N)), j = 1..N (0-based here)."""
    return 2.0 * np.sin(np.arange(n, dtype=np.float64) * np.pi / (2.0 * n))


def inv_lap_symbol(rows: int, cols: int) -> np.ndarray:
    """Diagonal of the spectral pseudo-inverse (tilde Delta)^dagger.

    Entry (i, j) is -1/(sigma_{R,i}^2 + sigma_{C,j}^2) with the zero frequency
    mapped to 0.  The row frequency pairs with the row count R (= N2+1) and the
    column frequency with the column count C (= N1+1); on a square grid this
    is the printed formula, on a non-square grid it is the only pairing under
    which the result is the pseudo-inverse (the printed indices would pair the
    row index with N1).
    """
    s2 = sigma(rows) ** 2
    s1 = sigma(cols) ** 2
    den = s2[:, None] + s1[None, :]
    out = np.zeros_like(den)
    nz = den > 0
    out[nz] = -1.0 / den[nz]
    return out


def dct2(u: np.ndarray) -> np.ndarray:
    """2-D DCT C_R u C_C^T (eq:DCT2D) through SciPy's orthonormal DCT-II."""
    return scipy.fft.dctn(u, type=2, norm="ortho", axes=(-2, -1))


def idct2(u: np.ndarray) -> np.ndarray:
    """Inverse 2-D DCT C_R^T u C_C (eq:DCT2Dinv)."""
    return scipy.fft.idctn(u, type=2, norm="ortho", axes=(-2, -1))


def inv_lap(s: np.ndarray) -> np.ndarray:
    """Moore-Penrose inverse of the Neumann Laplacian, eq. form:DiscInvLapl."""
    r, c = s.shape[-2:]
    return idct2(inv_lap_symbol(r, c) * dct2(s))


def inv_lap_dense(s: np.ndarray) -> np.ndarray:
    """Same operator with the explicit matrices C_N (small grids)."""
    r, c = s.shape
    cr, cc = dct_matrix(r), dct_matrix(c)
    return cr.T @ (inv_lap_symbol(r, c) * (cr @ s @ cc.T)) @ cc


def proj_k(tau: np.ndarray) -> np.ndarray:
    """P_K = I - grad Delta^dagger div, eq. formula:PKh (2-vector field)."""
    phi = inv_lap(div(tau))
    return tau - grad(phi)


# --------------------------------------------------------------------------
# Scalar products and norms with h = 1 (Section 4.1).
# --------------------------------------------------------------------------


def dot(a: np.ndarray, b: np.ndarray) -> float:
    return float(np.sum(a * b))


def sqnorm(a: np.ndarray) -> float:
    return float(np.sum(a * a))
