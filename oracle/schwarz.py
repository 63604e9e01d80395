"""Overlapping Schwarz decomposition of the duals, Section 6 (FP64).

Test infrastructure only (see the package header).

* ``Decomp`` -- M2 x M1 overlapping rectangles and the partition of unity
  theta_m (Section 6.1).  The paper fixes only the properties of theta
  (sums to one, non-negative, supported in the subdomain, gradient O(1/s)).
  Reading used: cores split each axis as evenly as integers allow (core m
  along an axis of N pixels is [floor(mN/M), floor((m+1)N/M))); two
  neighbouring subdomains share a strip of exactly s pixels around their
  core boundary b, namely [b - ceil(s/2), b + floor(s/2)); on that strip the
  lower subdomain's weight falls linearly, theta = (b - ceil(s/2) + s - x - 1/2)/s
  at pixel x, and the upper one's is 1 minus that; theta = 1 elsewhere in the
  subdomain.  The 2-D weight is the product of the two 1-D weights.  Steps 1
  and 2 share the cores (Omega_m = tilde Omega_m restricted to Omega); the
  extra last row/column of the extended grid belongs to the last subdomain.
* ``schwarz_irv1`` -- Algorithm 2 with Algorithm 3 for eq. ir1dualdis.
* ``schwarz_tfs`` -- Algorithm 2 with Algorithm 4 (global arrays) or with the
  fully localized Algorithm 5 (``localized=True``), whose local projection is
  evaluated with the block formula eq. invLaplLowCapLong inside eq.
  locglobprojpart1, and whose omega is assembled from the pieces
  R P_K E over all subdomains.

Readings: the inner stopping rule is not specified, so every inner solve runs
a fixed number of updates k and is warm-started from the previous outer
iterate's q_m (q_m = 0 initially).  Where theta_m = 0 and psi = 0 the update
0/0 is taken as 0 (the feasible set forces |v| <= theta_m = 0 there).  The
damping alpha_hat follows the colouring rule of Section 6.1: 1 for one
subdomain, 1/2 for strips, 1/4 for a 2-D grid.

Parity: pinned by the partition-of-unity properties, by the locality
identities resDiv/resGrad, by the localized projection equalling the global
projection restricted, by Algorithm 5 reproducing Algorithm 4, by the single
subdomain case reproducing k global iterations per outer iteration exactly,
and by the Schwarz iterates converging to the global minimiser
(tests/test_oracle_schwarz.py).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import ops
from .tvs import chambolle_update, tfs_problem, tfs_report, irv1_report


# --------------------------------------------------------------------------
# Decomposition and partition of unity (Section 6.1)
# --------------------------------------------------------------------------


def axis_cores(n: int, m: int) -> list[int]:
    return [(k * n) // m for k in range(m + 1)]


def axis_parts(n: int, m: int, s: int, extended: bool):
    """1-D subdomain extents [start, end) and weights theta (length n or n+1)."""
    if m < 1 or s < 0:
        raise ValueError("need m >= 1 and s >= 0")
    b = axis_cores(n, m)
    if any(b[k + 1] - b[k] < max(s, 1) for k in range(m)):
        raise ValueError("every core must be at least max(s, 1) pixels wide")
    length = n + 1 if extended else n
    lo, hi = (s + 1) // 2, s // 2
    extents, thetas = [], []
    x = np.arange(length, dtype=np.float64)
    for k in range(m):
        start = 0 if k == 0 else b[k] - lo
        end = length if k == m - 1 else b[k + 1] + hi
        th = np.zeros(length)
        th[start:end] = 1.0
        if k > 0 and s > 0:
            a = b[k] - lo
            sl = slice(a, a + s)
            th[sl] = 1.0 - (a + s - x[sl] - 0.5) / s
        if k < m - 1 and s > 0:
            a = b[k + 1] - lo
            sl = slice(a, a + s)
            th[sl] = (a + s - x[sl] - 0.5) / s
        extents.append((start, end))
        thetas.append(th)
    return extents, thetas


def colouring_alpha_hat(m2: int, m1: int) -> float:
    if m2 == 1 and m1 == 1:
        return 1.0
    if m2 == 1 or m1 == 1:
        return 0.5
    return 0.25


@dataclass
class Decomp:
    n2: int
    n1: int
    m2: int
    m1: int
    s: int
    extended: bool      # True: grid is the extended (N2+1) x (N1+1) grid

    def __post_init__(self):
        self.ext_y, self.th_y = axis_parts(self.n2, self.m2, self.s, self.extended)
        self.ext_x, self.th_x = axis_parts(self.n1, self.m1, self.s, self.extended)
        self.rows = self.n2 + 1 if self.extended else self.n2
        self.cols = self.n1 + 1 if self.extended else self.n1

    def subdomains(self):
        return [(a, b) for a in range(self.m2) for b in range(self.m1)]

    def theta(self, m) -> np.ndarray:
        return np.outer(self.th_y[m[0]], self.th_x[m[1]])

    def box(self, m):
        """(y0, y1, x0, x1) of Gamma_m, half-open."""
        (y0, y1), (x0, x1) = self.ext_y[m[0]], self.ext_x[m[1]]
        return y0, y1, x0, x1

    def box_plus(self, m):
        """Gamma_{m,+}: one more row below and column right, where possible."""
        y0, y1, x0, x1 = self.box(m)
        return y0, min(y1 + 1, self.rows), x0, min(x1 + 1, self.cols)

    def alpha_hat(self) -> float:
        return colouring_alpha_hat(self.m2, self.m1)


def theta_update(v: np.ndarray, psi: np.ndarray, th: np.ndarray, t: float) -> np.ndarray:
    """v <- (theta v + t theta psi) / (theta + t |psi|), per channel (Alg. 3).

    0/0 (theta = 0 and psi = 0) is taken as 0.
    """
    if v.ndim == 4:
        return np.stack([theta_update(v[k], psi[k], th, t) for k in range(v.shape[0])])
    nrm = np.sqrt(psi[0] ** 2 + psi[1] ** 2)
    den = th + t * nrm
    num = th * v + t * th * psi
    out = np.zeros_like(v)
    nz = den > 0
    out[:, nz] = num[:, nz] / den[nz]
    return out


# --------------------------------------------------------------------------
# Step 2: Algorithm 2 + Algorithm 3 with Lambda = div, f = f_2
# --------------------------------------------------------------------------


def schwarz_irv1(f2: np.ndarray, alpha: float, dd: Decomp, t: float = 0.125,
                 outer: int = 10, k_inner: int = 10, alpha_hat: float | None = None,
                 p0: np.ndarray | None = None, q0=None, return_state: bool = False):
    """Algorithm 2 with the inner Algorithm 3; returns (d, p, report)."""
    if dd.extended:
        raise ValueError("step 2 lives on the image grid")
    ah = dd.alpha_hat() if alpha_hat is None else alpha_hat
    subs = dd.subdomains()
    thetas = {m: dd.theta(m) for m in subs}
    others = {m: sum((thetas[l] for l in subs if l != m), np.zeros_like(f2)) for m in subs}
    p = np.zeros((2,) + f2.shape) if p0 is None else p0.copy()
    q = {m: np.zeros_like(p) for m in subs} if q0 is None else {m: q0[m].copy() for m in subs}
    for _ in range(outer):
        for m in subs:
            w = others[m] * p                       # sum_{l != m} theta_l p^n
            v = q[m]
            for _ in range(k_inner):
                psi = ops.grad(ops.div(v + w) - f2)  # Lambda^*(-Lambda(v + w) + f)
                v = theta_update(v, psi, thetas[m], t)
            q[m] = v
        p = (1.0 - ah) * p + ah * sum(q[m] for m in subs)
    d = (f2 - ops.div(p)) / alpha
    rep = irv1_report(f2, p, alpha, outer)
    if return_state:
        return d, p, rep, q
    return d, p, rep


# --------------------------------------------------------------------------
# Localized projection, eqs. locglobprojpart1, locglobprojpart3,
# invLaplLowCapLong (Section 6.2)
# --------------------------------------------------------------------------


def _plus(box, rows, cols):
    y0, y1, x0, x1 = box
    return y0, min(y1 + 1, rows), x0, min(x1 + 1, cols)


def _split(n: int, parts: int):
    b = axis_cores(n, parts)
    return [(b[k], b[k + 1]) for k in range(parts)]


def local_inv_lap_blocks(s_a: np.ndarray, a_box, b_box, rows: int, cols: int,
                         lam_parts=(2, 2)) -> np.ndarray:
    """R_B Delta^dagger E_A s by the block formula eq. invLaplLowCapLong.

    The frequency rectangles tilde A_lambda split the extended grid into
    lam_parts[0] x lam_parts[1] disjoint blocks; only the matrix blocks
    [C_{N2}]^{k2}_{lambda2} (rows lambda2, columns A_y) and their B-counterparts
    are formed, and the diagonal (tilde Delta)^dagger acts block by block.
    """
    c2, c1 = ops.dct_matrix(rows), ops.dct_matrix(cols)
    sym = ops.inv_lap_symbol(rows, cols)
    ay0, ay1, ax0, ax1 = a_box
    by0, by1, bx0, bx1 = b_box
    out = np.zeros((by1 - by0, bx1 - bx0))
    for l2a, l2b in _split(rows, min(lam_parts[0], rows)):
        for l1a, l1b in _split(cols, min(lam_parts[1], cols)):
            fwd = c2[l2a:l2b, ay0:ay1] @ s_a @ c1[l1a:l1b, ax0:ax1].T
            fwd = sym[l2a:l2b, l1a:l1b] * fwd
            out += c2[l2a:l2b, by0:by1].T @ fwd @ c1[l1a:l1b, bx0:bx1]
    return out


def local_projection(u: np.ndarray, k_plus, m_plus, rows: int, cols: int,
                     lam_parts=(2, 2)) -> np.ndarray:
    """R_{Omega_{m,+}} P_K E_{Omega_{k,+}} u for u on Omega_{k,+} (2-vector).

    Follows eq. locglobprojpart1: with A_k = (Omega_{k,+})_+ and
    B_m = (Omega_{m,+})_+, the local divergence on A_k of the zero-extended u,
    the block-formula inverse Laplacian from A_k to B_m, and the local gradient
    on B_m restricted to Omega_{m,+}.
    """
    a_box = _plus(k_plus, rows, cols)
    b_box = _plus(m_plus, rows, cols)
    ay0, ay1, ax0, ax1 = a_box
    ky0, ky1, kx0, kx1 = k_plus
    ua = np.zeros((2, ay1 - ay0, ax1 - ax0))
    ua[:, ky0 - ay0:ky1 - ay0, kx0 - ax0:kx1 - ax0] = u
    s_a = ops.div(ua)                                   # div_{A_k} on the subgrid
    phi_b = local_inv_lap_blocks(s_a, a_box, b_box, rows, cols, lam_parts)
    g_b = ops.grad(phi_b)                               # grad_{B_m} on the subgrid
    by0, by1, bx0, bx1 = b_box
    my0, my1, mx0, mx1 = m_plus
    grad_part = g_b[:, my0 - by0:my1 - by0, mx0 - bx0:mx1 - bx0]
    # R_{m,+} E_{k,+} u: the overlap of the two boxes
    direct = np.zeros((2, my1 - my0, mx1 - mx0))
    oy0, oy1 = max(my0, ky0), min(my1, ky1)
    ox0, ox1 = max(mx0, kx0), min(mx1, kx1)
    if oy0 < oy1 and ox0 < ox1:
        direct[:, oy0 - my0:oy1 - my0, ox0 - mx0:ox1 - mx0] = \
            u[:, oy0 - ky0:oy1 - ky0, ox0 - kx0:ox1 - kx0]
    return direct - grad_part


# --------------------------------------------------------------------------
# Step 1: Algorithm 2 + Algorithm 4 (global) or Algorithm 5 (localized)
# --------------------------------------------------------------------------


def _pk_vecdiv(p: np.ndarray) -> np.ndarray:
    return ops.proj_k(ops.vecdiv(p))


def _local_vecdiv(v_plus: np.ndarray) -> np.ndarray:
    """vecdiv on a subgrid for a (2, 2, r, c) field."""
    return np.stack([ops.div(v_plus[0]), ops.div(v_plus[1])])


def _local_vecgrad(z: np.ndarray) -> np.ndarray:
    return np.stack([ops.grad(z[0]), ops.grad(z[1])])


def omega_by_pieces(prob_f1: np.ndarray, p: np.ndarray, dd: Decomp, m, thetas,
                    lam_parts=(2, 2)) -> np.ndarray:
    """R_{m,+}(f - P_K vecdiv sum_{l != m} theta_l p) from local pieces.

    Each piece R_{m,+} P_K E_{l,+} vecdiv_{l,+}(R_{l,+} E_l R_l theta_l p) is a
    localized projection, so no global operator is applied (end of Sec. 6.2).
    """
    rows, cols = dd.rows, dd.cols
    mp = dd.box_plus(m)
    my0, my1, mx0, mx1 = mp
    acc = prob_f1[:, my0:my1, mx0:mx1].copy()
    for l in dd.subdomains():
        if l == m:
            continue
        y0, y1, x0, x1 = dd.box(l)
        lp = dd.box_plus(l)
        ly0, ly1, lx0, lx1 = lp
        piece = np.zeros((2, 2, ly1 - ly0, lx1 - lx0))
        piece[:, :, y0 - ly0:y1 - ly0, x0 - lx0:x1 - lx0] = \
            thetas[l][y0:y1, x0:x1] * p[:, :, y0:y1, x0:x1]
        acc -= local_projection(_local_vecdiv(piece), lp, mp, rows, cols, lam_parts)
    return acc


def schwarz_tfs(d0: np.ndarray, delta: float, dd: Decomp, t: float = 0.125,
                outer: int = 10, k_inner: int = 10, alpha_hat: float | None = None,
                localized: bool = False, omega_pieces: bool = True,
                lam_parts=(2, 2), p0: np.ndarray | None = None):
    """Algorithm 2 for eq. tfsdualdis; inner loop Algorithm 4 or Algorithm 5.

    Returns (tau, p, report).
    """
    if not dd.extended:
        raise ValueError("step 1 lives on the extended grid")
    prob = tfs_problem(d0, delta)
    ah = dd.alpha_hat() if alpha_hat is None else alpha_hat
    subs = dd.subdomains()
    thetas = {m: dd.theta(m) for m in subs}
    others = {m: sum((thetas[l] for l in subs if l != m), np.zeros((dd.rows, dd.cols)))
              for m in subs}
    p = np.zeros((2, 2, dd.rows, dd.cols)) if p0 is None else p0.copy()
    q = {m: np.zeros_like(p) for m in subs}
    rows, cols = dd.rows, dd.cols
    for _ in range(outer):
        for m in subs:
            if not localized:
                w = others[m] * p
                omega0 = prob.f1 - _pk_vecdiv(w)
                v = q[m]
                for _ in range(k_inner):
                    psi = ops.vecgrad(_pk_vecdiv(v) - omega0)
                    v = theta_update(v, psi, thetas[m], t)
                q[m] = v
            else:
                y0, y1, x0, x1 = dd.box(m)
                mp = dd.box_plus(m)
                py0, py1, px0, px1 = mp
                if omega_pieces:
                    om = omega_by_pieces(prob.f1, p, dd, m, thetas, lam_parts)
                else:
                    om = (prob.f1 - _pk_vecdiv(others[m] * p))[:, py0:py1, px0:px1]
                v_loc = q[m][:, :, y0:y1, x0:x1].copy()
                th_loc = thetas[m][y0:y1, x0:x1]
                for _ in range(k_inner):
                    v_plus = np.zeros((2, 2, py1 - py0, px1 - px0))
                    v_plus[:, :, y0 - py0:y1 - py0, x0 - px0:x1 - px0] = v_loc
                    pk = local_projection(_local_vecdiv(v_plus), mp, mp, rows, cols, lam_parts)
                    g = _local_vecgrad(pk - om)
                    psi = g[:, :, y0 - py0:y1 - py0, x0 - px0:x1 - px0]
                    v_loc = theta_update(v_loc, psi, th_loc, t)
                qm = np.zeros_like(p)
                qm[:, :, y0:y1, x0:x1] = v_loc
                q[m] = qm
        p = (1.0 - ah) * p + ah * sum(q[m] for m in subs)
    tau = prob.ptau0 - delta * _pk_vecdiv(p)
    return tau, p, tfs_report(prob, p, outer)


# re-exported for tests that compare against the global iteration
__all__ = ["Decomp", "axis_parts", "theta_update", "schwarz_irv1", "schwarz_tfs",
           "local_projection", "local_inv_lap_blocks", "omega_by_pieces",
           "colouring_alpha_hat", "chambolle_update"]
