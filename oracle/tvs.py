"""Global (non-decomposed) TV-Stokes iterations in FP64.

Test infrastructure only (see the package header).

Step 1, tangent field smoothing (TFS), solves the discrete dual eq.
tfsdualdis on the extended grid with Chambolle's semi-implicit iteration,
Algorithm 1.  Step 2, image reconstruction variant 1 (IRV1), solves eq.
ir1dualdis on the image grid with the same iteration (Section 4.2).

Readings of the paper taken here (each stated where it is used):

* Algorithm 1 prints ``vecgrad(P_K vecdiv p - tau_0/delta)`` while the dual
  eq. tfsdualdis and the recovery of tau use ``P_K tau_0 / delta``.  The
  gradient of the dual objective is the same for either data term, namely
  ``-vecgrad(P_K vecdiv p - P_K tau_0/delta)``, so the projected data
  ``f_1 = P_K tau_0 / delta`` is used (``literal_alg1=True`` gives the printed
  form for comparison).
* The primal energies and duality gaps follow Appendix A: every problem is
  ``min_u TV(u) + (beta/2)||u - g||^2`` whose dual value for p is
  ``(beta/2)||g||^2 - D(p)/(2 beta)``; with ``u = g - Lambda p / beta`` the gap
  equals ``sum_k sum_ij (|grad u_k| + grad u_k . p_k)`` (non-negative on the
  feasible set).  TFS: beta = 1/delta, g = P_K tau_0.  IRV1: beta = alpha,
  g = d_0 - div(xi)/alpha.

Parity: pinned by invariants (adjointness, projection, feasibility,
monotone dual energy, gap identity, gap -> 0), by special cases (constant
image is a fixed point; xi = 0 reduces IRV1 to Chambolle's ROF iteration;
IRV2 with the noisy image's own tangent field returns the image), by
hand-derived values of xi, div xi and f_2 on a 2x3 image, by the identity
that the normal field of tau_0 is the eps-normalised backward gradient of
d_0, by brute-force dense solves on 8x8 images (FISTA, a different
algorithm, on the explicit matrices; for W^{1,1} on the shifted ball
|p - xi| <= 1 straight from eq. IRW11:dual) and, for the IRV2 potential, by
exact recovery of a known potential and numpy's least-squares solve
(tests/test_oracle_tvs.py, tests/test_oracle_irv2.py).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import ops


@dataclass
class Report:
    iters: int
    dual_D: float        # D(p) = ||Lambda p - f||^2
    primal_E: float      # E(u)
    gap: float           # pointwise duality gap
    rel_gap: float       # gap / E
    div_res_max: float   # max |div u| (TFS only, else 0)
    max_p: float         # max over channels and pixels of |p_k|
    history: list = field(default_factory=list)


# --------------------------------------------------------------------------
# Chambolle's semi-implicit update (Algorithm 1 line for p; Section 4.2)
# --------------------------------------------------------------------------


def chambolle_update(p: np.ndarray, psi: np.ndarray, t: float) -> np.ndarray:
    """p_k <- (p_k + t psi_k) / (1 + t |psi_k|), channel by channel.

    ``p`` and ``psi`` have shape (2, R, C) (one channel) or (c, 2, R, C).
    """
    if p.ndim == 3:
        nrm = np.sqrt(psi[0] ** 2 + psi[1] ** 2)
        return (p + t * psi) / (1.0 + t * nrm)
    out = np.empty_like(p)
    for k in range(p.shape[0]):
        out[k] = chambolle_update(p[k], psi[k], t)
    return out


def tv(u: np.ndarray) -> float:
    """Isotropic discrete TV: sum_ij |grad u|_ij (scalar field)."""
    g = ops.grad(u)
    return float(np.sum(np.sqrt(g[0] ** 2 + g[1] ** 2)))


def pointwise_gap(u: np.ndarray, p: np.ndarray) -> float:
    """sum_ij (|grad u| + grad u . p) for a scalar u and a 2-vector p."""
    g = ops.grad(u)
    return float(np.sum(np.sqrt(g[0] ** 2 + g[1] ** 2) + g[0] * p[0] + g[1] * p[1]))


# --------------------------------------------------------------------------
# Step 1: tangent field smoothing
# --------------------------------------------------------------------------


@dataclass
class TFSProblem:
    d0: np.ndarray
    delta: float
    tau0: np.ndarray      # (2, N2+1, N1+1)
    ptau0: np.ndarray     # P_K tau0
    f1: np.ndarray        # P_K tau0 / delta


def tfs_problem(d0: np.ndarray, delta: float) -> TFSProblem:
    tau0 = ops.tangent(d0)
    ptau0 = ops.proj_k(tau0)
    return TFSProblem(d0=d0, delta=delta, tau0=tau0, ptau0=ptau0, f1=ptau0 / delta)


def _pk2(w: np.ndarray) -> np.ndarray:
    """P_K applied to vecdiv p.

    vecdiv p = (div p_1, div p_2) is one 2-vector field on the extended grid
    whose components play the roles of (tau_1, tau_2); P_K projects it onto
    the divergence-free fields (eq. tfsdualdis).
    """
    return ops.proj_k(w)


def tfs_residual(prob: TFSProblem, p: np.ndarray) -> np.ndarray:
    """z = P_K vecdiv p - f_1 (the argument of the gradient in Algorithm 1)."""
    return _pk2(ops.vecdiv(p)) - prob.f1


def tfs_tau(prob: TFSProblem, p: np.ndarray) -> np.ndarray:
    """tau = P_K tau_0 - delta P_K vecdiv p (Section 4.2, after eq. ir2dualdis)."""
    return prob.ptau0 - prob.delta * _pk2(ops.vecdiv(p))


def tfs_report(prob: TFSProblem, p: np.ndarray, iters: int) -> Report:
    z = _pk2(ops.vecdiv(p)) - prob.f1
    tau = -prob.delta * z
    dual_D = ops.sqnorm(z)
    tvs = tv(tau[0]) + tv(tau[1])
    energy = tvs + ops.sqnorm(tau - prob.ptau0) / (2.0 * prob.delta)
    gap = pointwise_gap(tau[0], p[0]) + pointwise_gap(tau[1], p[1])
    maxp = float(np.max(np.sqrt(p[:, 0] ** 2 + p[:, 1] ** 2)))
    return Report(iters=iters, dual_D=dual_D, primal_E=energy, gap=gap,
                  rel_gap=gap / energy if energy > 0 else 0.0,
                  div_res_max=float(np.max(np.abs(ops.div(tau)))), max_p=maxp)


def tfs_step(prob: TFSProblem, p: np.ndarray, t: float, literal_alg1: bool = False) -> np.ndarray:
    """One iteration of Algorithm 1 (projected data term, see module header)."""
    data = prob.tau0 / prob.delta if literal_alg1 else prob.f1
    z = _pk2(ops.vecdiv(p)) - data
    psi = ops.vecgrad(z)
    return chambolle_update(p, psi, t)


def tfs(d0: np.ndarray, delta: float, t: float = 0.125, iters: int = 300,
        p0: np.ndarray | None = None, rel_gap_tol: float = 0.0,
        check_every: int = 0, literal_alg1: bool = False):
    """Run Algorithm 1 from p = p0 (zero by default) for ``iters`` updates.

    Stops early when ``rel_gap_tol > 0`` and the relative gap, checked every
    ``check_every`` updates, falls below it.  Returns (tau, p, report).
    """
    prob = tfs_problem(d0, delta)
    n2, n1 = d0.shape
    p = np.zeros((2, 2, n2 + 1, n1 + 1)) if p0 is None else p0.copy()
    hist = []
    n = 0
    while n < iters:
        p = tfs_step(prob, p, t, literal_alg1)
        n += 1
        if check_every and n % check_every == 0:
            rep = tfs_report(prob, p, n)
            hist.append((n, rep.rel_gap, rep.dual_D))
            if rel_gap_tol > 0 and rep.rel_gap <= rel_gap_tol:
                break
    rep = tfs_report(prob, p, n)
    rep.history = hist
    return tfs_tau(prob, p), p, rep


# --------------------------------------------------------------------------
# Normal field and IRV1 data, eq. defXi2:discrete and eq. ir1dualdis
# --------------------------------------------------------------------------


def normal_field(tau: np.ndarray, n2: int, n1: int, eps: float) -> np.ndarray:
    """xi = tau_perp / sqrt(|tau_perp|^2 + eps), tau_perp = R_Omega(tau_2, -tau_1)."""
    tp1 = tau[1][:n2, :n1]
    tp2 = -tau[0][:n2, :n1]
    den = np.sqrt(tp1 ** 2 + tp2 ** 2 + eps)
    return np.stack([tp1 / den, tp2 / den])


def irv1_data(d0: np.ndarray, xi: np.ndarray, alpha: float) -> np.ndarray:
    """f_2 = alpha d_0 - div xi (eq. ir1dualdis)."""
    return alpha * d0 - ops.div(xi)


# --------------------------------------------------------------------------
# Step 2: IRV1 Chambolle iteration (Section 4.2, eq. ir1dualdis)
# --------------------------------------------------------------------------


def irv1_image(f2: np.ndarray, p: np.ndarray, alpha: float) -> np.ndarray:
    """d = d_0 - (div p + div xi)/alpha = (f_2 - div p)/alpha (eq. tau_hat)."""
    return (f2 - ops.div(p)) / alpha


def irv1_report(f2: np.ndarray, p: np.ndarray, alpha: float, iters: int) -> Report:
    z = ops.div(p) - f2
    d = -z / alpha
    g = f2 / alpha
    energy = tv(d) + 0.5 * alpha * ops.sqnorm(d - g)
    gap = pointwise_gap(d, p)
    maxp = float(np.max(np.sqrt(p[0] ** 2 + p[1] ** 2)))
    return Report(iters=iters, dual_D=ops.sqnorm(z), primal_E=energy, gap=gap,
                  rel_gap=gap / energy if energy > 0 else 0.0, div_res_max=0.0, max_p=maxp)


def irv1_step(f2: np.ndarray, p: np.ndarray, t: float) -> np.ndarray:
    psi = ops.grad(ops.div(p) - f2)
    return chambolle_update(p, psi, t)


def irv1(f2: np.ndarray, alpha: float, t: float = 0.125, iters: int = 300,
         p0: np.ndarray | None = None, rel_gap_tol: float = 0.0, check_every: int = 0):
    """Chambolle's iteration for eq. ir1dualdis.  Returns (d, p, report)."""
    p = np.zeros((2,) + f2.shape) if p0 is None else p0.copy()
    hist = []
    n = 0
    while n < iters:
        p = irv1_step(f2, p, t)
        n += 1
        if check_every and n % check_every == 0:
            rep = irv1_report(f2, p, alpha, n)
            hist.append((n, rep.rel_gap, rep.dual_D))
            if rel_gap_tol > 0 and rep.rel_gap <= rel_gap_tol:
                break
    rep = irv1_report(f2, p, alpha, n)
    rep.history = hist
    return irv1_image(f2, p, alpha), p, rep


# --------------------------------------------------------------------------
# W^{1,1} variant of step 2 (Remark IRPW11, eq. IRW11:dual)
# --------------------------------------------------------------------------


def w11(d0: np.ndarray, xi: np.ndarray, alpha: float, t: float = 0.125, iters: int = 300,
        p0: np.ndarray | None = None, rel_gap_tol: float = 0.0, check_every: int = 0):
    """Dual eq. IRW11:dual, min ||div p - alpha d0||^2 over |p - xi| <= 1.

    Reading: with q = p - xi the problem is eq. IRPXi_dual / ir1dualdis
    (``||div q - (alpha d0 - div xi)||^2`` over |q| <= 1), so Chambolle's
    iteration runs on q exactly as for IRV1 and p = q + xi.  Both give
    ``d = d0 - div p / alpha`` (the first optimality condition of the
    proposition after eq. IRW11:dual).  ``p0`` is a warm start of p.
    Returns (d, p, report); the report is the IRV1 report of q.
    """
    f2 = irv1_data(d0, xi, alpha)
    q0 = None if p0 is None else p0 - xi
    d, q, rep = irv1(f2, alpha, t, iters, q0, rel_gap_tol, check_every)
    return d, q + xi, rep


# --------------------------------------------------------------------------
# IRV2, the alternative step 2 (Section 3.3: eqs. modifiedStep2,
# modifiedStep2_2, modifiedStep2_2_dual; discrete eq. ir2dualdis)
# --------------------------------------------------------------------------


def potential(tau: np.ndarray, n2: int, n1: int) -> np.ndarray:
    """Image g with grad g = tau_perp, tau_perp = R_Omega(tau_2, -tau_1).

    The paper asks for (D^-_x g, D^-_y g) = tau_perp on the image grid.  The
    backward differences between neighbouring image pixels are the equations
        g[i, j] - g[i, j-1] = tau_2[i, j]     (1 <= j <= N1-1),
        g[i, j] - g[i-1, j] = -tau_1[i, j]    (1 <= i <= N2-1),
    which are consistent exactly when div tau = D^-_x tau_1 + D^-_y tau_2
    vanishes at the extended-grid points 1 <= i <= N2-1, 1 <= j <= N1-1
    (the paper's condition div tau = 0).  The rows of D^- at
    the first and last index (zero extension) are not consistent in general,
    so, reading: g is the least-squares solution of the pixel-difference
    equations above, fixed to mean zero.  These equations are
    grad g = v with the forward-edge field v_x[i, j] = tau_2[i, j+1],
    v_y[i, j] = -tau_1[i+1, j] (zero in the last column / row, where grad has
    no equation), so the least-squares g solves the normal equations
    div grad g = div v, i.e. g = Delta^dagger div v on the N2 x N1 grid
    (eq. form:DiscInvLapl on that grid; the paper constructs g "with the help
    of the Fourier transform").  Where an exact potential exists this is it,
    up to the constant, which cancels in d (see ``irv2``).
    """
    a = tau[1][:n2, :n1]
    b = -tau[0][:n2, :n1]
    v = np.zeros((2, n2, n1))
    v[0][:, :-1] = a[:, 1:]
    v[1][:-1, :] = b[1:, :]
    return ops.inv_lap(ops.div(v))


def irv2_data(d0: np.ndarray, g: np.ndarray, alpha: float) -> np.ndarray:
    """f = alpha (d_0 - g), the data of eq. ir2dualdis."""
    return alpha * (d0 - g)


def irv2(d0: np.ndarray, tau: np.ndarray, alpha: float, t: float = 0.125, iters: int = 300,
         p0: np.ndarray | None = None, rel_gap_tol: float = 0.0, check_every: int = 0):
    """IRV2: g from tau, the ROF problem eq. modifiedStep2_2 in u = d - g by
    Chambolle's iteration on its dual eq. ir2dualdis, then d = u + g.

    A constant added to g shifts d_0 - g and u by opposite amounts and leaves
    d (and p) unchanged.  Returns (d, p, report, g); the report is that of
    the ROF problem in u (beta = alpha, data d_0 - g).
    """
    n2, n1 = d0.shape
    g = potential(tau, n2, n1)
    f = irv2_data(d0, g, alpha)
    u, p, rep = irv1(f, alpha, t, iters, p0, rel_gap_tol, check_every)
    return u + g, p, rep, g


# --------------------------------------------------------------------------
# Whole two-step pipeline (Section 4.2)
# --------------------------------------------------------------------------


def denoise(d0: np.ndarray, delta: float = 0.05, alpha: float = 10.0, eps: float = 1e-3,
            t: float = 0.125, iters1: int = 300, iters2: int = 300):
    """d0 -> tau (TFS) -> xi, f_2 -> d (IRV1).  Returns (d, tau, rep1, rep2)."""
    n2, n1 = d0.shape
    tau, _, rep1 = tfs(d0, delta, t, iters1)
    xi = normal_field(tau, n2, n1, eps)
    f2 = irv1_data(d0, xi, alpha)
    d, _, rep2 = irv1(f2, alpha, t, iters2)
    return d, tau, rep1, rep2
