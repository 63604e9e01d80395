"""Pins for oracle.tvs: Algorithm 1 (TFS), the normal field and IRV1 (Section 4.2),
and the energies and gaps of Appendix A.

Independent references used here: dense operator matrices assembled entry by
entry (tests/test_oracle_ops.py), the projector onto Null(div) from SciPy's
null_space, and a FISTA projected-gradient solve of the same duals on those
matrices -- a different algorithm from Chambolle's, run to a certified gap.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import ops, tvs
from synth import SceneSpec, noisy_scene
from test_oracle_ops import dense_ops

RNG = np.random.default_rng(99)


def image(rows=16, cols=20, seed=0, sigma=0.1):
    return noisy_scene(SceneSpec(rows, cols, seed, sigma))[1]


# ---- special cases -------------------------------------------------------

def test_constant_image_is_a_fixed_point():
    d0 = np.full((9, 13), 0.37)
    tau, p, rep = tvs.tfs(d0, 0.05, iters=20)
    assert np.all(tau == 0.0) and np.all(p == 0.0)
    xi = tvs.normal_field(tau, 9, 13, 1e-3)
    assert np.all(xi == 0.0)
    f2 = tvs.irv1_data(d0, xi, 10.0)
    d, p2, _ = tvs.irv1(f2, 10.0, iters=20)
    assert np.all(p2 == 0.0)
    np.testing.assert_array_equal(d, d0)


def test_irv1_with_zero_normal_field_is_chambolle_rof():
    # xi = 0 reduces eq. ir1dualdis to the ROF dual ||div p - alpha d0||^2, whose
    # textbook Chambolle iteration (u = d0 - div p / alpha) is written out here.
    d0 = image(10, 12, 4)
    alpha, t = 10.0, 0.125
    f2 = tvs.irv1_data(d0, np.zeros((2,) + d0.shape), alpha)
    np.testing.assert_array_equal(f2, alpha * d0)
    d, _, _ = tvs.irv1(f2, alpha, t, iters=50)
    grad_m, div_m = dense_ops(*d0.shape)
    p = np.zeros(2 * d0.size)
    g = d0.reshape(-1)
    for _ in range(50):
        psi = grad_m @ (div_m @ p - alpha * g)
        nrm = np.sqrt(psi[: d0.size] ** 2 + psi[d0.size:] ** 2)
        p = (p + t * psi) / (1.0 + t * np.concatenate([nrm, nrm]))
    np.testing.assert_allclose(d.reshape(-1), g - div_m @ p / alpha, atol=1e-12)


# ---- invariants of the iterations ---------------------------------------

def test_tfs_feasible_monotone_and_gap_identity():
    d0 = image(14, 17, 1)
    prob = tvs.tfs_problem(d0, 0.05)
    p = np.zeros((2, 2, 15, 18))
    last = np.inf
    for n in range(60):
        p = tvs.tfs_step(prob, p, 0.125)
        rep = tvs.tfs_report(prob, p, n + 1)
        assert rep.max_p <= 1.0 + 1e-12
        assert rep.dual_D <= last + 1e-10
        last = rep.dual_D
        assert rep.gap >= -1e-10
        assert rep.div_res_max < 1e-11
    # gap identity: E(u) - dual(p) = pointwise gap, dual = (beta/2)||g||^2 - D/(2 beta)
    beta = 1.0 / prob.delta
    dual = 0.5 * beta * ops.sqnorm(prob.ptau0) - rep.dual_D / (2 * beta)
    assert abs((rep.primal_E - dual) - rep.gap) < 1e-9 * rep.primal_E


def test_irv1_feasible_monotone_and_gap_identity():
    d0 = image(14, 17, 2)
    tau, _, _ = tvs.tfs(d0, 0.05, iters=30)
    xi = tvs.normal_field(tau, 14, 17, 1e-3)
    assert np.max(np.sqrt(xi[0] ** 2 + xi[1] ** 2)) < 1.0
    alpha = 10.0
    f2 = tvs.irv1_data(d0, xi, alpha)
    p = np.zeros((2, 14, 17))
    last = np.inf
    for n in range(60):
        p = tvs.irv1_step(f2, p, 0.125)
        rep = tvs.irv1_report(f2, p, alpha, n + 1)
        assert rep.max_p <= 1.0 + 1e-12
        assert rep.dual_D <= last + 1e-10
        last = rep.dual_D
        assert rep.gap >= -1e-10
    g = f2 / alpha
    dual = 0.5 * alpha * ops.sqnorm(g) - rep.dual_D / (2 * alpha)
    assert abs((rep.primal_E - dual) - rep.gap) < 1e-9 * rep.primal_E


def test_gaps_go_to_zero():
    d0 = image(12, 12, 5)
    _, _, r1 = tvs.tfs(d0, 0.05, iters=4000)
    assert r1.rel_gap < 1e-6
    tau, _, _ = tvs.tfs(d0, 0.05, iters=300)
    f2 = tvs.irv1_data(d0, tvs.normal_field(tau, 12, 12, 1e-3), 10.0)
    _, _, r2a = tvs.irv1(f2, 10.0, iters=1000)
    _, _, r2 = tvs.irv1(f2, 10.0, iters=4000)
    assert r2.rel_gap < 1e-5 and r2.rel_gap < 0.25 * r2a.rel_gap


def test_literal_alg1_differs_but_shares_the_minimiser_objective():
    # The printed data term tau0/delta changes the iterates (vecgrad of the
    # removed gradient part is not zero), see the module header of oracle.tvs.
    d0 = image(10, 11, 6)
    prob = tvs.tfs_problem(d0, 0.05)
    p = np.zeros((2, 2, 11, 12))
    a = tvs.tfs_step(prob, p, 0.125)
    b = tvs.tfs_step(prob, p, 0.125, literal_alg1=True)
    assert np.abs(a - b).max() > 1e-6


# ---- brute force on 8x8 images --------------------------------------------

def _ball(p, nch, npx):
    q = p.reshape(nch, 2, npx)
    n = np.maximum(np.sqrt(q[:, 0] ** 2 + q[:, 1] ** 2), 1.0)
    return (q / n[:, None, :]).reshape(-1)


def _fista(lam, f, nch, npx, iters):
    lip = 2.0 * np.linalg.norm(lam, 2) ** 2
    p = np.zeros(lam.shape[1])
    y, tk = p.copy(), 1.0
    for _ in range(iters):
        pn = _ball(y - 2.0 * lam.T @ (lam @ y - f) / lip, nch, npx)
        tn = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * tk * tk))
        y = pn + (tk - 1.0) / tn * (pn - p)
        p, tk = pn, tn
    return p


def _dense_gap(grad_m, u, p, npx):
    g = grad_m @ u
    return float(np.sum(np.sqrt(g[:npx] ** 2 + g[npx:] ** 2) + g[:npx] * p[:npx] + g[npx:] * p[npx:]))


def test_irv1_agrees_with_bruteforce_dense_solve():
    d0 = image(8, 8, 3)
    tau, _, _ = tvs.tfs(d0, 0.05, iters=200)
    alpha = 10.0
    f2 = tvs.irv1_data(d0, tvs.normal_field(tau, 8, 8, 1e-3), alpha)
    grad_m, div_m = dense_ops(8, 8)
    p_bf = _fista(div_m, f2.reshape(-1), 1, 64, 20000)
    d_bf = (f2.reshape(-1) - div_m @ p_bf) / alpha
    gap_bf = _dense_gap(grad_m, d_bf, p_bf, 64)
    d_or, _, rep = tvs.irv1(f2, alpha, iters=20000)
    assert gap_bf < 1e-8 and rep.gap < 1e-8
    bound = np.sqrt(2 * gap_bf / alpha) + np.sqrt(2 * rep.gap / alpha)
    assert np.linalg.norm(d_or.reshape(-1) - d_bf) <= bound + 1e-12
    assert np.abs(d_or.reshape(-1) - d_bf).max() < 1e-6


def test_tfs_agrees_with_bruteforce_dense_solve():
    d0 = image(8, 8, 7)
    delta = 0.05
    r, c = 9, 9
    npx = r * c
    grad_m, div_m = dense_ops(r, c)
    q = scipy.linalg.null_space(div_m)
    proj = q @ q.T                                        # projector onto K
    vecdiv_m = scipy.linalg.block_diag(div_m, div_m)      # (2 npx) x (4 npx)
    lam = proj @ vecdiv_m
    tau0 = ops.tangent(d0).reshape(-1)
    f = proj @ tau0 / delta
    p_bf = _fista(lam, f, 2, npx, 30000)
    tau_bf = proj @ tau0 - delta * lam @ p_bf
    gap_bf = (_dense_gap(grad_m, tau_bf[:npx], p_bf[: 2 * npx], npx)
              + _dense_gap(grad_m, tau_bf[npx:], p_bf[2 * npx:], npx))
    tau_or, _, rep = tvs.tfs(d0, delta, iters=30000)
    assert gap_bf < 1e-9 and rep.gap < 1e-9
    bound = np.sqrt(2 * gap_bf * delta) + np.sqrt(2 * rep.gap * delta)
    assert np.linalg.norm(tau_or.reshape(-1) - tau_bf) <= bound + 1e-12
    assert np.abs(tau_or.reshape(-1) - tau_bf).max() < 1e-6


def test_denoise_pipeline_reduces_error():
    gt, d0 = noisy_scene(SceneSpec(32, 32, 0, 0.1))
    d, tau, r1, r2 = tvs.denoise(d0, iters1=300, iters2=300)
    assert np.mean((d - gt) ** 2) < 0.5 * np.mean((d0 - gt) ** 2)
    assert r1.div_res_max < 1e-11


# ---- the normal field xi and the data f_2 (eq. defXi2:discrete, eq. ir1dualdis) ----

def test_normal_field_and_f2_match_hand_values(golden):
    d0 = np.asarray(golden["image_2x3"], dtype=np.float64)
    tau0 = np.stack([np.asarray(golden["tau0_2x3_component1"], dtype=np.float64),
                     np.asarray(golden["tau0_2x3_component2"], dtype=np.float64)])
    xi = tvs.normal_field(tau0, 2, 3, 4.0)
    np.testing.assert_allclose(xi[0], golden["xi_2x3_eps4_component1"], atol=1e-15)
    np.testing.assert_allclose(xi[1], golden["xi_2x3_eps4_component2"], atol=1e-15)
    np.testing.assert_allclose(ops.div(xi), golden["div_xi_2x3_eps4"], atol=1e-15)
    np.testing.assert_allclose(tvs.irv1_data(d0, xi, 1.0), golden["f2_2x3_eps4_alpha1"], atol=1e-14)


@pytest.mark.parametrize("rows,cols,eps", [(7, 9, 1e-3), (12, 5, 0.5), (16, 16, 1e-3)])
def test_normal_field_of_tau0_is_the_normalised_backward_gradient(rows, cols, eps):
    # tau_0 = (-D^{neum-}_y d0, D^{neum-}_x d0), so tau_0^perp = (tau_0,2, -tau_0,1)
    # = (D^{neum-}_x d0, D^{neum-}_y d0) on Omega: the normal field points along
    # the backward-difference gradient of d0 (the direction in which the
    # intensity grows), which is what the alignment term of Section 5.1
    # rewards.  A swapped or sign-flipped xi fails this.
    d0 = image(rows, cols, 11)
    xi = tvs.normal_field(ops.tangent(d0), rows, cols, eps)
    gx = ops.dx_neum(d0)[:rows, :cols]
    gy = ops.dy_neum(d0)[:rows, :cols]
    den = np.sqrt(gx ** 2 + gy ** 2 + eps)
    np.testing.assert_allclose(xi[0], gx / den, atol=1e-15)
    np.testing.assert_allclose(xi[1], gy / den, atol=1e-15)
    assert np.all(xi[0] * gx + xi[1] * gy >= 0.0)
    assert np.max(np.sqrt(xi[0] ** 2 + xi[1] ** 2)) < 1.0


def test_irv1_minimises_the_w11_functional_written_out():
    # eq. IRW11 (and IRPXi) as printed: J(d) = ||grad d||_1 - <grad d, xi> + (alpha/2)||d - d0||^2.
    # The IRV1 result, run to a small certified gap, must minimise J: random
    # feasible perturbations never lower it, and the minimiser for the other
    # sign of xi (what a sign error in f_2 = alpha d0 - div xi would give) is worse.
    d0 = image(10, 11, 12)
    tau, _, _ = tvs.tfs(d0, 0.05, iters=200)
    xi = tvs.normal_field(tau, 10, 11, 1e-3)
    alpha = 10.0

    def J(d):
        g = ops.grad(d)
        return (float(np.sum(np.sqrt(g[0] ** 2 + g[1] ** 2))) - float(np.sum(g * xi))
                + 0.5 * alpha * float(np.sum((d - d0) ** 2)))

    d, _, rep = tvs.irv1(tvs.irv1_data(d0, xi, alpha), alpha, iters=20000)
    assert rep.rel_gap < 1e-9
    j0 = J(d)
    rng = np.random.default_rng(5)
    for _ in range(20):
        h = rng.standard_normal(d.shape)
        for s in (1e-2, 1e-4):
            assert J(d + s * h) >= j0 - 1e-9
    d_flip, _, _ = tvs.irv1(tvs.irv1_data(d0, -xi, alpha), alpha, iters=20000)
    assert J(d_flip) > j0 + 1e-3


def test_w11_dual_agrees_with_projected_gradient_on_the_shifted_ball():
    # eq. IRW11:dual solved by FISTA on the explicit matrices with the
    # projection onto |p - xi| <= 1 (no reduction to IRV1 involved), against
    # the oracle's reading (Chambolle on q = p - xi, p = q + xi).
    d0 = image(8, 8, 13)
    tau, _, _ = tvs.tfs(d0, 0.05, iters=200)
    xi = tvs.normal_field(tau, 8, 8, 1e-3)
    alpha = 10.0
    grad_m, div_m = dense_ops(8, 8)
    xiv = xi.reshape(-1)
    f = alpha * d0.reshape(-1)
    lip = 2.0 * np.linalg.norm(div_m, 2) ** 2
    p = xiv.copy()
    y, tk = p.copy(), 1.0
    for _ in range(30000):
        pn = xiv + _ball(y - 2.0 * div_m.T @ (div_m @ y - f) / lip - xiv, 1, 64)
        tn = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * tk * tk))
        y = pn + (tk - 1.0) / tn * (pn - p)
        p, tk = pn, tn
    d_pg = d0.reshape(-1) - div_m @ p / alpha          # -div p = alpha (d - d0)
    # gap of eq. IRW11 at (d, p): sum |grad d| + grad d . (p - xi) >= 0
    g = grad_m @ d_pg
    gap_pg = float(np.sum(np.sqrt(g[:64] ** 2 + g[64:] ** 2)) + np.sum(g * (p - xiv)))
    d_or, p_or, rep = tvs.w11(d0, xi, alpha, iters=30000)
    assert gap_pg < 1e-8 and rep.gap < 1e-8
    assert np.max(np.sqrt((p_or[0] - xi[0]) ** 2 + (p_or[1] - xi[1]) ** 2)) <= 1.0 + 1e-12
    bound = np.sqrt(2 * gap_pg / alpha) + np.sqrt(2 * rep.gap / alpha)
    assert np.linalg.norm(d_or.reshape(-1) - d_pg) <= bound + 1e-12
    assert np.abs(d_or.reshape(-1) - d_pg).max() < 1e-6
    # first optimality condition of the proposition: -div p = alpha (d - d0)
    np.testing.assert_allclose(-ops.div(p_or), alpha * (d_or - d0), atol=1e-12)
    # second: where |grad d| > 0, (xi - p) |grad d| = grad d
    gd = ops.grad(d_or)
    nd = np.sqrt(gd[0] ** 2 + gd[1] ** 2)
    big = nd > 1e-3
    for c in range(2):
        np.testing.assert_allclose(((xi[c] - p_or[c]) * nd)[big], gd[c][big], atol=1e-5)
