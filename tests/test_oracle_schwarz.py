"""Pins for oracle.schwarz: Section 6 (partition of unity, Algorithms 2-5,
locality identities resDiv/resGrad, the localized projection).
"""
import numpy as np
import pytest

from oracle import ops, schwarz, tvs
from synth import SceneSpec, noisy_scene

RNG = np.random.default_rng(7)


@pytest.mark.parametrize("n,m,s,ext", [(64, 4, 8, False), (64, 4, 8, True), (30, 3, 3, False),
                                       (31, 3, 4, True), (20, 1, 4, False), (17, 2, 5, True),
                                       (64, 8, 0, False)])
def test_partition_of_unity_properties(n, m, s, ext):
    ext_list, th = schwarz.axis_parts(n, m, s, ext)
    total = np.sum(th, axis=0)
    np.testing.assert_allclose(total, 1.0, atol=1e-15)
    for (a, b), t in zip(ext_list, th):
        assert np.all(t >= 0)
        assert np.all(t[:a] == 0) and np.all(t[b:] == 0)     # supp theta_m in Gamma_m
        assert np.all(t[a:b] > 0)
        if s > 0:
            assert np.abs(np.diff(t)).max() <= 1.0 / s + 1e-15   # |grad theta| <= C0/s, C0 = 1
    # consecutive subdomains overlap in exactly s pixels
    for k in range(m - 1):
        assert ext_list[k][1] - ext_list[k + 1][0] == s


def test_steps_share_cores():
    # Omega_m = tilde Omega_m restricted to Omega (Section 6.1)
    a = schwarz.Decomp(40, 52, 3, 4, 6, False)
    b = schwarz.Decomp(40, 52, 3, 4, 6, True)
    for m in a.subdomains():
        y0, y1, x0, x1 = b.box(m)
        assert a.box(m) == (y0, min(y1, 40), x0, min(x1, 52))
        np.testing.assert_array_equal(b.theta(m)[:40, :52], a.theta(m))


@pytest.mark.parametrize("box", [(2, 7, 3, 9), (0, 5, 0, 4), (6, 11, 8, 13), (0, 11, 0, 13)])
def test_locality_identities(box):
    # resDiv: div(E_{A-} u) = E_A div_A R_A E_{A-} u ; resGrad: R_{A-} grad d = R_{A-} E_A grad_A R_A d
    rows, cols = 11, 13
    y0, y1, x0, x1 = box          # A
    am = (y0, y1 - 1 if y1 < rows else y1, x0, x1 - 1 if x1 < cols else x1)   # A_-
    u = np.zeros((2, rows, cols))
    u[:, am[0]:am[1], am[2]:am[3]] = RNG.standard_normal((2, am[1] - am[0], am[3] - am[2]))
    lhs = ops.div(u)
    rhs = np.zeros((rows, cols))
    rhs[y0:y1, x0:x1] = ops.div(u[:, y0:y1, x0:x1])
    np.testing.assert_array_equal(lhs, rhs)
    d = RNG.standard_normal((rows, cols))
    g_glob = ops.grad(d)[:, am[0]:am[1], am[2]:am[3]]
    g_loc = ops.grad(d[y0:y1, x0:x1])[:, am[0] - y0:am[1] - y0, am[2] - x0:am[3] - x0]
    np.testing.assert_array_equal(g_glob, g_loc)


@pytest.mark.parametrize("rows,cols,m2,m1,s", [(17, 21, 2, 3, 2), (25, 25, 3, 3, 4), (13, 30, 1, 3, 3)])
def test_localized_projection_equals_global_projection(rows, cols, m2, m1, s):
    dd = schwarz.Decomp(rows - 1, cols - 1, m2, m1, s, True)
    for k in dd.subdomains():
        kp = dd.box_plus(k)
        ky0, ky1, kx0, kx1 = kp
        u = RNG.standard_normal((2, ky1 - ky0, kx1 - kx0))
        full = np.zeros((2, rows, cols))
        full[:, ky0:ky1, kx0:kx1] = u
        glob = ops.proj_k(full)
        for m in dd.subdomains():
            mp = dd.box_plus(m)
            my0, my1, mx0, mx1 = mp
            loc = schwarz.local_projection(u, kp, mp, rows, cols, lam_parts=(m2, m1))
            np.testing.assert_allclose(loc, glob[:, my0:my1, mx0:mx1], atol=1e-12)


def test_block_formula_independent_of_frequency_split():
    rows, cols = 19, 23
    s = RNG.standard_normal((6, 7))
    a_box, b_box = (3, 9, 10, 17), (8, 15, 2, 12)
    ref = schwarz.local_inv_lap_blocks(s, a_box, b_box, rows, cols, (1, 1))
    full = np.zeros((rows, cols))
    full[3:9, 10:17] = s
    np.testing.assert_allclose(ref, ops.inv_lap(full)[8:15, 2:12], atol=1e-12)
    for parts in [(2, 3), (5, 4), (19, 23)]:
        np.testing.assert_allclose(
            schwarz.local_inv_lap_blocks(s, a_box, b_box, rows, cols, parts), ref, atol=1e-12)


def _f2(rows, cols, seed):
    d0 = noisy_scene(SceneSpec(rows, cols, seed, 0.1))[1]
    tau, _, _ = tvs.tfs(d0, 0.05, iters=100)
    return d0, tvs.irv1_data(d0, tvs.normal_field(tau, rows, cols, 1e-3), 10.0)


def test_single_subdomain_is_k_global_iterations():
    d0, f2 = _f2(15, 18, 1)
    dd = schwarz.Decomp(15, 18, 1, 1, 4, False)
    _, p_s, _ = schwarz.schwarz_irv1(f2, 10.0, dd, outer=4, k_inner=5)
    _, p_g, _ = tvs.irv1(f2, 10.0, iters=20)
    np.testing.assert_array_equal(p_s, p_g)
    dt = schwarz.Decomp(15, 18, 1, 1, 4, True)
    _, p1s, _ = schwarz.schwarz_tfs(d0, 0.05, dt, outer=3, k_inner=4)
    _, p1g, _ = tvs.tfs(d0, 0.05, iters=12)
    np.testing.assert_allclose(p1s, p1g, atol=1e-13)


def test_algorithm5_reproduces_algorithm4():
    d0 = noisy_scene(SceneSpec(14, 12, 3, 0.1))[1]
    dd = schwarz.Decomp(14, 12, 2, 2, 2, True)
    _, pa, _ = schwarz.schwarz_tfs(d0, 0.05, dd, outer=5, k_inner=3)
    _, pb, _ = schwarz.schwarz_tfs(d0, 0.05, dd, outer=5, k_inner=3, localized=True)
    assert np.abs(pa).max() > 0.1
    np.testing.assert_allclose(pb, pa, atol=1e-12)


def test_schwarz_irv1_feasible_and_reaches_global_minimiser():
    d0, f2 = _f2(24, 20, 2)
    dd = schwarz.Decomp(24, 20, 2, 2, 4, False)
    d_s, p_s, r_s = schwarz.schwarz_irv1(f2, 10.0, dd, outer=300, k_inner=10)
    d_g, _, r_g = tvs.irv1(f2, 10.0, iters=3000)
    assert r_s.max_p <= 1.0 + 1e-12
    assert r_s.rel_gap < 1e-4
    bound = np.sqrt(2 * r_s.gap / 10.0) + np.sqrt(2 * r_g.gap / 10.0)
    assert np.linalg.norm(d_s - d_g) <= bound


def test_schwarz_tfs_reaches_global_minimiser():
    d0 = noisy_scene(SceneSpec(12, 10, 1, 0.1))[1]
    dd = schwarz.Decomp(12, 10, 2, 2, 2, True)
    t_s, p_s, r_s = schwarz.schwarz_tfs(d0, 0.05, dd, outer=300, k_inner=5)
    t_g, _, r_g = tvs.tfs(d0, 0.05, iters=3000)
    assert r_s.max_p <= 1.0 + 1e-12
    assert r_s.rel_gap < 1e-5
    bound = np.sqrt(2 * r_s.gap * 0.05) + np.sqrt(2 * r_g.gap * 0.05)
    assert np.linalg.norm(t_s - t_g) <= bound
