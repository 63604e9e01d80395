"""Pins for IRV2 in oracle.tvs (Section 3.3: eqs. modifiedStep2, modifiedStep2_2,
modifiedStep2_2_dual; discrete eq. ir2dualdis).

The potential g of tau_perp is the one reading the paper leaves open (see
oracle.tvs.potential): the least-squares solution of the backward differences
between neighbouring image pixels.  It is pinned by exact recovery of a known
potential, by numpy's least-squares solve of the assembled equations, and by
the paper's remark that backward differences put g in the coordinates of d0
(the potential of the noisy image's own tangent field is the image).  The
ROF part is pinned by a brute-force FISTA solve and by the primal functional
of eq. modifiedStep2 written out.
"""
import numpy as np
import pytest

from oracle import ops, tvs
from synth import SceneSpec, noisy_scene
from test_oracle_ops import dense_ops
from test_oracle_tvs import _fista, _dense_gap

RNG = np.random.default_rng(2024)


def image(rows, cols, seed, sigma=0.1):
    return noisy_scene(SceneSpec(rows, cols, seed, sigma))[1]


def tau_of_potential(g):
    """An extended-grid tau whose tau_perp has g's backward differences
    between image pixels; everything else (first column of tau_2, first row
    of tau_1, the extra row and column) is random."""
    n2, n1 = g.shape
    tau = RNG.standard_normal((2, n2 + 1, n1 + 1))
    tau[1][:n2, 1:n1] = g[:, 1:] - g[:, :-1]          # tau_2 = D^-_x g between pixels
    tau[0][1:n2, :n1] = -(g[1:, :] - g[:-1, :])        # -tau_1 = D^-_y g between pixels
    return tau


@pytest.mark.parametrize("n2,n1", [(3, 3), (7, 12), (16, 9), (33, 40)])
def test_potential_recovers_a_known_potential(n2, n1):
    g = RNG.standard_normal((n2, n1))
    got = tvs.potential(tau_of_potential(g), n2, n1)
    np.testing.assert_allclose(got, g - g.mean(), atol=1e-11)


@pytest.mark.parametrize("n2,n1", [(5, 6), (12, 7), (20, 20)])
def test_potential_of_the_tangent_field_is_the_image(n2, n1):
    # tau_0 = (-D^{neum-}_y d0, D^{neum-}_x d0): its pixel differences are d0's
    d0 = image(n2, n1, 3)
    got = tvs.potential(ops.tangent(d0), n2, n1)
    np.testing.assert_allclose(got, d0 - d0.mean(), atol=1e-12)


@pytest.mark.parametrize("n2,n1", [(4, 5), (6, 6), (9, 4)])
def test_potential_is_the_least_squares_solution(n2, n1):
    tau = RNG.standard_normal((2, n2 + 1, n1 + 1))
    a = tau[1][:n2, :n1]
    b = -tau[0][:n2, :n1]
    rows, rhs = [], []
    idx = lambda i, j: i * n1 + j
    for i in range(n2):
        for j in range(1, n1):
            r = np.zeros(n2 * n1)
            r[idx(i, j)], r[idx(i, j - 1)] = 1.0, -1.0
            rows.append(r)
            rhs.append(a[i, j])
    for i in range(1, n2):
        for j in range(n1):
            r = np.zeros(n2 * n1)
            r[idx(i, j)], r[idx(i - 1, j)] = 1.0, -1.0
            rows.append(r)
            rhs.append(b[i, j])
    sol = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)[0]    # minimum norm: mean zero
    np.testing.assert_allclose(tvs.potential(tau, n2, n1).reshape(-1), sol, atol=1e-12)


def test_irv2_with_the_images_own_tangent_field_returns_the_image():
    # g = d0 - mean, so the ROF data alpha (d0 - g) is constant (up to the
    # rounding of g): p stays 0 and d = d0
    d0 = image(11, 13, 4)
    d, p, rep, g = tvs.irv2(d0, ops.tangent(d0), 10.0, iters=50)
    assert np.abs(p).max() < 1e-12
    np.testing.assert_allclose(d, d0, atol=1e-12)


def test_irv2_is_invariant_to_a_constant_in_the_potential():
    d0 = image(10, 12, 5)
    tau, _, _ = tvs.tfs(d0, 0.05, iters=100)
    d, p, _, g = tvs.irv2(d0, tau, 10.0, iters=200)
    u2, p2, _ = tvs.irv1(tvs.irv2_data(d0, g + 0.37, 10.0), 10.0, iters=200)
    np.testing.assert_allclose(u2 + g + 0.37, d, atol=1e-12)
    np.testing.assert_allclose(p2, p, atol=1e-12)


def test_irv2_agrees_with_bruteforce_and_minimises_the_printed_functional():
    d0 = image(8, 8, 6)
    tau, _, _ = tvs.tfs(d0, 0.05, iters=200)
    alpha = 10.0
    d_or, p_or, rep, g = tvs.irv2(d0, tau, alpha, iters=20000)
    grad_m, div_m = dense_ops(8, 8)
    f = (alpha * (d0 - g)).reshape(-1)
    p_bf = _fista(div_m, f, 1, 64, 20000)
    u_bf = (f - div_m @ p_bf) / alpha
    gap_bf = _dense_gap(grad_m, u_bf, p_bf, 64)
    assert gap_bf < 1e-8 and rep.gap < 1e-8
    bound = np.sqrt(2 * gap_bf / alpha) + np.sqrt(2 * rep.gap / alpha)
    assert np.linalg.norm(d_or.reshape(-1) - (u_bf + g.reshape(-1))) <= bound + 1e-12
    # eq. modifiedStep2 as printed: TV(d - g) + (alpha/2) ||d - d0||^2
    J = lambda d: tvs.tv(d - g) + 0.5 * alpha * float(np.sum((d - d0) ** 2))
    j0 = J(d_or)
    for _ in range(20):
        h = RNG.standard_normal(d0.shape)
        for s in (1e-2, 1e-4):
            assert J(d_or + s * h) >= j0 - 1e-9
    # d = d0 - div p / alpha (the relation printed after eq. modifiedStep2_2_dual)
    np.testing.assert_allclose(d_or, d0 - ops.div(p_or) / alpha, atol=1e-12)
