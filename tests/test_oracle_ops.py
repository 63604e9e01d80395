"""Pins for oracle.ops: the operators of Section 4.1 and the projection of Appendix B.

Each check compares the oracle with something other than itself: hand-derived
values (tests/golden/tiny_operators.json), dense matrices assembled here
entry by entry from the definitions, library routines (SciPy DCT, numpy pinv,
SciPy null_space), or identities the paper proves.
"""
import numpy as np
import pytest
import scipy.fft
import scipy.linalg

from oracle import ops

RNG = np.random.default_rng(1234)
SHAPES = [(2, 2), (2, 5), (3, 4), (5, 9), (9, 14), (13, 7)]


def a(x):
    return np.asarray(x, dtype=np.float64)


# ---- hand-derived values -------------------------------------------------

def test_differences_match_hand_values(golden):
    u = a(golden["image_2x3"])
    np.testing.assert_array_equal(ops.dxp(u), a(golden["dxp_2x3"]))
    np.testing.assert_array_equal(ops.dyp(u), a(golden["dyp_2x3"]))
    np.testing.assert_array_equal(ops.dxm(u), a(golden["dxm_2x3"]))
    np.testing.assert_array_equal(ops.dym(u), a(golden["dym_2x3"]))


def test_neumann_differences_and_tangent_match_hand_values(golden):
    d = a(golden["image_2x3"])
    np.testing.assert_array_equal(ops.dx_neum(d), a(golden["dx_neum_2x3"]))
    np.testing.assert_array_equal(ops.dy_neum(d), a(golden["dy_neum_2x3"]))
    t0 = ops.tangent(d)
    np.testing.assert_array_equal(t0[0], a(golden["tau0_2x3_component1"]))
    np.testing.assert_array_equal(t0[1], a(golden["tau0_2x3_component2"]))


def test_dct_matrix_and_sigma_match_hand_values(golden):
    np.testing.assert_allclose(ops.dct_matrix(2), a(golden["dct_C2"]), atol=1e-15)
    np.testing.assert_allclose(ops.dct_matrix(3), a(golden["dct_C3"]), atol=1e-15)
    np.testing.assert_allclose(ops.sigma(2) ** 2, a(golden["sigma_sq_N2"]), atol=1e-15)
    np.testing.assert_allclose(ops.sigma(3) ** 2, a(golden["sigma_sq_N3"]), atol=1e-15)


def test_inverse_laplacian_and_projection_match_hand_values(golden):
    s = np.zeros((2, 2))
    s[0, 0] = 1.0
    np.testing.assert_allclose(ops.inv_lap(s), a(golden["inv_lap_2x2_of_delta00"]), atol=1e-15)
    g = golden["proj_2x2_of_e00_x"]
    tau = np.stack([a(g["input_component1"]), a(g["input_component2"])])
    out = ops.proj_k(tau)
    np.testing.assert_allclose(out[0], a(g["output_component1"]), atol=1e-15)
    np.testing.assert_allclose(out[1], a(g["output_component2"]), atol=1e-15)


# ---- dense matrices assembled from the definitions ----------------------

def d_plus_1d(n):
    m = np.zeros((n, n))
    for j in range(n - 1):
        m[j, j + 1] = 1.0
        m[j, j] = -1.0
    return m


def d_minus_1d(n):
    m = np.zeros((n, n))
    m[0, 0] = 1.0
    for j in range(1, n - 1):
        m[j, j] = 1.0
        m[j, j - 1] = -1.0
    m[n - 1, n - 2] = -1.0
    return m


def dense_ops(r, c):
    """Row-major vec: index = i*c + j.  x acts on columns, y on rows."""
    dxp = np.kron(np.eye(r), d_plus_1d(c))
    dyp = np.kron(d_plus_1d(r), np.eye(c))
    dxm = np.kron(np.eye(r), d_minus_1d(c))
    dym = np.kron(d_minus_1d(r), np.eye(c))
    grad = np.vstack([dxp, dyp])
    div = np.hstack([dxm, dym])
    return grad, div


@pytest.mark.parametrize("shape", SHAPES)
def test_operators_equal_dense_definitions(shape):
    r, c = shape
    grad_m, div_m = dense_ops(r, c)
    u = RNG.standard_normal((r, c))
    v = RNG.standard_normal((2, r, c))
    np.testing.assert_allclose(ops.grad(u).reshape(-1), grad_m @ u.reshape(-1), atol=1e-13)
    np.testing.assert_allclose(ops.div(v).reshape(-1), div_m @ v.reshape(-1), atol=1e-13)


@pytest.mark.parametrize("shape", SHAPES)
def test_div_is_minus_grad_adjoint(shape):
    # div = -grad^* (Section 4.1, after eq. defDivDis); vecdiv = -vecgrad^*
    r, c = shape
    grad_m, div_m = dense_ops(r, c)
    np.testing.assert_array_equal(div_m, -grad_m.T)
    u = RNG.standard_normal((2, r, c))
    p = RNG.standard_normal((2, 2, r, c))
    lhs = ops.dot(ops.vecgrad(u), p)
    rhs = -ops.dot(u, ops.vecdiv(p))
    assert abs(lhs - rhs) <= 1e-12 * (1 + abs(lhs))


# ---- DCT and the Laplacian pseudo-inverse --------------------------------

@pytest.mark.parametrize("n", [2, 3, 5, 8, 13, 65])
def test_dct_matrix_orthogonal_and_equals_textbook_dct2(n):
    c = ops.dct_matrix(n)
    np.testing.assert_allclose(c @ c.T, np.eye(n), atol=1e-13)
    x = RNG.standard_normal(n)
    np.testing.assert_allclose(c @ x, scipy.fft.dct(x, type=2, norm="ortho"), atol=1e-13)


@pytest.mark.parametrize("shape", SHAPES)
def test_inverse_laplacian_equals_pinv(shape):
    r, c = shape
    grad_m, div_m = dense_ops(r, c)
    lap = div_m @ grad_m
    pinv = np.linalg.pinv(lap, rcond=1e-10, hermitian=True)
    s = RNG.standard_normal((r, c))
    np.testing.assert_allclose(ops.inv_lap(s).reshape(-1), pinv @ s.reshape(-1), atol=1e-11)
    np.testing.assert_allclose(ops.inv_lap_dense(s), ops.inv_lap(s), atol=1e-12)
    # Delta Delta^dagger Delta = Delta
    u = RNG.standard_normal((r, c))
    np.testing.assert_allclose(ops.laplacian(ops.inv_lap(ops.laplacian(u))), ops.laplacian(u), atol=1e-11)


def test_printed_eigenvalue_pairing_breaks_non_square_grids():
    # The printed symbol pairs row index i with sigma_{N1+1, i} and column
    # index j with sigma_{N2+1, j}.  On a non-square grid that is not the
    # pseudo-inverse; pairing the row frequency with the row count is.
    r, c = 9, 14
    grad_m, div_m = dense_ops(r, c)
    pinv = np.linalg.pinv(div_m @ grad_m, rcond=1e-10, hermitian=True)
    s = RNG.standard_normal((r, c))
    i = np.arange(r)[:, None]
    j = np.arange(c)[None, :]
    den = (2 * np.sin(i * np.pi / (2 * c))) ** 2 + (2 * np.sin(j * np.pi / (2 * r))) ** 2
    printed = np.where(den > 0, -1.0 / np.where(den > 0, den, 1.0), 0.0)
    wrong = ops.idct2(printed * ops.dct2(s))
    assert np.abs(wrong.reshape(-1) - pinv @ s.reshape(-1)).max() > 1e-3
    right = ops.idct2(ops.inv_lap_symbol(r, c) * ops.dct2(s))
    assert np.abs(right.reshape(-1) - pinv @ s.reshape(-1)).max() < 1e-11


# ---- the projection P_K (formula:PKh, Appendix B) -------------------------

@pytest.mark.parametrize("shape", SHAPES)
def test_projection_equals_orthogonal_projector_onto_null_div(shape):
    r, c = shape
    _, div_m = dense_ops(r, c)
    q = scipy.linalg.null_space(div_m)
    proj = q @ q.T
    tau = RNG.standard_normal((2, r, c))
    np.testing.assert_allclose(ops.proj_k(tau).reshape(-1), proj @ tau.reshape(-1), atol=1e-11)


@pytest.mark.parametrize("shape", [(3, 4), (9, 14), (33, 47), (65, 65)])
def test_projection_properties(shape):
    r, c = shape
    t1 = RNG.standard_normal((2, r, c))
    t2 = RNG.standard_normal((2, r, c))
    p1 = ops.proj_k(t1)
    np.testing.assert_allclose(ops.proj_k(p1), p1, atol=1e-11)           # idempotent
    assert abs(ops.dot(p1, t2) - ops.dot(t1, ops.proj_k(t2))) < 1e-10    # self-adjoint
    assert np.abs(ops.div(p1)).max() < 1e-12                              # lands in K
    phi = RNG.standard_normal((r, c))
    assert np.abs(ops.proj_k(ops.grad(phi))).max() < 1e-11               # kills gradients
    # identity on K: (-D^-_y chi, D^-_x chi) is divergence free for any chi
    chi = RNG.standard_normal((r, c))
    k_field = np.stack([-ops.dym(chi), ops.dxm(chi)])
    assert np.abs(ops.div(k_field)).max() < 1e-13
    np.testing.assert_allclose(ops.proj_k(k_field), k_field, atol=1e-11)


def test_norm_of_projected_vecdiv_at_most_8():
    # ||P_K vecdiv||^2 <= ||vecdiv||^2 <= 8 (proof of the convergence theorem, Sec. 4.2)
    r, c = 17, 23
    p = RNG.standard_normal((2, 2, r, c))
    lam = 0.0
    for _ in range(300):
        w = ops.proj_k(ops.vecdiv(p))
        p2 = -ops.vecgrad(ops.proj_k(w))     # (P_K vecdiv)^* (P_K vecdiv) p
        lam = np.sqrt(ops.sqnorm(p2))
        p = p2 / lam
    assert 7.0 < lam <= 8.0 + 1e-9


def test_tangent_divergence_vanishes_inside_but_not_on_the_ring():
    # Section 4.2: tau_0 need not lie in K.  Inside the extended grid the mixed
    # differences cancel; on the boundary ring they do not in general.
    d = RNG.standard_normal((12, 15))
    dv = ops.div(ops.tangent(d))
    assert np.abs(dv[1:-1, 1:-1]).max() < 1e-13
    assert np.abs(dv).max() > 1e-3
    ptau = ops.proj_k(ops.tangent(d))
    assert np.abs(ptau - ops.tangent(d)).max() > 1e-3
