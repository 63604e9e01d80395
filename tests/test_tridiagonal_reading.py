"""The y pass of Delta^dagger as Neumann tridiagonal solves (CPU, FP64).

The GPU path applies the pseudo-inverse of eqs. form:DiscInvLapl /
form:DiscInvLaplTild as a DCT along x and, for every x frequency k, the
operator C_R^T diag(Lambda(., k)) C_R along y.  It evaluates that operator as
-(T + lambda_k I)^{-1} (the Neumann second difference T, lambda_k =
sigma_{C,k}^2; the pseudo-inverse -T^dagger for k = 0) by two first-order
recursions with closed-form start values.  These tests pin both statements
against the oracle's DCT matrices and symbol, so that the equivalence the
column kernel relies on is checked independently of the GPU.
"""
import numpy as np
import pytest

from oracle import ops


def neumann_t(n: int) -> np.ndarray:
    """tridiag(-1, 2, -1) with 1 in both corners: -Laplacian with the D^- / D^+ pairing."""
    t = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    t[0, 0] = t[-1, -1] = 1.0
    return t


def column_operator(rows: int, cols: int, k: int) -> np.ndarray:
    """C_R^T diag(Lambda(:, k)) C_R with the oracle's DCT matrix and symbol."""
    c = ops.dct_matrix(rows)
    lam = ops.inv_lap_symbol(rows, cols)[:, k]
    return c.T @ np.diag(lam) @ c


def recursions(b: np.ndarray, lam: float) -> np.ndarray:
    """-(T + lam I)^{-1} b (lam > 0) or -T^dagger b (lam = 0) by the two recursions."""
    n = len(b)
    if lam == 0.0:
        c = np.cumsum(b - b.mean())                 # c_{-1} = 0
        w = np.cumsum(c[::-1])[::-1]                # w_L = 0
        return -(w - w.mean())
    q = 0.5 * (np.sqrt(lam * (4.0 + lam)) - lam)    # 1 - r
    r = 1.0 - q
    j = np.arange(n)
    u0 = np.sum(b * (r ** j + r ** (2 * n - 1 - j))) / (1.0 - r ** (2 * n))
    c = np.empty(n)
    prev = u0
    for i in range(n):
        prev = b[i] + r * prev
        c[i] = prev
    w = np.empty(n)
    nxt = c[-1] / q                                 # w_L = w_{L-1} = c_{L-1} / (1 - r)
    for i in range(n - 1, -1, -1):
        nxt = c[i] + r * nxt
        w[i] = nxt
    return -r * w


@pytest.mark.parametrize("rows,cols", [(3, 3), (4, 9), (17, 17), (65, 33), (129, 257)])
def test_column_operator_is_the_shifted_neumann_inverse(rows, cols):
    t = neumann_t(rows)
    lam = ops.sigma(cols) ** 2
    for k in sorted({0, 1, 2, cols // 2, cols - 1}):
        a = column_operator(rows, cols, k)
        if k == 0:
            ref = -np.linalg.pinv(t, rtol=1e-10, hermitian=True)
        else:
            ref = -np.linalg.inv(t + lam[k] * np.eye(rows))
        assert np.abs(a - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("rows,cols", [(3, 3), (4, 9), (17, 17), (65, 33), (257, 1025), (1025, 1025)])
def test_recursions_apply_the_column_operator(rows, cols):
    rng = np.random.default_rng(rows * 7 + cols)
    lam = ops.sigma(cols) ** 2
    for k in sorted({0, 1, 2, cols // 2, cols - 1}):
        b = rng.standard_normal(rows)
        got = recursions(b, float(lam[k]))
        ref = column_operator(rows, cols, k) @ b
        assert np.abs(got - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max())


def test_rows_then_columns_reproduce_the_oracle_pseudo_inverse():
    """DCT along x, the recursions along y, inverse DCT along x == ops.inv_lap."""
    rng = np.random.default_rng(3)
    rows, cols = 33, 20
    s = rng.standard_normal((rows, cols))
    cx = ops.dct_matrix(cols)
    sx = s @ cx.T                                   # x transform of every row
    lam = ops.sigma(cols) ** 2
    y = np.stack([recursions(sx[:, k], float(lam[k])) for k in range(cols)], axis=1)
    phi = y @ cx
    assert np.abs(phi - ops.inv_lap(s)).max() <= 1e-10 * np.abs(phi).max()
