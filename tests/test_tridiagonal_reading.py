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


def chunked(b: np.ndarray, lam: float, chunk: int = 32, ranges: int = 24) -> np.ndarray:
    """The same solve in the chunked form of the long-column kernels.

    Per chunk of `chunk` rows, summaries from a zero carry: h = sum r^(i-i0) b_i,
    the causal end value a, g = sum r^(i-i0) c_i over the causal values from
    zero and (k = 0) K = sum (i-i0+1) c_i.  Per column, the chunks are grouped
    into `ranges` consecutive ranges (the warps of the scan kernel) whose
    composites are combined, then the carries C (into a chunk) and W (after
    it) are formed and every chunk reruns both recursions from its carries.
    For k = 0 (r = 1) the input mean enters as corrections of a, g and K.
    """
    n = len(b)
    if lam == 0.0:
        q = 0.0
    else:
        q = 0.5 * (np.sqrt(lam * (4.0 + lam)) - lam)
    r = 1.0 - q
    nch = (n + chunk - 1) // chunk
    lens = [min(chunk, n - c * chunk) for c in range(nch)]
    h, a, g, kk = np.zeros(nch), np.zeros(nch), np.zeros(nch), np.zeros(nch)
    for c in range(nch):
        seg = b[c * chunk: c * chunk + lens[c]]
        p, loc = 0.0, []
        for x in seg:
            p = x + r * p
            loc.append(p)
        a[c] = p
        h[c] = sum(r ** i * x for i, x in enumerate(seg))
        g[c] = sum(r ** i * x for i, x in enumerate(loc))
        kk[c] = sum((i + 1) * x for i, x in enumerate(loc))
    zero = lam == 0.0
    S1 = sum(r ** (c * chunk) * h[c] for c in range(nch))
    R2 = sum(r ** (n - c * chunk - lens[c]) * a[c] for c in range(nch))
    mu = S1 / n if zero else 0.0
    ap = np.array([a[c] - mu * lens[c] for c in range(nch)]) if zero else a
    gp = np.array([g[c] - mu * lens[c] * (lens[c] + 1) / 2 for c in range(nch)]) if zero else g
    kn = [sum(r ** (2 * m + 1) for m in range(lens[c])) for c in range(nch)]
    u0 = 0.0 if zero else (S1 + r ** n * R2) / (1.0 - r ** (2 * n))
    cpw = (nch + ranges - 1) // ranges
    rng_of = [(min(nch, w * cpw), min(nch, w * cpw + cpw)) for w in range(ranges)]
    # forward composites per range, then the carries
    comp = []
    for c0, c1 in rng_of:
        f, m = 0.0, 1.0
        for c in range(c0, c1):
            f = ap[c] + r ** lens[c] * f
            m *= r ** lens[c]
        comp.append((f, m))
    carry, cin = u0, np.zeros(nch)
    for w, (c0, c1) in enumerate(rng_of):
        for c in range(c0, c1):
            cin[c] = carry
            carry = ap[c] + r ** lens[c] * carry
    wL = 0.0 if zero else carry / q
    # backward composites per range, then the carries after each chunk
    bcomp = []
    for (c0, c1), (_, m) in zip(rng_of, comp):
        s = 0.0
        for c in range(c1 - 1, c0 - 1, -1):
            s = gp[c] + cin[c] * kn[c] + r ** lens[c] * s
        bcomp.append((s, m))
    win = np.zeros(nch)
    wa = wL
    for w in range(ranges - 1, -1, -1):
        c0, c1 = rng_of[w]
        for c in range(c1 - 1, c0 - 1, -1):
            win[c] = wa
            wa = gp[c] + cin[c] * kn[c] + r ** lens[c] * wa
    shift = 0.0
    if zero:
        tot = 0.0
        for c in range(nch):
            m = lens[c]
            kc = kk[c] - mu * m * (m + 1) * (2 * m + 1) / 6
            tot += kc + cin[c] * m * (m + 1) / 2 + m * win[c]
        shift = tot / n
    out = np.zeros(n)
    for c in range(nch):
        seg = b[c * chunk: c * chunk + lens[c]] - mu
        p, cv = cin[c], []
        for x in seg:
            p = x + r * p
            cv.append(p)
        wv = win[c]
        for i in range(lens[c] - 1, -1, -1):
            wv = cv[i] + r * wv
            out[c * chunk + i] = -r * wv + shift
    return out


@pytest.mark.parametrize("ranges", [24, 16, 7])
@pytest.mark.parametrize("rows,cols", [(1537, 64), (2049, 2049), (1601, 33), (40, 7)])
def test_chunked_recursions_equal_the_one_pass_recursions(rows, cols, ranges):
    rng = np.random.default_rng(rows + cols)
    lam = ops.sigma(cols) ** 2
    for k in sorted({0, 1, 2, cols // 2, cols - 1}):
        b = rng.standard_normal(rows)
        got = chunked(b, float(lam[k]), ranges=ranges)
        ref = recursions(b, float(lam[k]))
        assert np.abs(got - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max())
