"""GPU (libtvs, FP32) versus the FP64 oracle, through the C ABI.

Tolerances: the FP32 path must match the FP64 oracle within 1e-4 max-abs per
pixel on [0, 1] intensities (tau, d and the dual p) at equal iteration count,
and energies within a relative 1e-6 (dual energy and primal energy).  Inputs
are the seeded synthetic scenes of ``synth``.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import ops, schwarz as osch, tvs as otvs  # noqa: E402
from synth import SceneSpec, noisy_scene  # noqa: E402

TOL = 1e-4
EREL = 1e-6


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_17494_gb300 import build
    build.build()
    from paper_2602_17494_gb300 import binding
    return binding


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def image(n2, n1, seed=0, sigma=0.1, texture=False):
    return noisy_scene(SceneSpec(n2, n1, seed, sigma, texture))[1]


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


# ---------------------------------------------------------------------------
# the divergence-free projection
# ---------------------------------------------------------------------------
# (2049, 70), (4097, 33), (8193, 24): long columns, 9, 17 and 33 rows per thread in the
# tridiagonal column pass; (24, 8193): 16384-point Bluestein row transforms
@pytest.mark.parametrize("shape", [(3, 3), (3, 17), (9, 14), (65, 65), (66, 131), (257, 130), (1025, 1025),
                                   (2049, 70), (4097, 33), (8193, 24), (24, 8193)])
def test_projection_matches_oracle(B, shape):
    rng = np.random.default_rng(sum(shape))
    tau = rng.standard_normal((2,) + shape)
    out = host(B.tvs_project(cuda(tau)))
    ref = ops.proj_k(tau)
    scale = np.abs(tau).max()
    assert np.abs(out - ref).max() <= 2e-5 * scale
    # lands in K and is idempotent on the GPU too
    assert np.abs(ops.div(out)).max() <= 2e-5 * scale
    again = host(B.tvs_project(cuda(out)))
    assert np.abs(again - out).max() <= 2e-5 * scale


# ---------------------------------------------------------------------------
# step 1, step 2 and the pipeline at equal iteration counts
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n2,n1,seed,iters", [(64, 64, 0, 300), (64, 64, 1, 300), (37, 53, 2, 120), (2, 9, 3, 50),
                                              (96, 40, 4, 200)])
def test_step1_matches_oracle(B, n2, n1, seed, iters):
    d0 = image(n2, n1, seed)
    tau_o, p_o, rep_o = otvs.tfs(d0, 0.05, 0.125, iters)
    p = torch.zeros((4, n2 + 1, n1 + 1), dtype=torch.float32, device="cuda")
    res = B.tvs_step1(cuda(d0), 0.05, B.make_iter(iters), p=p)
    assert np.abs(host(res.out) - tau_o).max() <= TOL
    assert np.abs(host(p).reshape(2, 2, n2 + 1, n1 + 1) - p_o).max() <= TOL
    r = res.report
    assert r["iters"] == iters
    assert rel(r["dual_D"], rep_o.dual_D) <= EREL * 10 or abs(r["dual_D"] - rep_o.dual_D) <= 1e-6
    assert rel(r["primal_E"], rep_o.primal_E) <= EREL
    assert abs(r["gap"] - rep_o.gap) <= 1e-5 * rep_o.primal_E
    assert r["max_p"] <= 1.0 + 1e-6
    assert r["div_res_max"] <= 1e-4


@pytest.mark.parametrize("n2,n1,seed,iters", [(64, 64, 0, 300), (37, 53, 2, 150), (2, 2, 5, 20), (130, 67, 6, 100)])
def test_step2_matches_oracle(B, n2, n1, seed, iters):
    d0 = image(n2, n1, seed)
    tau, _, _ = otvs.tfs(d0, 0.05, 0.125, 60)
    tau32 = tau.astype(np.float32).astype(np.float64)       # both sides see the same FP32 tau
    xi = otvs.normal_field(tau32, n2, n1, 1e-3)
    f2 = otvs.irv1_data(d0.astype(np.float32).astype(np.float64), xi, 10.0)
    d_o, p_o, rep_o = otvs.irv1(f2, 10.0, 0.125, iters)
    p = torch.zeros((2, n2, n1), dtype=torch.float32, device="cuda")
    res = B.tvs_step2(cuda(d0), cuda(tau32), 10.0, 1e-3, B.make_iter(iters), p=p)
    assert np.abs(host(res.out) - d_o).max() <= TOL
    assert np.abs(host(p) - p_o).max() <= TOL
    r = res.report
    assert rel(r["primal_E"], rep_o.primal_E) <= EREL
    assert abs(r["gap"] - rep_o.gap) <= 1e-5 * rep_o.primal_E
    assert r["max_p"] <= 1.0 + 1e-6


def test_denoise_matches_oracle_config1(B):
    # 64x64 scene, sigma 0.1, delta 0.05, alpha 10 (mu 0.1), eps 1e-3, 300 iterations per step
    d0 = image(64, 64, 0)
    d_o, tau_o, r1, r2 = otvs.denoise(d0, 0.05, 10.0, 1e-3, 0.125, 300, 300)
    tau = torch.empty((2, 65, 65), dtype=torch.float32, device="cuda")
    d, _, reps, st = B.tvs_denoise(cuda(d0), 0.05, 10.0, 1e-3, B.make_iter(300), B.make_iter(300), tau=tau)
    assert np.abs(host(tau) - tau_o).max() <= TOL
    assert np.abs(host(d) - d_o).max() <= TOL
    assert rel(reps[0]["primal_E"], r1.primal_E) <= EREL
    assert rel(reps[1]["primal_E"], r2.primal_E) <= EREL


# ---------------------------------------------------------------------------
# edge cases and host logic on the device
# ---------------------------------------------------------------------------
def test_constant_image_is_a_fixed_point(B):
    d0 = np.full((33, 47), 0.4375)       # exactly representable
    d, tau, reps, st = B.tvs_denoise(cuda(d0), 0.05, 10.0, 1e-3, B.make_iter(20), B.make_iter(20),
                                     tau=torch.empty((2, 34, 48), device="cuda"))
    assert torch.count_nonzero(tau).item() == 0
    assert np.abs(host(d) - d0).max() <= 1e-6


def test_warm_start_continues_exactly(B):
    d0 = image(48, 40, 7)
    p = torch.zeros((4, 49, 41), dtype=torch.float32, device="cuda")
    B.tvs_step1(cuda(d0), 0.05, B.make_iter(40), p=p)
    B.tvs_step1(cuda(d0), 0.05, B.make_iter(60), p=p)
    q = torch.zeros_like(p)
    B.tvs_step1(cuda(d0), 0.05, B.make_iter(100), p=q)
    assert torch.equal(p, q)


def test_deterministic(B):
    d0 = cuda(image(100, 120, 8))
    a = B.tvs_step1(d0, 0.05, B.make_iter(30, rel_gap_tol=1e-9, check_every=10))
    b = B.tvs_step1(d0, 0.05, B.make_iter(30, rel_gap_tol=1e-9, check_every=10))
    assert torch.equal(a.out, b.out) and a.report == b.report


def test_gap_stopping(B):
    d0 = cuda(image(64, 64, 9))
    r = B.tvs_step1(d0, 0.05, B.make_iter(5000, rel_gap_tol=1e-3, check_every=10))
    assert r.status == 0
    assert r.report["rel_gap"] <= 1e-3
    assert r.report["iters"] < 5000
    tau = r.out
    r2 = B.tvs_step2(d0, tau, 10.0, 1e-3, B.make_iter(20, rel_gap_tol=1e-12, check_every=5))
    assert r2.status == B.TVS_ERR_NOT_CONVERGED


# ---------------------------------------------------------------------------
# 16-bit storage of the step-2 dual (FP32 arithmetic; stochastic rounding)
# ---------------------------------------------------------------------------
# Bounds on max|d - d_oracle| after 300 updates, each about 2.5x the error
# measured on GB300 (s16 3e-5, f16 4e-4, bf16 2e-3).  The 16-bit fixed point
# on [-1, 1] keeps the FP32 tolerances.
NARROW_TOL = {3: (1e-4, EREL), 2: (1e-3, 5e-5), 1: (5e-3, 1e-3)}
# stored components may sit a few units above 1 (stochastic rounding of a
# value next to the bound); the fixed-point code is clamped to [-1, 1]
NARROW_PMAX = {3: 1.0, 2: 1.0 + 2.0 ** -8, 1: 1.0 + 2.0 ** -5}


@pytest.mark.parametrize("storage", [3, 2, 1])
@pytest.mark.parametrize("decomp", [False, True])
def test_step2_16bit_storage_error_against_oracle(B, storage, decomp):
    n2, n1, iters = 64, 72, 300
    d0 = image(n2, n1, 31, texture=True)
    tau = otvs.tfs(d0, 0.05, 0.125, 40)[0].astype(np.float32).astype(np.float64)
    f2 = otvs.irv1_data(d0.astype(np.float32).astype(np.float64), otvs.normal_field(tau, n2, n1, 1e-3), 10.0)
    p = torch.zeros((2, n2, n1), dtype=torch.float32, device="cuda")
    if decomp:
        dd = osch.Decomp(n2, n1, 2, 2, 4, False)
        d_o, _, rep_o = osch.schwarz_irv1(f2, 10.0, dd, 0.125, 40, 4)
        res = B.tvs_schwarz(2, cuda(d0), cuda(tau), 10.0, 1e-3, B.make_decomp(2, 2, 4, 4),
                            B.make_iter(40, storage=storage), p=p)
    else:
        d_o, _, rep_o = otvs.irv1(f2, 10.0, 0.125, iters)
        res = B.tvs_step2(cuda(d0), cuda(tau), 10.0, 1e-3, B.make_iter(iters, storage=storage), p=p)
    dtol, etol = NARROW_TOL[storage]
    assert np.abs(host(res.out) - d_o).max() <= dtol
    assert rel(res.report["primal_E"], rep_o.primal_E) <= etol
    assert np.abs(host(p)).max() <= NARROW_PMAX[storage]


def test_step2_16bit_storage_is_reproducible(B):
    d0 = cuda(image(96, 80, 32))
    tau = B.tvs_step1(d0, 0.05, B.make_iter(20)).out
    a = B.tvs_step2(d0, tau, 10.0, 1e-3, B.make_iter(50, storage=2)).out
    b = B.tvs_step2(d0, tau, 10.0, 1e-3, B.make_iter(50, storage=2)).out
    assert torch.equal(a, b)


def test_step2_fixed_point_storage_converges_like_fp32(B):
    # stochastic rounding keeps updates below one unit in expectation, so the
    # iteration reaches the gap tolerance in about as many updates as FP32
    d0 = cuda(image(256, 256, 33, texture=True))
    tau = B.tvs_step1(d0, 0.05, B.make_iter(30)).out
    its = {}
    for st in (0, 3):
        r = B.tvs_step2(d0, tau, 10.0, 1e-3, B.make_iter(5000, rel_gap_tol=1e-4, check_every=10, storage=st))
        assert r.status == 0 and r.report["rel_gap"] <= 1e-4
        its[st] = r.report["iters"]
    assert its[3] <= 1.1 * its[0] + 20


# ---------------------------------------------------------------------------
# Schwarz step 2 (Algorithm 2 with Algorithm 3)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n2,n1,m2,m1,s,k,outer", [(48, 40, 2, 2, 4, 5, 20), (64, 64, 4, 4, 8, 4, 10),
                                                   (37, 53, 1, 3, 3, 6, 12), (30, 30, 1, 1, 4, 7, 5),
                                                   (70, 90, 3, 2, 5, 3, 8)])
def test_schwarz2_matches_oracle(B, n2, n1, m2, m1, s, k, outer):
    d0 = image(n2, n1, 11)
    tau, _, _ = otvs.tfs(d0, 0.05, 0.125, 40)
    tau32 = tau.astype(np.float32).astype(np.float64)
    f2 = otvs.irv1_data(d0.astype(np.float32).astype(np.float64), otvs.normal_field(tau32, n2, n1, 1e-3), 10.0)
    dd = osch.Decomp(n2, n1, m2, m1, s, False)
    d_o, p_o, rep_o = osch.schwarz_irv1(f2, 10.0, dd, 0.125, outer, k)
    p = torch.zeros((2, n2, n1), dtype=torch.float32, device="cuda")
    res = B.tvs_schwarz(2, cuda(d0), cuda(tau32), 10.0, 1e-3, B.make_decomp(m2, m1, s, k), B.make_iter(outer), p=p)
    assert np.abs(host(p) - p_o).max() <= TOL
    assert np.abs(host(res.out) - d_o).max() <= TOL
    assert rel(res.report["primal_E"], rep_o.primal_E) <= EREL


@pytest.mark.parametrize("n2,n1,k", [(256, 256, 4), (200, 262, 3)])
def test_schwarz2_64px_tiles_match_oracle(B, n2, n1, k):
    # subdomains of about 64 x 64 with overlap 4: one CTA per subdomain
    m2, m1 = (n2 + 63) // 64, (n1 + 63) // 64
    d0 = image(n2, n1, 14, texture=True)
    tau = otvs.tfs(d0, 0.05, 0.125, 20)[0].astype(np.float32).astype(np.float64)
    f2 = otvs.irv1_data(d0.astype(np.float32).astype(np.float64), otvs.normal_field(tau, n2, n1, 1e-3), 10.0)
    dd = osch.Decomp(n2, n1, m2, m1, 4, False)
    d_o, p_o, rep_o = osch.schwarz_irv1(f2, 10.0, dd, 0.125, 6, k)
    p = torch.zeros((2, n2, n1), dtype=torch.float32, device="cuda")
    res = B.tvs_schwarz(2, cuda(d0), cuda(tau), 10.0, 1e-3, B.make_decomp(m2, m1, 4, k), B.make_iter(6), p=p)
    assert np.abs(host(p) - p_o).max() <= TOL
    assert np.abs(host(res.out) - d_o).max() <= TOL
    assert rel(res.report["primal_E"], rep_o.primal_E) <= EREL


def test_schwarz2_single_subdomain_equals_global(B):
    d0 = image(40, 44, 12)
    tau = cuda(otvs.tfs(d0, 0.05, 0.125, 30)[0])
    g = B.tvs_step2(cuda(d0), tau, 10.0, 1e-3, B.make_iter(24))
    s = B.tvs_schwarz(2, cuda(d0), tau, 10.0, 1e-3, B.make_decomp(1, 1, 0, 6), B.make_iter(4))
    assert torch.abs(g.out - s.out).max().item() <= 1e-6


@pytest.mark.parametrize("n2,n1,m2,m1,s,k,outer", [
    # ~264^2 subdomains: clusters of 14 CTAs of 67 x 5 threads, two CTAs per SM
    (1024, 1024, 4, 4, 8, 4, 3),
    # 250 x 392 subdomains: clusters of 13 CTAs of 99 x 5 threads, one CTA per SM
    (250, 780, 1, 2, 4, 5, 4),
    # 1200 x 102 subdomains: taller than 16 such CTAs -> the shared-memory band kernel
    (1200, 200, 1, 2, 4, 3, 3),
])
def test_schwarz2_large_subdomains_use_clusters(B, n2, n1, m2, m1, s, k, outer):
    # subdomains too large for one CTA span a cluster of CTAs; compare with
    # the oracle after a few outer iterations
    d0 = image(n2, n1, 13, texture=True)
    tau = otvs.tfs(d0, 0.05, 0.125, 5)[0].astype(np.float32).astype(np.float64)
    f2 = otvs.irv1_data(d0.astype(np.float32).astype(np.float64), otvs.normal_field(tau, n2, n1, 1e-3), 10.0)
    dd = osch.Decomp(n2, n1, m2, m1, s, False)
    d_o, p_o, _ = osch.schwarz_irv1(f2, 10.0, dd, 0.125, outer, k)
    p = torch.zeros((2, n2, n1), dtype=torch.float32, device="cuda")
    res = B.tvs_schwarz(2, cuda(d0), cuda(tau), 10.0, 1e-3, B.make_decomp(m2, m1, s, k), B.make_iter(outer), p=p)
    assert np.abs(host(p) - p_o).max() <= TOL
    assert np.abs(host(res.out) - d_o).max() <= TOL


# ---------------------------------------------------------------------------
# full-size launches (the sizes the benchmark times)
# ---------------------------------------------------------------------------
def test_step1_one_iteration_full_size_1024(B):
    n = 1024
    d0 = image(n, n, 21, texture=True)
    rng = np.random.default_rng(5)
    p0 = rng.uniform(-0.7, 0.7, (2, 2, n + 1, n + 1))
    prob = otvs.tfs_problem(d0.astype(np.float32).astype(np.float64), 0.05)
    p0 = p0.astype(np.float32).astype(np.float64)
    p1 = otvs.tfs_step(prob, p0, 0.125)
    tau1 = otvs.tfs_tau(prob, p1)
    p = cuda(p0.reshape(4, n + 1, n + 1))
    res = B.tvs_step1(cuda(d0), 0.05, B.make_iter(1), p=p)
    assert np.abs(host(p).reshape(2, 2, n + 1, n + 1) - p1).max() <= TOL
    assert np.abs(host(res.out) - tau1).max() <= TOL


@pytest.mark.parametrize("n", [4096, 8192])
def test_step2_full_size_window_parity(B, n):
    # After m updates a pixel of p depends only on f2 within distance 2m, so a
    # window padded by 2m + 2 gives the exact oracle values in its centre.
    d0 = image(n, n, 31, texture=True)
    t0 = torch.zeros((2, n + 1, n + 1), dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(1)
    tau_h = (0.2 * rng.standard_normal((2, n + 1, n + 1))).astype(np.float32)
    t0.copy_(torch.from_numpy(tau_h))
    m = 30
    p = torch.zeros((2, n, n), dtype=torch.float32, device="cuda")
    res = B.tvs_step2(cuda(d0), t0, 10.0, 1e-3, B.make_iter(m), p=p)
    ph = host(p)
    assert res.report["max_p"] <= 1.0 + 1e-6
    pad = 2 * m + 2
    for (cy, cx) in [(n // 2, n // 3), (0, 0), (n - 16, n - 16), (5, n // 2)]:
        y0, y1 = max(cy - pad, 0), min(cy + 16 + pad, n)
        x0, x1 = max(cx - pad, 0), min(cx + 16 + pad, n)
        tau_w = tau_h[:, y0:y1 + 1, x0:x1 + 1].astype(np.float64)
        d_w = d0[y0:y1, x0:x1].astype(np.float32).astype(np.float64)
        xi = otvs.normal_field(tau_w, y1 - y0, x1 - x0, 1e-3)
        # div xi must see the true neighbours: build it on a one-pixel larger window
        f2 = 10.0 * d_w - ops.div(xi)
        _, p_w, _ = otvs.irv1(f2, 10.0, 0.125, m)
        iy0 = cy - y0 + (0 if y0 == 0 else 0)
        sl = (slice(None), slice(cy - y0, cy - y0 + 16), slice(cx - x0, cx - x0 + 16))
        ref = p_w[sl]
        got = ph[:, cy:cy + 16, cx:cx + 16]
        # pixels further than 2m+1 from an artificial window edge are exact
        assert np.abs(got - ref).max() <= TOL, (cy, cx, iy0)


# ---------------------------------------------------------------------------
# Schwarz step 1 (Algorithm 2 with the localized Algorithm 5)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n2,n1,m2,m1,s,k,outer", [(14, 12, 2, 2, 2, 3, 5), (40, 36, 2, 3, 4, 4, 6),
                                                   (33, 47, 3, 1, 3, 2, 4), (64, 64, 4, 4, 8, 3, 3)])
def test_schwarz1_matches_oracle(B, n2, n1, m2, m1, s, k, outer):
    d0 = image(n2, n1, 17)
    dd = osch.Decomp(n2, n1, m2, m1, s, True)
    tau_o, p_o, rep_o = osch.schwarz_tfs(d0.astype(np.float32).astype(np.float64), 0.05, dd, 0.125, outer, k)
    p = torch.zeros((4, n2 + 1, n1 + 1), dtype=torch.float32, device="cuda")
    res = B.tvs_schwarz(1, cuda(d0), None, 0.05, 1e-3, B.make_decomp(m2, m1, s, k), B.make_iter(outer), p=p)
    assert np.abs(host(p).reshape(2, 2, n2 + 1, n1 + 1) - p_o).max() <= TOL
    assert np.abs(host(res.out) - tau_o).max() <= TOL
    assert rel(res.report["primal_E"], rep_o.primal_E) <= EREL


def test_schwarz1_single_subdomain_equals_global(B):
    d0 = cuda(image(30, 26, 18))
    g = B.tvs_step1(d0, 0.05, B.make_iter(12))
    s = B.tvs_schwarz(1, d0, None, 0.05, 1e-3, B.make_decomp(1, 1, 0, 4), B.make_iter(3))
    assert torch.abs(g.out - s.out).max().item() <= 2e-6


@pytest.mark.parametrize("n,k", [(8192, 4), (2048, 16)])
def test_schwarz2_full_size_reaches_global_minimiser(B, n, k):
    # Strong convexity of the primal (Appendix A) certifies ||d - d*|| <= sqrt(2 gap / alpha);
    # both runs stop on their own duality gap, so their distance is bounded by the sum.
    d0 = cuda(image(n, n, 41, texture=True))
    tau = B.tvs_step1(d0, 0.05, B.make_iter(30)).out
    g = B.tvs_step2(d0, tau, 10.0, 1e-3, B.make_iter(20000, rel_gap_tol=2e-5, check_every=50))
    s = B.tvs_schwarz(2, d0, tau, 10.0, 1e-3, B.make_decomp(n // 64, n // 64, 4, k),
                      B.make_iter(20000, rel_gap_tol=2e-5, check_every=max(1, 50 // k)))
    assert g.status == 0 and s.status == 0
    # |q| <= theta holds exactly only in exact arithmetic: once t|psi| drops below
    # half an ulp of theta the FP32 denominator rounds to theta while q still
    # moves by t psi, so each inner update may overshoot by about one ulp.
    assert s.report["max_p"] <= 1.0 + 1.2e-7 * s.report["iters"] * k
    dist = torch.linalg.vector_norm((g.out - s.out).double()).item()
    bound = np.sqrt(2 * g.report["gap"] / 10.0) + np.sqrt(2 * s.report["gap"] / 10.0)
    assert dist <= bound * 1.05 + 1e-6 * n, (dist, bound)   # + FP32 rounding of d


# ---------------------------------------------------------------------------
# quality measures (Section 5.3)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n2,n1", [(64, 64), (257, 130), (1024, 1024)])
def test_quality_matches_oracle(B, n2, n1):
    import oracle.quality as oq
    clean, noisy = noisy_scene(SceneSpec(n2, n1, 7, 0.1, True))
    d = noisy.astype(np.float32)
    gt = clean.astype(np.float32)
    ps, ms = B.tvs_quality(cuda(d), cuda(gt))
    assert ps == pytest.approx(oq.psnr(d, gt), rel=1e-6)
    assert ms == pytest.approx(oq.mssim(d, gt), rel=1e-6)
    ps2, ms2 = B.tvs_quality(cuda(gt), cuda(gt))
    assert ps2 == float("inf") and ms2 == pytest.approx(1.0, abs=1e-6)
