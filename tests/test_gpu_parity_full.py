"""GPU parity at the sizes and in the configurations the benchmark runs.

* tvs_denoise with the step-2 Schwarz decomposition (the benchmarked call) on
  the 1024 x 1024 textured scene, 4 x 4 subdomains, overlap 8, k = 10;
* many global TFS updates at 1024^2 and a few at 4096^2 (16384-point
  Bluestein rows at 8192^2 are covered by the projection at 8193 x 8193);
* Schwarz step 1 (Algorithm 5) on 256^2 with 4 x 4 subdomains;
* the 16-bit dual formats at 512^2;
* the chunked tridiagonal column pass (long columns) in the projection.
Tolerances as in test_gpu_parity.py: 1e-4 max-abs on tau, d and p, energies
within a relative 1e-6.
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


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def test_benchmarked_denoise_with_schwarz_matches_oracle(B):
    # the benchmark's call on its 1024^2 scene with fewer iterations: TFS
    # (Algorithm 1), xi and f2, then Algorithm 2 with Algorithm 3
    n, it1, outer = 1024, 20, 3
    d0 = f32(image(n, n, 0, 0.1, True))
    tau_o, _, r1 = otvs.tfs(d0, 0.05, 0.125, it1)
    f2 = otvs.irv1_data(d0, otvs.normal_field(tau_o, n, n, 1e-3), 10.0)
    dd = osch.Decomp(n, n, 4, 4, 8, False)
    d_o, _, r2 = osch.schwarz_irv1(f2, 10.0, dd, 0.125, outer, 10)
    tau = torch.empty((2, n + 1, n + 1), dtype=torch.float32, device="cuda")
    d, _, reps, st = B.tvs_denoise(cuda(d0), 0.05, 10.0, 1e-3, B.make_iter(it1), B.make_iter(outer),
                                   B.make_decomp(4, 4, 8, 10), tau=tau)
    assert st == 0
    assert np.abs(host(tau) - tau_o).max() <= TOL
    assert np.abs(host(d) - d_o).max() <= TOL
    assert rel(reps[0]["primal_E"], r1.primal_E) <= EREL
    assert rel(reps[1]["primal_E"], r2.primal_E) <= EREL


def test_step1_many_updates_full_size_1024(B):
    n, iters = 1024, 24
    d0 = f32(image(n, n, 21, texture=True))
    tau_o, p_o, rep_o = otvs.tfs(d0, 0.05, 0.125, iters)
    p = torch.zeros((4, n + 1, n + 1), dtype=torch.float32, device="cuda")
    res = B.tvs_step1(cuda(d0), 0.05, B.make_iter(iters), p=p)
    assert np.abs(host(res.out) - tau_o).max() <= TOL
    assert np.abs(host(p).reshape(2, 2, n + 1, n + 1) - p_o).max() <= TOL
    assert rel(res.report["primal_E"], rep_o.primal_E) <= EREL
    assert abs(res.report["gap"] - rep_o.gap) <= 1e-5 * rep_o.primal_E


def test_step1_full_size_4096(B):
    # 4097^2 extended grid: 8192-point Bluestein rows and the chunked column pass
    n, iters = 4096, 2
    d0 = f32(image(n, n, 22, texture=True))
    tau_o, p_o, rep_o = otvs.tfs(d0, 0.05, 0.125, iters)
    p = torch.zeros((4, n + 1, n + 1), dtype=torch.float32, device="cuda")
    res = B.tvs_step1(cuda(d0), 0.05, B.make_iter(iters), p=p)
    assert np.abs(host(res.out) - tau_o).max() <= TOL
    assert np.abs(host(p).reshape(2, 2, n + 1, n + 1) - p_o).max() <= TOL
    assert rel(res.report["primal_E"], rep_o.primal_E) <= EREL


def test_step1_full_size_8192_invariants(B):
    # the benchmark's step-1 size: the divergence-free constraint, feasibility,
    # a non-negative gap and a dual energy that does not increase
    n = 8192
    d0 = cuda(image(n, n, 23, texture=True))
    p = torch.zeros((4, n + 1, n + 1), dtype=torch.float32, device="cuda")
    last = None
    for _ in range(3):
        r = B.tvs_step1(d0, 0.05, B.make_iter(4), p=p)
        assert r.report["max_p"] <= 1.0 + 1e-6
        assert r.report["gap"] >= -1e-6 * r.report["primal_E"]
        assert r.report["div_res_max"] <= 1e-3
        if last is not None:
            assert r.report["dual_D"] <= last * (1 + 1e-6)
        last = r.report["dual_D"]


@pytest.mark.parametrize("shape", [(1537, 40), (1601, 97), (2049, 2049), (3000, 70), (8193, 8193)])
def test_projection_long_columns_match_oracle(B, shape):
    # columns of at least 1537 rows go through the chunked column pass
    rng = np.random.default_rng(sum(shape) + 1)
    tau = rng.standard_normal((2,) + shape).astype(np.float32).astype(np.float64)
    out = host(B.tvs_project(cuda(tau)))
    ref = ops.proj_k(tau)
    scale = np.abs(tau).max()
    assert np.abs(out - ref).max() <= 2e-5 * scale
    assert np.abs(ops.div(out)).max() <= 2e-5 * scale


def test_schwarz1_4x4_on_256(B):
    n2 = n1 = 256
    d0 = f32(image(n2, n1, 24, texture=True))
    dd = osch.Decomp(n2, n1, 4, 4, 8, True)
    tau_o, p_o, rep_o = osch.schwarz_tfs(d0, 0.05, dd, 0.125, 3, 3)
    p = torch.zeros((4, n2 + 1, n1 + 1), dtype=torch.float32, device="cuda")
    res = B.tvs_schwarz(1, cuda(d0), None, 0.05, 1e-3, B.make_decomp(4, 4, 8, 3), B.make_iter(3), p=p)
    assert np.abs(host(p).reshape(2, 2, n2 + 1, n1 + 1) - p_o).max() <= TOL
    assert np.abs(host(res.out) - tau_o).max() <= TOL
    assert rel(res.report["primal_E"], rep_o.primal_E) <= EREL


# error bounds of the 16-bit formats as in test_gpu_parity.py (S16 keeps the FP32 bounds)
NARROW_TOL = {3: (1e-4, EREL), 2: (1e-3, 5e-5)}


@pytest.mark.parametrize("storage", [3, 2])
@pytest.mark.parametrize("decomp", [False, True])
def test_step2_16bit_formats_at_512(B, storage, decomp):
    n2, n1 = 512, 520
    d0 = f32(image(n2, n1, 25, texture=True))
    tau = f32(otvs.tfs(d0, 0.05, 0.125, 10)[0])
    f2 = otvs.irv1_data(d0, otvs.normal_field(tau, n2, n1, 1e-3), 10.0)
    p = torch.zeros((2, n2, n1), dtype=torch.float32, device="cuda")
    if decomp:
        m2, m1 = n2 // 64, (n1 + 63) // 64
        dd = osch.Decomp(n2, n1, m2, m1, 4, False)
        d_o, _, rep_o = osch.schwarz_irv1(f2, 10.0, dd, 0.125, 10, 8)
        res = B.tvs_schwarz(2, cuda(d0), cuda(tau), 10.0, 1e-3, B.make_decomp(m2, m1, 4, 8),
                            B.make_iter(10, storage=storage), p=p)
    else:
        d_o, _, rep_o = otvs.irv1(f2, 10.0, 0.125, 300)
        res = B.tvs_step2(cuda(d0), cuda(tau), 10.0, 1e-3, B.make_iter(300, storage=storage), p=p)
    dtol, etol = NARROW_TOL[storage]
    assert np.abs(host(res.out) - d_o).max() <= dtol
    assert rel(res.report["primal_E"], rep_o.primal_E) <= etol
    assert np.abs(host(p)).max() <= 1.0 + 2.0 ** -8


# ---------------------------------------------------------------------------
# 16-bit storage of the step-1 dual (and of tau kept inside tvs_denoise)
# ---------------------------------------------------------------------------
# bounds on max|tau - tau_oracle| and the relative primal energy after 300 updates
STEP1_NARROW = {3: (1e-4, EREL), 2: (1e-3, 5e-5), 1: (5e-3, 1e-3)}


@pytest.mark.parametrize("storage", [3, 2, 1])
def test_step1_16bit_storage_error_against_oracle(B, storage):
    n2, n1, iters = 64, 72, 300
    d0 = f32(image(n2, n1, 26, texture=True))
    tau_o, _, rep_o = otvs.tfs(d0, 0.05, 0.125, iters)
    p = torch.zeros((4, n2 + 1, n1 + 1), dtype=torch.float32, device="cuda")
    res = B.tvs_step1(cuda(d0), 0.05, B.make_iter(iters, storage=storage), p=p)
    ttol, etol = STEP1_NARROW[storage]
    assert np.abs(host(res.out) - tau_o).max() <= ttol
    assert rel(res.report["primal_E"], rep_o.primal_E) <= etol
    assert res.report["div_res_max"] <= 1e-4
    assert np.abs(host(p)).max() <= 1.0 + 2.0 ** -5


@pytest.mark.parametrize("storage", [3, 2, 1])
def test_denoise_16bit_step1_and_tau(B, storage):
    # tvs_denoise with a 16-bit step-1 dual and no tau buffer keeps tau in 16
    # bits (FP16, or BF16 for a BF16 dual); d against the FP64 pipeline
    n, it = 64, 200
    d0 = f32(image(n, n, 27, texture=True))
    d_o, _, _, r2 = otvs.denoise(d0, 0.05, 10.0, 1e-3, 0.125, it, it)
    d, _, reps, st = B.tvs_denoise(cuda(d0), 0.05, 10.0, 1e-3, B.make_iter(it, storage=storage), B.make_iter(it))
    dtol = {3: 2e-4, 2: 1e-3, 1: 5e-3}[storage]
    assert np.abs(host(d) - d_o).max() <= dtol
    assert rel(reps[1]["primal_E"], r2.primal_E) <= 10 * STEP1_NARROW[storage][1]


def test_step1_16bit_is_reproducible_and_converges(B):
    d0 = cuda(image(256, 256, 28, texture=True))
    a = B.tvs_step1(d0, 0.05, B.make_iter(40, storage=3)).out
    b = B.tvs_step1(d0, 0.05, B.make_iter(40, storage=3)).out
    assert torch.equal(a, b)
    its = {}
    for st in (0, 3):
        r = B.tvs_step1(d0, 0.05, B.make_iter(5000, rel_gap_tol=1e-4, check_every=10, storage=st))
        assert r.status == 0 and r.report["rel_gap"] <= 1e-4
        its[st] = r.report["iters"]
    assert its[3] <= 1.1 * its[0] + 20
