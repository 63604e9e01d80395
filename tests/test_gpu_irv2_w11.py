"""IRV2 (Section 3.3, eq. ir2dualdis) and the W^{1,1} dual (eq. IRW11:dual)
on the GPU against the FP64 oracle (oracle.tvs.irv2, oracle.tvs.w11), at equal
iteration counts; tolerances as in test_gpu_parity.py."""
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


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def image(n2, n1, seed=0, sigma=0.1, texture=False):
    return f32(noisy_scene(SceneSpec(n2, n1, seed, sigma, texture))[1])


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.mark.parametrize("n2,n1,seed,iters", [(64, 64, 0, 300), (37, 53, 2, 150), (3, 5, 4, 20), (130, 67, 6, 100)])
def test_irv2_matches_oracle(B, n2, n1, seed, iters):
    d0 = image(n2, n1, seed)
    tau = f32(otvs.tfs(d0, 0.05, 0.125, 60)[0])
    d_o, p_o, rep_o, g_o = otvs.irv2(d0, tau, 10.0, 0.125, iters)
    p = torch.zeros((2, n2, n1), dtype=torch.float32, device="cuda")
    d, g, rep, st = B.tvs_irv2(cuda(d0), cuda(tau), 10.0, B.make_iter(iters), p=p)
    assert st == 0
    assert np.abs(host(g) - g_o).max() <= TOL
    assert np.abs(host(d) - d_o).max() <= TOL
    assert np.abs(host(p) - p_o).max() <= TOL
    assert rel(rep["primal_E"], rep_o.primal_E) <= EREL
    assert abs(rep["gap"] - rep_o.gap) <= 1e-5 * rep_o.primal_E


def test_irv2_at_4096(B):
    # The potential's Poisson solve on a 4096^2 image grid (chunked column
    # pass).  tau is the scene's own tangent field plus noise, so g is
    # image-like with an inconsistent part.  g's lowest frequencies carry the
    # FP32 rounding of the transforms amplified by 1/lambda_min (about 1.7e6
    # at this size): an FP32 DCT solve of the same data on the CPU
    # (scipy.fft in float32) is 1.9e-4 off the FP64 potential, so g is held
    # to 4e-4.  In d = u + g that smooth error cancels (u absorbs it), and d
    # is held to the 1e-4 of every result.
    n, iters = 4096, 20
    rng = np.random.default_rng(8)
    d0 = image(n, n, 9, texture=True)
    tau = f32(ops.tangent(d0) + 0.02 * rng.standard_normal((2, n + 1, n + 1)))
    d_o, _, rep_o, g_o = otvs.irv2(d0, tau, 10.0, 0.125, iters)
    d, g, rep, st = B.tvs_irv2(cuda(d0), cuda(tau), 10.0, B.make_iter(iters))
    assert np.abs(host(g) - g_o).max() <= 4e-4
    assert np.abs(host(d) - d_o).max() <= TOL
    # the energy is that of u = d - g, which carries g's smooth error into TV(u)
    assert rel(rep["primal_E"], rep_o.primal_E) <= 5 * EREL


def test_irv2_of_the_images_own_tangent_field_returns_the_image(B):
    n2, n1 = 96, 80
    d0 = image(n2, n1, 10)
    tau0 = f32(ops.tangent(d0))
    d, g, rep, st = B.tvs_irv2(cuda(d0), cuda(tau0), 10.0, B.make_iter(50))
    assert np.abs(host(g) - (d0 - d0.mean())).max() <= 1e-5
    assert np.abs(host(d) - d0).max() <= 1e-5


def test_irv2_under_schwarz_matches_oracle(B):
    n2, n1, k, outer = 128, 136, 4, 6
    d0 = image(n2, n1, 11, texture=True)
    tau = f32(otvs.tfs(d0, 0.05, 0.125, 40)[0])
    g_o = otvs.potential(tau, n2, n1)
    dd = osch.Decomp(n2, n1, 2, 2, 4, False)
    u_o, p_o, rep_o = osch.schwarz_irv1(otvs.irv2_data(d0, g_o, 10.0), 10.0, dd, 0.125, outer, k)
    p = torch.zeros((2, n2, n1), dtype=torch.float32, device="cuda")
    d, g, rep, st = B.tvs_irv2(cuda(d0), cuda(tau), 10.0, B.make_iter(outer), B.make_decomp(2, 2, 4, k), p=p)
    assert np.abs(host(d) - (u_o + g_o)).max() <= TOL
    assert np.abs(host(p) - p_o).max() <= TOL
    assert rel(rep["primal_E"], rep_o.primal_E) <= EREL


@pytest.mark.parametrize("n2,n1,seed,iters", [(64, 72, 0, 300), (37, 53, 3, 120), (130, 67, 5, 100)])
def test_w11_matches_oracle(B, n2, n1, seed, iters):
    d0 = image(n2, n1, seed)
    tau = f32(otvs.tfs(d0, 0.05, 0.125, 60)[0])
    xi = otvs.normal_field(tau, n2, n1, 1e-3)
    d_o, p_o, rep_o = otvs.w11(d0, xi, 10.0, 0.125, iters)
    d, p, rep, st = B.tvs_step2_w11(cuda(d0), cuda(tau), 10.0, 1e-3, B.make_iter(iters))
    assert st == 0
    assert np.abs(host(d) - d_o).max() <= TOL
    assert np.abs(host(p) - p_o).max() <= TOL
    assert rel(rep["primal_E"], rep_o.primal_E) <= EREL
    # the shifted ball |p - xi| <= 1 of eq. IRW11:dual
    ph = host(p)
    assert np.sqrt((ph[0] - xi[0]) ** 2 + (ph[1] - xi[1]) ** 2).max() <= 1.0 + 1e-5
    # and d equals the IRV1 result of tvs_step2
    r2 = B.tvs_step2(cuda(d0), cuda(tau), 10.0, 1e-3, B.make_iter(iters))
    assert torch.equal(r2.out, d)


def test_w11_warm_start(B):
    n2, n1 = 48, 56
    d0 = image(n2, n1, 7)
    tau = cuda(f32(otvs.tfs(d0, 0.05, 0.125, 30)[0]))
    _, p1, _, _ = B.tvs_step2_w11(cuda(d0), tau, 10.0, 1e-3, B.make_iter(40))
    d2, p2, _, _ = B.tvs_step2_w11(cuda(d0), tau, 10.0, 1e-3, B.make_iter(60), p0=p1.clone())
    d3, p3, _, _ = B.tvs_step2_w11(cuda(d0), tau, 10.0, 1e-3, B.make_iter(100))
    assert torch.abs(p2 - p3).max().item() <= 1e-5
    assert torch.abs(d2 - d3).max().item() <= 1e-5
