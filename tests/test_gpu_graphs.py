"""Graph replay of the iteration runs: the cached CUDA graphs make exactly
the launches the drivers would make, so every result is bit-identical with
graphs on (first call: capture; second call: cache hit) and off."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import SceneSpec, noisy_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_17494_gb300 import build
    build.build()
    from paper_2602_17494_gb300 import binding
    return binding


def image(n2, n1, seed):
    return torch.from_numpy(noisy_scene(SceneSpec(n2, n1, seed, 0.1, True))[1].astype(np.float32)).cuda()


def three_ways(B, fn):
    """fn() with graphs off, then twice with graphs on (capture, then replay)."""
    prev = B.tvs_set_graphs(False)
    try:
        ref = fn()
        B.tvs_set_graphs(True)
        first = fn()
        second = fn()
    finally:
        B.tvs_set_graphs(prev)
    return ref, first, second


def same(a, b):
    return torch.equal(a, b)


@pytest.mark.parametrize("n2,n1", [(96, 130), (257, 200)])
def test_step1_graph_runs_are_bit_identical(B, n2, n1):
    d0 = image(n2, n1, 71)
    # checks every 10 updates (never converged): runs of 10 and 8 plain updates
    it = B.make_iter(57, 0.125, 1e-12, 10)

    def fn():
        r = B.tvs_step1(d0, 0.05, it)
        return r.out.clone(), r.report["iters"]

    (a, ia), (b, ib), (c, ic) = three_ways(B, fn)
    assert same(a, b) and same(a, c)
    assert ia == ib == ic == 57


def test_step2_graph_runs_are_bit_identical(B):
    d0 = image(180, 211, 72)
    tau = B.tvs_step1(d0, 0.05, B.make_iter(20)).out
    it = B.make_iter(131, 0.125, 0.0, 0)       # one plain run of 64, 64 and the rest

    def fn():
        return B.tvs_step2(d0, tau, 10.0, 1e-3, it).out.clone()

    a, b, c = three_ways(B, fn)
    assert same(a, b) and same(a, c)


@pytest.mark.parametrize("m,k", [(3, 4), (1, 6)])
def test_schwarz2_graph_runs_are_bit_identical(B, m, k):
    d0 = image(200, 180, 73)
    tau = B.tvs_step1(d0, 0.05, B.make_iter(20)).out
    dd = B.make_decomp(m, m, 4, k)
    it = B.make_iter(13, 0.125, 1e-12, 4)      # runs of 4 outer iterations between checks

    def fn():
        return B.tvs_schwarz(2, d0, tau, 10.0, 1e-3, dd, it).out.clone()

    a, b, c = three_ways(B, fn)
    assert same(a, b) and same(a, c)


def test_denoise_graph_runs_are_bit_identical(B):
    d0 = image(128, 128, 74)
    dd = B.make_decomp(2, 2, 4, 5)

    def fn():
        return B.tvs_denoise(d0, 0.05, 10.0, 1e-3, B.make_iter(30), B.make_iter(8), dd)[0].clone()

    a, b, c = three_ways(B, fn)
    assert same(a, b) and same(a, c)
