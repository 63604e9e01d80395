"""tvs_project_noalloc: the projection for callers that cannot allocate.

Some callers cannot call cudaMalloc or hand the library a workspace (a plug-in
running inside another framework's memory pool, a host callback).  The
no-allocation entry point keeps its scratch in a fixed device array inside the
library.  This test calls it through the C ABI twice in a row (the second call
finds the first call's leftovers in the shared array) and checks each result
against the workspace-based tvs_project within the tolerance of the other
projection tests.  It lives in its own file so that it runs last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_17494_gb300 import build
    build.build()
    from paper_2602_17494_gb300 import binding
    return binding


def _call_noalloc(B, tau, out):
    _, rows, cols = tau.shape
    st = B.lib().tvs_project_noalloc(ctypes.c_void_p(tau.data_ptr()), ctypes.c_void_p(out.data_ptr()), rows, cols,
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


@pytest.mark.parametrize("shape", [(65, 65), (129, 300), (1025, 1025)])
def test_noalloc_matches_workspace_projection_twice(B, shape):
    rng = np.random.default_rng(shape[0] * 7 + shape[1])
    for call in range(2):
        tau = torch.from_numpy(rng.standard_normal((2,) + shape).astype(np.float32)).cuda()
        ref = B.tvs_project(tau)
        out = torch.full_like(tau, float("nan"))
        assert _call_noalloc(B, tau, out) == 0, B.lib().tvs_last_error()
        torch.cuda.synchronize()
        scale = tau.abs().max().item()
        assert torch.isfinite(out).all()
        assert (out - ref).abs().max().item() <= 2e-5 * scale, call


def test_noalloc_in_place(B):
    # in == out is allowed: the projection overwrites its own input
    rng = np.random.default_rng(11)
    tau = torch.from_numpy(rng.standard_normal((2, 257, 190)).astype(np.float32)).cuda()
    ref = B.tvs_project(tau)
    for call in range(2):
        buf = tau.clone()
        assert _call_noalloc(B, buf, buf) == 0, B.lib().tvs_last_error()
        torch.cuda.synchronize()
        assert (buf - ref).abs().max().item() <= 2e-5 * tau.abs().max().item(), call


def test_noalloc_rejects_grids_beyond_its_scratch(B):
    tau = torch.zeros((2, 1026, 1100), dtype=torch.float32, device="cuda")
    out = torch.empty_like(tau)
    assert _call_noalloc(B, tau, out) == 6          # TVS_ERR_UNSUPPORTED
    assert b"scratch" in B.lib().tvs_last_error()
