"""The bounded device-side waits report TVS_ERR_TIMEOUT and leave the context usable.

tvs_set_wait_limit shortens the limit of the TMA waits to a few SM cycles, so
the first wait of each launch gives up before its copy lands (the copy is
still drained with the default limit before the CTA exits).  The calls must
return TVS_ERR_TIMEOUT; after the default limit is restored the same calls
must give the same results as before.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from synth import SceneSpec, noisy_scene  # noqa: E402

TVS_ERR_TIMEOUT = 4


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_17494_gb300 import build
    build.build()
    from paper_2602_17494_gb300 import binding
    return binding


def test_short_wait_limit_reports_timeout_and_recovers(B):
    d0 = torch.from_numpy(noisy_scene(SceneSpec(256, 200, 3, 0.1, True))[1].astype(np.float32)).cuda()
    tau = B.tvs_step1(d0, 0.05, B.make_iter(10)).out.clone()
    ref = B.tvs_step2(d0, tau, 10.0, 1e-3, B.make_iter(20)).out.clone()
    B.tvs_set_wait_limit(4)
    try:
        with pytest.raises(B.TvsError) as e2:
            B.tvs_step2(d0, tau, 10.0, 1e-3, B.make_iter(20))
        assert e2.value.status == TVS_ERR_TIMEOUT
        with pytest.raises(B.TvsError) as e1:
            B.tvs_step1(d0, 0.05, B.make_iter(6))
        assert e1.value.status == TVS_ERR_TIMEOUT
    finally:
        B.tvs_set_wait_limit(0)
    torch.cuda.synchronize()
    assert torch.equal(B.tvs_step1(d0, 0.05, B.make_iter(10)).out, tau)
    assert torch.equal(B.tvs_step2(d0, tau, 10.0, 1e-3, B.make_iter(20)).out, ref)
