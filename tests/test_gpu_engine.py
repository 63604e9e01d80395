"""Batching / serving engine (tvs_engine_*): shared launches, admission by the
device-memory budget, and per-request results that do not depend on the mix."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle.schwarz as osch
import oracle.tvs as otvs
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


def image(n2, n1, seed, sigma=0.1):
    return noisy_scene(SceneSpec(n2, n1, seed, sigma, True))[1]


def cfg(B, it1=(40, 20), it2=(6, 3), storage=0, tile=32, overlap=4, k=4, max_live=16):
    # rel_gap_tol 0: every request stops at max_iter, so runs are comparable
    return B.make_engine_config(0.05, 10.0, 1e-3, B.make_iter(it1[0], 0.125, 0.0, it1[1]),
                                B.make_iter(it2[0], 0.125, 0.0, it2[1], storage=storage), tile, overlap, k, max_live)


def run(B, c, imgs, pool=1 << 30, stagger=False):
    eng = B.Engine(c, pool)
    outs, reps = {}, {}
    pending = list(enumerate(imgs))
    if not stagger:
        for i, im in pending:
            eng.submit(i, torch.from_numpy(im.astype(np.float32)).cuda())
        pending = []
    steps = 0
    while eng.pending() or pending:
        if pending:                           # one new arrival per engine step
            i, im = pending.pop(0)
            eng.submit(i, torch.from_numpy(im.astype(np.float32)).cuda())
        for rid, d, r1, r2 in eng.step():
            outs[rid] = d.cpu().numpy()
            reps[rid] = (r1, r2)
        steps += 1
        assert steps < 1000
    eng.close()
    return outs, reps


SIZES = [(64, 80), (100, 70), (130, 131), (47, 200), (96, 96)]


def test_engine_result_same_alone_and_in_mix(B):
    imgs = [image(n2, n1, 50 + i) for i, (n2, n1) in enumerate(SIZES)]
    c = cfg(B)
    mix, rmix = run(B, c, imgs)
    mix2, _ = run(B, c, imgs, stagger=True)
    for i, im in enumerate(imgs):
        alone, ralone = run(B, c, [im])
        assert np.array_equal(alone[0], mix[i]), i
        assert np.array_equal(alone[0], mix2[i]), i
        assert ralone[0][1]["iters"] == rmix[i][1]["iters"]


def test_engine_matches_single_image_calls(B):
    imgs = [image(n2, n1, 60 + i) for i, (n2, n1) in enumerate(SIZES[:3])]
    outs, reps = run(B, cfg(B), imgs)
    for i, im in enumerate(imgs):
        n2, n1 = im.shape
        d0 = torch.from_numpy(im.astype(np.float32)).cuda()
        tau = B.tvs_step1(d0, 0.05, B.make_iter(40)).out
        dd = B.make_decomp(max(1, (n2 + 31) // 32), max(1, (n1 + 31) // 32), 4, 4)
        ref = B.tvs_schwarz(2, d0, tau, 10.0, 1e-3, dd, B.make_iter(6)).out.cpu().numpy()
        assert np.abs(outs[i] - ref).max() <= 1e-6
        assert reps[i][0]["iters"] == 39 and reps[i][1]["iters"] == 6


def test_engine_matches_oracle(B):
    n2, n1 = 48, 56
    im = image(n2, n1, 70)
    outs, _ = run(B, cfg(B), [im])
    d0 = im.astype(np.float32).astype(np.float64)
    tau = otvs.tfs(d0, 0.05, 0.125, 40)[0].astype(np.float32).astype(np.float64)
    f2 = otvs.irv1_data(d0, otvs.normal_field(tau, n2, n1, 1e-3), 10.0)
    dd = osch.Decomp(n2, n1, 2, 2, 4, False)
    d_o, _, _ = osch.schwarz_irv1(f2, 10.0, dd, 0.125, 6, 4)
    assert np.abs(outs[0] - d_o).max() <= 1e-4


def test_engine_admits_by_memory_budget(B):
    imgs = [image(96, 96, 80 + i) for i in range(5)]
    c = cfg(B)
    eng = B.Engine(c, 1 << 20)
    one = eng.request_bytes(96, 96)
    eng.close()
    # room for two requests at a time: all five still finish, with the same results
    pool = B.lib().tvs_engine_pool_overhead(c) + 2 * one + 4096
    small, _ = run(B, c, imgs, pool=pool)
    big, _ = run(B, c, imgs)
    for i in range(5):
        assert np.array_equal(small[i], big[i])
    eng = B.Engine(c, pool)
    with pytest.raises(B.TvsError):          # could never fit
        eng.submit(0, torch.zeros((1024, 1024), device="cuda"))
    eng.close()


def test_engine_16bit_storage_close_to_fp32(B):
    imgs = [image(n2, n1, 90 + i) for i, (n2, n1) in enumerate(SIZES[:3])]
    f32, _ = run(B, cfg(B), imgs)
    s16, _ = run(B, cfg(B, storage=3), imgs)
    for i in range(3):
        assert np.abs(f32[i] - s16[i]).max() <= 1e-4


def test_autotuner_picks_a_converging_candidate(B):
    d0 = torch.from_numpy(image(160, 192, 95).astype(np.float32)).cuda()
    tau = B.tvs_step1(d0, 0.05, B.make_iter(30)).out
    it = B.make_iter(400, 0.125, 1e-4, 2)
    (tile, s, k), ms = B.tvs_tune_schwarz2(d0, tau, 10.0, 1e-3, it, tiles=(32, 64), overlaps=(2, 4), ks=(4, 16))
    assert tile in (32, 64) and s in (2, 4) and k in (4, 16) and ms > 0
    dd = B.make_decomp((160 + tile - 1) // tile, (192 + tile - 1) // tile, s, k)
    r = B.tvs_schwarz(2, d0, tau, 10.0, 1e-3, dd, it)
    assert r.status == 0 and r.report["rel_gap"] <= 1e-4


def test_engine_graph_replay_matches_direct_launches(B):
    # an even check interval: the step-2 chunk of a set of requests is
    # captured into a CUDA graph the second time the set comes round and then
    # replayed; results must equal direct launches bit for bit (FP32 and the
    # fixed-point dual, whose rounding seeds come from a device counter)
    imgs = [image(n2, n1, 100 + i) for i, (n2, n1) in enumerate(SIZES[:4])]
    for storage in (0, 3):
        c = cfg(B, it2=(12, 2), storage=storage)
        on, ron = run(B, c, imgs)
        prev = B.tvs_set_graphs(False)
        try:
            off, roff = run(B, c, imgs)
        finally:
            B.tvs_set_graphs(prev)
        for i in range(len(imgs)):
            assert np.array_equal(on[i], off[i]), (storage, i)
            assert ron[i][1]["iters"] == roff[i][1]["iters"] == 12
    outs, _ = run(B, cfg(B, it2=(12, 2)), imgs)
    for i, im in enumerate(imgs):
        n2, n1 = im.shape
        d0 = torch.from_numpy(im.astype(np.float32)).cuda()
        tau = B.tvs_step1(d0, 0.05, B.make_iter(40)).out
        dd = B.make_decomp(max(1, (n2 + 31) // 32), max(1, (n1 + 31) // 32), 4, 4)
        ref = B.tvs_schwarz(2, d0, tau, 10.0, 1e-3, dd, B.make_iter(12)).out.cpu().numpy()
        assert np.abs(outs[i] - ref).max() <= 1e-6
