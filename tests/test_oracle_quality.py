"""Pins of the quality measures (oracle/quality.py, Section 5.3)."""
import numpy as np
import pytest

import oracle.quality as q
from synth import SceneSpec, noisy_scene


def test_psnr_of_constant_offset():
    gt = noisy_scene(SceneSpec(20, 30, 1, 0.1, False))[0]
    for c in (0.1, 0.01, 0.25):
        assert q.psnr(gt + c, gt) == pytest.approx(-20 * np.log10(c), rel=1e-12)
    assert q.psnr(gt, gt) == float("inf")


def test_mssim_identity_and_symmetry():
    clean, noisy = noisy_scene(SceneSpec(24, 17, 2, 0.1, True))
    assert q.mssim(clean, clean) == pytest.approx(1.0, abs=1e-15)
    assert q.mssim(noisy, clean) == pytest.approx(q.mssim(clean, noisy), rel=1e-14)
    assert q.mssim(noisy, clean) < 1.0


def test_mssim_affine_closed_form():
    # d = a gt + b: m_d = a m + b, s_d^2 = a^2 s^2, s_dg = a s^2
    gt = noisy_scene(SceneSpec(16, 21, 3, 0.1, True))[0]
    m, s2 = gt.mean(), gt.var()
    c1, c2 = 1e-4, 9e-4
    for a, b in ((1.0, 0.05), (0.7, 0.1), (1.3, -0.2)):
        md = a * m + b
        want = (2 * md * m + c1) * (2 * a * s2 + c2) / ((md ** 2 + m ** 2 + c1) * (a * a * s2 + s2 + c2))
        assert q.mssim(a * gt + b, gt) == pytest.approx(want, rel=1e-12)


def test_against_brute_force_loops():
    rng = np.random.default_rng(4)
    d, gt = rng.random((5, 7)), rng.random((5, 7))
    n = d.size
    se = sum((d[i, j] - gt[i, j]) ** 2 for i in range(5) for j in range(7))
    assert q.psnr(d, gt) == pytest.approx(-10 * np.log10(se / n), rel=1e-12)
    md = sum(d.flat) / n
    mg = sum(gt.flat) / n
    sd = sum((x - md) ** 2 for x in d.flat) / n
    sg = sum((x - mg) ** 2 for x in gt.flat) / n
    sdg = sum((x - md) * (y - mg) for x, y in zip(d.flat, gt.flat)) / n
    want = (2 * md * mg + 1e-4) * (2 * sdg + 9e-4) / ((md * md + mg * mg + 1e-4) * (sd + sg + 9e-4))
    assert q.mssim(d, gt) == pytest.approx(want, rel=1e-12)
