"""Piecewise-constant test scenes with optional ramp and textures, plus noise.

The paper evaluates on twelve photographs and phantoms in [0, 1] with additive
Gaussian noise (Section 5.2).  Those images are not available, so every
workload here is drawn from a seeded generator with the same structure:

* background intensity ~ U[0, 1];
* six axis-aligned rectangles, side lengths U[N/8, N/2] per axis, top-left
  corner uniform over the valid range, intensity U[0, 1];
* four discs, centre uniform, radius U[min(N)/16, min(N)/6], intensity U[0, 1];
* shapes are painted in that order, later ones overwrite earlier ones;
* optionally (``texture=True``) a linear ramp spanning 0.2 in a random
  direction and two sinusoids ``0.1*sin(2*pi*(x cos phi + y sin phi)/P + psi)``
  with P ~ U[8, 32] and phi, psi ~ U[0, 2*pi);
* i.i.d. Gaussian noise of standard deviation sigma, no clipping.

All draws come from ``numpy.random.Generator(PCG64(seed))`` in a fixed order,
so a (shape, seed, options) triple always gives the same bytes.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class SceneSpec:
    rows: int            # N2, image height (y)
    cols: int            # N1, image width (x)
    seed: int = 0
    sigma: float = 0.1   # noise standard deviation
    texture: bool = False


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def scene(rows: int, cols: int, seed: int = 0, texture: bool = False) -> np.ndarray:
    """Noise-free scene, float64, shape (rows, cols), row index = y."""
    if rows < 1 or cols < 1:
        raise ValueError("scene needs rows, cols >= 1")
    g = _rng(seed)
    img = np.full((rows, cols), g.uniform(0.0, 1.0), dtype=np.float64)
    yy, xx = np.meshgrid(np.arange(rows, dtype=np.float64),
                         np.arange(cols, dtype=np.float64), indexing="ij")
    for _ in range(6):
        h = int(round(g.uniform(rows / 8.0, rows / 2.0)))
        w = int(round(g.uniform(cols / 8.0, cols / 2.0)))
        h = min(max(h, 1), rows)
        w = min(max(w, 1), cols)
        y0 = int(g.integers(0, rows - h + 1))
        x0 = int(g.integers(0, cols - w + 1))
        img[y0:y0 + h, x0:x0 + w] = g.uniform(0.0, 1.0)
    n = float(min(rows, cols))
    for _ in range(4):
        cy = g.uniform(0.0, rows)
        cx = g.uniform(0.0, cols)
        r = g.uniform(n / 16.0, n / 6.0)
        val = g.uniform(0.0, 1.0)
        mask = (yy + 0.5 - cy) ** 2 + (xx + 0.5 - cx) ** 2 <= r * r
        img[mask] = val
    if texture:
        ang = g.uniform(0.0, 2.0 * np.pi)
        proj = xx * np.cos(ang) + yy * np.sin(ang)
        span = proj.max() - proj.min()
        if span > 0:
            img += 0.2 * (proj - proj.min()) / span - 0.1
        for _ in range(2):
            period = g.uniform(8.0, 32.0)
            phi = g.uniform(0.0, 2.0 * np.pi)
            psi = g.uniform(0.0, 2.0 * np.pi)
            img += 0.1 * np.sin(2.0 * np.pi * (xx * np.cos(phi) + yy * np.sin(phi)) / period + psi)
    return img


def noisy_scene(spec: SceneSpec) -> tuple[np.ndarray, np.ndarray]:
    """(ground truth, noisy observation), both float64 (rows, cols)."""
    gt = scene(spec.rows, spec.cols, spec.seed, spec.texture)
    g = _rng(spec.seed + 7_000_003)
    noisy = gt + spec.sigma * g.standard_normal(gt.shape)
    return gt, noisy


def mixed_batch_sizes(count: int, lo: int, hi: int, seed: int = 1000) -> list[tuple[int, int, float]]:
    """(rows, cols, sigma) for a batch of uneven images.

    Sides are independently log-uniform in [lo, hi]; sigma ~ U[0.05, 0.15].
    """
    g = _rng(seed)
    out = []
    for _ in range(count):
        r = int(round(np.exp(g.uniform(np.log(lo), np.log(hi)))))
        c = int(round(np.exp(g.uniform(np.log(lo), np.log(hi)))))
        s = float(g.uniform(0.05, 0.15))
        out.append((r, c, s))
    return out


def poisson_arrivals(count: int, rate_per_s: float, seed: int = 2000) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson process with the given rate."""
    g = _rng(seed)
    return np.cumsum(g.exponential(1.0 / rate_per_s, size=count))
