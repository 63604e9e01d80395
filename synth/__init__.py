"""Seeded synthetic grayscale scenes for the TV-Stokes denoising workloads.

This module only draws pixels.  It holds none of the denoising arithmetic, so
both the FP64 oracle and the GPU path may take their inputs from it.
"""
from .images import (  # noqa: F401
    SceneSpec,
    scene,
    noisy_scene,
    mixed_batch_sizes,
    poisson_arrivals,
)
