"""Image quality measures of Section 5.3 (FP64): PSNR and single-window MSSIM.

Test infrastructure only (see the package header).

For a reconstruction d and ground truth gt on an N2 x N1 grid with intensities
in [0, 1] (so the largest pixel value R is 1):

* MSE  = mean((d - gt)^2),  PSNR = -10 log10(MSE);
* MSSIM = (2 m_d m_gt + c1)(2 s_dgt + c2) / ((m_d^2 + m_gt^2 + c1)(s_d^2 + s_gt^2 + c2))
  over the whole image as one window, with population variances and covariance
  (divisor N1 N2) and c1 = (k1 R)^2, c2 = (k2 R)^2, k1 = 0.01, k2 = 0.03.

Pins (tests/test_oracle_quality.py): PSNR of a constant offset c is -20 log10|c|;
MSSIM(x, x) = 1 and is symmetric; the closed form for an affine image
d = a gt + b written out from the moments; the brute-force loop on a small image.
"""
from __future__ import annotations

import numpy as np

K1, K2, RMAX = 0.01, 0.03, 1.0


def psnr(d: np.ndarray, gt: np.ndarray) -> float:
    """-10 log10 of the mean squared error (Section 5.3)."""
    mse = float(np.mean((np.asarray(d, np.float64) - np.asarray(gt, np.float64)) ** 2))
    return float("inf") if mse == 0.0 else -10.0 * np.log10(mse)


def mssim(d: np.ndarray, gt: np.ndarray) -> float:
    """Single-window structural similarity over the whole image (Section 5.3)."""
    d = np.asarray(d, np.float64)
    gt = np.asarray(gt, np.float64)
    md, mg = d.mean(), gt.mean()
    sd2 = np.mean((d - md) ** 2)
    sg2 = np.mean((gt - mg) ** 2)
    sdg = np.mean((d - md) * (gt - mg))
    c1, c2 = (K1 * RMAX) ** 2, (K2 * RMAX) ** 2
    return float((2 * md * mg + c1) * (2 * sdg + c2) / ((md * md + mg * mg + c1) * (sd2 + sg2 + c2)))
