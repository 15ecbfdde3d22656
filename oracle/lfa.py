"""Local Fourier analysis tools of Sec. 3-4 (symbols, symbol ratios, Gauss-Seidel amplification).

Test infrastructure only: these formulas are not on the solver's path; the tests use them to
tie the oracle's relaxations to the paper's printed rates.
"""
from __future__ import annotations

import numpy as np

__all__ = ["helmholtz_symbol", "symbol_ratio", "gs_amplification", "smoothing_factor", "overall_rate", "theta_grid"]


def helmholtz_symbol(theta1, theta2, kh: float, h: float = 1.0, beta: float = 0.0):
    """Symbol of L^h (beta = 0) or M^h on the Fourier mode with angles (theta1, theta2) = omega h:
    ``(2 cos theta1 + 2 cos theta2 - 4 + (kh)^2 (1 + i beta)) / h^2`` (Sec. 3, Eqs. for tau)."""
    return (2 * np.cos(theta1) + 2 * np.cos(theta2) - 4 + kh * kh * (1 + 1j * beta)) / (h * h)


def symbol_ratio(omega1, omega2, k: float, h: float, H: float, beta: float = 0.0):
    """``tau_H = L~^h / A~^H`` for A = L (beta = 0, tau^HLM) or A = M (tau^SL), Sec. 3."""
    fine = helmholtz_symbol(omega1 * h, omega2 * h, k * h, h, 0.0)
    coarse = helmholtz_symbol(omega1 * H, omega2 * H, k * H, H, beta)
    return fine / coarse


def gs_amplification(theta1, theta2, kH: float, beta: float = 0.0):
    """Lexicographic Gauss-Seidel amplification of a Fourier mode (Sec. 4):
    ``|(e^{-i th1} + e^{-i th2}) / (e^{i th1} + e^{i th2} - 4 + (kH)^2 (1 + i beta))|``;
    beta = 0 gives mu^HLM, beta > 0 mu^SL."""
    num = np.exp(-1j * theta1) + np.exp(-1j * theta2)
    den = np.exp(1j * theta1) + np.exp(1j * theta2) - 4 + kH * kH * (1 + 1j * beta)
    return np.abs(num / den)


def theta_grid(points: int = 721):
    """Angles on [-pi, pi]^2 (both ends and 0, pi/2 included when points = 4 m + 1)."""
    t = np.linspace(-np.pi, np.pi, points)
    return np.meshgrid(t, t, indexing="ij")


def smoothing_factor(kH: float, beta: float = 0.0, points: int = 721) -> float:
    """``mu~_H``: the largest amplification over oscillatory modes, pi/2 <= max |theta| <= pi (Sec. 4)."""
    t1, t2 = theta_grid(points)
    mask = np.maximum(np.abs(t1), np.abs(t2)) >= np.pi / 2 - 1e-12
    return float(gs_amplification(t1, t2, kH, beta)[mask].max())


def overall_rate(kH: float, beta: float = 0.0, points: int = 721) -> float:
    """``mu^_H``: the largest amplification over all modes, 0 <= max |theta| <= pi (Sec. 4)."""
    t1, t2 = theta_grid(points)
    return float(gs_amplification(t1, t2, kH, beta).max())
