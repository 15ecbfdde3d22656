"""Local Fourier analysis tools of Sec. 3-4 (symbols, symbol ratios, Gauss-Seidel amplification).

Test infrastructure only: these formulas are not on the solver's path; the tests use them to
tie the oracle's relaxations to the paper's printed rates.
"""
from __future__ import annotations

import numpy as np

__all__ = ["helmholtz_symbol", "symbol_ratio", "gs_amplification", "smoothing_factor", "overall_rate", "theta_grid",
           "jacobi_amplification", "jacobi_smoothing_factor", "rb_sor_two_harmonic", "rb_smoothing_factor"]


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


# ----------------------------------------------------------------- the alternatives of Sec. 4's remark
# Symbols below are of the h^2-scaled 5-point row: neighbours 1, diagonal d = -4 + (kH)^2 (1 + i beta).


def jacobi_amplification(theta1, theta2, kH: float, beta: float = 0.0, omega: float = 0.8):
    """Damped Jacobi ``u + omega D^-1 (f - A u)`` multiplies the Fourier mode by
    ``1 - omega (2 cos th1 + 2 cos th2 + d) / d``; returns the modulus."""
    d = -4 + kH * kH * (1 + 1j * beta)
    return np.abs(1 - omega * (2 * np.cos(theta1) + 2 * np.cos(theta2) + d) / d)


def jacobi_smoothing_factor(kH: float, beta: float = 0.0, omega: float = 0.8, points: int = 721) -> float:
    """Largest damped-Jacobi amplification over oscillatory modes, pi/2 <= max |theta| <= pi."""
    t1, t2 = theta_grid(points)
    mask = np.maximum(np.abs(t1), np.abs(t2)) >= np.pi / 2 - 1e-12
    return float(jacobi_amplification(t1, t2, kH, beta, omega)[mask].max())


def rb_sor_two_harmonic(theta1: float, theta2: float, kH: float, beta: float = 0.0, omega: float = 1.0):
    """One red-black SOR sweep (red first, f = 0) on span{e_th, e_(th + (pi, pi))} as a 2 x 2 matrix in
    that basis. On red nodes (i + j even) u = a e_th + b e_(th+(pi,pi)) equals R e_th with R = a + b,
    on black nodes K e_th with K = a - b; the neighbours of a node of one colour sum to S = 2 cos th1 +
    2 cos th2 times the other colour's amplitude, so with q = omega S / d:
    R' = (1 - omega) R - q K and K' = (1 - omega) K - q R'. omega = 1 is red-black Gauss-Seidel."""
    d = -4 + kH * kH * (1 + 1j * beta)
    q = omega * (2 * np.cos(theta1) + 2 * np.cos(theta2)) / d
    Mrk = np.array([[1 - omega, -q], [-q * (1 - omega), (1 - omega) + q * q]], dtype=complex)
    to_rk = np.array([[1, 1], [1, -1]], dtype=complex)  # (a, b) -> (R, K)
    return np.linalg.solve(to_rk, Mrk @ to_rk)


def _high(t):
    t = (np.asarray(t) + np.pi) % (2 * np.pi) - np.pi
    return np.max(np.abs(t), axis=0) >= np.pi / 2 - 1e-12


def rb_smoothing_factor(kH: float, beta: float = 0.0, omega: float = 1.0, points: int = 128) -> float:
    """Red-black smoothing factor: the largest spectral radius of Q S over the pairs {th, th + (pi, pi)},
    S the two-harmonic sweep matrix and Q the projection onto the pair's oscillatory members (both
    when both are oscillatory), i.e. a sweep followed by an ideal coarse-grid correction."""
    t = np.linspace(-np.pi, np.pi, points, endpoint=False)
    worst = 0.0
    for a in t:
        for b in t:
            h = _high(np.array([[a, a + np.pi], [b, b + np.pi]]))
            if not h.any():
                continue
            QS = np.diag(h.astype(float)) @ rb_sor_two_harmonic(a, b, kH, beta, omega)
            worst = max(worst, float(np.abs(np.linalg.eigvals(QS)).max()))
    return worst
