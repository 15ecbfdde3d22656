"""Ray correction (Sec. 6, Table 7): FP64 reference, test infrastructure only.

Like the rest of this package it is imported only by the test suite, ``__graft_entry__.smoke()``
and the benchmark's CPU legs; the CUDA library never imports it and it imports nothing from the
library.

Sec. 6 writes the near-kernel error as a sum of eight plane waves ``exp(i k d_j . x)``, directions
``d_j = (cos j pi/4, sin j pi/4)``, each times a smooth ray function, and corrects it by
approximating the ray functions on a coarse scale; Table 7 uses a V-cycle followed by this
correction as a stand-alone solver. The paper defers the construction to its [BL97] reference.
Reading taken here (each point also listed in the design notes):

* Ray functions are bilinear on a ray grid of spacing ``H = m h`` (the same vertex grid with every
  m-th node); ``m`` is the largest power of two with ``k_ref H <= 2.5`` (the paper's coarsest scale
  ladder value) that divides n and leaves at least two ray cells.
* The eight ray functions are unknowns of ONE coarse problem: the correction is the Galerkin
  projection ``x += P (P^H A P)^{-1} P^H (b - A x)``, ``P = [diag(exp(i k d_j . x)) I_H^h]_j``
  (bilinear interpolation I_H^h), with the Helmholtz operator A itself. Treating each direction
  on its own (the eight projections added, or applied one after another with the residual updated
  between them) diverges or stalls on Table 7's problems, so the coupled form is the reading.
* The wavenumber of the plane waves is the problem's k_ref (Table 7's media are constant).
* A cycle of the stand-alone solver is one V-cycle on the residual, then one ray correction on the
  new residual; the solve stops at relres <= tol on b - A x after a full cycle.

Unknowns of the ray problem are ordered node-major: column ``8 C + j`` for ray node
``C = J (n/m + 1) + I`` and direction j.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .helmholtz import vcycle

__all__ = ["RAY_DIRECTIONS", "RAY_KH", "ray_spacing", "linear_interpolation_1d", "ray_phases", "ray_prolongation",
           "RayCorrection", "ray_galerkin", "ray_setup", "cycle_solve", "CycleResult"]

_S = math.sqrt(0.5)
# (cos j pi/4, sin j pi/4), j = 0..7, written with the exactly rounded sqrt(1/2)
RAY_DIRECTIONS = ((1.0, 0.0), (_S, _S), (0.0, 1.0), (-_S, _S), (-1.0, 0.0), (-_S, -_S), (0.0, -1.0), (_S, -_S))
RAY_KH = 2.5


def ray_spacing(n: int, k_ref: float, kH: float = RAY_KH) -> int:
    """Ray-grid factor m: the largest power of two with ``k_ref m / n <= kH``, ``n % m == 0`` and
    ``n / m >= 2`` (1 if none larger qualifies)."""
    m = 1
    while n % (2 * m) == 0 and n // (2 * m) >= 2 and k_ref * (2 * m) / n <= kH * (1 + 1e-12):
        m *= 2
    return m


def linear_interpolation_1d(nc: int, m: int) -> sp.csr_matrix:
    """``(nc m + 1) x (nc + 1)`` linear interpolation: fine node ``i = m I + t`` takes
    ``(1 - t/m)`` of coarse node I and ``t/m`` of node I + 1."""
    rows, cols, vals = [], [], []
    for i in range(nc * m + 1):
        c, t = divmod(i, m)
        rows += [i]
        cols += [c]
        vals += [1.0 - t / m]
        if t:
            rows += [i]
            cols += [c + 1]
            vals += [t / m]
    return sp.csr_matrix((vals, (rows, cols)), shape=(nc * m + 1, nc + 1))


def ray_phases(n: int, k: float) -> np.ndarray:
    """``(8, (n+1)^2)`` plane waves ``exp(i k (d_x x + d_y y))`` at node ``(x, y) = (i h, j h)``."""
    h = 1.0 / n
    J, I = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    x, y = (I * h).ravel(), (J * h).ravel()
    return np.stack([np.exp(1j * (k * (dx * x + dy * y))) for dx, dy in RAY_DIRECTIONS])


def ray_prolongation(n: int, m: int, k: float) -> sp.csr_matrix:
    """``P``: ``(n+1)^2 x 8 (n/m+1)^2``, column ``8 C + j`` = plane wave j times the bilinear hat of
    ray node C (Sec. 6's sum of plane waves with ray-function envelopes)."""
    assert n % m == 0
    nc = n // m
    I1 = linear_interpolation_1d(nc, m)
    I2 = sp.kron(I1, I1).tocsr()  # row j(n+1)+i, column J(nc+1)+I
    ph = ray_phases(n, k)
    Nc = (nc + 1) ** 2
    blocks = [sp.diags(ph[j]) @ I2 for j in range(8)]
    P = sp.hstack(blocks).tocsc()  # column j Nc + C
    perm = np.arange(8 * Nc).reshape(8, Nc).T.ravel()  # new column 8 C + j <- old column j Nc + C
    return P[:, perm].tocsr()


@dataclass
class RayCorrection:
    n: int
    m: int
    k: float
    P: sp.csr_matrix
    PH: sp.csr_matrix
    Ac: sp.csc_matrix  # P^H A P
    lu: object = field(repr=False, default=None)

    def restrict(self, r: np.ndarray) -> np.ndarray:
        """``P^H r``: each ray node and direction gathers the residual times the conjugate plane wave
        under its hat."""
        return self.PH @ r

    def correct(self, r: np.ndarray) -> np.ndarray:
        """The correction ``P (P^H A P)^{-1} P^H r`` to add to the iterate whose residual is r."""
        return self.P @ self.lu.solve(self.restrict(r))


def ray_galerkin(A: sp.csr_matrix, P: sp.csr_matrix):
    """``(P^H, P^H A P)``: the restriction and the Galerkin ray operator."""
    PH = P.conj().T.tocsr()
    return PH, (PH @ (A @ P)).tocsc()


def ray_setup(A: sp.csr_matrix, n: int, k: float, m: int = 0) -> RayCorrection:
    """Galerkin ray problem of the operator A on the ray grid of factor m (0: :func:`ray_spacing`)."""
    if m <= 0:
        m = ray_spacing(n, k)
    P = ray_prolongation(n, m, k)
    PH, Ac = ray_galerkin(A, P)
    rc = RayCorrection(n, m, float(k), P, PH, Ac)
    rc.lu = spla.splu(Ac)
    return rc


@dataclass
class CycleResult:
    x: np.ndarray
    cycles: int
    history: list  # relres after each cycle
    status: str  # converged | maxit | diverged


def cycle_solve(A, b: np.ndarray, hierarchy, ray: RayCorrection | None = None, tol: float = 1e-7,
                maxc: int = 100, blowup: float = 1e8) -> CycleResult:
    """Table 7's stand-alone solver from x = 0: each cycle adds a V-cycle of the residual, then (with
    ``ray``) the ray correction of the new residual; stops when ``|b - A x| <= tol |b|`` after a
    cycle, or reports divergence once the residual exceeds ``blowup |b|``."""
    x = np.zeros_like(b)
    bn = np.linalg.norm(b)
    hist = []
    for c in range(1, maxc + 1):
        x = x + vcycle(hierarchy, b - A @ x)
        if ray is not None:
            x = x + ray.correct(b - A @ x)
        rr = float(np.linalg.norm(b - A @ x) / bn)
        hist.append(rr)
        if not math.isfinite(rr) or rr > blowup:
            return CycleResult(x, c, hist, "diverged")
        if rr <= tol:
            return CycleResult(x, c, hist, "converged")
    return CycleResult(x, maxc, hist, "maxit")
