"""FP64 reference solver: discretisation, relaxations, transfers, V-cycle, Bi-CGSTAB.

Test infrastructure only (see the package docstring): the CUDA library never
imports this module and this module imports nothing from the library.

Everything is built on explicit sparse matrices of the paper's operators, so
each step is ordinary linear algebra on those matrices and can be checked
against the paper by eye. Units are physical (rows carry the 1/h^2 factor).
Grid: ``(n+1)^2`` vertex nodes of the unit square, ``h = 1/n``, node ``(i, j)``
at ``(i h, j h)``, flat index ``p = j (n+1) + i``; boundary nodes are unknowns.

Readings of points the paper leaves open (each one also listed in the design notes):

* Boundary rows (Sec. 1 says only "first-order Sommerfeld" and "standard
  discretization"): each out-of-domain neighbour (ghost) of a boundary node is
  eliminated with the centred difference of ``du/dn - i k u = 0``, i.e.
  ``u_ghost = u_mirror + 2 i k h u_b``, with the node's own k.
* The shift ``M^h = L^h + i k^2 beta`` (Eq. 3) adds ``i k(x)^2 beta`` to every row's diagonal.
* Coarse operators are rediscretised with k injected to the coarse nodes (Sec. 5).
* Full weighting mirrors fine nodes across the boundary (``r_{-1} = r_1``);
  bilinear interpolation needs no boundary rule on a vertex grid.
* Gauss-Seidel is red-black ((i+j) even first on the way down, odd first on the
  way up); "GS on the normal equations" (Sec. 4-5) is row-action Kaczmarz with
  colours ``(i + 2j) mod 5`` (0..4 on the way down, 4..0 on the way up).
* Level roles (Sec. 5): a level relaxes by Kaczmarz (GS on the normal equations)
  when the local scales ``k(x) H`` of its nodes reach into the band
  ``[0.625 sqrt 2, 2 sqrt 2)`` where red-black GS fails as a smoother (Sec. 4);
  other levels use GS, with the operator binned by ``c = k_ref H`` around the
  paper's scales 0.3125, 0.625, 1.25, 2.5 (geometric-midpoint edges), plus a
  guard that relaxes with M where red-black GS on L would amplify oscillatory
  error (any node with ``1 < k H < 2 sqrt 2``). The earlier reading, Kaczmarz
  on the ``c ~ 1.25`` bin only, is kept as ``rule="bins"``.
* Bi-CGSTAB is right-preconditioned, x0 = 0, shadow residual r^_0 a fixed
  pseudo-random vector (r^_0 = b degenerates: after a final red-black sweep
  with the Krylov operator itself, ``(A K v)_p = v_p`` on the last colour, so a
  point source's shadow space collapses),
  first argument of the inner product conjugated; convergence is tested after
  the half step (counted .5, as Table 1 prints) and after the full step; a
  recurrence-converged iterate is confirmed on the true residual b - A x.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

__all__ = [
    "grid_index", "helmholtz_matrix", "full_weighting", "bilinear_prolongation", "inject",
    "red_black_colours", "kaczmarz_colours", "gs_update_rows", "rb_gs_sweep", "lex_gs_sweep",
    "kaczmarz_update_rows", "kaczmarz_sweep", "jacobi_sweep", "rb_sor_sweep", "level_policy", "OracleLevel",
    "OracleHierarchy", "DEFAULT_OMEGA",
    "build_hierarchy", "vcycle", "bicgstab", "BicgstabResult", "true_relres",
    "BIN_EDGES", "GUARD_BAND", "KACZ_BAND", "level_count", "schedule", "renewed_shadow_seed",
    "STALL_COS2", "STALL_STEP2", "MAX_SHADOW_RESTARTS", "MAX_TRUE_RESTARTS", "shadow_residual", "splitmix64_u01",
]

# --------------------------------------------------------------------------- grid and operator (Sec. 1)


def grid_index(n: int) -> np.ndarray:
    """Flat index of node (i, j) stored at ``[j, i]``."""
    return np.arange((n + 1) * (n + 1)).reshape(n + 1, n + 1)


def helmholtz_matrix(n: int, kfield: np.ndarray, shift: float = 0.0) -> sp.csr_matrix:
    """The 5-point Helmholtz matrix ``L^h`` (``shift = 0``, Eq. 2) or ``M^h = L^h + i k^2 shift`` (Eq. 3).

    Interior rows: ``(u_E + u_W + u_N + u_S - 4 u_p) / h^2 + k_p^2 (1 + i shift) u_p``, the standard
    second-order discretisation of ``Delta u + k^2 u`` (Eq. 1). A neighbour that falls outside the
    square is a ghost; the first-order Sommerfeld condition ``du/dn - i k u = 0`` (Sec. 1), written
    with a centred difference across the boundary, gives ``u_ghost = u_mirror + 2 i k_p h u_p``, so
    the ghost's ``1/h^2`` coefficient moves onto the mirror node and ``2 i k_p / h`` onto the diagonal.
    """
    h = 1.0 / n
    k = np.asarray(kfield, dtype=np.float64)
    assert k.shape == (n + 1, n + 1)
    idx = grid_index(n)
    J, I = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    diag = (-4.0 / h**2 + k**2 * (1.0 + 1j * shift)).astype(np.complex128)
    rows, cols, vals = [], [], []
    for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
        qi, qj = I + di, J + dj
        inside = (qi >= 0) & (qi <= n) & (qj >= 0) & (qj <= n)
        rows.append(idx[inside])
        cols.append(idx[qj[inside], qi[inside]])
        vals.append(np.full(int(inside.sum()), 1.0 / h**2, dtype=np.complex128))
        ghost = ~inside
        rows.append(idx[ghost])
        cols.append(idx[J[ghost] - dj, I[ghost] - di])  # mirror node
        vals.append(np.full(int(ghost.sum()), 1.0 / h**2, dtype=np.complex128))
        diag[ghost] += 2j * k[ghost] / h
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    N = (n + 1) ** 2
    A = sp.coo_matrix(
        (np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N)
    ).tocsr()
    A.sum_duplicates()
    return A


# --------------------------------------------------------------------------- transfers (Sec. 5)


def _reflect(i: np.ndarray, n: int) -> np.ndarray:
    i = np.where(i < 0, -i, i)
    return np.where(i > n, 2 * n - i, i)


def _fw_1d(n: int) -> sp.csr_matrix:
    m = n // 2
    rows, cols, vals = [], [], []
    for a, w in ((-1, 0.25), (0, 0.5), (1, 0.25)):
        I = np.arange(m + 1)
        rows.append(I)
        cols.append(_reflect(2 * I + a, n))
        vals.append(np.full(m + 1, w))
    R = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(m + 1, n + 1))
    return R.tocsr()


def _bilinear_1d(n: int) -> sp.csr_matrix:
    m = n // 2
    rows, cols, vals = [], [], []
    I = np.arange(m + 1)
    rows.append(2 * I); cols.append(I); vals.append(np.ones(m + 1))
    I = np.arange(m)
    rows += [2 * I + 1, 2 * I + 1]; cols += [I, I + 1]; vals += [np.full(m, 0.5), np.full(m, 0.5)]
    P = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n + 1, m + 1))
    return P.tocsr()


def full_weighting(n: int) -> sp.csr_matrix:
    """Full weighting from the (n+1)^2 grid to the (n/2+1)^2 grid: weights 1/16 [1 2 1; 2 4 2; 1 2 1]
    centred on the coincident fine node, fine nodes outside the square mirrored back inside."""
    assert n % 2 == 0
    R1 = _fw_1d(n)
    return sp.kron(R1, R1, format="csr")


def bilinear_prolongation(n: int) -> sp.csr_matrix:
    """Bilinear interpolation from the (n/2+1)^2 grid to the (n+1)^2 grid."""
    assert n % 2 == 0
    P1 = _bilinear_1d(n)
    return sp.kron(P1, P1, format="csr")


def inject(field2d: np.ndarray) -> np.ndarray:
    """Coarse-grid values of a nodal field by injection (coarse node (I, J) = fine node (2I, 2J))."""
    return np.ascontiguousarray(field2d[::2, ::2])


# --------------------------------------------------------------------------- relaxations (Sec. 4-5)


def red_black_colours(n: int) -> np.ndarray:
    """0 (red) where i + j is even, 1 (black) where it is odd; flat order."""
    J, I = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    return ((I + J) % 2).ravel()


def kaczmarz_colours(n: int) -> np.ndarray:
    """Colour ``(i + 2 j) mod 5``: two nodes of one colour never share a 5-point stencil entry."""
    J, I = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    return ((I + 2 * J) % 5).ravel()


def gs_update_rows(A_off_rows: sp.csr_matrix, diag_rows: np.ndarray, f: np.ndarray, u: np.ndarray,
                   rows: np.ndarray) -> np.ndarray:
    """Gauss-Seidel update of a set of mutually uncoupled unknowns: each one solves its own
    equation with every other unknown held at its current value (Sec. 4)."""
    u = u.copy()
    u[rows] = (f[rows] - A_off_rows @ u) / diag_rows
    return u


def kaczmarz_update_rows(A_rows: sp.csr_matrix, A_rows_H: sp.csr_matrix, rownorm2: np.ndarray,
                         f: np.ndarray, u: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """Row-action Kaczmarz step for a set of rows with pairwise disjoint supports: each row's
    equation is satisfied by the smallest change of u, ``u += a_p^H (f_p - a_p u) / |a_p|^2``.
    This is Gauss-Seidel on ``A A^H y = f`` with ``u = A^H y`` (the normal-equation relaxation
    of Sec. 4-5)."""
    delta = (f[rows] - A_rows @ u) / rownorm2
    return u + A_rows_H @ delta


def sor_update_rows(A_off_rows: sp.csr_matrix, diag_rows: np.ndarray, f: np.ndarray, u: np.ndarray,
                    rows: np.ndarray, omega: float) -> np.ndarray:
    """Over-relaxed Gauss-Seidel update of uncoupled unknowns: ``(1 - omega) u + omega g`` with g the
    Gauss-Seidel value (omega = 1 is Gauss-Seidel)."""
    u = u.copy()
    u[rows] = (1.0 - omega) * u[rows] + omega * ((f[rows] - A_off_rows @ u) / diag_rows)
    return u


def lex_gs_sweep(A: sp.csr_matrix, f: np.ndarray, u: np.ndarray, order: np.ndarray | None = None) -> np.ndarray:
    """One Gauss-Seidel sweep over the unknowns in ``order`` (lexicographic by default):
    ``u <- (D + L)^{-1} (f - U u)`` with D, L, U taken in that ordering. A general triangular
    solve, used to check the colour-parallel sweeps and the Fourier analysis of Sec. 4."""
    if order is None:
        order = np.arange(A.shape[0])
    Ap = A[order][:, order].tocsr()
    lower = sp.tril(Ap, format="csr")
    upper = sp.triu(Ap, k=1, format="csr")
    up = spla.spsolve_triangular(lower, f[order] - upper @ u[order], lower=True)
    out = np.empty_like(u)
    out[order] = up
    return out


# --------------------------------------------------------------------------- level policy (Sec. 5)

# Bin edges in c = k_ref H: geometric midpoints between the paper's scales 0.3125, 0.625, 1.25, 2.5.
BIN_EDGES = (0.625 / math.sqrt(2.0), 0.625 * math.sqrt(2.0), 1.25 * math.sqrt(2.0))
# Guard band in local k H where red-black Gauss-Seidel on L is not a usable smoother (see level_policy).
GUARD_BAND = (1.0, 2.0 * math.sqrt(2.0))
# Band of local k H where Gauss-Seidel is replaced by Kaczmarz (rule "band" of level_policy): from the
# geometric midpoint of the paper's 0.625 and 1.25 scales up to the end of the guard band.
KACZ_BAND = (0.625 * math.sqrt(2.0), 2.0 * math.sqrt(2.0))


def level_policy(variant: str, c: float, c_local: np.ndarray, guard: bool = True, rule: str = "band"):
    """(relaxation operator, smoother, residual operator) for a non-coarsest level.

    ``c = k_ref H`` picks the scale bin; ``c_local`` holds ``k(x) H`` at the level's nodes.
    Sec. 5: one GS pre/post sweep on every scale except ``kH ~ 1.25``, where four sweeps of
    GS on the normal equations (Kaczmarz) are used; HLM-V uses L for relaxation (A) and for the
    residual (B); SL-V uses M for both; HYB-V uses L for (B) always and for (A) except on
    ``0.625 <~ kH <~ 1.25``, where M replaces it. ``sl_plain`` is M with GS on every level.

    Which levels count as the ``kH ~ 1.25`` scale (reading): Sec. 4 finds GS a good smoother for
    ``kH <~ 0.625`` and ``kH >~ 2.5`` only, and brings in GS on the normal equations where it is not.
    With ``rule="band"`` (default) a level is such a scale when any node's ``k(x) H`` lies in
    :data:`KACZ_BAND`, ``[0.625 sqrt 2, 2 sqrt 2)``: the lower edge is the bin edge between the
    paper's 0.625 and 1.25 scales, the upper edge the ``kH`` below which one red-black sweep
    still amplifies some oscillatory Fourier pair (the guard analysis below). In a heterogeneous
    medium one level spans the scales ``k_min H .. k_max H``, so several levels can reach the band.
    Kaczmarz relaxes with M (HYB, SL) or L (HLM). With ``rule="bins"`` only levels with
    ``c = k_ref H`` in ``[0.625 sqrt 2, 1.25 sqrt 2)`` do.

    Guard (reading): HYB relaxes with L on coarse scales because Gauss-Seidel converges fast
    there (Sec. 5). For red-black GS one sweep maps the Fourier pair {theta, theta + (pi, pi)}
    by a rank-one matrix with eigenvalue ``(S/d)^2``, ``S = 2 cos th1 + 2 cos th2`` in [-4, 4],
    ``d = -4 + (kH)^2``: every pair converges once ``|d| >= 4`` (``kH >= 2 sqrt 2``), and on
    fine scales (``kH <= 1``) only the smoothest pairs grow, which the coarse grid handles.
    In between, L-GS amplifies oscillatory error (at kH = 2.5 by about 2.5 per sweep), so an
    HYB L-GS level with any node in that band relaxes with M instead.
    """
    lo, mid, hi = BIN_EDGES
    if variant == "sl_plain":
        return "M", "gs", "M"
    if rule == "band":
        c_local = np.asarray(c_local)
        kacz = bool(np.any((c_local >= KACZ_BAND[0]) & (c_local < KACZ_BAND[1])))
    elif rule == "bins":
        kacz = mid <= c < hi
    else:
        raise ValueError(rule)
    smoother = "kaczmarz" if kacz else "gs"
    if variant == "sl":
        return "M", smoother, "M"
    if variant == "hlm":
        return "L", smoother, "L"
    if variant != "hyb":
        raise ValueError(variant)
    op = "M" if (lo <= c < hi or kacz) else "L"
    if op == "L" and guard:
        c_local = np.asarray(c_local)
        if np.any((c_local > GUARD_BAND[0]) & (c_local < GUARD_BAND[1])):
            op = "M"
    return op, smoother, "L"


@dataclass
class OracleLevel:
    n: int
    H: float
    k: np.ndarray
    relax_op: str
    smoother: str  # gs | jacobi | sor | kaczmarz | direct
    resid_op: str
    nu: int
    A: sp.csr_matrix  # relaxation operator (or the direct-solve operator on the coarsest level)
    B: sp.csr_matrix | None = None  # residual operator
    R: sp.csr_matrix | None = None  # full weighting to the next level
    P: sp.csr_matrix | None = None  # bilinear interpolation from the next level
    omega: float = 1.0  # relaxation factor of a jacobi or sor level
    cache: dict = field(default_factory=dict)


@dataclass
class OracleHierarchy:
    n: int
    beta: float
    variant: str
    k_ref: float
    levels: list


# Default relaxation factors of the alternative smoothers: damped Jacobi at the usual 4/5 of
# two-dimensional 5-point smoothing; SOR at 1, i.e. Gauss-Seidel.
DEFAULT_OMEGA = {"jacobi": 0.8, "sor": 1.0}


def level_count(n: int, levels: int = 0) -> int:
    """Number of grids: ``levels``, or (0) coarsen while the grid count is even and larger than 8."""
    if levels <= 0:
        levels, m = 1, n
        while m % 2 == 0 and m > 8:
            m //= 2
            levels += 1
    assert n % (1 << (levels - 1)) == 0 and n >> (levels - 1) >= 2, "grid not divisible for the requested levels"
    return levels


def schedule(n: int, kfield: np.ndarray, k_ref: float, variant: str = "hyb", levels: int = 0, guard: bool = True,
             rule: str = "band") -> list:
    """(n_l, relax_op, smoother, resid_op) of every level, as :func:`build_hierarchy` assigns them,
    without building any operator (k injected level by level, Sec. 5)."""
    levels = level_count(n, levels)
    out = []
    k = np.asarray(kfield, dtype=np.float64)
    for l in range(levels):
        nl = n >> l
        if l > 0:
            k = inject(k)
        if l == levels - 1:
            op = "M" if variant in ("sl", "sl_plain") else "L"
            out.append((nl, op, "direct", op))
        else:
            out.append((nl,) + tuple(level_policy(variant, k_ref / nl, k / nl, guard, rule)))
    return out


def build_hierarchy(n: int, kfield: np.ndarray, k_ref: float, variant: str = "hyb", levels: int = 0,
                    beta: float = 0.5, nu_gs: int = 1, nu_kacz: int = 4, guard: bool = True,
                    ops: list | None = None, gs_smoother: str = "gs", omega: float | None = None,
                    rule: str = "band") -> OracleHierarchy:
    """Grids n, n/2, ... with rediscretised operators and the per-level roles of :func:`level_policy`.

    ``levels = 0`` coarsens while the grid count is even and larger than 8. The coarsest level is
    solved directly with L (HYB, HLM) or M (SL variants). ``ops`` optionally overrides
    (relax_op, smoother, resid_op) per non-coarsest level; ``rule`` selects which levels relax by
    Kaczmarz (see :func:`level_policy`). ``gs_smoother`` replaces red-black
    Gauss-Seidel on the levels that use it by damped Jacobi ("jacobi") or red-black SOR ("sor")
    with relaxation factor ``omega`` (the alternatives the remark of Sec. 4 names).
    """
    levels = level_count(n, levels)
    out = []
    k = np.asarray(kfield, dtype=np.float64)
    for l in range(levels):
        nl = n >> l
        H = 1.0 / nl
        if l > 0:
            k = inject(k)
        L = helmholtz_matrix(nl, k, 0.0)
        M = helmholtz_matrix(nl, k, beta)
        if l == levels - 1:
            op = "M" if variant in ("sl", "sl_plain") else "L"
            lv = OracleLevel(nl, H, k, op, "direct", op, 0, M if op == "M" else L)
            lv.cache["lu"] = sla.lu_factor(lv.A.toarray())
        else:
            relax, smoother, resid = level_policy(variant, k_ref * H, k * H, guard, rule) if ops is None else ops[l]
            if smoother == "gs" and gs_smoother != "gs":
                smoother = gs_smoother
            nu = nu_kacz if smoother == "kaczmarz" else nu_gs
            lv = OracleLevel(nl, H, k, relax, smoother, resid, nu, M if relax == "M" else L,
                             M if resid == "M" else L, full_weighting(nl), bilinear_prolongation(nl))
            if smoother in DEFAULT_OMEGA:
                lv.omega = DEFAULT_OMEGA[smoother] if omega is None else float(omega)
            _prepare_relaxation(lv)
        out.append(lv)
    return OracleHierarchy(n, beta, variant, k_ref, out)


def _prepare_relaxation(lv: OracleLevel) -> None:
    A = lv.A
    if lv.smoother == "jacobi":
        lv.cache["diag"] = A.diagonal()
    elif lv.smoother in ("gs", "sor"):
        diag = A.diagonal()
        A_off = (A - sp.diags(diag)).tocsr()
        col = red_black_colours(lv.n)
        for c in (0, 1):
            rows = np.nonzero(col == c)[0]
            lv.cache[("gs", c)] = (rows, A_off[rows], diag[rows])
    else:
        col = kaczmarz_colours(lv.n)
        for c in range(5):
            rows = np.nonzero(col == c)[0]
            Ar = A[rows]
            rownorm2 = np.asarray(abs(Ar).power(2).sum(axis=1)).ravel()
            lv.cache[("kz", c)] = (rows, Ar, Ar.conj().T.tocsr(), rownorm2)


def rb_gs_sweep(lv: OracleLevel, f: np.ndarray, u: np.ndarray, first: int = 0) -> np.ndarray:
    """One red-black Gauss-Seidel sweep with the level's relaxation operator; ``first`` = 0 starts with red."""
    for c in (first, 1 - first):
        rows, A_off_rows, diag_rows = lv.cache[("gs", c)]
        u = gs_update_rows(A_off_rows, diag_rows, f, u, rows)
    return u


def rb_sor_sweep(lv: OracleLevel, f: np.ndarray, u: np.ndarray, first: int = 0) -> np.ndarray:
    """One red-black SOR sweep with the level's relaxation operator and factor ``lv.omega``."""
    for c in (first, 1 - first):
        rows, A_off_rows, diag_rows = lv.cache[("gs", c)]
        u = sor_update_rows(A_off_rows, diag_rows, f, u, rows, lv.omega)
    return u


def jacobi_sweep(lv: OracleLevel, f: np.ndarray, u: np.ndarray) -> np.ndarray:
    """One damped Jacobi sweep, every unknown at once: ``u + omega D^-1 (f - A u)``."""
    return u + lv.omega * (f - lv.A @ u) / lv.cache["diag"]


def kaczmarz_sweep(lv: OracleLevel, f: np.ndarray, u: np.ndarray, order=(0, 1, 2, 3, 4)) -> np.ndarray:
    """One Kaczmarz sweep over the five colours in ``order`` with the level's relaxation operator."""
    for c in order:
        rows, Ar, ArH, rn2 = lv.cache[("kz", c)]
        u = kaczmarz_update_rows(Ar, ArH, rn2, f, u, rows)
    return u


def relax(lv: OracleLevel, f: np.ndarray, u: np.ndarray, post: bool) -> np.ndarray:
    """The level's pre (``post=False``) or post relaxation: nu sweeps of its smoother."""
    for _ in range(lv.nu):
        if lv.smoother == "gs":
            u = rb_gs_sweep(lv, f, u, first=1 if post else 0)
        elif lv.smoother == "sor":
            u = rb_sor_sweep(lv, f, u, first=1 if post else 0)
        elif lv.smoother == "jacobi":
            u = jacobi_sweep(lv, f, u)
        else:
            u = kaczmarz_sweep(lv, f, u, order=(4, 3, 2, 1, 0) if post else (0, 1, 2, 3, 4))
    return u


# --------------------------------------------------------------------------- V-cycle (Sec. 5)


def vcycle(h: OracleHierarchy, f: np.ndarray, level: int = 0, trace: dict | None = None) -> np.ndarray:
    """One V-cycle from a zero initial guess on ``level``: relax (A), residual with (B), full weighting,
    recursion, bilinear correction, relax (A); the coarsest level is solved directly."""
    lv = h.levels[level]
    if lv.smoother == "direct":
        return sla.lu_solve(lv.cache["lu"], f)
    u = relax(lv, f, np.zeros_like(f), post=False)
    r = f - lv.B @ u
    fc = lv.R @ r
    if trace is not None:
        trace[(level, "pre")] = u.copy()
        trace[(level, "fc")] = fc.copy()
    ec = vcycle(h, fc, level + 1, trace)
    u = u + lv.P @ ec
    u = relax(lv, f, u, post=True)
    if trace is not None:
        trace[(level, "ec")] = ec.copy()
        trace[(level, "post")] = u.copy()
    return u


# --------------------------------------------------------------------------- Bi-CGSTAB (Sec. 6)

SHADOW_SEED = 0x5EED1312


def splitmix64_u01(seed: int, counters: np.ndarray) -> np.ndarray:
    """Counter-based SplitMix64 (Steele, Lea, Flood 2014): output number ``c + 1`` of the generator
    started from state ``seed``, for each counter ``c``, mapped to [0, 1) by its top 53 bits."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + np.uint64(0x9E3779B97F4A7C15) * (counters.astype(np.uint64) + np.uint64(1))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * 2.0**-53


def shadow_residual(N: int, seed: int = SHADOW_SEED) -> np.ndarray:
    """Pseudo-random shadow residual: ``r^_p = (u_{2p} - 1/2) + i (u_{2p+1} - 1/2)``."""
    c = np.arange(2 * N, dtype=np.uint64)
    u = splitmix64_u01(seed, c)
    return (u[0::2] - 0.5) + 1j * (u[1::2] - 0.5)


@dataclass
class BicgstabResult:
    x: np.ndarray
    iterations: float  # full iterations; a stop after the half step counts .5
    history: list  # relative residual after each half and each full step
    status: str  # converged | maxit | breakdown
    true_relres: float
    restarts: int = 0  # restarts from the true residual (recurrence converged, b - A x did not)
    shadow_restarts: int = 0  # renewals of the shadow residual (stalled recurrences)


def true_relres(A, b, x) -> float:
    return float(np.linalg.norm(b - A @ x) / np.linalg.norm(b))


# Shadow-residual renewal after stalled recurrences (reading, not in the paper): seeds of the
# renewed shadow residuals, and the default thresholds and cap.
SHADOW_SEED_STEP = 0x2545F4914F6CDD1D
STALL_COS2 = 1e-12
STALL_STEP2 = 1e-8
MAX_SHADOW_RESTARTS = 16
# Restarts from the true residual that one solve may take.
MAX_TRUE_RESTARTS = 8


def renewed_shadow_seed(k: int) -> int:
    """Seed of the k-th renewed shadow residual (k = 1, 2, ...): ``SHADOW_SEED + k * SHADOW_SEED_STEP``
    modulo 2^64."""
    return (SHADOW_SEED + k * SHADOW_SEED_STEP) % (1 << 64)


def bicgstab(A, b: np.ndarray, precond=None, tol: float = 1e-6, maxit: int = 1000, callback=None,
             rhat: np.ndarray | None = None, stall_cos2: float = STALL_COS2, stall_step2: float = STALL_STEP2,
             max_shadow_restarts: int = MAX_SHADOW_RESTARTS,
             max_true_restarts: int = MAX_TRUE_RESTARTS, renew_shadow=None) -> BicgstabResult:
    """Right-preconditioned Bi-CGSTAB (van der Vorst 1992) from ``x0 = 0``; the shadow residual
    ``rhat`` defaults to :func:`shadow_residual`.

    Each iteration applies the preconditioner twice (Sec. 6). Stops when ``|r| / |b| <= tol`` after
    the half step (``s``) or the full step. Two readings complete the method where the paper is
    silent:

    * A recurrence-converged iterate is accepted only when the true residual ``b - A x`` also
      meets ``tol``. If it does not, the iteration restarts from it: ``r = b - A x``, the next
      direction is ``p = r`` and ``rho = <rhat, r>``; at most ``max_true_restarts`` times and
      below ``maxit`` iterations, else the solve ends unconfirmed (status ``maxit``).
    * Stalled recurrences: after a full step with ``|<rhat, r>|^2 < stall_cos2 |rhat|^2 |r|^2``
      and ``|omega|^2 |t|^2 < stall_step2 |r|^2``, the next iteration renews the shadow residual
      (:func:`shadow_residual` with seed :func:`renewed_shadow_seed` of the renewal's number),
      takes ``p = r`` and ``rho = <rhat, r>``; at most ``max_shadow_restarts`` times.

    ``callback(x)`` is called after every full step. ``renew_shadow(k, r)``, if given, supplies the
    k-th renewed shadow residual instead of the seeded one (used to check the renewal against a
    fresh start of an independent implementation).
    """
    K = (lambda v: v) if precond is None else precond
    x = np.zeros_like(b)
    r = b.copy()
    rhat = shadow_residual(b.size) if rhat is None else np.asarray(rhat, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    tol2 = (tol * bnorm) ** 2
    hist = []
    p = np.zeros_like(b)
    v = np.zeros_like(b)
    alpha = omega = beta = 1.0 + 0j
    if bnorm == 0:
        return BicgstabResult(x, 0.0, hist, "converged", 0.0)
    rho = np.vdot(rhat, r)
    restarts = renewals = 0
    first, renew = True, False
    it = 1

    def result(status, iterations, xx):
        return BicgstabResult(xx, float(iterations), hist, status, true_relres(A, b, xx), restarts, renewals)

    if rho == 0:
        return result("breakdown", 0, x)
    while it <= maxit:
        if renew:  # a new shadow residual and a fresh direction
            renewals += 1
            rhat = (shadow_residual(b.size, renewed_shadow_seed(renewals)) if renew_shadow is None
                    else np.asarray(renew_shadow(renewals, r), dtype=np.complex128))
            rho = np.vdot(rhat, r)
            p = r.copy()
            renew = False
            if rho == 0:
                return result("breakdown", it - 1, x)
        elif first:
            p = r.copy()
        else:
            p = r + beta * (p - omega * v)
        y = K(p)
        v = A @ y
        rv = np.vdot(rhat, v)
        if rv == 0:
            return result("breakdown", it - 1, x)
        alpha = rho / rv
        s = r - alpha * v
        ss = np.vdot(s, s).real
        hist.append(math.sqrt(ss) / bnorm)
        stop = None
        if ss <= tol2:  # stop after the half step
            x = x + alpha * y
            stop = it - 0.5
        else:
            z = K(s)
            t = A @ z
            tt = np.vdot(t, t).real
            if tt == 0:
                return result("breakdown", it - 1, x)
            omega = np.vdot(t, s) / tt
            x = x + alpha * y + omega * z
            r = s - omega * t
            rho_new = np.vdot(rhat, r)
            rr = np.vdot(r, r).real
            hist.append(math.sqrt(rr) / bnorm)
            if callback:
                callback(x)
            if omega == 0:
                return result("breakdown", it, x)
            if rr <= tol2:
                stop = float(it)
            elif rho_new == 0:
                return result("breakdown", it, x)
            else:
                cos2 = abs(rho_new) ** 2 / (np.vdot(rhat, rhat).real * rr)
                step2 = abs(omega) ** 2 * tt / rr
                if cos2 < stall_cos2 and step2 < stall_step2 and renewals < max_shadow_restarts:
                    renew = True
                else:
                    beta = (rho_new / rho) * (alpha / omega)
                    rho = rho_new
                    first = False
                it += 1
                continue
        # the recurrence says converged: confirm on the true residual b - A x
        tr = b - A @ x
        if np.vdot(tr, tr).real <= tol2:
            if stop != int(stop) and callback:
                callback(x)
            return result("converged", stop, x)
        if restarts >= max_true_restarts or it >= maxit:
            return result("maxit", stop, x)
        restarts += 1
        r = tr
        rho = np.vdot(rhat, r)
        first = True
        it += 1
        if rho == 0:
            return result("breakdown", it - 1, x)
    return result("maxit", maxit, x)
