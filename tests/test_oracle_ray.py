"""Pins of the oracle's ray correction (Sec. 6: the near-kernel error as eight plane waves with smooth
ray functions; Table 7: V-cycle plus ray correction as a stand-alone solver).

The Galerkin ray operator is pinned by two closed forms that do not go through the oracle's
construction: the plane-wave eigenvalue of the 5-point stencil summed against a bilinear hat (a
Fejer kernel), and the textbook Galerkin coarse Laplacian of bilinear interpolation. A dropped
conjugate, a wrong direction, phase sign or hat weight, or a transposed operand changes one of them.
"""
import math

import numpy as np
import pytest

import oracle as o
from paper_1312_2880_gb300 import inputs as I


def _fejer(phi, m):
    """sum_{t=-(m-1)}^{m-1} (1 - |t|/m) e^{i t phi} = sin^2(m phi / 2) / (m sin^2(phi / 2))."""
    s = math.sin(phi / 2)
    return float(m) if abs(s) < 1e-300 else math.sin(m * phi / 2) ** 2 / (m * s * s)


def test_ray_spacing_rule():
    # Table 7's kh = 0.3125: H = 8 h, k H = 2.5; kh = 0.2: H = 8 h (k H = 1.6; 16 h would be 3.2)
    assert [o.ray_spacing(n, k) for k, n in I.PAPER_TABLE7] == [8, 8, 8, 8]
    assert o.ray_spacing(640, 128.0) == 8
    assert o.ray_spacing(16, 20.0) == 2  # at least two ray cells: 16 / 8 = 2 allowed only if k H <= 2.5
    assert o.ray_spacing(12, 1.0) == 4  # 12 / 8 is not an integer


def test_directions_are_the_eight_unit_vectors():
    for j, (dx, dy) in enumerate(o.RAY_DIRECTIONS):
        assert dx == pytest.approx(math.cos(j * math.pi / 4), abs=2.5e-16)
        assert dy == pytest.approx(math.sin(j * math.pi / 4), abs=2.5e-16)
        assert dx * dx + dy * dy == pytest.approx(1.0, abs=4.5e-16)


def test_prolongation_columns_are_hats_times_plane_waves():
    n, m, k = 12, 4, 3.7
    P = o.ray_prolongation(n, m, k).toarray()
    nc = n // m
    for C in range(0, (nc + 1) ** 2, 5):
        Ic, Jc = C % (nc + 1), C // (nc + 1)
        for j in (0, 3, 6):
            dx, dy = math.cos(j * math.pi / 4), math.sin(j * math.pi / 4)
            col = np.zeros((n + 1, n + 1), complex)
            for jj in range(n + 1):
                for i in range(n + 1):
                    w = max(0.0, 1 - abs(i - Ic * m) / m) * max(0.0, 1 - abs(jj - Jc * m) / m)
                    col[jj, i] = w * complex(math.cos(k * (dx * i + dy * jj) / n), math.sin(k * (dx * i + dy * jj) / n))
            assert np.allclose(P[:, 8 * C + j], col.ravel(), rtol=0, atol=1e-13)


def test_galerkin_row_sums_are_fejer_closed_form():
    # interior ray node C = (4, 4) of n = 64, m = 8: its hat and the stencil around it stay inside
    n, m, k = 64, 8, 20.0
    h = 1.0 / n
    A = o.helmholtz_matrix(n, I.constant_k(n, k))
    ray = o.ray_setup(A, n, k, m)
    Ac = ray.Ac.toarray()
    nc = n // m
    C = 4 * (nc + 1) + 4
    X = np.array([4 * m * h, 4 * m * h])
    d = np.array(o.RAY_DIRECTIONS)
    for j in range(8):
        row = Ac[8 * C + j].reshape(-1, 8)  # [C', j']
        for jp in range(8):
            lam = (2 * math.cos(k * d[jp, 0] * h) + 2 * math.cos(k * d[jp, 1] * h) - 4) / h**2 + k * k
            w = k * (d[jp] - d[j])
            expect = lam * np.exp(1j * (w @ X)) * _fejer(w[0] * h, m) * _fejer(w[1] * h, m)
            got = row[:, jp].sum()
            assert abs(got - expect) <= 1e-9 * n * n, (j, jp, got, expect)


def test_galerkin_of_the_laplacian_is_the_textbook_coarse_operator():
    # k = 0: every plane wave is 1, and the (j, j) block is P1^T-Galerkin of the 5-point Laplacian:
    # (1/h^2) [t(dI) s(dJ) + s(dI) t(dJ)], t = (1, -2, 1)/m, s = ((m^2-1)/(6m), (2m^2+1)/(3m), (m^2-1)/(6m))
    n, m = 32, 4
    h = 1.0 / n
    A = o.helmholtz_matrix(n, np.zeros((n + 1, n + 1)))
    _, Ac = o.ray_galerkin(A, o.ray_prolongation(n, m, 0.0))
    Ac = Ac.toarray()
    nc = n // m
    t = {0: -2.0 / m, 1: 1.0 / m}
    s = {0: (2 * m * m + 1) / (3.0 * m), 1: (m * m - 1) / (6.0 * m)}
    for Ic, Jc in ((2, 3), (4, 4), (5, 2)):
        C = Jc * (nc + 1) + Ic
        for dI in (-1, 0, 1):
            for dJ in (-1, 0, 1):
                Cp = (Jc + dJ) * (nc + 1) + Ic + dI
                expect = (t[abs(dI)] * s[abs(dJ)] + s[abs(dI)] * t[abs(dJ)]) / h**2
                for j in (0, 5):
                    assert Ac[8 * C + j, 8 * Cp + j] == pytest.approx(expect, rel=1e-12, abs=1e-9)


def test_correction_reproduces_its_range_and_leaves_an_orthogonal_residual():
    n, k = 64, 20.0
    kf = I.constant_k(n, k) * (1 + 0.1 * np.sin(np.arange((n + 1) ** 2).reshape(n + 1, n + 1)))
    A = o.helmholtz_matrix(n, kf)
    ray = o.ray_setup(A, n, k)
    rng = np.random.default_rng(7)
    c = rng.normal(size=ray.Ac.shape[0]) + 1j * rng.normal(size=ray.Ac.shape[0])
    e = ray.P @ c
    got = ray.correct(A @ e)
    assert np.abs(got - e).max() <= 1e-8 * np.abs(e).max()
    r = rng.normal(size=A.shape[0]) + 1j * rng.normal(size=A.shape[0])
    after = r - A @ ray.correct(r)
    assert np.abs(ray.PH @ after).max() <= 1e-9 * np.abs(ray.PH @ r).max()


def test_table7_hlm_v_converges_only_with_the_ray_correction():
    # Sec. 6: HLM-V alone is no solver; with the ray correction it is (Table 7, k = 20: 16 cycles)
    _, w = I.paper_table7_workloads(max_n=64)[0]
    A = o.helmholtz_matrix(w.n, w.kfield)
    b = w.rhs.ravel()
    H = o.build_hierarchy(w.n, w.kfield, w.k_ref, variant="hlm")
    alone = o.cycle_solve(A, b, H, None, tol=w.tol, maxc=80)
    assert alone.status == "diverged"
    res = o.cycle_solve(A, b, H, o.ray_setup(A, w.n, w.k_ref), tol=w.tol, maxc=40)
    assert res.status == "converged" and res.cycles <= 16
    assert o.true_relres(A, b, res.x) <= w.tol


@pytest.mark.parametrize("variant", ["hlm", "sl", "hyb"])
def test_table7_cycle_counts_do_not_grow_with_k(variant):
    counts = []
    for _, w in I.paper_table7_workloads(max_n=128):
        A = o.helmholtz_matrix(w.n, w.kfield)
        H = o.build_hierarchy(w.n, w.kfield, w.k_ref, variant=variant)
        res = o.cycle_solve(A, w.rhs.ravel(), H, o.ray_setup(A, w.n, w.k_ref), tol=w.tol, maxc=40)
        assert res.status == "converged"
        counts.append(res.cycles)
    assert counts[1] <= counts[0] + 1


def test_cycle_solver_with_an_exact_cycle_stops_after_one(monkeypatch):
    # with the V-cycle replaced by the exact inverse, the first cycle reaches the solution (the ray
    # correction of a zero residual adds nothing), so the loop must stop after one cycle
    import oracle.ray as R
    import scipy.sparse.linalg as spla

    _, w = I.paper_table7_workloads(max_n=64)[0]
    A = o.helmholtz_matrix(w.n, w.kfield)
    lu = spla.splu(A.tocsc())
    monkeypatch.setattr(R, "vcycle", lambda h, r: lu.solve(r))
    res = o.cycle_solve(A, w.rhs.ravel(), None, o.ray_setup(A, w.n, w.k_ref), tol=1e-10, maxc=5)
    assert res.status == "converged" and res.cycles == 1 and res.history[0] <= 1e-12
