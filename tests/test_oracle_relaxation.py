"""Pins of the oracle's transfers (Sec. 5), Gauss-Seidel (Sec. 4) and Kaczmarz (Sec. 4-5)."""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grid(n):
    J, I = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    return I, J


def _level(n, k, op="L", smoother="gs", beta=0.5):
    kf = np.full((n + 1, n + 1), k) if np.isscalar(k) else k
    A = o.helmholtz_matrix(n, kf, beta if op == "M" else 0.0)
    lv = o.OracleLevel(n, 1.0 / n, kf, op, smoother, op, 1, A, A, o.full_weighting(n), o.bilinear_prolongation(n))
    o.helmholtz._prepare_relaxation(lv)
    return lv


# --------------------------------------------------------------------------- transfers


def test_prolongation_is_exact_on_bilinear_functions():
    n = 16
    Ic, Jc = _grid(n // 2)
    If, Jf = _grid(n)
    f = lambda x, y: 1.5 - 2.0 * x + 0.7 * y + 3.1 * x * y  # noqa: E731
    coarse = f(Ic * 2.0 / n, Jc * 2.0 / n).ravel()
    fine = f(If / n, Jf / n).ravel()
    np.testing.assert_allclose(o.bilinear_prolongation(n) @ coarse, fine, rtol=0, atol=1e-13)


def test_full_weighting_preserves_constants_and_is_quarter_transpose_inside():
    n = 16
    R = o.full_weighting(n)
    P = o.bilinear_prolongation(n)
    np.testing.assert_allclose(R @ np.ones((n + 1) ** 2), 1.0, atol=1e-15)
    Ic, Jc = _grid(n // 2)
    inner = ((Ic > 0) & (Ic < n // 2) & (Jc > 0) & (Jc < n // 2)).ravel()
    np.testing.assert_allclose(R.toarray()[inner], 0.25 * P.T.toarray()[inner], atol=1e-15)
    # weights of an interior row: 1/16 [1 2 1; 2 4 2; 1 2 1]
    row = R.toarray()[(n // 4) * (n // 2 + 1) + n // 4].reshape(n + 1, n + 1)
    c = n // 2
    np.testing.assert_allclose(row[c - 1:c + 2, c - 1:c + 2] * 16, [[1, 2, 1], [2, 4, 2], [1, 2, 1]])
    assert abs(row.sum() - 1) < 1e-15 and np.count_nonzero(row) == 9


def test_full_weighting_mirrors_at_the_boundary():
    n = 8
    R = o.full_weighting(n).toarray()
    # coarse corner (0, 0): fine (0,0) 4/16, (1,0) and (0,1) 2*2/16 each, (1,1) 4*1/16
    row = R[0].reshape(n + 1, n + 1)
    np.testing.assert_allclose(row[:2, :2] * 16, [[4, 4], [4, 4]])


# --------------------------------------------------------------------------- Gauss-Seidel


@pytest.mark.parametrize("op", ["L", "M"])
@pytest.mark.parametrize("first", [0, 1])
def test_red_black_sweep_equals_gauss_seidel_in_colour_order(op, first):
    """The colour-parallel sweep is Gauss-Seidel in the ordering 'all of one colour, then the other',
    computed here by a general triangular solve in that ordering."""
    n = 12
    rng = np.random.default_rng(2)
    k = 10 + 20 * rng.random((n + 1, n + 1))
    lv = _level(n, k, op)
    f = rng.standard_normal((n + 1) ** 2) + 1j * rng.standard_normal((n + 1) ** 2)
    u = rng.standard_normal((n + 1) ** 2) + 1j * rng.standard_normal((n + 1) ** 2)
    col = o.red_black_colours(n)
    order = np.concatenate([np.nonzero(col == first)[0], np.nonzero(col == 1 - first)[0]])
    got = o.rb_gs_sweep(lv, f, u, first=first)
    ref = o.lex_gs_sweep(lv.A, f, u, order)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    # the colour relaxed last has zero residual
    last = col == 1 - first
    res = f - lv.A @ got
    assert np.abs(res[last]).max() < 1e-10 * np.abs(f).max()


@pytest.mark.parametrize("kH,beta", [(0.3125, 0.0), (0.3125, 0.5), (5.0, 0.0), (5.0, 0.5)])
@pytest.mark.parametrize("theta", [(2.0, 2.5), (np.pi / 2, 3.0), (-2.2, 1.7), (2.9, -0.4)])
def test_lexicographic_gs_reproduces_the_fourier_amplification(kH, beta, theta):
    """One lexicographic sweep on f = 0 multiplies a Fourier mode by the factor of Sec. 4
    away from the boundaries where the sweep starts. The sweep runs in +i, +j, so its factor
    is the printed formula at -theta (identical modulus for HLM; reading for SL)."""
    n = 160
    k = kH * n
    A = o.helmholtz_matrix(n, np.full((n + 1, n + 1), k), beta)
    I, J = _grid(n)
    e0 = np.exp(1j * (theta[0] * I + theta[1] * J)).ravel()
    e1 = o.lex_gs_sweep(A, np.zeros_like(e0), e0)
    m = 60
    win = ((I >= m) & (I <= n - 2) & (J >= m) & (J <= n - 2)).ravel()
    ratio = np.abs(e1[win] / e0[win])
    mu = o.gs_amplification(-theta[0], -theta[1], kH, beta)
    np.testing.assert_allclose(ratio, mu, rtol=1e-9)


def test_printed_gauss_seidel_rates():
    """The paper's printed rates (Sec. 4) from its own formula; the golden file cites each entry."""
    g = json.load(open(os.path.join(GOLDEN, "lfa_printed.json")))
    for e in g["pinned"]:
        for var, beta in (("hlm", 0.0), ("sl", 0.5)):
            if e["quantity"] == "smoothing_factor":
                val = o.smoothing_factor(e["kH"], beta)
                assert abs(val - e[var]) <= 0.08 * e[var], (e, var, val)
            elif e["quantity"] == "overall_rate":
                val = o.overall_rate(e["kH"], beta)
                assert abs(val - e[var]) <= 0.08 * e[var], (e, var, val)
            else:  # printed as an upper bound
                val = o.overall_rate(e["kH"], beta)
                assert val <= e[var] * 1.005, (e, var, val)


def test_overall_rate_closed_form_on_fine_scales():
    """For L on fine scales the worst mode is the smoothest, theta = 0: mu^ = 2 / |2 - k^2 H^2|.
    For M the value at theta = 0, 2 / |2 - k^2 H^2 (1 + i beta)|, is a lower bound within 1%."""
    for kH in (0.1, 0.2, 0.3125):
        assert abs(o.overall_rate(kH, 0.0) - 2.0 / abs(2 - kH * kH)) < 1e-12
        at0 = 2.0 / abs(2 - kH * kH * (1 + 0.5j))
        assert at0 * (1 - 1e-14) <= o.overall_rate(kH, 0.5) <= 1.01 * at0


def test_shifted_symbol_ratio_imaginary_part_on_fine_scales():
    """Sec. 3, first bullet: for kH <= 0.625, oscillatory components have Im tau^SL <= .1 and
    Re tau^SL close to tau^HLM. Fig. 1, which the bullet summarises, shows omega_1 = omega_2 only."""
    k, h = 20.0, 1.0 / 64
    H = 2 * h
    t = np.linspace(np.pi / 2, np.pi, 257) / H
    sl = o.symbol_ratio(t, t, k, h, H, 0.5)
    hlm = o.symbol_ratio(t, t, k, h, H, 0.0)
    assert np.abs(sl.imag).max() <= 0.1
    assert np.abs(sl.real - hlm.real).max() <= 0.05


def test_red_black_two_colour_analysis_behind_the_guard():
    """On a periodic grid one red-black sweep (f = 0) maps span{e_th, e_(th+(pi,pi))} into itself by a
    rank-one matrix with eigenvalue (S/d)^2, S = 2 cos th1 + 2 cos th2, d the diagonal. This is the
    analysis that places the L-relaxation guard at 1 < kH < 2 sqrt 2."""
    m = 16
    N = m * m
    idx = np.arange(N).reshape(m, m)
    for kH in (0.3, 2.5, 3.2):
        d = -4 + kH * kH
        rows, cols, vals = [], [], []
        for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            rows.append(idx.ravel()); cols.append(np.roll(np.roll(idx, -dj, 0), -di, 1).ravel()); vals.append(np.ones(N))
        rows.append(idx.ravel()); cols.append(idx.ravel()); vals.append(np.full(N, d))
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N)).tocsr()
        J, I = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
        col = ((I + J) % 2).ravel()
        order = np.concatenate([np.nonzero(col == 0)[0], np.nonzero(col == 1)[0]])
        th = (2 * np.pi * 3 / m, 2 * np.pi * 2 / m)
        e1 = np.exp(1j * (th[0] * I + th[1] * J)).ravel()
        e2 = np.exp(1j * ((th[0] + np.pi) * I + (th[1] + np.pi) * J)).ravel()
        G = np.zeros((2, 2), complex)
        for c, e in enumerate((e1, e2)):
            out = o.lex_gs_sweep(A, np.zeros(N, complex), e, order)
            coef = np.linalg.lstsq(np.stack([e1, e2], 1), out, rcond=None)[0]
            assert np.linalg.norm(np.stack([e1, e2], 1) @ coef - out) < 1e-10
            G[:, c] = coef
        S = 2 * math.cos(th[0]) + 2 * math.cos(th[1])
        ev = np.linalg.eigvals(G)
        np.testing.assert_allclose(sorted(np.abs(ev)), sorted([0.0, (S / d) ** 2]), atol=1e-12)


# --------------------------------------------------------------------------- Kaczmarz


def test_kaczmarz_colours_separate_stencils():
    n = 20
    col = o.kaczmarz_colours(n).reshape(n + 1, n + 1)
    A = o.helmholtz_matrix(n, np.full((n + 1, n + 1), 30.0))
    S = (abs(A) > 0).astype(int)
    C = (S @ S.T).tocoo()  # rows that share a column
    same = col.ravel()[C.row] == col.ravel()[C.col]
    assert np.all(C.row[same] == C.col[same])


@pytest.mark.parametrize("op", ["L", "M"])
def test_kaczmarz_sweep_equals_sequential_projections(op):
    """The colour-parallel sweep equals one-row-at-a-time Kaczmarz projections taken in colour order
    (rows of a colour in index order)."""
    n = 8
    rng = np.random.default_rng(3)
    k = 20 + 10 * rng.random((n + 1, n + 1))
    lv = _level(n, k, op, "kaczmarz")
    A = lv.A.toarray()
    f = rng.standard_normal((n + 1) ** 2) + 1j * rng.standard_normal((n + 1) ** 2)
    u0 = rng.standard_normal((n + 1) ** 2) + 1j * rng.standard_normal((n + 1) ** 2)
    for order in ((0, 1, 2, 3, 4), (4, 3, 2, 1, 0)):
        col = o.kaczmarz_colours(n)
        u = u0.copy()
        for c in order:
            for p in np.nonzero(col == c)[0]:
                a = A[p]
                u = u + np.conj(a) * (f[p] - a @ u) / np.vdot(a, a).real
        got = o.kaczmarz_sweep(lv, f, u0, order)
        np.testing.assert_allclose(got, u, rtol=1e-12, atol=1e-12 * np.abs(u).max())


def test_kaczmarz_error_is_monotone_on_consistent_systems():
    """Each row step is an orthogonal projection onto that row's solution hyperplane, so the
    Euclidean error never grows (Kaczmarz convergence), even at kH ~ 1.25 where GS diverges."""
    n = 16
    k = 1.25 * n
    lv = _level(n, k, "M", "kaczmarz")
    rng = np.random.default_rng(4)
    xs = rng.standard_normal((n + 1) ** 2) + 1j * rng.standard_normal((n + 1) ** 2)
    f = lv.A @ xs
    u = np.zeros_like(f)
    errs = [np.linalg.norm(u - xs)]
    for _ in range(6):
        u = o.kaczmarz_sweep(lv, f, u)
        errs.append(np.linalg.norm(u - xs))
    assert all(b <= a * (1 + 1e-14) for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < errs[0]
    # the rows of the last colour have zero residual after the sweep
    res = f - lv.A @ u
    last = o.kaczmarz_colours(n) == 4
    assert np.abs(res[last]).max() < 1e-9 * np.abs(f).max()


# --------------------------------------------------------------------------- Jacobi and SOR
# The alternatives the remark of Sec. 4 names: damped Jacobi and (red-black) SOR.


def _periodic_level(m, kH, beta, smoother, omega):
    """An m x m periodic grid with the h^2-scaled 5-point row (neighbours 1, diagonal
    -4 + (kH)^2 (1 + i beta)) wrapped in an OracleLevel, so the oracle's own sweeps run on it."""
    N = m * m
    idx = np.arange(N).reshape(m, m)
    d = -4 + kH * kH * (1 + 1j * beta)
    rows, cols, vals = [], [], []
    for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
        rows.append(idx.ravel()); cols.append(np.roll(np.roll(idx, -dj, 0), -di, 1).ravel()); vals.append(np.ones(N))
    rows.append(idx.ravel()); cols.append(idx.ravel()); vals.append(np.full(N, d))
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N)).tocsr()
    lv = o.OracleLevel(m - 1, 1.0, np.zeros((m, m)), "L", smoother, "L", 1, A, omega=omega)
    o.helmholtz._prepare_relaxation(lv)
    J, I = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    return lv, I, J


@pytest.mark.parametrize("kH,beta,omega", [(0.3125, 0.0, 0.8), (1.25, 0.5, 0.8), (2.5, 0.0, 0.6), (5.0, 0.5, 1.0)])
def test_jacobi_sweep_multiplies_each_fourier_mode(kH, beta, omega):
    from oracle import lfa

    m = 16
    lv, I, J = _periodic_level(m, kH, beta, "jacobi", omega)
    for th in ((2 * np.pi * 3 / m, 2 * np.pi * 1 / m), (2 * np.pi * 7 / m, 2 * np.pi * 6 / m)):
        e = np.exp(1j * (th[0] * I + th[1] * J)).ravel()
        out = o.jacobi_sweep(lv, np.zeros_like(e), e)
        d = -4 + kH * kH * (1 + 1j * beta)
        g = 1 - omega * (2 * math.cos(th[0]) + 2 * math.cos(th[1]) + d) / d
        np.testing.assert_allclose(out, g * e, rtol=0, atol=1e-12)
        assert abs(abs(g) - lfa.jacobi_amplification(th[0], th[1], kH, beta, omega)) < 1e-13


@pytest.mark.parametrize("kH,beta,omega", [(0.3, 0.0, 1.0), (1.25, 0.5, 1.2), (2.5, 0.0, 0.7), (3.2, 0.5, 1.0)])
def test_red_black_sor_sweep_is_the_two_harmonic_matrix(kH, beta, omega):
    """One red-black SOR sweep of the oracle maps span{e_th, e_(th+(pi,pi))} into itself by exactly the
    2 x 2 matrix derived in lfa.rb_sor_two_harmonic (omega = 1: the Gauss-Seidel analysis above)."""
    from oracle import lfa

    m = 16
    lv, I, J = _periodic_level(m, kH, beta, "sor", omega)
    th = (2 * np.pi * 3 / m, 2 * np.pi * 2 / m)
    e1 = np.exp(1j * (th[0] * I + th[1] * J)).ravel()
    e2 = np.exp(1j * ((th[0] + np.pi) * I + (th[1] + np.pi) * J)).ravel()
    G = np.zeros((2, 2), complex)
    for c, e in enumerate((e1, e2)):
        out = o.rb_sor_sweep(lv, np.zeros_like(e), e, first=0)
        coef = np.linalg.lstsq(np.stack([e1, e2], 1), out, rcond=None)[0]
        assert np.linalg.norm(np.stack([e1, e2], 1) @ coef - out) < 1e-10
        G[:, c] = coef
    np.testing.assert_allclose(G, lfa.rb_sor_two_harmonic(th[0], th[1], kH, beta, omega), atol=1e-12)


def test_textbook_smoothing_factors_of_the_laplacian():
    """kH = 0 is the Poisson 5-point stencil, whose factors are textbook values: damped Jacobi with
    omega = 4/5 smooths by 3/5, red-black Gauss-Seidel by 1/4."""
    from oracle import lfa

    assert abs(lfa.jacobi_smoothing_factor(0.0, 0.0, 0.8) - 0.6) < 1e-12
    assert abs(lfa.rb_smoothing_factor(0.0, 0.0, 1.0) - 0.25) < 1e-12


def test_sor_with_omega_one_is_gauss_seidel():
    n, k = 32, 12.0
    kf = np.full((n + 1, n + 1), k)
    f = np.random.default_rng(3).standard_normal((n + 1) ** 2) + 0j
    z_gs = o.vcycle(o.build_hierarchy(n, kf, k, "hyb"), f)
    z_sor = o.vcycle(o.build_hierarchy(n, kf, k, "hyb", gs_smoother="sor", omega=1.0), f)
    assert np.array_equal(z_gs, z_sor)
    H = o.build_hierarchy(n, kf, k, "hyb", gs_smoother="jacobi")
    assert [lv.smoother for lv in H.levels] == ["jacobi" if s == "gs" else s
                                                for s in (lv.smoother for lv in o.build_hierarchy(n, kf, k, "hyb").levels)]
    assert all(lv.omega == 0.8 for lv in H.levels if lv.smoother == "jacobi")
