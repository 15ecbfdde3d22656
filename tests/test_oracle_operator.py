"""Pins of the oracle's discretisation (Sec. 1, Eqs. 1-3; symbols of Sec. 3) to closed forms."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as o


def _grid(n):
    J, I = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    return I, J


def _boundary_mask(n):
    I, J = _grid(n)
    return ((I == 0) | (I == n) | (J == 0) | (J == n)).ravel()


@pytest.mark.parametrize("shift", [0.0, 0.5])
@pytest.mark.parametrize("theta", [(0.3, 1.1), (np.pi / 2, -2.0), (3.0, 0.0)])
def test_interior_rows_reproduce_the_symbol(shift, theta):
    """On a plane wave e^{i(th1 i + th2 j)} every interior row returns the symbol of Sec. 3,
    (2 cos th1 + 2 cos th2 - 4 + k^2 h^2 (1 + i beta)) / h^2, times the wave."""
    n, k = 24, 17.0
    h = 1.0 / n
    A = o.helmholtz_matrix(n, np.full((n + 1, n + 1), k), shift)
    I, J = _grid(n)
    wave = np.exp(1j * (theta[0] * I + theta[1] * J)).ravel()
    symbol = o.helmholtz_symbol(theta[0], theta[1], k * h, h, shift)
    interior = ~_boundary_mask(n)
    got = (A @ wave)[interior]
    np.testing.assert_allclose(got, symbol * wave[interior], rtol=1e-12, atol=1e-9 / h**2)


def test_boundary_weighted_operator_is_complex_symmetric_with_boundary_damping():
    """With trapezoid weights W (1 inside, 1/2 on edges, 1/4 at corners) the discrete Sommerfeld
    problem is the Galerkin form of Delta + k^2 with the boundary term i k u: W L is complex
    symmetric and Im(W L) = diag(k / h on boundary nodes, 0 inside). A wrong inward factor,
    a wrong sign of i k, or a wrong corner term breaks one of the two statements."""
    n = 12
    rng = np.random.default_rng(5)
    k = 5.0 + 10.0 * rng.random((n + 1, n + 1))
    h = 1.0 / n
    L = o.helmholtz_matrix(n, k, 0.0).toarray()
    I, J = _grid(n)
    w = np.ones((n + 1, n + 1))
    w[(I == 0) | (I == n)] *= 0.5
    w[(J == 0) | (J == n)] *= 0.5
    WL = w.ravel()[:, None] * L
    np.testing.assert_allclose(WL, WL.T, atol=1e-9)
    expect_im = np.where(_boundary_mask(n), k.ravel() / h, 0.0)
    np.testing.assert_allclose(np.imag(WL), np.diag(expect_im), atol=1e-9)
    # The shift adds i k^2 beta on every row (Eq. 3), so Im(W M) gains W k^2 beta.
    M = o.helmholtz_matrix(n, k, 0.5).toarray()
    np.testing.assert_allclose(M - L, np.diag(1j * 0.5 * k.ravel() ** 2), atol=1e-9)


def test_boundary_rows_are_consistent_with_the_sommerfeld_condition():
    """u = exp(i k x) solves Delta u + k^2 u = 0 and meets du/dn - i k u = 0 exactly on x = 1.
    The discrete rows there must vanish as h -> 0 at first order (the ghost elimination has an
    O(h^3) defect, divided by h^2); interior rows vanish at second order."""
    k = 6.0
    errs_b, errs_i = [], []
    for n in (16, 32, 64, 128):
        I, J = _grid(n)
        x = I / n
        u = np.exp(1j * k * x).ravel()
        A = o.helmholtz_matrix(n, np.full((n + 1, n + 1), k), 0.0)
        res = np.abs(A @ u)
        edge = ((I == n) & (J > 0) & (J < n)).ravel()
        inner = ((I > 0) & (I < n) & (J > 0) & (J < n)).ravel()
        errs_b.append(res[edge].max())
        errs_i.append(res[inner].max())
    ratios_b = np.array(errs_b[:-1]) / np.array(errs_b[1:])
    ratios_i = np.array(errs_i[:-1]) / np.array(errs_i[1:])
    assert np.all(np.abs(ratios_b - 2.0) < 0.1), ratios_b
    assert np.all(np.abs(ratios_i - 4.0) < 0.1), ratios_i


def test_ghost_elimination_equals_padded_interior_stencil():
    """A boundary row equals the interior 5-point row applied to the grid extended by ghost nodes
    whose values come from the centred difference of du/dn - i k u = 0 across the boundary."""
    n = 10
    h = 1.0 / n
    rng = np.random.default_rng(1)
    k = 3.0 + rng.random((n + 1, n + 1)) * 20
    u = rng.standard_normal((n + 1, n + 1)) + 1j * rng.standard_normal((n + 1, n + 1))
    ext = np.zeros((n + 3, n + 3), dtype=complex)
    ext[1:-1, 1:-1] = u
    # outward normal derivative by a centred difference: (u_ghost - u_mirror) / (2h) = i k u_b
    ext[1:-1, 0] = u[:, 1] + 2j * k[:, 0] * h * u[:, 0]
    ext[1:-1, -1] = u[:, -2] + 2j * k[:, -1] * h * u[:, -1]
    ext[0, 1:-1] = u[1, :] + 2j * k[0, :] * h * u[0, :]
    ext[-1, 1:-1] = u[-2, :] + 2j * k[-1, :] * h * u[-1, :]
    lap = (ext[1:-1, 2:] + ext[1:-1, :-2] + ext[2:, 1:-1] + ext[:-2, 1:-1] - 4 * u) / h**2
    expect = (lap + k**2 * u).ravel()
    got = o.helmholtz_matrix(n, k, 0.0) @ u.ravel()
    np.testing.assert_allclose(got, expect, rtol=1e-12, atol=1e-9)


def test_l_is_nonsingular_and_matches_dense_solution():
    n, k = 16, 20.0
    A = o.helmholtz_matrix(n, np.full((n + 1, n + 1), k))
    b = np.zeros((n + 1) ** 2, complex)
    b[(n // 2) * (n + 1) + n // 2] = n * n
    x = sp.linalg.spsolve(A.tocsc(), b)
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) < 1e-12
    assert np.linalg.cond(A.toarray()) < 1e6
