"""Pins of the oracle's V-cycle (Sec. 5), level policy (Sec. 5) and Bi-CGSTAB (Sec. 6)."""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import oracle as o
from paper_1312_2880_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- dense restatement


def _gs_affine(A, n, first):
    """Dense (G, S) of one Gauss-Seidel sweep u <- G u + S f in the ordering colour `first`, then the other:
    with D + L the lower triangle and U the strict upper triangle of the permuted matrix,
    u_new = (D + L)^{-1} (f - U u)."""
    col = o.red_black_colours(n)
    perm = np.concatenate([np.nonzero(col == first)[0], np.nonzero(col == 1 - first)[0]])
    Ap = A[np.ix_(perm, perm)]
    T = np.tril(Ap)
    Uu = np.triu(Ap, 1)
    Ti = sla.solve_triangular(T, np.eye(len(perm)), lower=True)
    Pm = np.eye(len(perm))[perm]  # Pm @ u = u[perm]
    return -Pm.T @ Ti @ Uu @ Pm, Pm.T @ Ti @ Pm


def _kaczmarz_affine(A, n, order):
    """Dense (G, S) of one sweep of row projections u <- u + a_p^H (f_p - a_p u) / |a_p|^2, rows in colour order."""
    N = A.shape[0]
    G, S = np.eye(N, dtype=complex), np.zeros((N, N), complex)
    col = o.kaczmarz_colours(n)
    for c in order:
        for p in np.nonzero(col == c)[0]:
            a = A[p]
            w = np.conj(a) / np.vdot(a, a).real
            G = G - np.outer(w, a @ G)
            S = S - np.outer(w, a @ S)
            S[:, p] += w
    return G, S


def _dense_vcycle(h, level=0):
    lv = h.levels[level]
    if lv.smoother == "direct":
        return np.linalg.inv(lv.A.toarray())
    A, B = lv.A.toarray(), lv.B.toarray()
    N = A.shape[0]
    if lv.smoother == "gs":
        pre, post = _gs_affine(A, lv.n, 0), _gs_affine(A, lv.n, 1)
    else:
        pre, post = _kaczmarz_affine(A, lv.n, (0, 1, 2, 3, 4)), _kaczmarz_affine(A, lv.n, (4, 3, 2, 1, 0))
    U = np.zeros((N, N), complex)
    for _ in range(lv.nu):
        U = pre[0] @ U + pre[1]
    Kc = _dense_vcycle(h, level + 1)
    U = U + lv.P.toarray() @ Kc @ lv.R.toarray() @ (np.eye(N) - B @ U)
    for _ in range(lv.nu):
        U = post[0] @ U + post[1]
    return U


@pytest.mark.parametrize(
    "n,levels,ops",
    [
        (8, 2, [("M", "gs", "M")]),
        (8, 2, [("M", "gs", "L")]),
        (16, 3, [("L", "gs", "L"), ("M", "kaczmarz", "L")]),
        (16, 3, [("M", "kaczmarz", "M"), ("L", "gs", "L")]),
    ],
)
def test_vcycle_equals_product_of_dense_operators(n, levels, ops):
    """From a zero guess the V-cycle is linear in f; its matrix equals the composition
    S_post (u + P K_c R (f - B u)) of S_pre, built here from dense triangular solves and
    dense row projections, with K_c the next level's operator (the inverse on the coarsest)."""
    rng = np.random.default_rng(7)
    kf = 1.1 * n + 0.3 * n * rng.random((n + 1, n + 1))
    h = o.build_hierarchy(n, kf, k_ref=1.25 * n, variant="hyb", levels=levels, ops=ops)
    N = (n + 1) ** 2
    Kv = np.stack([o.vcycle(h, np.eye(N, dtype=complex)[:, j]) for j in range(N)], axis=1)
    Kd = _dense_vcycle(h)
    np.testing.assert_allclose(Kv, Kd, rtol=1e-10, atol=1e-10 * np.abs(Kd).max())


def test_coarsest_lu_backward_error():
    n = 8
    kf = np.full((n + 1, n + 1), 40.0)
    h = o.build_hierarchy(n, kf, 40.0, "hyb", levels=1)
    A = h.levels[0].A.toarray()
    f = np.random.default_rng(0).standard_normal(A.shape[0]) + 0j
    u = o.vcycle(h, f)
    assert np.linalg.norm(A @ u - f) <= 1e-13 * np.linalg.norm(A) * np.linalg.norm(u)


# --------------------------------------------------------------------------- policy


def _sched(h):
    return [(lv.relax_op, lv.smoother, lv.resid_op) for lv in h.levels]


def test_policy_table1_setting():
    """k = 40, h = 1/64 (Table 1): scales kH = 0.625, 1.25, 2.5, 5. HYB relaxes M at 0.625 and 1.25
    (Kaczmarz at 1.25, and with the band rule also at 2.5 < 2 sqrt 2), L residuals everywhere, L on
    the coarsest; SL is M throughout; HLM is L."""
    kf = I.constant_k(64, 40.0)
    hyb = _sched(o.build_hierarchy(64, kf, 40.0, "hyb", 4))
    assert hyb[0] == ("M", "gs", "L") and hyb[1] == ("M", "kaczmarz", "L")
    assert hyb[2] == ("M", "kaczmarz", "L")  # band: kH = 2.5 in [0.625 sqrt 2, 2 sqrt 2)
    assert hyb[3] == ("L", "direct", "L")
    assert _sched(o.build_hierarchy(64, kf, 40.0, "sl", 4)) == [("M", "gs", "M"), ("M", "kaczmarz", "M"), ("M", "kaczmarz", "M"), ("M", "direct", "M")]
    assert _sched(o.build_hierarchy(64, kf, 40.0, "hlm", 4)) == [("L", "gs", "L"), ("L", "kaczmarz", "L"), ("L", "kaczmarz", "L"), ("L", "direct", "L")]
    bins = _sched(o.build_hierarchy(64, kf, 40.0, "hyb", 4, rule="bins"))
    assert bins[2] == ("M", "gs", "L")  # bins: Gauss-Seidel, guard 1 < kH = 2.5 < 2 sqrt 2 gives M
    assert o.build_hierarchy(64, kf, 40.0, "hyb", 4, guard=False, rule="bins").levels[2].relax_op == "L"


def test_policy_wedge_n512():
    """Layers k * {1.0, 1.5, 0.75}: level l spans k H from 75/n_l to 150/n_l. Band rule: Kaczmarz on
    n_l = 128 (0.59 .. 1.17), 64 (1.17 .. 2.34) and 32 (2.34 .. 4.69); bins: on n_l = 64 only."""
    wl = I.wedge_n512()
    h = o.build_hierarchy(wl.n, wl.kfield, wl.k_ref, wl.variant, wl.levels)
    assert [lv.n for lv in h.levels] == [512, 256, 128, 64, 32, 16, 8, 4]
    ops = [(a[0] + ("k" if a[1] == "kaczmarz" else "")) for a in _sched(h)]
    assert ops == ["L", "L", "Mk", "Mk", "Mk", "L", "L", "L"]
    assert all(lv.resid_op == "L" for lv in h.levels)
    sch = o.schedule(wl.n, wl.kfield, wl.k_ref, wl.variant, wl.levels, rule="bins")
    assert [a[1] + ("k" if a[2] == "kaczmarz" else "") for a in sch] == ["L", "L", "M", "Mk", "M", "L", "L", "L"]


def test_kaczmarz_band_edges_follow_the_red_black_analysis():
    """The band rule's upper edge: one red-black sweep on L maps the Fourier pair {theta, theta+(pi,pi)}
    with eigenvalue (S/d)^2, d = -4 + (kH)^2, |S| <= 4 reached by the smoothest pair and its
    oscillatory partner; it exceeds 1 for some pair exactly when |d| < 4, i.e. kH < 2 sqrt 2 (for
    kH > 0). The lower edge is the geometric midpoint of the paper's 0.625 and 1.25 scales. A level
    relaxes by Kaczmarz exactly when some node's k H lies in [lower, upper)."""
    lo, hi = o.KACZ_BAND
    assert lo == pytest.approx(math.sqrt(0.625 * 1.25)) and hi == pytest.approx(2 * math.sqrt(2))
    # measured: growth per red-black sweep (f = 0) of a random error on a periodic 16 x 16 grid,
    # whose Fourier pairs include S = 4 and -4; the analysis gives the rate (4/d)^2
    m, N = 16, 256
    idx = np.arange(N).reshape(m, m)
    J, Ii = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    col = ((Ii + J) % 2).ravel()
    order = np.concatenate([np.nonzero(col == 0)[0], np.nonzero(col == 1)[0]])
    for kH in (2.6, 2.75, 2.9, 3.2):
        d = -4 + kH * kH
        rows, cols, vals = [], [], []
        for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            rows.append(idx.ravel()); cols.append(np.roll(np.roll(idx, -dj, 0), -di, 1).ravel()); vals.append(np.ones(N))
        rows.append(idx.ravel()); cols.append(idx.ravel()); vals.append(np.full(N, d))
        import scipy.sparse as sp
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N)).tocsr()
        e = np.random.default_rng(1).standard_normal(N) + 0j
        for _ in range(400):
            e = o.lex_gs_sweep(A, np.zeros(N, complex), e, order)
            e /= np.linalg.norm(e)
        rate = np.linalg.norm(o.lex_gs_sweep(A, np.zeros(N, complex), e, order))
        assert rate == pytest.approx((4 / d) ** 2, rel=1e-6)
        assert (rate > 1.0) == (kH < hi)
    rng = np.random.default_rng(3)
    for variant in ("hyb", "sl", "hlm"):
        for _ in range(200):
            c = float(rng.uniform(0.05, 6.0))
            c_local = c * rng.uniform(0.6, 1.4, size=7)
            expect = bool(np.any((c_local >= lo) & (c_local < hi)))
            assert (o.level_policy(variant, c, c_local)[1] == "kaczmarz") == expect
            if variant == "hyb" and expect:
                assert o.level_policy(variant, c, c_local)[0] == "M"


def test_schedule_matches_built_hierarchy():
    for wl in (I.wedge_n512(), I.grf_n4096(n=256, k=62.5), I.plain_n64()):
        for rule in ("band", "bins"):
            h = o.build_hierarchy(wl.n, wl.kfield, wl.k_ref, wl.variant, wl.levels, rule=rule)
            assert o.schedule(wl.n, wl.kfield, wl.k_ref, wl.variant, wl.levels, rule=rule) == [
                (lv.n, lv.relax_op, lv.smoother, lv.resid_op) for lv in h.levels]


def test_policy_fine_hyb_uses_l():
    """kH = 0.3125 (Table 2 finest scales): HYB relaxes with L."""
    kf = I.constant_k(128, 40.0)
    assert o.build_hierarchy(128, kf, 40.0, "hyb", 5).levels[0].relax_op == "L"


def test_auto_levels():
    assert [lv.n for lv in o.build_hierarchy(96, I.constant_k(96, 50.0), 50.0).levels] == [96, 48, 24, 12, 6]
    assert [lv.n for lv in o.build_hierarchy(64, I.constant_k(64, 20.0), 20.0).levels] == [64, 32, 16, 8]


# --------------------------------------------------------------------------- Bi-CGSTAB


def _problem(n=32, k=20.0):
    kf = I.constant_k(n, k)
    A = o.helmholtz_matrix(n, kf)
    b = I.centre_source_rhs(n).ravel()
    return n, kf, A, b


def test_bicgstab_with_exact_preconditioner_stops_at_the_first_half_step():
    n, kf, A, b = _problem()
    lu = spla.splu(A.tocsc())
    res = o.bicgstab(A, b, lu.solve, tol=1e-10)
    assert res.iterations == 0.5 and res.status == "converged"
    np.testing.assert_allclose(res.x, lu.solve(b), rtol=1e-12)


@pytest.mark.parametrize("precond", ["none", "sl_vcycle"])
def test_bicgstab_iterates_match_an_independent_implementation(precond):
    """With the same shadow residual (r^ = b, as scipy uses) the iterates equal scipy's Bi-CGSTAB,
    which is also right-preconditioned with the inner product conjugated in its first argument."""
    n, kf, A, b = _problem()
    if precond == "none":
        K = None
        M = None
    else:
        h = o.build_hierarchy(n, kf, 20.0, "sl")
        K = lambda v: o.vcycle(h, v)  # noqa: E731
        M = spla.LinearOperator(A.shape, matvec=K, dtype=complex)
    mine, ref = [], []
    o.bicgstab(A, b, K, tol=1e-30, maxit=8, callback=lambda x: mine.append(x.copy()), rhat=b)
    spla.bicgstab(A, b, M=M, rtol=1e-30, atol=0, maxiter=8, callback=lambda x: ref.append(x.copy()))
    assert len(mine) == len(ref) == 8
    for a, r in zip(mine, ref):
        np.testing.assert_allclose(a, r, rtol=1e-9, atol=1e-9 * np.abs(r).max())


def test_shadow_renewal_is_a_fresh_start_of_an_independent_implementation():
    """Renewing the shadow residual after a full step (forced here: every step, up to the cap) takes
    p = r and rho = <rhat_new, r>, i.e. Bi-CGSTAB starts afresh from the current iterate. With the
    renewed shadow residual set to the current residual (scipy's choice of r^ at a start), the
    iterates equal a chain of one-iteration scipy solves, each started from the previous iterate."""
    n, kf, A, b = _problem()
    h = o.build_hierarchy(n, kf, 20.0, "sl")
    K = lambda v: o.vcycle(h, v)  # noqa: E731
    M = spla.LinearOperator(A.shape, matvec=K, dtype=complex)
    mine = []
    res = o.bicgstab(A, b, K, tol=1e-30, maxit=6, callback=lambda x: mine.append(x.copy()), rhat=b,
                     stall_cos2=2.0, stall_step2=np.inf, max_shadow_restarts=4,
                     renew_shadow=lambda k, r: r.copy())
    assert res.shadow_restarts == 4 and res.status == "maxit" and len(mine) == 6
    ref, x = [], np.zeros_like(b)
    for it in range(6):
        if it <= 4:  # renewed before iterations 2..5: each one a fresh start from the last iterate
            x, _ = spla.bicgstab(A, b, x0=x, M=M, rtol=1e-30, atol=0, maxiter=1)
            ref.append(x.copy())
    # iteration 6 continues iteration 5's recurrence (renewals used up): two scipy iterations from x4
    two = []
    spla.bicgstab(A, b, x0=ref[3], M=M, rtol=1e-30, atol=0, maxiter=2, callback=lambda z: two.append(z.copy()))
    ref[4:] = two
    for a, r in zip(mine, ref):
        np.testing.assert_allclose(a, r, rtol=1e-9, atol=1e-9 * np.abs(r).max())


def test_seeded_shadow_renewals_follow_the_generator():
    """The k-th renewed shadow residual is SplitMix64 started from SHADOW_SEED + k * step (mod 2^64)."""
    assert o.renewed_shadow_seed(1) == (0x5EED1312 + 0x2545F4914F6CDD1D) % 2**64
    assert o.renewed_shadow_seed(7) == (0x5EED1312 + 7 * 0x2545F4914F6CDD1D) % 2**64
    n, kf, A, b = _problem(16, 10.0)
    seen = []
    o.bicgstab(A, b, None, tol=1e-30, maxit=3, stall_cos2=2.0, stall_step2=np.inf, max_shadow_restarts=2,
               renew_shadow=lambda k, r: (seen.append(k), o.shadow_residual(b.size, o.renewed_shadow_seed(k)))[1])
    assert seen == [1, 2]
    a = o.bicgstab(A, b, None, tol=1e-30, maxit=3, stall_cos2=2.0, stall_step2=np.inf, max_shadow_restarts=2)
    c = o.bicgstab(A, b, None, tol=1e-30, maxit=3, stall_cos2=2.0, stall_step2=np.inf, max_shadow_restarts=2,
                   renew_shadow=lambda k, r: o.shadow_residual(b.size, o.renewed_shadow_seed(k)))
    assert np.array_equal(a.x, c.x)


def test_true_residual_restart_below_the_attainable_accuracy():
    """A tolerance below what FP64 can reach: the recurrence residual keeps falling while b - A x
    stalls, so every recurrence stop is refused by the true residual and the solve restarts from it
    (r = b - A x, p = r) until the cap; it then ends unconfirmed (status maxit) with x still at the
    attainable accuracy. After each restart the recurrence residual starts again from the true one."""
    n, kf, A, b = _problem()
    h = o.build_hierarchy(n, kf, 20.0, "sl")
    res = o.bicgstab(A, b, lambda v: o.vcycle(h, v), tol=1e-18, maxit=400)
    assert res.restarts == o.MAX_TRUE_RESTARTS and res.status == "maxit"
    assert res.true_relres <= 1e-13
    xs = spla.spsolve(A.tocsc(), b)
    assert np.linalg.norm(res.x - xs) / np.linalg.norm(xs) < 1e-10
    # the history drops below 1e-18 once per stop (restarts + 1 times), rising again after each
    below = [q for q, v in enumerate(res.history) if v <= 1e-18]
    assert len(below) == o.MAX_TRUE_RESTARTS + 1
    for q in below[:-1]:
        assert res.history[q + 1] > 1e2 * res.history[q]
    # with the cap at zero the first refused stop ends the solve
    one = o.bicgstab(A, b, lambda v: o.vcycle(h, v), tol=1e-18, maxit=400, max_true_restarts=0)
    assert one.restarts == 0 and one.status == "maxit" and one.history[-1] <= 1e-18


def test_bicgstab_solution_matches_direct_solve():
    n, kf, A, b = _problem(48, 30.0)
    h = o.build_hierarchy(n, kf, 30.0, "hyb")
    res = o.bicgstab(A, b, lambda v: o.vcycle(h, v), tol=1e-8, maxit=200)
    assert res.status == "converged" and res.true_relres <= 1e-8
    xs = spla.spsolve(A.tocsc(), b)
    assert np.linalg.norm(res.x - xs) / np.linalg.norm(xs) < 1e-5
    # history: one entry per half step, the last at or below tol
    assert len(res.history) == int(2 * res.iterations)
    assert res.history[-1] <= 1e-8


def test_shadow_residual_generator_matches_published_vectors():
    g = json.load(open(os.path.join(GOLDEN, "splitmix64_vectors.json")))
    for v in g["vectors"]:
        outs = [int(x, 0) for x in v["outputs"]]
        u = o.splitmix64_u01(v["seed"], np.arange(len(outs)))
        np.testing.assert_array_equal(u, [(x >> 11) * 2.0**-53 for x in outs])
        np.testing.assert_array_equal(I.splitmix64(v["seed"], len(outs)), np.array(outs, dtype=np.uint64))
    r = o.shadow_residual(5)
    assert r.dtype == np.complex128 and np.all(np.abs(r.real) <= 0.5) and np.all(np.abs(r.imag) <= 0.5)


def test_paper_trends():
    """Table 1 trends (iteration counts themselves are not pinned): HYB-V needs no more iterations
    than SL-V, and counts grow with k at fixed kh = 0.625."""
    t = json.load(open(os.path.join(GOLDEN, "paper_iterations.json")))["table1"]
    counts = {}
    for k, n in zip(t["k"][:3:2], t["n"][:3:2]):  # k = 40 and 80
        kf = I.constant_k(n, k)
        A = o.helmholtz_matrix(n, kf)
        b = I.centre_source_rhs(n, 1.0).ravel()
        for var in ("sl", "hyb"):
            h = o.build_hierarchy(n, kf, k, var)
            counts[(k, var)] = o.bicgstab(A, b, lambda v: o.vcycle(h, v), tol=1e-7, maxit=300).iterations
    assert counts[(40, "hyb")] <= counts[(40, "sl")]
    assert counts[(80, "hyb")] <= counts[(80, "sl")]
    assert counts[(80, "sl")] > counts[(40, "sl")] and counts[(80, "hyb")] > counts[(40, "hyb")]


def test_paper_table_workloads():
    """The runs behind Tables 1, 2 and 6: kh = 0.625 (Table 1), k = 40 (Table 2), k_ref h = 15/64
    with k between k_ref and 2 k_ref (Table 6), unit sources at the centre or at (0.5, 1)."""
    runs = I.paper_table_workloads(max_n=256)
    assert [c for t, c, _ in runs if t == "table1"] == ["k=40,h=1/64", "k=50,h=1/80", "k=80,h=1/128",
                                                       "k=100,h=1/160", "k=150,h=1/240"]
    for table, _, wl in runs:
        assert wl.tol == 1e-7 and wl.rhs.sum() == 1.0
        (j, i), = np.argwhere(wl.rhs != 0)
        if table == "table6":
            assert (i, j) == (wl.n // 2, wl.n)
            assert abs(wl.k_ref / wl.n - 15.0 / 64) < 1e-12
            assert wl.kfield.min() == wl.k_ref and wl.kfield.max() == 2 * wl.k_ref
        else:
            assert (i, j) == (wl.n // 2, wl.n // 2)
            assert np.all(wl.kfield == wl.k_ref)
            if table == "table1":
                assert abs(wl.k_ref / wl.n - 0.625) < 1e-12
            else:
                assert wl.k_ref == 40.0
