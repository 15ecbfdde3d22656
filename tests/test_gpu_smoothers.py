"""Damped Jacobi and red-black SOR on the Gauss-Seidel levels (the alternatives of Sec. 4's remark),
CUDA path against the oracle through the C ABI: every level step at the FP64 step tolerance
(1e-12), including the ping-pong of several Jacobi sweeps, a whole V-cycle at 1e-11 (FP64) and
2e-5 (FP32), solves that reach the tolerance in both forms, and batched solves equal to single
ones bit for bit.
"""
import numpy as np
import pytest

import oracle as o
from paper_1312_2880_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1312_2880_gb300 import build

    build.build()


def wedge(n=128, k=25.0):
    kf = I.wedge_k(n, k, I.SEED_BASE + 2)
    rhs = I.point_source_rhs(n, I.random_interior_nodes(n, 3, 11))
    return I.Workload(f"wedge_n{n}", n, k, kf, rhs, variant="hyb", levels=0)


SMOOTHERS = [("jacobi", 0.0, 0.8), ("jacobi", 0.6, 0.6), ("sor", 1.2, 1.2), ("sor", 0.0, 1.0)]


def rand_c(shape, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def dev(x, n):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, dtype=np.complex128).reshape(n + 1, n + 1))).cuda()


def rel(a, b):
    a = a.cpu().numpy() if hasattr(a, "cpu") else a
    return float(np.abs(np.asarray(a).ravel() - np.asarray(b).ravel()).max() / np.abs(b).max())


def pair(wl, sm, omega, precision="fp64", nu_gs=1, batch=1, rule="band"):
    from paper_1312_2880_gb300 import hz

    P = hz.Problem(wl.n, wl.kfield, 0.5, variant=wl.variant, precision=precision, levels=wl.levels, k_ref=wl.k_ref,
                   nu_gs=nu_gs, gs_smoother=sm, omega=omega, batch=batch, kacz_rule=rule)
    H = o.build_hierarchy(wl.n, wl.kfield, wl.k_ref, wl.variant, wl.levels, nu_gs=nu_gs, gs_smoother=sm,
                          omega=None if omega == 0.0 else omega, rule=rule)
    assert [d["smoother"] for d in P.schedule()] == [lv.smoother for lv in H.levels]
    return P, H


@pytest.mark.parametrize("nu_gs", [1, 2, 3])
@pytest.mark.parametrize("sm,omega,expect", SMOOTHERS)
def test_level_steps_match_the_oracle(sm, omega, expect, nu_gs):
    wl = wedge()
    # the bins rule leaves three of the wedge's levels to the smoother under test (the band rule two)
    P, H = pair(wl, sm, omega, nu_gs=nu_gs, rule="bins")
    try:
        checked = 0
        for l, lv in enumerate(H.levels[:-1]):
            if lv.smoother != sm:
                continue
            assert abs(lv.omega - expect) < 1e-15
            checked += 1
            f = rand_c((lv.n + 1) ** 2, 10 + l)
            u_ref = o.helmholtz.relax(lv, f, np.zeros_like(f), post=False)
            u, fc = P.level_presmooth(l, dev(f, lv.n))
            assert rel(u, u_ref) <= 1e-12, (l, "pre")
            assert rel(fc, lv.R @ (f - lv.B @ u_ref)) <= 1e-12, (l, "restriction")
            nc = H.levels[l + 1].n
            u0, ec = rand_c((lv.n + 1) ** 2, 20 + l), rand_c((nc + 1) ** 2, 30 + l)
            ref = o.helmholtz.relax(lv, f, u0 + lv.P @ ec, post=True)
            assert rel(P.level_postsmooth(l, dev(f, lv.n), dev(u0, lv.n), dev(ec, nc)), ref) <= 1e-12, (l, "post")
        assert checked >= 3
    finally:
        P.close()


@pytest.mark.parametrize("sm,omega,expect", SMOOTHERS)
def test_vcycle_matches_the_oracle(sm, omega, expect):
    wl = wedge()
    r = rand_c((wl.n + 1) ** 2, 5)
    P, H = pair(wl, sm, omega)
    try:
        ref = o.vcycle(H, r)
        assert rel(P.vcycle(dev(r, wl.n)), ref) <= 1e-11
    finally:
        P.close()
    P, _ = pair(wl, sm, omega, precision="fp32")
    try:
        assert rel(P.vcycle(dev(r, wl.n)), ref) <= 2e-5
    finally:
        P.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("sm,omega", [("jacobi", 0.0), ("sor", 1.2)])
def test_solves_reach_the_tolerance(sm, omega, precision):
    wl = wedge()
    P, _ = pair(wl, sm, omega, precision=precision)
    try:
        x, info, _ = P.solve(dev(wl.rhs, wl.n), tol=1e-6, maxit=1000)
    finally:
        P.close()
    A = o.helmholtz_matrix(wl.n, wl.kfield)
    assert info["status"] == 0 and o.true_relres(A, wl.rhs.ravel(), x.cpu().numpy().ravel()) <= 1e-6


def test_batched_jacobi_solves_equal_single_solves():
    wl = wedge()
    n = wl.n
    rhs = np.stack([I.point_source_rhs(n, I.random_interior_nodes(n, 2, s)) for s in (7, 8)])
    P, _ = pair(wl, "jacobi", 0.0, precision="fp32", nu_gs=2, batch=2)
    try:
        xb, infos = P.solve_batch(torch.from_numpy(rhs).cuda(), tol=1e-6, maxit=1000)
        xb = xb.cpu().numpy()
    finally:
        P.close()
    for q in range(2):
        S, _ = pair(wl, "jacobi", 0.0, precision="fp32", nu_gs=2)
        try:
            x, info, _ = S.solve(torch.from_numpy(rhs[q]).cuda(), tol=1e-6, maxit=1000)
        finally:
            S.close()
        assert info["iterations"] == infos[q]["iterations"]
        assert np.array_equal(x.cpu().numpy().view(np.uint64), xb[q].view(np.uint64))


def test_invalid_smoother_options_are_refused():
    from paper_1312_2880_gb300 import hz

    wl = wedge(64, 10.0)
    with pytest.raises(hz.HzError):
        hz.Problem(wl.n, wl.kfield, 0.5, k_ref=wl.k_ref, gs_smoother="jacobi", omega=2.5)
