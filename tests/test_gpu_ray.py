"""Ray correction and the stand-alone cycle solver (Sec. 6, Table 7), CUDA path against the oracle
through the C ABI: the restriction P^H r and the assembled Galerkin ray operator at the FP64 step
tolerance, the block-LU ray solve by its residual and against the oracle's sparse LU, the whole
correction, and Table 7's cycle solves (cycle counts equal to the oracle's, iterates close).

Tolerances: restriction and assembly are sums of a few hundred products, 1e-12 of the largest
entry. The ray solve is checked by its residual (1e-11) and against the oracle's sparse LU within
the ray operator's condition number (about 3e5 at k H = 2.5, 2e3 at k H = 5) times the FP64 unit
roundoff with room: 1e-8 of the largest entry. At k H = 1.25 (condition about 2e11) only the
residual is checked.
"""
import json
import os

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


def t7(k):
    return next(w for c, w in I.paper_table7_workloads() if c == f"k={k:g}")


def medium(n=96, k=30.0):
    # a variable medium on a grid whose ray blocks (13 ray rows, 104 unknowns a block row) are not
    # a multiple of the 32-wide GEMM tiles
    kf = I.wedge_k(n, k, I.SEED_BASE + 9, (1.0, 1.2, 0.9))
    return I.Workload(f"wedge_n{n}_k{k:g}", n, k, kf, I.centre_source_rhs(n, 1.0), variant="hlm", tol=1e-7)


CASES = [("t7_k20", lambda: t7(20.0), 0), ("wedge_n96", medium, 0), ("t7_k20_m16", lambda: t7(20.0), 16),
         ("t7_k20_m4", lambda: t7(20.0), 4)]


def rand_c(shape, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, dtype=np.complex128))).cuda()


def rel(a, b):
    a = a.cpu().numpy() if hasattr(a, "cpu") else a
    return float(np.abs(np.asarray(a).ravel() - np.asarray(b).ravel()).max() / np.abs(b).max())


def pair(wl, m=0, variant=None, precision="fp64"):
    from paper_1312_2880_gb300 import hz

    v = variant or wl.variant
    P = hz.Problem(wl.n, wl.kfield, 0.5, variant=v, precision=precision, levels=wl.levels, k_ref=wl.k_ref)
    R = hz.Ray(P, wl.k_ref, m)
    A = o.helmholtz_matrix(wl.n, wl.kfield)
    ray = o.ray_setup(A, wl.n, wl.k_ref, m)
    assert R.m == ray.m and R.unknowns == ray.Ac.shape[0]
    return P, R, A, ray


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request):
    _, make, m = request.param
    wl = make()
    P, R, A, ray = pair(wl, m)
    yield wl, P, R, A, ray
    R.close()
    P.close()


def test_restriction_matches_oracle(case):
    wl, P, R, A, ray = case
    r = rand_c((wl.n + 1) ** 2, 1)
    g = R.restrict(dev(r.reshape(wl.n + 1, wl.n + 1)))
    assert rel(g, ray.restrict(r)) <= 1e-12


def test_assembled_blocks_match_oracle(case):
    wl, P, R, A, ray = case
    Lb, Db, Ub = (b.cpu().numpy() for b in R.blocks())
    Nr, Bs = R.nc + 1, 8 * (R.nc + 1)
    dense = np.zeros((Nr * Bs, Nr * Bs), complex)
    for J in range(Nr):
        dense[J * Bs:(J + 1) * Bs, J * Bs:(J + 1) * Bs] = Db[J]
        if J > 0:
            dense[J * Bs:(J + 1) * Bs, (J - 1) * Bs:J * Bs] = Lb[J]
        if J < Nr - 1:
            dense[J * Bs:(J + 1) * Bs, (J + 1) * Bs:(J + 2) * Bs] = Ub[J]
    assert not Lb[0].any() and not Ub[Nr - 1].any()
    assert rel(dense, ray.Ac.toarray()) <= 1e-12


def test_ray_solve_by_residual_and_against_sparse_lu(case):
    wl, P, R, A, ray = case
    g = rand_c(R.unknowns, 2)
    z = R.coarse_solve(dev(g)).cpu().numpy()
    Ac = ray.Ac
    if R.m == 4:
        # k H = 1.25: the eight plane-wave bases are nearly dependent (condition ~2e11), so only the
        # residual is defined to a few digits (the floor is unit roundoff times the condition)
        assert np.linalg.norm(Ac @ z - g) <= 1e-4 * np.linalg.norm(g)
        return
    assert np.linalg.norm(Ac @ z - g) <= 1e-11 * np.linalg.norm(g)
    assert rel(z, ray.lu.solve(g)) <= 1e-8


def test_correction_matches_oracle(case):
    wl, P, R, A, ray = case
    if R.m == 4:
        pytest.skip("ill-conditioned ray basis at k H = 1.25: compared by residual only")
    n = wl.n
    r = rand_c((n + 1) ** 2, 3)
    x0 = rand_c((n + 1) ** 2, 4)
    x = dev(x0.reshape(n + 1, n + 1))
    R.correct(dev(r.reshape(n + 1, n + 1)), x)
    want = x0 + ray.correct(r)
    assert rel(x, want) <= 1e-8


def test_correction_is_exact_on_the_ray_space(case):
    wl, P, R, A, ray = case
    if R.m == 4:
        pytest.skip("ill-conditioned ray basis at k H = 1.25")
    n = wl.n
    e = ray.P @ rand_c(R.unknowns, 5)
    x = torch.zeros((n + 1, n + 1), dtype=torch.complex128, device="cuda")
    R.correct(dev((A @ e).reshape(n + 1, n + 1)), x)
    assert rel(x, e) <= 1e-8


@pytest.mark.parametrize("k,variant", [(20.0, "hlm"), (20.0, "sl"), (20.0, "hyb"), (40.0, "hlm")])
def test_table7_cycle_solve_matches_oracle(k, variant):
    from paper_1312_2880_gb300 import hz

    wl = t7(k)
    P, R, A, ray = pair(wl, 0, variant)
    H = o.build_hierarchy(wl.n, wl.kfield, wl.k_ref, variant)
    b = wl.rhs.ravel()
    ref = o.cycle_solve(A, b, H, ray, tol=wl.tol, maxc=40)
    x, info, hist = P.cycle_solve(dev(wl.rhs), R, tol=wl.tol, maxc=40)
    assert ref.status == "converged" and info["status"] == hz.HZ_OK
    assert info["cycles"] == ref.cycles
    assert np.allclose(hist, ref.history, rtol=1e-6, atol=0)
    assert rel(x, ref.x) <= 1e-8
    assert o.true_relres(A, b, x.cpu().numpy().ravel()) <= wl.tol
    R.close()
    P.close()


@pytest.mark.parametrize("variant", ["hlm", "sl", "hyb"])
def test_table7_every_column_takes_the_stored_oracle_cycle_count(variant):
    # k = 20 .. 160 (n = 64 .. 512): the oracle's counts, histories and sampled solutions from
    # make_table7_oracle.py
    from paper_1312_2880_gb300 import hz

    golden = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table7_oracle.json")))
    for ci, (col, wl) in enumerate(I.paper_table7_workloads()):
        ref = golden["oracle"][variant][ci]
        P = hz.Problem(wl.n, wl.kfield, 0.5, variant=variant, k_ref=wl.k_ref)
        R = hz.Ray(P, wl.k_ref)
        assert R.m == golden["columns"][ci]["m"]
        x, info, hist = P.cycle_solve(dev(wl.rhs), R, tol=wl.tol, maxc=60)
        assert info["status"] == hz.HZ_OK and info["cycles"] == ref["cycles"], col
        assert np.allclose(hist, ref["history"], rtol=1e-6, atol=0), col
        # the solution on the stored lattice of nodes (every n/8-th node each way)
        smp = np.array(ref["sampled"])
        xs = x.cpu().numpy()[smp[:, 1].astype(int), smp[:, 0].astype(int)]
        assert np.abs(xs - (smp[:, 2] + 1j * smp[:, 3])).max() <= 1e-8 * ref["max_abs_x"], col
        R.close()
        P.close()


def test_hlm_cycle_solve_without_ray_diverges_like_the_oracle():
    from paper_1312_2880_gb300 import hz

    wl = t7(20.0)
    P = hz.Problem(wl.n, wl.kfield, 0.5, variant="hlm", k_ref=wl.k_ref)
    A = o.helmholtz_matrix(wl.n, wl.kfield)
    H = o.build_hierarchy(wl.n, wl.kfield, wl.k_ref, "hlm")
    ref = o.cycle_solve(A, wl.rhs.ravel(), H, None, tol=wl.tol, maxc=80)
    x, info, hist = P.cycle_solve(dev(wl.rhs), None, tol=wl.tol, maxc=80, allow_fail=True)
    assert ref.status == "diverged" and info["status"] == hz.HZ_EMAXIT
    assert abs(info["cycles"] - ref.cycles) <= 1
    n = min(len(hist), len(ref.history)) - 3
    assert np.allclose(hist[:n], ref.history[:n], rtol=1e-5, atol=0)
    P.close()


def test_fp32_vcycle_with_ray_converges():
    from paper_1312_2880_gb300 import hz

    wl = t7(40.0)
    P, R, A, ray = pair(wl, 0, "hlm", precision="fp32")
    x, info, hist = P.cycle_solve(dev(wl.rhs), R, tol=wl.tol, maxc=40)
    assert info["status"] == hz.HZ_OK and info["cycles"] <= 12
    assert o.true_relres(A, wl.rhs.ravel(), x.cpu().numpy().ravel()) <= wl.tol
    R.close()
    P.close()


def test_bad_ray_arguments_are_refused():
    from paper_1312_2880_gb300 import hz

    wl = t7(20.0)
    P = hz.Problem(wl.n, wl.kfield, 0.5, variant="hlm", k_ref=wl.k_ref)
    for k_ref, m in ((20.0, 3), (20.0, 128), (0.0, 0), (float("nan"), 0), (20.0, 256)):
        with pytest.raises(hz.HzError) as ei:
            hz.Ray(P, k_ref, m)
        assert ei.value.status == hz.HZ_EINVAL
    # outputs that share bytes with inputs are refused before anything is launched
    R = hz.Ray(P, wl.k_ref)
    r = dev(rand_c((wl.n + 1, wl.n + 1), 12))
    for call in (lambda: R.correct(r, r), lambda: P.cycle_solve(r, R, x=r)):
        with pytest.raises(hz.HzError) as ei:
            call()
        assert ei.value.status == hz.HZ_EINVAL
    R.close()
    P.close()
