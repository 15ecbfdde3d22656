"""Batched form on the GPU: many right-hand sides per launch (hz_solve_batch) and several
problems of different grids in one graph per iteration (hz_group_solve). Each right-hand side
runs exactly the arithmetic of its own single solve, so results are compared bitwise."""
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


def _rhs(n, count, seed):
    nodes = I.random_interior_nodes(n, count, seed)
    return np.stack([I.point_source_rhs(n, [nd]) for nd in nodes])


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_equals_single_solves(precision):
    from paper_1312_2880_gb300 import hz

    n, k = 96, 0.2 * 96
    kf = I.wedge_k(n, k, 5)
    rhs = _rhs(n, 3, 21)
    rhs[1] = 0.0  # retires at once: x = 0 after zero iterations
    PB = hz.Problem(n, kf, 0.5, precision=precision, k_ref=k, batch=3)
    xb, infos = PB.solve_batch(torch.from_numpy(rhs).cuda(), tol=1e-6)
    P1 = hz.Problem(n, kf, 0.5, precision=precision, k_ref=k)
    for b in range(3):
        x1, i1, _ = P1.solve(torch.from_numpy(rhs[b]).cuda(), tol=1e-6)
        assert infos[b]["iterations"] == i1["iterations"], b
        assert torch.equal(xb[b], x1), b
    assert infos[1]["iterations"] == 0 and torch.count_nonzero(xb[1]) == 0
    A = o.helmholtz_matrix(n, kf)
    for b in (0, 2):
        assert o.true_relres(A, rhs[b].ravel(), xb[b].cpu().numpy().ravel()) <= 1e-6


def test_group_of_batched_problems_equals_separate_solves():
    from paper_1312_2880_gb300 import hz

    specs = [(48, 0.2 * 48, 2), (96, 0.2 * 96, 3), (64, 0.2 * 64, 2)]
    probs, rhss = [], []
    for q, (n, k, B) in enumerate(specs):
        kf = I.grf_k(n, k, 30 + q, corr=0.2)
        probs.append(hz.Problem(n, kf, 0.5, precision="fp32", k_ref=k, batch=B))
        rhss.append(torch.from_numpy(_rhs(n, B, 40 + q)).cuda())
    G = hz.Group(probs)
    xs, infos = G.solve(rhss, tol=1e-6)
    G.close()
    q = 0
    for P, r, x in zip(probs, rhss, xs):
        xb, ib = P.solve_batch(r, tol=1e-6)
        assert torch.equal(x, xb)
        for b in range(P.batch):
            assert infos[q]["iterations"] == ib[b]["iterations"] and infos[q]["status"] == 0
            q += 1


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batched_workload_matches_the_oracle(precision):
    """The batched workload itself (64 right-hand sides over n = 96, 192, 384, 576 at kh = 2 pi / 12,
    one group solve): right-hand side 0 of the two smaller grids against the oracle's own solves.
    FP64 form: iterations within the oracle's spread under one-ulp rescalings of b, solution within max(1e-10, 10 x that
    spread); FP32 form: relres 1e-6 on the oracle's operator and within 1e-4 of the oracle."""
    from paper_1312_2880_gb300 import hz

    wls = I.batch_problems(rhs_per_k=16)
    probs = [hz.Problem(w.n, w.kfield, 0.5, variant=w.variant, precision=precision, k_ref=w.k_ref,
                        batch=w.rhs.shape[0]) for w in wls]
    G = hz.Group(probs)
    xs, infos = G.solve([torch.from_numpy(w.rhs).cuda() for w in wls], tol=1e-6, maxit=3000)
    G.close()
    for P in probs:
        P.close()
    assert all(i["status"] == 0 for i in infos)
    for pi in (0, 1):
        w = wls[pi]
        b = w.rhs[0].ravel()
        A = o.helmholtz_matrix(w.n, w.kfield)
        H = o.build_hierarchy(w.n, w.kfield, w.k_ref, w.variant, w.levels)
        ref = o.bicgstab(A, b, lambda v: o.vcycle(H, v), tol=1e-6, maxit=3000)
        x = xs[pi][0].cpu().numpy().ravel()
        err = float(np.abs(x - ref.x).max() / np.abs(ref.x).max())
        assert o.true_relres(A, b, x) <= 1e-6
        it = infos[16 * pi]["iterations"]
        if precision == "fp64":
            # the oracle's own spread: its solution and iteration count under three one-ulp-scale
            # rescalings of b
            spread, spread_it = 0.0, 0.0
            for sc in (1 + 2.0**-52, 1 - 2.0**-53, 1 + 2.0**-51):
                alt = o.bicgstab(A, b * sc, lambda v: o.vcycle(H, v), tol=1e-6, maxit=3000)
                spread = max(spread, float(np.abs(alt.x / sc - ref.x).max() / np.abs(ref.x).max()))
                spread_it = max(spread_it, abs(alt.iterations - ref.iterations))
            assert abs(it - ref.iterations) <= max(2.0, 2 * spread_it)
            assert err <= max(1e-10, 10 * spread), (err, spread)
        else:
            assert err <= 1e-4, (w.n, err)
