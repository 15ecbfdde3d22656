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
