"""The one-block coarse tail: the smallest levels of the V-cycle in one launch.

With the tail the V-cycle must give the same bits as without it (the tail and the per-level
kernels take the same fixed-rounding operations for one-sweep Gauss-Seidel levels and for every
Kaczmarz form), in FP32 and FP64, and the FP64 tail stays within the V-cycle tolerance of the
oracle. Cases: all
Gauss-Seidel levels (plain n = 64), a Kaczmarz level inside the tail (wedge n = 256, k = 50:
kH = 1.56 on the n = 32 level), batches, and the tail's level flags.
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


def hzmod():
    from paper_1312_2880_gb300 import hz

    return hz


def wedge(n, k):
    kf = I.wedge_k(n, k, I.SEED_BASE + 2)
    rhs = I.point_source_rhs(n, I.random_interior_nodes(n, 3, 11))
    return I.Workload(f"wedge_n{n}", n, k, kf, rhs, variant="hyb", levels=0)


CASES = {"plain64": I.plain_n64, "wedge256": lambda: wedge(256, 50.0), "wedge512": I.wedge_n512}


def rand_c(shape, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def vcycle(wl, precision, tail, r, batch=1):
    P = hzmod().Problem(wl.n, wl.kfield, 0.5, variant=wl.variant, precision=precision, levels=wl.levels,
                        k_ref=wl.k_ref, coarse_tail=tail, batch=batch)
    try:
        sched = P.schedule()
        z = P.vcycle(torch.from_numpy(r.reshape(wl.n + 1, wl.n + 1)).cuda()).cpu().numpy()
    finally:
        P.close()
    return z, sched


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("name", list(CASES))
def test_tail_is_bitwise_the_per_level_cycle(name, precision):
    wl = CASES[name]()
    r = rand_c((wl.n + 1) ** 2, 95)
    z1, s1 = vcycle(wl, precision, True, r)
    z0, s0 = vcycle(wl, precision, False, r)
    tail = [l for l, d in enumerate(s1) if d["in_tail"]]
    assert tail and tail[-1] == len(s1) - 1 and tail[0] >= 1, tail
    assert not any(d["in_tail"] for d in s0)
    assert np.array_equal(z1.view(np.uint64), z0.view(np.uint64)), np.abs(z1 - z0).max()


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_tail_matches_the_oracle(name):
    wl = CASES[name]()
    r = rand_c((wl.n + 1) ** 2, 96)
    H = o.build_hierarchy(wl.n, wl.kfield, wl.k_ref, wl.variant, wl.levels)
    ref = o.vcycle(H, r.ravel())
    z, s = vcycle(wl, "fp64", True, r)
    assert any(d["in_tail"] for d in s)
    err = np.abs(z.ravel() - ref).max() / np.abs(ref).max()
    assert err <= 1e-11, err


def test_tail_with_a_kaczmarz_level():
    wl = CASES["wedge256"]()
    _, s = vcycle(wl, "fp32", True, rand_c((wl.n + 1) ** 2, 97))
    assert any(d["in_tail"] and d["smoother"] == "kaczmarz" for d in s), s


def test_batched_tail_solve_equals_single_solves_without_tail():
    hz = hzmod()
    wl = wedge(128, 25.0)
    n = wl.n
    rhs = np.stack([I.point_source_rhs(n, I.random_interior_nodes(n, 2, s)) for s in (4, 5)])
    P = hz.Problem(n, wl.kfield, 0.5, variant="hyb", precision="fp32", k_ref=wl.k_ref, batch=2)
    xb, infos = P.solve_batch(torch.from_numpy(rhs).cuda(), tol=1e-6, maxit=1000)
    xb = xb.cpu().numpy()
    P.close()
    for q in range(2):
        S = hz.Problem(n, wl.kfield, 0.5, variant="hyb", precision="fp32", k_ref=wl.k_ref, coarse_tail=False)
        x, info, _ = S.solve(torch.from_numpy(rhs[q]).cuda(), tol=1e-6, maxit=1000)
        S.close()
        assert info["iterations"] == infos[q]["iterations"]
        assert np.array_equal(x.cpu().numpy().view(np.uint64), xb[q].view(np.uint64))
