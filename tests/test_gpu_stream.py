"""Kernel forms of the fused Gauss-Seidel passes, in FP32 and FP64: shared-memory tiles (form 0)
and register streaming with 2 .. 256 rows per warp (forms 1..8), and the tile autotuner that picks
one per level.

Every form takes the same fixed-rounding operations in the same order on every node, so the
V-cycle must be bitwise identical across forms (and therefore whatever the autotuner picks); form
0 itself is held to the FP64 oracle in test_gpu_parity.py, and each form is checked against the
oracle here as well. The grids cover one-strip levels (both grid edges in one warp), several
strips with a ragged last one, ragged last row segments, batches, and the smallest level the
streaming form accepts (n_l = 4).
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


def grf(n, k, seed=17):
    return I.Workload(f"grf_n{n}", n, k, I.grf_k(n, k, seed), I.centre_source_rhs(n), variant="hyb", levels=0)


def wedge(n, k):
    kf = I.wedge_k(n, k, I.SEED_BASE + 2)
    rhs = I.point_source_rhs(n, I.random_interior_nodes(n, 3, 11))
    return I.Workload(f"wedge_n{n}", n, k, kf, rhs, variant="hyb", levels=0)


CASES = {
    "plain64": I.plain_n64,
    "grf200": lambda: grf(200, 60.0),
    "wedge256": lambda: wedge(256, 50.0),
    "sl_plain_n16": lambda: I.Workload("plain16", 16, 5.0, I.constant_k(16, 5.0), I.centre_source_rhs(16),
                                       variant="sl_plain", levels=3),
}


def rand_c(shape, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def vcycle(wl, form, r, batch=1, precision="fp32"):
    P = hzmod().Problem(wl.n, wl.kfield, 0.5, variant=wl.variant, precision=precision, levels=wl.levels,
                        k_ref=wl.k_ref, pass_variant=form, batch=batch)
    try:
        sched = P.schedule()
        z = P.vcycle(torch.from_numpy(r.reshape(wl.n + 1, wl.n + 1)).cuda()).cpu().numpy()
    finally:
        P.close()
    return z, sched


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("name", list(CASES))
def test_forms_are_bitwise_identical(name, precision):
    wl = CASES[name]()
    r = rand_c((wl.n + 1) ** 2, 91)
    z0, sched0 = vcycle(wl, 0, r, precision=precision)
    fused = [l for l, d in enumerate(sched0) if d["pass_down"] >= 0]
    assert fused, "no fused level in this hierarchy"
    assert all(sched0[l]["pass_down"] == 0 and sched0[l]["pass_up"] == 0 for l in fused)
    for form in range(1, 9):
        z, sched = vcycle(wl, form, r, precision=precision)
        for l in fused:
            want = form if sched[l]["n"] >= 4 else 0
            assert (sched[l]["pass_down"], sched[l]["pass_up"]) == (want, want)
        assert np.array_equal(z.view(np.uint64), z0.view(np.uint64)), (name, form, np.abs(z - z0).max())


@pytest.mark.parametrize("precision,tol", [("fp32", 2e-5), ("fp64", 1e-11)])
@pytest.mark.parametrize("name", ["plain64", "grf200"])
def test_streaming_form_matches_oracle(name, precision, tol):
    wl = CASES[name]()
    H = o.build_hierarchy(wl.n, wl.kfield, wl.k_ref, wl.variant, wl.levels)
    r = rand_c((wl.n + 1) ** 2, 92)
    ref = o.vcycle(H, r.ravel())
    for form in (1, 3, 6):
        z, _ = vcycle(wl, form, r, precision=precision)
        err = np.abs(z.ravel() - ref).max() / np.abs(ref).max()
        assert err <= tol, (form, err)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_autotuned_forms_are_valid_and_bitwise_equal(precision):
    wl = CASES["grf200"]()
    r = rand_c((wl.n + 1) ** 2, 93)
    z0, _ = vcycle(wl, 0, r, precision=precision)
    z, sched = vcycle(wl, -1, r, precision=precision)
    for d in sched:
        if d["pass_down"] >= 0:
            assert 0 <= d["pass_down"] <= 6 and 0 <= d["pass_up"] <= 6
    assert np.array_equal(z.view(np.uint64), z0.view(np.uint64))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batched_streaming_solve_equals_single_tile_solves(precision):
    """Batch of 3 right-hand sides with the streaming form == three single solves with tiles."""
    hz = hzmod()
    wl = wedge(128, 25.0)
    n = wl.n
    rhs = np.stack([I.point_source_rhs(n, I.random_interior_nodes(n, 2, s)) for s in (1, 2, 3)])
    P = hz.Problem(n, wl.kfield, 0.5, variant="hyb", precision=precision, k_ref=wl.k_ref, batch=3, pass_variant=4)
    xb, infos = P.solve_batch(torch.from_numpy(rhs).cuda(), tol=1e-6, maxit=1000)
    xb = xb.cpu().numpy()
    P.close()
    for q in range(3):
        S = hz.Problem(n, wl.kfield, 0.5, variant="hyb", precision=precision, k_ref=wl.k_ref, pass_variant=0)
        x, info, _ = S.solve(torch.from_numpy(rhs[q]).cuda(), tol=1e-6, maxit=1000)
        S.close()
        assert info["iterations"] == infos[q]["iterations"]
        assert np.array_equal(x.cpu().numpy().view(np.uint64), xb[q].view(np.uint64))
