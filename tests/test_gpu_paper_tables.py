"""Sec. 6, Tables 1, 2 and 6 re-run on the GPU (Bi-CGSTAB to relres 1e-7, x0 = 0, unit point source).

The paper's counts are not pinned (it leaves the boundary scheme, smoother ordering, coarsest
solve and shadow residual unstated; tests/golden/paper_iterations.json holds them as context).
Checked here: on the smallest columns the GPU FP64 form takes the oracle's iteration count (the
same algorithm, so the counts agree up to rounding of the last half step); over Tables 1 and 2
two of the trends the paper reports hold on the GPU: counts grow with k at fixed kh and do not grow
as h shrinks at fixed k = 40. The third, HYB-V ahead of SL-V in every column, does not hold in this
reading (the two stay within a few iterations, either ahead), so it is not asserted.
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


def gpu_iterations(wl, variant, precision="fp64", maxit=400):
    from paper_1312_2880_gb300 import hz

    P = hz.Problem(wl.n, wl.kfield, 0.5, variant=variant, precision=precision, k_ref=wl.k_ref)
    try:
        _, info, _ = P.solve(torch.from_numpy(wl.rhs).cuda(), tol=wl.tol, maxit=maxit, allow_fail=True)
    finally:
        P.close()
    assert info["status"] == 0, info
    assert info["relres_true"] <= wl.tol
    return info["iterations"]


def columns(table, variant, max_n):
    return [(col, wl) for t, col, wl in I.paper_table_workloads((table,), variant=variant, max_n=max_n)]


@pytest.mark.parametrize("variant", ["hyb", "sl"])
@pytest.mark.parametrize("table", ["table1", "table6"])
def test_smallest_column_takes_the_oracles_iteration_count(table, variant):
    (col, wl), = columns(table, variant, 64)
    A = o.helmholtz_matrix(wl.n, wl.kfield)
    H = o.build_hierarchy(wl.n, wl.kfield, wl.k_ref, variant, wl.levels)
    ref = o.bicgstab(A, wl.rhs.ravel(), lambda v: o.vcycle(H, v), tol=wl.tol, maxit=400)
    assert abs(gpu_iterations(wl, variant) - ref.iterations) <= 1.0, (col, ref.iterations)


def test_table1_and_table2_trends():
    counts = {}
    for table, max_n in (("table1", 160), ("table2", 512)):
        for variant in ("hyb", "sl"):
            counts[(table, variant)] = [gpu_iterations(wl, variant) for _, wl in columns(table, variant, max_n)]
    # The paper's HYB-V < SL-V in every column is not asserted: in this reading the two variants are
    # within a few iterations of each other on Tables 1 and 2, either one ahead (reported beside
    # the paper's counts by `bench.py --tables`). The k and h trends below do hold.
    for variant in ("hyb", "sl"):
        t1 = counts[("table1", variant)]
        assert all(b > a for a, b in zip(t1, t1[1:])), t1  # more iterations as k grows at fixed kh
        t2 = counts[("table2", variant)]
        assert t2[-1] <= t2[0], t2  # no growth as h shrinks at fixed k


def test_fp32_form_reaches_the_table1_tolerance():
    for variant in ("hyb", "sl"):
        for _, wl in columns("table1", variant, 128):
            assert gpu_iterations(wl, variant, "fp32") > 0
