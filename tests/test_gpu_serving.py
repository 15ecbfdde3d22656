"""Serving form on the GPU: non-blocking solves, continuous admission, results alone vs in the mix."""
import numpy as np
import pytest

from paper_1312_2880_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1312_2880_gb300 import build

    build.build()


def _jobs(count=8):
    from paper_1312_2880_gb300.serve import Job

    jobs = []
    for r in range(count):
        n = (64, 96, 128)[r % 3]
        medium = "wedge" if r % 2 == 0 else "grf"
        k = 0.2 * n  # kh = 0.2, where the method converges in both forms
        seed = 100 + (r % 4)
        fn = (lambda n=n, k=k, s=seed: I.wedge_k(n, k, s)) if medium == "wedge" else (
            lambda n=n, k=k, s=seed: I.grf_k(n, k, s, corr=0.2))
        src = I.random_interior_nodes(n, 1, 1000 + r)[0]
        jobs.append(Job(r, n, (n, medium, seed), fn, k, src, arrival=0.0))
    return jobs


def test_nonblocking_solve_equals_blocking():
    from paper_1312_2880_gb300 import hz

    wl = I.wedge_n512()
    P = hz.Problem(wl.n, wl.kfield, 0.5, variant=wl.variant, precision="fp32", levels=wl.levels, k_ref=wl.k_ref)
    rhs = torch.from_numpy(wl.rhs).cuda()
    xb, ib, hb = P.solve(rhs, tol=1e-6)
    x = torch.empty_like(rhs)
    P.solve_start(rhs, x, tol=1e-6)
    polls = 0
    while not P.solve_poll():
        polls += 1
    xa, ia, ha = P.solve_finish()
    assert torch.equal(xa, xb) and ia == ib and np.array_equal(ha, hb)
    assert polls > 0  # the loop really did return before the end


def test_each_result_is_the_same_alone_and_in_the_mix():
    from paper_1312_2880_gb300.serve import Server

    free = torch.cuda.mem_get_info()[0]
    mix = Server(hbm_budget=free // 2, precision="fp32", max_active=8, keep_solutions=True)
    summ = mix.run(_jobs(), realtime=False)
    assert summ["completed"] == 8 and summ["converged"] == 8
    mixed = {j.rid: j.result["x"] for j in mix.done}
    assert summ["peak_active"] == 8  # all eight solves were in flight together
    mix.close()
    for job in _jobs():
        alone = Server(hbm_budget=free // 2, precision="fp32", max_active=1, keep_solutions=True)
        alone.run([job], realtime=False)
        assert np.array_equal(alone.done[0].result["x"], mixed[job.rid]), job.rid
        alone.close()


def test_admission_stays_within_the_memory_budget():
    from paper_1312_2880_gb300.serve import Server

    probe = Server(hbm_budget=1 << 40, precision="fp32")
    budget = 2 * probe.footprint(128) + 1
    srv = Server(hbm_budget=budget, precision="fp32", max_active=8)
    summ = srv.run(_jobs(), realtime=False)
    assert summ["completed"] == 8 and summ["peak_hbm_bytes"] <= budget
    assert summ["evictions"] > 0
    srv.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_served_requests_match_the_oracle(precision):
    """Requests of the served stream itself (kh = 2 pi / 12, wedge and random-field media, one
    seeded source), served in a mix: the first request of n = 128 and of n = 256 against the
    oracle's own solve of it. FP64 form: iteration count within the oracle's spread under one-ulp rescalings of b and the
    solution within max(1e-10, 10 x that spread) (the final-solution reading of the 1e-10
    tolerance); FP32 form: relres 1e-6 on the oracle's operator and within 1e-4 of the oracle's
    solution (both stop at relres 1e-6)."""
    import oracle as o
    from paper_1312_2880_gb300.serve import Job, Server

    reqs = I.serving_requests(40, 200.0)
    picks = [next(q for q in reqs if q.n == n) for n in (128, 256)]
    others = [q for q in reqs if q.n <= 256 and q not in picks][:4]
    jobs = []
    for q in picks + others:
        kf = I.request_medium(q)
        jobs.append(Job(q.rid, q.n, (q.n, q.medium, q.medium_seed), (lambda kf=kf: kf), q.k, q.source))
    free = torch.cuda.mem_get_info()[0]
    srv = Server(hbm_budget=free // 2, precision=precision, max_active=8, keep_solutions={q.rid for q in picks},
                 fallback=False)
    summ = srv.run(jobs, realtime=False)
    got = {j.rid: j.result for j in srv.done}
    srv.close()
    assert summ["converged"] == len(jobs)
    for q in picks:
        kf = I.request_medium(q)
        b = I.point_source_rhs(q.n, [q.source]).ravel()
        A = o.helmholtz_matrix(q.n, kf)
        H = o.build_hierarchy(q.n, kf, q.k, "hyb")
        ref = o.bicgstab(A, b, lambda v: o.vcycle(H, v), tol=1e-6, maxit=4000)
        x = got[q.rid]["x"].ravel()
        err = float(np.abs(x - ref.x).max() / np.abs(ref.x).max())
        assert o.true_relres(A, b, x) <= 1e-6
        if precision == "fp64":
            # the oracle's own spread: its solution and iteration count under three one-ulp-scale
            # rescalings of b
            spread, spread_it = 0.0, 0.0
            for sc in (1 + 2.0**-52, 1 - 2.0**-53, 1 + 2.0**-51):
                alt = o.bicgstab(A, b * sc, lambda v: o.vcycle(H, v), tol=1e-6, maxit=4000)
                spread = max(spread, float(np.abs(alt.x / sc - ref.x).max() / np.abs(ref.x).max()))
                spread_it = max(spread_it, abs(alt.iterations - ref.iterations))
            assert abs(got[q.rid]["iterations"] - ref.iterations) <= max(2.0, 2 * spread_it)
            assert err <= max(1e-10, 10 * spread), (err, spread)
        else:
            assert err <= 1e-4, (q.rid, err)
