"""Host logic of the serving scheduler (admission by memory, reuse of resident problems, eviction,
latency accounting) against a fake backend: no GPU needed."""
import pytest

from paper_1312_2880_gb300 import serve


class FakeProblem:
    built = 0

    def __init__(self, n, kfield, beta, **kw):
        FakeProblem.built += 1
        self.n = n
        self.polls = 0
        self.closed = False

    def solve_start(self, rhs, x, tol, maxit):
        self.polls = 3 + self.n // 64  # finishes after a few polls

    def solve_poll(self):
        self.polls -= 1
        return self.polls <= 0

    def solve_finish(self, history_cap=0, allow_fail=False):
        return None, {"status": 0, "iterations": 10.0, "relres_true": 1e-7, "restarts": 0}, []

    def close(self):
        self.closed = True


class FakeHz:
    Problem = FakeProblem

    @staticmethod
    def footprint_bytes(n, **kw):
        return 1000 * n


@pytest.fixture
def server():
    def make(budget, max_active=4):
        return serve.Server(hbm_budget=budget, max_active=max_active, backend=FakeHz,
                            make_io=lambda n, src: (None, None))

    return make


def _job(rid, n, key, arrival=0.0):
    return serve.Job(rid, n, key, lambda: None, 1.0, (1, 1), arrival=arrival)


def test_resident_problems_are_reused(server):
    FakeProblem.built = 0
    s = server(budget=10**9, max_active=1)
    out = s.run([_job(r, 64, ("a",)) for r in range(5)], realtime=False)
    assert out["completed"] == 5 and FakeProblem.built == 1


def test_memory_budget_bounds_admission_and_evicts_idle(server):
    FakeProblem.built = 0
    foot = 1000 * 64 + 2 * 16 * 65 ** 2
    s = server(budget=2 * foot, max_active=8)
    jobs = [_job(r, 64, (r % 4,)) for r in range(8)]
    out = s.run(jobs, realtime=False)
    assert out["completed"] == 8
    assert out["peak_hbm_bytes"] <= 2 * foot
    assert out["evictions"] >= 2 and FakeProblem.built >= 4


def test_latency_counts_from_arrival(server):
    s = server(budget=10**9)
    out = s.run([_job(0, 64, ("a",), arrival=0.0), _job(1, 64, ("b",), arrival=0.05)], realtime=True)
    assert out["completed"] == 2 and out["p50_ms"] is not None
    for j in s.done:
        assert j.end >= j.arrival and j.start >= j.arrival


def test_request_larger_than_the_budget_is_rejected_not_queued_forever(server):
    FakeProblem.built = 0
    foot64 = 1000 * 64 + 2 * 16 * 65 ** 2
    s = server(budget=foot64, max_active=4)
    jobs = [_job(0, 64, ("a",)), _job(1, 512, ("big",)), _job(2, 64, ("a",))]
    out = s.run(jobs, realtime=False, time_limit=30.0)
    assert out["completed"] == 3 and out["converged"] == 2
    assert out["statuses"] == {0: 2, serve.Server.ENOMEM: 1}
    big = [j for j in s.done if j.rid == 1][0]
    assert big.result["status"] == serve.Server.ENOMEM and "budget" in big.result["error"]


class StallingFp32Problem(FakeProblem):
    """FP32-form solves of odd request sizes end at maxit; FP64 ones converge."""

    def __init__(self, n, kfield, beta, precision="fp32", **kw):
        super().__init__(n, kfield, beta, **kw)
        self.precision = precision

    def solve_finish(self, history_cap=0, allow_fail=False):
        if self.precision == "fp32" and self.n == 96:
            return None, {"status": 6, "iterations": 4000.0, "relres_true": 1e-3, "restarts": 0}, []
        return None, {"status": 0, "iterations": 10.0, "relres_true": 1e-7, "restarts": 0}, []


class StallingHz(FakeHz):
    Problem = StallingFp32Problem


def test_fp32_solve_that_does_not_converge_falls_back_to_fp64():
    s = serve.Server(hbm_budget=10**9, max_active=4, backend=StallingHz, make_io=lambda n, src: (None, None))
    jobs = [_job(0, 64, ("a",)), _job(1, 96, ("b",)), _job(2, 64, ("a",))]
    out = s.run(jobs, realtime=False, time_limit=30.0)
    assert out["completed"] == 3 and out["converged"] == 3 and out["fp64_fallbacks"] == 1
    j1 = [j for j in s.done if j.rid == 1][0]
    assert j1.precision == "fp64" and j1.result["fp32_attempt"]["status"] == 6
    assert all(j.precision is None for j in s.done if j.rid != 1)
    off = serve.Server(hbm_budget=10**9, max_active=4, backend=StallingHz, make_io=lambda n, src: (None, None),
                       fallback=False)
    assert off.run([_job(1, 96, ("b",))], realtime=False, time_limit=30.0)["converged"] == 0
