"""hz_apply_dot_noalloc, the entry point for callers that cannot allocate device memory at call
time (hosts whose own pool owns the device; latency-critical loops where cudaMalloc may
synchronise): its v = A u and <w, v> must equal hz_apply's result and the dot product of that
result, within the per-step tolerance of the other GPU tests (1e-12), on two calls in a row
(the second call reuses the shared scratch the first one left behind); hz_apply is itself checked
against the oracle's operator at the same tolerance."""
from ctypes import c_void_p

import numpy as np
import pytest

from paper_1312_2880_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("n", [96, 1024])
def test_noalloc_apply_dot_matches_apply_twice(n):
    from paper_1312_2880_gb300 import build, hz

    build.build()
    L = hz.lib()
    kf = I.grf_k(n, n * 0.5, 5)
    P = hz.Problem(n, kf, 0.5, variant="hyb")
    g = np.random.default_rng(n)
    u = torch.from_numpy(g.standard_normal((n + 1, n + 1)) + 1j * g.standard_normal((n + 1, n + 1))).cuda()
    w = torch.from_numpy(g.standard_normal((n + 1, n + 1)) + 1j * g.standard_normal((n + 1, n + 1))).cuda()
    kh = torch.from_numpy(np.ascontiguousarray(kf * (1.0 / n))).cuda()
    stream = c_void_p(torch.cuda.current_stream().cuda_stream)
    import oracle as o

    for beta, op in ((0.0, "L"), (0.5, "M")):
        ref_v = P.apply(u, op).cpu().numpy()
        ref_dot = np.vdot(w.cpu().numpy().ravel(), ref_v.ravel())
        # hz_apply itself against the oracle's operator (the per-step bound of the other tests)
        oracle_v = (o.helmholtz_matrix(n, kf, beta) @ u.cpu().numpy().ravel()).reshape(n + 1, n + 1)
        assert _rel(ref_v, oracle_v) <= 1e-12
        for _ in range(2):
            v = torch.full_like(u, complex("nan"))
            dot = torch.full((1,), complex("nan"), dtype=torch.complex128, device="cuda")
            st = L.hz_apply_dot_noalloc(n, c_void_p(kh.data_ptr()), beta, c_void_p(u.data_ptr()),
                                        c_void_p(w.data_ptr()), c_void_p(v.data_ptr()), c_void_p(dot.data_ptr()),
                                        stream)
            assert st == hz.HZ_OK
            torch.cuda.synchronize()
            assert _rel(v.cpu().numpy(), ref_v) <= 1e-12
            assert abs(complex(dot.cpu().numpy()[0]) - ref_dot) <= 1e-12 * abs(ref_dot)
    P.close()


def test_noalloc_rejects_sizes_beyond_its_limit():
    from paper_1312_2880_gb300 import build, hz

    build.build()
    L = hz.lib()
    t = torch.zeros(4, dtype=torch.complex128, device="cuda")
    p = c_void_p(t.data_ptr())
    q = c_void_p(t[2:].data_ptr())
    assert L.hz_apply_dot_noalloc(32769, p, 0.0, p, p, q, q, None) == hz.HZ_EINVAL
    assert L.hz_apply_dot_noalloc(1, p, 0.0, p, p, q, q, None) == hz.HZ_EINVAL
