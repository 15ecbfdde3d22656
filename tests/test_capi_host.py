"""C-ABI checks that need no GPU: the library loads, exports every declared function, validates
arguments, sizes its arena, and computes the same level schedule as the oracle's policy."""
import ctypes

import numpy as np
import pytest

import oracle as o
from paper_1312_2880_gb300 import inputs as I

hz = pytest.importorskip("paper_1312_2880_gb300.hz")


@pytest.fixture(scope="module")
def L():
    from paper_1312_2880_gb300 import build

    build.build()
    return hz.lib()


def test_every_declared_function_is_exported(L):
    names = hz.header_functions()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_create_problem_validates_arguments(L):
    h = ctypes.c_void_p()
    dp = ctypes.POINTER(ctypes.c_double)
    k = np.full((9, 9), 10.0)
    assert L.hz_create_problem(8, k.ctypes.data_as(dp), 0.5, 0, ctypes.byref(h)) == hz.HZ_OK
    L.hz_destroy(h)
    assert L.hz_create_problem(1, k.ctypes.data_as(dp), 0.5, 0, ctypes.byref(h)) == hz.HZ_EINVAL
    assert L.hz_create_problem(8, k.ctypes.data_as(dp), 0.5, 7, ctypes.byref(h)) == hz.HZ_EINVAL
    bad = k.copy()
    bad[3, 3] = np.nan
    assert L.hz_create_problem(8, bad.ctypes.data_as(dp), 0.5, 0, ctypes.byref(h)) == hz.HZ_EINVAL
    bad[3, 3] = -1.0
    assert L.hz_create_problem(8, bad.ctypes.data_as(dp), 0.5, 0, ctypes.byref(h)) == hz.HZ_EINVAL
    assert L.hz_status_string(hz.HZ_EMAXIT) == b"HZ_EMAXIT"


def test_footprint(L):
    fp64 = hz.footprint_bytes(4096, levels=10, precision="fp64")
    fp32 = hz.footprint_bytes(4096, levels=10, precision="fp32")
    N = 4097**2
    # 11 complex FP64 vectors + FP64 k h, plus the level arrays
    assert fp64 > 11 * 16 * N and fp32 > 11 * 16 * N
    assert fp32 < fp64 < 20 * 16 * N
    assert hz.footprint_bytes(64, levels=9) == 0  # 64 / 2^8 < 2
    assert hz.footprint_bytes(100, levels=2) == 0  # coarsest 51^2 > 1089 unknowns


def _oracle_schedule(wl, variant=None, rule="band"):
    return o.schedule(wl.n, wl.kfield, wl.k_ref, variant or wl.variant, wl.levels, rule=rule)


def _lib_schedule(wl, variant=None, levels=None, rule="band"):
    sch = hz.describe_hierarchy(wl.n, wl.kfield, variant=variant or wl.variant,
                                levels=wl.levels if levels is None else levels, k_ref=wl.k_ref, kacz_rule=rule)
    return [(d["n"], d["relax_op"], d["smoother"], d["resid_op"]) for d in sch]


@pytest.mark.parametrize("rule", ["band", "bins"])
@pytest.mark.parametrize("variant", ["hyb", "sl", "hlm", "sl_plain"])
def test_schedule_matches_oracle_policy(L, variant, rule):
    cases = [I.plain_n64(), I.wedge_n512(), I.grf_n4096(n=512, k=125.0)]
    cases += I.batch_problems(rhs_per_k=1)
    cases += [wl for _, _, wl in I.paper_table_workloads(max_n=256)]
    for wl in cases:
        assert _lib_schedule(wl, variant, rule=rule) == _oracle_schedule(wl, variant, rule), (wl.name, variant)


def test_schedule_of_the_n4096_random_field(L):
    """n = 4096, k = 1000, k (1 + 0.3 g): local k H spans 0.7 .. 1.3 times k_ref H, so with the band
    rule the levels n_l = 1024, 512 and 256 (k_ref H = 0.98, 1.95, 3.9) relax by Kaczmarz."""
    wl = I.grf_n4096()
    for rule in ("band", "bins"):
        assert _lib_schedule(wl, rule=rule) == _oracle_schedule(wl, rule=rule)
    kacz = [s[0] for s in _oracle_schedule(wl) if s[2] == "kaczmarz"]
    assert kacz == [1024, 512, 256]


def test_schedule_of_table1_setting(L):
    kf = I.constant_k(64, 40.0)
    sch = hz.describe_hierarchy(64, kf, variant="hyb", levels=4, k_ref=40.0)
    assert [(d["relax_op"], d["smoother"], d["nu"]) for d in sch] == [
        ("M", "gs", 1), ("M", "kaczmarz", 4), ("M", "kaczmarz", 4), ("L", "direct", 0)]
    sch = hz.describe_hierarchy(64, kf, variant="hyb", levels=4, k_ref=40.0, kacz_rule="bins")
    assert [(d["relax_op"], d["smoother"], d["nu"]) for d in sch] == [
        ("M", "gs", 1), ("M", "kaczmarz", 4), ("M", "gs", 1), ("L", "direct", 0)]


def test_noalloc_rejects_overlapping_outputs_before_any_device_call(L):
    """The allocation-free entry point checks byte ranges on the host: an output that shares a byte
    with an input, or with the other output, is refused before anything touches the device (the
    addresses below are never dereferenced)."""
    from ctypes import c_void_p

    n = 8
    cb = 16 * (n + 1) ** 2  # bytes of one complex128 grid vector
    base = 1 << 40
    kh, u, w, v, dot = base, base + 4 * cb, base + 6 * cb, base + 8 * cb, base + 10 * cb

    def call(kh_, u_, w_, v_, dot_):
        return L.hz_apply_dot_noalloc(n, c_void_p(kh_), 0.5, c_void_p(u_), c_void_p(w_), c_void_p(v_),
                                      c_void_p(dot_), None)

    assert call(kh, u, w, u + 16, dot) == hz.HZ_EINVAL  # v starts inside u
    assert call(kh, u, w, w - cb + 16, dot) == hz.HZ_EINVAL  # v ends inside w
    assert call(kh, u, w, kh + 8, dot) == hz.HZ_EINVAL  # v inside kh
    assert call(kh, u, w, v, v + cb - 16) == hz.HZ_EINVAL  # dot is v's last element
    assert call(kh, u, w, v, u) == hz.HZ_EINVAL  # dot inside u
    assert call(kh, u, w, v, w + 8) == hz.HZ_EINVAL  # dot straddles w
    assert call(kh, u, w, v, kh) == hz.HZ_EINVAL  # dot inside kh


def test_ray_grid_rule_matches_the_oracle(L):
    # the library's host rule for hz_ray_create's m = 0 against oracle.ray_spacing, over the Table 7
    # columns and grids whose power-of-two factors are cut short by divisibility or the two-cell floor
    cases = [(n, k) for k, n in I.PAPER_TABLE7]
    cases += [(n, kh * n) for n in (2, 3, 4, 6, 12, 16, 24, 48, 96, 100, 640, 1024, 4096)
              for kh in (0.01, 0.156, 0.2, 0.3125, 0.625, 1.25, 2.5, 3.0)]
    for n, k in cases:
        assert hz.ray_spacing(n, k) == o.ray_spacing(n, k), (n, k)
    assert hz.ray_spacing(1, 1.0) == 0 and hz.ray_spacing(64, 0.0) == 0 and hz.ray_spacing(64, float("inf")) == 0


def test_ray_footprint_and_cycle_scratch_sizes(L):
    # six sets of (nc + 1) dense blocks of (8 (nc + 1))^2 complex128 dominate the ray arena; the
    # plane-wave table is 8 (n + 1)^2 complex128
    for k, n in I.PAPER_TABLE7:
        m = o.ray_spacing(n, k)
        Nr = n // m + 1
        blocks = 6 * Nr * (8 * Nr) ** 2 * 16
        waves = 8 * (n + 1) ** 2 * 16
        got = L.hz_ray_footprint_bytes(n, k, 0)
        assert got == L.hz_ray_footprint_bytes(n, k, m)
        vectors = 5 * 8 * Nr * Nr * 16  # five ray vectors of Nr rows of 8 Nr unknowns
        assert blocks + waves + vectors <= got <= blocks + waves + vectors + 64 * 1024
    assert L.hz_ray_footprint_bytes(64, 20.0, 3) == 0  # not a power of two
    assert L.hz_ray_footprint_bytes(64, 20.0, 128) == 0  # does not divide n
    assert L.hz_ray_footprint_bytes(1024, 20.0, 4) == 0  # n / m above HZ_RAY_MAX_NC
    n = 200
    assert L.hz_cycle_scratch_bytes(n) >= 3 * 16 * (n + 1) ** 2
    assert L.hz_cycle_scratch_bytes(1) == 0
