"""Kernel forms of a Kaczmarz level (Sec. 4): colour launches, one block, halo tiles, the whole
level over a thread-block cluster, and the whole level in global memory by one cooperative launch
with grid-wide barriers.

All five forms take the same fixed-rounding row actions in the same colour order, so V-cycles run
with any of them give the same bits, in FP32 and in FP64. The FP64 cluster form is also checked
against the oracle per level step (1e-12) and per V-cycle (1e-11). Kaczmarz levels of
n = 48 (49 rows: ragged bands), 64, 128, 256, 512 and 1024 (where the FP32 tiles take two sweeps
per launch), the coarse tail off so that the level runs in the form under test; batches retire
instances inside every form's launches.
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
    return I.Workload(f"wedge_n{n}_k{k:g}", n, k, kf, rhs, variant="hyb", levels=0)


def grf(n=96, k=50.0):
    return I.Workload(f"grf_n{n}", n, k, I.grf_k(n, k, 17), I.centre_source_rhs(n), variant="hyb", levels=0)


# name -> (workload, n of its Kaczmarz level)
CASES = {
    "grf96": (lambda: grf(), 48),
    "wedge512_k100": (lambda: wedge(512, 100.0), 64),
    "wedge512_k160": (lambda: wedge(512, 160.0), 128),
    "wedge1024_k320": (lambda: wedge(1024, 320.0), 256),
    # n_l = 512 and 1024: the FP32 tiles run two sweeps per launch on 32- and 64-node tiles
    "const1024_k600": (lambda: I.Workload("const_n1024", 1024, 600.0, I.constant_k(1024, 600.0),
                                          I.centre_source_rhs(1024), variant="hyb", levels=0), 512),
    "const2048_k1200": (lambda: I.Workload("const_n2048", 2048, 1200.0, I.constant_k(2048, 1200.0),
                                           I.centre_source_rhs(2048), variant="hyb", levels=0), 1024),
}


def rand_c(shape, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def problem(wl, precision, form, batch=1):
    return hzmod().Problem(wl.n, wl.kfield, 0.5, variant=wl.variant, precision=precision, levels=wl.levels,
                           k_ref=wl.k_ref, coarse_tail=False, kacz_form=form, batch=batch)


def kacz_level(sched, nk):
    """Index of the Kaczmarz level of n_l = nk (the band rule can make further levels Kaczmarz)."""
    ls = [l for l, d in enumerate(sched) if d["smoother"] == "kaczmarz" and d["n"] == nk]
    assert len(ls) == 1, sched
    return ls[0]


def vcycle(wl, precision, form, r):
    P = problem(wl, precision, form)
    try:
        sched = P.schedule()
        z = P.vcycle(torch.from_numpy(r.reshape(wl.n + 1, wl.n + 1)).cuda()).cpu().numpy()
    finally:
        P.close()
    return z, sched


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("name", list(CASES))
def test_kaczmarz_forms_give_the_same_bits(name, precision):
    make, nk = CASES[name]
    wl = make()
    r = rand_c((wl.n + 1) ** 2, 77)
    out = {}
    # the cluster form holds levels up to n = 256 in FP32 and 128 in FP64 (28 or 56 bytes a node
    # in 16 x 200 KB)
    cluster_fits = nk <= (256 if precision == "fp32" else 128)
    for form in ("colour", "level", "tile", "cluster", "grid"):
        z, s = vcycle(wl, precision, form, r)
        got = s[kacz_level(s, nk)]["kacz_form"]
        if form in ("colour", "grid") or (form == "cluster" and cluster_fits):
            assert got == form, s
        out[got] = z
    assert len(out) >= (2 if cluster_fits else 1), out.keys()
    ref = out["colour"]
    for form, z in out.items():
        assert np.array_equal(z.view(np.uint64), ref.view(np.uint64)), (form, np.abs(z - ref).max())


@pytest.mark.parametrize("name", ["grf96", "wedge512_k100", "wedge512_k160"])
def test_fp64_cluster_level_steps_match_the_oracle(name):
    make, nk = CASES[name]
    wl = make()
    P = problem(wl, "fp64", "cluster")
    try:
        l = kacz_level(P.schedule(), nk)
        assert P.schedule()[l]["kacz_form"] == "cluster"
        H = o.build_hierarchy(wl.n, wl.kfield, wl.k_ref, wl.variant, wl.levels)
        lv, nc = H.levels[l], H.levels[l + 1].n
        f = rand_c((lv.n + 1) ** 2, 5)
        u_ref = o.helmholtz.relax(lv, f, np.zeros_like(f), post=False)
        fc_ref = lv.R @ (f - lv.B @ u_ref)
        u, fc = P.level_presmooth(l, torch.from_numpy(f.reshape(lv.n + 1, -1)).cuda())
        for got, ref in ((u, u_ref), (fc, fc_ref)):
            err = np.abs(got.cpu().numpy().ravel() - ref).max() / np.abs(ref).max()
            assert err <= 1e-12, err
        u0, ec = rand_c((lv.n + 1) ** 2, 6), rand_c((nc + 1) ** 2, 7)
        ref = o.helmholtz.relax(lv, f, u0 + lv.P @ ec, post=True)
        dv = lambda a, m: torch.from_numpy(a.reshape(m + 1, m + 1)).cuda()
        got = P.level_postsmooth(l, dv(f, lv.n), dv(u0, lv.n), dv(ec, nc)).cpu().numpy().ravel()
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= 1e-12, err
    finally:
        P.close()


@pytest.mark.parametrize("name", ["grf96", "wedge512_k100"])
def test_fp64_cluster_vcycle_matches_the_oracle(name):
    make, nk = CASES[name]
    wl = make()
    r = rand_c((wl.n + 1) ** 2, 78)
    H = o.build_hierarchy(wl.n, wl.kfield, wl.k_ref, wl.variant, wl.levels)
    ref = o.vcycle(H, r.ravel())
    for form in ("cluster", "colour", "grid"):
        z, s = vcycle(wl, "fp64", form, r)
        assert s[kacz_level(s, nk)]["kacz_form"] == form
        err = np.abs(z.ravel() - ref).max() / np.abs(ref).max()
        assert err <= 1e-11, (form, err)


def test_fp64_form_defaults_to_the_cluster():
    wl = CASES["wedge512_k100"][0]()
    P = hzmod().Problem(wl.n, wl.kfield, 0.5, variant="hyb", precision="fp64", k_ref=wl.k_ref, coarse_tail=False)
    try:
        s = P.schedule()
        assert s[kacz_level(s, 64)]["kacz_form"] == "cluster"
        assert all(d["kacz_form"] is None for d in s if d["smoother"] != "kaczmarz")
    finally:
        P.close()


def test_fp64_form_takes_tiles_on_levels_the_cluster_cannot_hold():
    # the random medium at n = 2048 (config 3's kh): Kaczmarz levels 512, 256 (tiles) and 128 (cluster)
    wl = I.grf_n4096(n=2048, k=500.0)
    P = hzmod().Problem(wl.n, wl.kfield, 0.5, variant="hyb", precision="fp64", levels=wl.levels, k_ref=wl.k_ref)
    try:
        forms = {d["n"]: d["kacz_form"] for d in P.schedule() if d["smoother"] == "kaczmarz" and not d["in_tail"]}
        assert forms.get(512) == "tile" and forms.get(256) == "tile", forms
        assert forms.get(128, "cluster") == "cluster", forms
    finally:
        P.close()


@pytest.mark.parametrize("form,precision", [("cluster", "fp32"), ("cluster", "fp64"), ("level", "fp32"),
                                            ("level", "fp64"), ("tile", "fp32"), ("colour", "fp64")])
def test_batched_solves_equal_single_solves(form, precision):
    """Instances of a batch converge at different iterations; a retired instance's blocks leave each
    Kaczmarz launch at its stop flag while the others go on, and every instance keeps the bits of
    its single solve."""
    hz = hzmod()
    wl = wedge(256, 50.0)  # Kaczmarz on n = 32, outside the tail when the tail is off
    n = wl.n
    rhs = np.stack([I.point_source_rhs(n, I.random_interior_nodes(n, 2, s)) for s in (4, 5, 6)])
    P = problem(wl, precision, form, batch=3)
    try:
        assert P.schedule()[kacz_level(P.schedule(), 32)]["kacz_form"] == form
        xb, infos = P.solve_batch(torch.from_numpy(rhs).cuda(), tol=1e-6, maxit=1000)
        xb = xb.cpu().numpy()
    finally:
        P.close()
    assert len({i["iterations"] for i in infos}) > 1, infos
    for q in range(3):
        S = problem(wl, precision, form)
        try:
            x, info, _ = S.solve(torch.from_numpy(rhs[q]).cuda(), tol=1e-6, maxit=1000)
        finally:
            S.close()
        assert info["status"] == 0 and info["iterations"] == infos[q]["iterations"]
        assert np.array_equal(x.cpu().numpy().view(np.uint64), xb[q].view(np.uint64))
