"""Seeded synthetic inputs: wavenumber fields k(x) and point-source right-hand sides.

This module holds no solver arithmetic. It only draws media and sources, so the
CUDA path, the CPU oracle, the tests and the benchmark can all be fed the same
arrays. Arrays are indexed ``[j, i]`` with ``i`` the x index (fastest) and
``j`` the y index, on the ``(n+1) x (n+1)`` vertex grid of the unit square,
``h = 1/n`` (boundary nodes included), matching the problem of Sec. 1, Eq. (1).

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) with Box-Muller normals, written
out here so that a seed gives the same field on every machine and numpy
version.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 13122880  # per-workload seeds are SEED_BASE + workload index

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """``count`` outputs of SplitMix64 started from state ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        inc = np.uint64(0x9E3779B97F4A7C15)
        z = state + inc * np.arange(1, count + 1, dtype=np.uint64)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normals by the Box-Muller transform of SplitMix64 uniforms."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
    return z[:count]


# --------------------------------------------------------------------------- media


def constant_k(n: int, k: float) -> np.ndarray:
    """Constant wavenumber on the (n+1)^2 grid."""
    return np.full((n + 1, n + 1), float(k), dtype=np.float64)


def wedge_k(n: int, k: float, seed: int, factors=(1.0, 1.5, 0.75)) -> np.ndarray:
    """Three-layer wedge medium (the heterogeneous test of Sec. 6, Fig. 3).

    The figure is not available, so the geometry is a seeded stand-in: two
    straight interfaces ``y = a_m + s_m (x - 1/2)`` with ``a = (2/3, 1/3)`` and
    slopes ``s_m ~ U[-0.5, 0.5]``; layers from top to bottom take
    ``k * factors``; a node on an interface takes the upper layer.
    """
    s = uniform01(seed, 2) - 0.5
    x = np.arange(n + 1) / n
    X, Y = np.meshgrid(x, x)  # [j, i]
    top = Y >= 2.0 / 3.0 + s[0] * (X - 0.5)
    mid = (~top) & (Y >= 1.0 / 3.0 + s[1] * (X - 0.5))
    out = np.full((n + 1, n + 1), k * factors[2])
    out[mid] = k * factors[1]
    out[top] = k * factors[0]
    return out


def gaussian_random_field(n: int, seed: int, corr: float = 0.05) -> np.ndarray:
    """Unit-variance Gaussian random field on the (n+1)^2 grid, clipped to [-1, 1].

    Circulant embedding on a periodic ``2n x 2n`` grid of spacing ``h = 1/n``
    with the Gaussian covariance ``exp(-d^2 / (2 corr^2))``: white noise is
    filtered by the square root of the covariance's discrete spectrum, so the
    field's variance is the covariance at zero lag, 1.
    """
    m = 2 * n
    h = 1.0 / n
    d = np.minimum(np.arange(m), m - np.arange(m)) * h
    cov = np.exp(-(d[:, None] ** 2 + d[None, :] ** 2) / (2.0 * corr * corr))
    spec = np.clip(np.fft.fft2(cov).real, 0.0, None)
    w = normal(seed, m * m).reshape(m, m)
    g = np.fft.ifft2(np.sqrt(spec) * np.fft.fft2(w)).real
    return np.clip(g[: n + 1, : n + 1], -1.0, 1.0)


def grf_k(n: int, k: float, seed: int, amp: float = 0.3, corr: float = 0.05) -> np.ndarray:
    """Smooth heterogeneous medium ``k (1 + amp * g(x))`` with ``g`` from :func:`gaussian_random_field`."""
    return k * (1.0 + amp * gaussian_random_field(n, seed, corr))


# --------------------------------------------------------------------------- sources


def point_source_rhs(n: int, nodes, value: float | None = None) -> np.ndarray:
    """Complex RHS that is zero except at the listed ``(i, j)`` nodes, where it is ``value`` (1/h^2 by default)."""
    f = np.zeros((n + 1, n + 1), dtype=np.complex128)
    v = float(n * n) if value is None else value
    for i, j in nodes:
        f[j, i] += v
    return f


def centre_source_rhs(n: int, value: float | None = None) -> np.ndarray:
    """The centre point source of Sec. 6, Tables 1-2 (``f(.5,.5)``), of value 1/h^2 by default."""
    return point_source_rhs(n, [(n // 2, n // 2)], value)


def random_interior_nodes(n: int, count: int, seed: int):
    """``count`` distinct interior nodes drawn uniformly from [1, n-1]^2."""
    out, seen, draw = [], set(), 0
    while len(out) < count:
        u = uniform01(seed + 7919 * draw, 2 * count)
        draw += 1
        for a, b in zip(u[0::2], u[1::2]):
            node = (1 + int(a * (n - 1)), 1 + int(b * (n - 1)))
            if node not in seen:
                seen.add(node)
                out.append(node)
                if len(out) == count:
                    break
    return out


# --------------------------------------------------------------------------- workloads


@dataclass
class Workload:
    """One solve: grid, medium, sources and the hierarchy settings that go with them."""

    name: str
    n: int
    k_ref: float
    kfield: np.ndarray
    rhs: np.ndarray
    variant: str = "hyb"  # hyb | sl | hlm | sl_plain
    levels: int = 0  # 0 = coarsen while n_l is even and larger than 8
    tol: float = 1e-6
    meta: dict = field(default_factory=dict)


def plain_n64() -> Workload:
    """n = 64, constant k = 20, centre source 1/h^2, all-M^h GS V(1,1), 4 levels."""
    n, k = 64, 20.0
    return Workload("plain_n64_k20", n, k, constant_k(n, k), centre_source_rhs(n), variant="sl_plain", levels=4,
                    meta={"medium": "constant k", "rhs": "centre point source 1/h^2"})


def wedge_n512(seed: int = SEED_BASE + 2) -> Workload:
    """n = 512, k = 100, seeded three-layer wedge, 8 seeded point sources, hybrid hierarchy, 8 levels."""
    n, k = 512, 100.0
    kf = wedge_k(n, k, seed)
    rhs = point_source_rhs(n, random_interior_nodes(n, 8, seed + 1))
    return Workload("wedge_n512_k100", n, k, kf, rhs, variant="hyb", levels=8,
                    meta={"medium": "three-layer wedge k*{1.0,1.5,0.75}", "rhs": "8 seeded point sources 1/h^2"})


def grf_n4096(seed: int = SEED_BASE + 3, n: int = 4096, k: float = 1000.0) -> Workload:
    """n = 4096, k = 1000, k(x) = k (1 + 0.3 g), centre source, hybrid hierarchy, 10 levels.

    ``n`` and ``k`` may be shrunk together (same kh) for quick runs.
    """
    kf = grf_k(n, k, seed)
    levels = max(2, int(round(math.log2(n))) - 2)
    return Workload(f"grf_n{n}_k{k:g}", n, k, kf, centre_source_rhs(n), variant="hyb", levels=levels,
                    meta={"medium": "k(1+0.3 g), g Gaussian random field", "rhs": "centre point source 1/h^2"})


# Sec. 6, Tables 1, 2 and 6: (k, n) of each column; Table 6 columns are k_ref with k_ref h = 15/64.
PAPER_TABLE1 = ((40.0, 64), (50.0, 80), (80.0, 128), (100.0, 160), (150.0, 240))
PAPER_TABLE2 = ((40.0, 64), (40.0, 128), (40.0, 256), (40.0, 512))
PAPER_TABLE6 = ((15.0, 64), (30.0, 128), (60.0, 256), (120.0, 512), (240.0, 1024))
# The Table 6 wedge: the figure is missing; its caption puts k between k_ref and 2 k_ref and the
# source at the middle of the upper boundary, so the layers read k_ref * {1, 1.5, 2} top to bottom.
PAPER_WEDGE_FACTORS = (1.0, 1.5, 2.0)
# Table 7: V-cycles with the ray correction used as a stand-alone solver, kh = 0.3125, centre source.
PAPER_TABLE7 = ((20.0, 64), (40.0, 128), (80.0, 256), (160.0, 512))
PAPER_TABLE7_CYCLES = {"hlm": (16, 16, 17, 18), "sl": (23, 34, 41, 48), "hyb": (26, 31, 37, 39)}


def paper_table_workloads(tables=("table1", "table2", "table6"), variant: str = "hyb", max_n: int = 1 << 30):
    """The Bi-CGSTAB runs behind Sec. 6, Tables 1, 2 and 6 (tolerance 1e-7, x0 = 0): constant k with
    a unit source at the centre (Tables 1-2), and the wedge with a unit source at the middle of
    the upper boundary (Table 6). Yields (table, column, Workload)."""
    out = []
    for name, spec in (("table1", PAPER_TABLE1), ("table2", PAPER_TABLE2), ("table6", PAPER_TABLE6)):
        if name not in tables:
            continue
        for k, n in spec:
            if n > max_n:
                continue
            if name == "table6":
                kf = wedge_k(n, k, SEED_BASE + 6, PAPER_WEDGE_FACTORS)
                rhs = point_source_rhs(n, [(n // 2, n)], 1.0)
                meta = {"medium": "wedge k_ref*{1,1.5,2}", "rhs": "unit source at (0.5, 1)"}
            else:
                kf = constant_k(n, k)
                rhs = centre_source_rhs(n, 1.0)
                meta = {"medium": "constant k", "rhs": "unit source at (0.5, 0.5)"}
            col = f"k_ref={k:g}" if name == "table6" else f"k={k:g},h=1/{n}"
            out.append((name, col, Workload(f"{name}_n{n}_k{k:g}", n, k, kf, rhs, variant=variant, levels=0,
                                             tol=1e-7, meta=meta)))
    return out


def paper_table7_workloads(max_n: int = 1 << 30):
    """The stand-alone cycle solves of Sec. 6, Table 7 (tolerance 1e-7, x0 = 0): constant k,
    kh = 0.3125, unit source at the centre. Yields (column, Workload)."""
    out = []
    for k, n in PAPER_TABLE7:
        if n > max_n:
            continue
        out.append((f"k={k:g}", Workload(f"table7_n{n}_k{k:g}", n, k, constant_k(n, k), centre_source_rhs(n, 1.0),
                                         variant="hlm", levels=0, tol=1e-7,
                                         meta={"medium": "constant k", "rhs": "unit source at (0.5, 0.5)"})))
    return out


BATCH_SPECS = ((50.0, 96), (100.0, 192), (200.0, 384), (300.0, 576))


def batch_problems(seed: int = SEED_BASE + 4, rhs_per_k: int = 16):
    """Four constant-k problems (k, n) with kh ~ 2 pi / 12, each with ``rhs_per_k`` seeded point sources."""
    out = []
    for idx, (k, n) in enumerate(BATCH_SPECS):
        nodes = random_interior_nodes(n, rhs_per_k, seed + 101 * idx)
        rhs = np.stack([point_source_rhs(n, [nd]) for nd in nodes])
        out.append(Workload(f"batch_n{n}_k{k:g}", n, k, constant_k(n, k), rhs, variant="hyb", levels=0))
    return out


SERVE_SIZES = (128, 256, 512, 1024, 2048)


@dataclass
class Request:
    rid: int
    arrival_s: float
    n: int
    k: float
    medium: str
    medium_seed: int
    source: tuple


def serving_requests(count: int = 2000, rate_hz: float = 200.0, seed: int = SEED_BASE + 5, media_pool: int = 4):
    """Poisson arrival stream of single-RHS requests.

    Gaps are exponential with mean ``1/rate_hz``; ``n`` is uniform over
    :data:`SERVE_SIZES`; ``k = (2 pi / 12) n`` so that ``kh = 2 pi / 12``; the
    medium is a wedge or a random field with equal odds. Media come from a pool
    of ``media_pool`` seeds per (n, medium) so that generating them does not
    dominate the client; the source node is seeded per request.
    """
    u = uniform01(seed, 4 * count)
    gaps = -np.log(1.0 - u[0::4]) / rate_hz
    t = np.cumsum(gaps) - gaps[0]
    reqs = []
    for r in range(count):
        n = SERVE_SIZES[min(len(SERVE_SIZES) - 1, int(u[4 * r + 1] * len(SERVE_SIZES)))]
        medium = "wedge" if u[4 * r + 2] < 0.5 else "grf"
        mseed = SEED_BASE + 1000 + int(u[4 * r + 3] * media_pool)
        src = random_interior_nodes(n, 1, seed + 17 * r + 3)[0]
        reqs.append(Request(r, float(t[r]), n, 2 * math.pi / 12 * n, medium, mseed, src))
    return reqs


def request_medium(req: Request) -> np.ndarray:
    if req.medium == "wedge":
        return wedge_k(req.n, req.k, req.medium_seed)
    return grf_k(req.n, req.k, req.medium_seed)
