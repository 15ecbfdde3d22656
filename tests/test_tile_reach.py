"""The geometry behind the tiled Kaczmarz kernel (Sec. 4-5: GS on the normal equations, colours
(i + 2j) mod 5), checked on the CPU by emulation.

A tile of KT x KT outputs holds a region with a halo of 6S columns on each side and 6S / 10S rows
on the near / far side of the sweep order (S sweeps per launch); colour phase ph of the launch
acts only on the rectangle of the region whose actions can still reach the outputs: with
R = 5S - 1 - ph phases after it, columns -1-R .. KT+R and rows -1-R .. KT+2R in tile coordinates
(order 0..4; -1-2R .. KT+R in the order 4..0). These are the constants of `TileGeo` and
`PhaseRect` in csrc/hz_kaczmarz.cu. The test runs whole-level sweeps and the tiled form, each as
a plain sequence of row actions on a small grid with first-order boundary rows (mirror neighbours
with coefficient 2), and requires equal bits on every output node: region values outside the
square are NaN, so a missing dependency shows. Tightening any bound by one node must break it.
"""
import numpy as np
import pytest


def _problem(n, seed):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n + 1, n + 1)) + 1j * rng.normal(size=(n + 1, n + 1)) - 4
    f = rng.normal(size=(n + 1, n + 1)) + 1j * rng.normal(size=(n + 1, n + 1))
    u0 = rng.normal(size=(n + 1, n + 1)) + 1j * rng.normal(size=(n + 1, n + 1))
    return d, f, u0


def _act(u, d, f, n, i, j):
    """One row action u += conj(a_p) (f_p - a_p u) / |a_p|^2 on row (i, j) (arrays indexed [j, i])."""
    iw = i - 1 if i > 0 else 1
    ie = i + 1 if i < n else n - 1
    js = j - 1 if j > 0 else 1
    jn = j + 1 if j < n else n - 1
    cx = 4 if i in (0, n) else 2
    cy = 4 if j in (0, n) else 2
    inv = 1 / (abs(d[j, i]) ** 2 + cx + cy)
    delta = (f[j, i] - (d[j, i] * u[j, i] + u[j, iw] + u[j, ie] + u[js, i] + u[jn, i])) * inv
    u[j, i] += np.conj(d[j, i]) * delta
    if iw == ie:
        u[j, iw] += 2 * delta
    else:
        u[j, iw] += delta
        u[j, ie] += delta
    if js == jn:
        u[js, i] += 2 * delta
    else:
        u[js, i] += delta
        u[jn, i] += delta


def _rect(KT, S, post, ph, shrink=None):
    R = 5 * S - 1 - ph
    b = {"xlo": -1 - R, "xhi": KT + R,
         "ylo": -1 - (2 if post else 1) * R, "yhi": KT + (1 if post else 2) * R}
    if shrink:
        b[shrink] += 1 if shrink.endswith("lo") else -1
    return b


def _tiled_equals_sweeps(n, KT, S, post, shrink=None):
    d, f, u0 = _problem(n, 1000 * n + 10 * KT + S + post)
    colours = ([4, 3, 2, 1, 0] if post else [0, 1, 2, 3, 4]) * S
    ref = u0.copy()
    for c in colours:
        for j in range(n + 1):
            for i in range(n + 1):
                if (i + 2 * j) % 5 == c:
                    _act(ref, d, f, n, i, j)
    HX, HN, HF = 6 * S, 6 * S, 10 * S
    below = HF if post else HN
    RX, RY = KT + 2 * HX, KT + HN + HF
    out = np.full_like(u0, np.nan)
    for y0 in range(0, n + 1, KT):
        for x0 in range(0, n + 1, KT):
            gx, gy = x0 - HX, y0 - below
            reg = np.full_like(u0, np.nan)
            j0, j1, i0, i1 = max(gy, 0), min(gy + RY, n + 1), max(gx, 0), min(gx + RX, n + 1)
            reg[j0:j1, i0:i1] = u0[j0:j1, i0:i1]
            for ph, c in enumerate(colours):
                b = _rect(KT, S, post, ph, shrink)
                for j in range(max(y0 + b["ylo"], 0), min(y0 + b["yhi"], n) + 1):
                    for i in range(max(x0 + b["xlo"], 0), min(x0 + b["xhi"], n) + 1):
                        if (i + 2 * j) % 5 != c:
                            continue
                        # the action's support (mirrors included) must lie in the region
                        assert gx <= i - 1 or i == 0
                        assert i + 1 < gx + RX or i == n
                        assert gy <= j - 1 or j == 0
                        assert j + 1 < gy + RY or j == n
                        _act(reg, d, f, n, i, j)
            out[y0:y0 + KT, x0:x0 + KT] = reg[y0:y0 + KT, x0:x0 + KT]
    return np.array_equal(out, ref)


@pytest.mark.parametrize("n,KT,S,post", [(40, 8, 1, False), (40, 8, 1, True), (44, 8, 2, False), (44, 8, 2, True),
                                         (47, 16, 2, False), (47, 16, 2, True)])
def test_tiles_with_reach_rectangles_give_the_bits_of_whole_level_sweeps(n, KT, S, post):
    assert _tiled_equals_sweeps(n, KT, S, post)


@pytest.mark.parametrize("shrink", ["xlo", "xhi", "ylo", "yhi"])
def test_every_reach_bound_is_tight(shrink):
    # columns and the far row bound of the order 0..4 (yhi) on a pre launch; the far row bound of
    # the order 4..0 (ylo) on a post launch
    post = shrink == "ylo"
    assert not _tiled_equals_sweeps(44, 8, 2, post, shrink)
