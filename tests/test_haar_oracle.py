"""The PCHT oracle against facts outside itself (CPU only), and planted mistakes
in it that those facts must catch."""
import numpy as np
import pytest

from oracle import haar
import pins
from synth import make_clip, RECT_ONLY


def haar_clips():
    """Small clips with power-of-two periods for the exact pins."""
    return [c for c in pins.tiny_clips() if c.T & (c.T - 1) == 0] + [
        make_clip(64, 12, 15, smin=3, smax=14, wmin=1, margin=1),
        make_clip(64, 6, 16, smin=4, smax=20, wmin=2, margin=1, mix=RECT_ONLY)]


def test_equals_dht_of_rasterisation():
    for c in haar_clips():
        assert pins.pin_haar_dht(c) == 0.0


def test_coarser_levels_equal_dht_corner():
    for c in haar_clips()[:3]:
        n = int(np.log2(c.T))
        for J in range(n):
            assert pins.pin_haar_dht(c, J) == 0.0, J


def test_parseval():
    for c in haar_clips():
        assert pins.pin_haar_parseval(c) < 1e-14


@pytest.mark.parametrize("N,J", [(16, 4), (64, 3), (8, 0)])
def test_half_tile(N, J):
    assert pins.pin_haar_half_tile(N, J) == 0.0


def test_intersection_area_of_rectangle():
    """Alg. 1 on one rectangle [2, 9) x [3, 7) against the clipped product of sides."""
    e = haar.horizontal_edges([2, 9, 9, 2], [7, 7, 3, 3])
    for (a1, a2, b1, b2) in [(0, 16, 0, 16), (4, 8, 0, 5), (9, 12, 0, 16), (0, 3, 6, 9), (5, 6, 7, 8)]:
        w = max(0, min(9, a2) - max(2, a1))
        h = max(0, min(7, b2) - max(3, b1))
        assert haar.intersection_area(e, a1, a2, b1, b2) == w * h


def test_rejects_bad_level():
    c = haar_clips()[0]
    with pytest.raises(ValueError):
        haar.pcht(c.x, c.y, c.poly_offsets, c.T, int(np.log2(c.T)) + 1)


# ---------------------------------------------------------------------------
# Planted mistakes
# ---------------------------------------------------------------------------
_orig_area = haar.intersection_area
_orig_scale = haar.level_scale
_orig_poly = haar._polygon


def _area_edge_sign(edges, a1, a2, b1, b2):
    x0, x1, ye = edges
    return _orig_area((x1, x0, ye), a1, a2, b1, b2)


def _area_height_from_top(edges, a1, a2, b1, b2):
    x0, x1, ye = edges
    u, v = np.minimum(x0, x1), np.maximum(x0, x1)
    keep = ~((a2 <= u) | (v <= a1) | (ye <= b1))
    return int(np.sum((np.sign(x1 - x0) * (np.minimum(v, a2) - np.maximum(u, a1)) * (b2 - ye))[keep]))


def _scale_level_up(J, N):
    return _orig_scale(J, N) * 2.0


def _make_poly(swap_bands=False, h_sign=False, shallow=False, child_transposed=False):
    def poly(edges, N, J, num):
        A0 = haar.intersection_area(edges, 0, N, 0, N)
        num[0, 0] += A0
        stack = [(0, 0, 0, A0)]
        while stack:
            j, kx, ky, A = stack.pop()
            side = N >> j
            if j >= J - (1 if shallow else 0) or A == 0 or A == side * side:
                continue
            half = side >> 1
            x0, y0 = kx * side, ky * side
            c = [[haar.intersection_area(edges, x0 + n * half, x0 + (n + 1) * half, y0 + m * half,
                                         y0 + (m + 1) * half) for m in (0, 1)] for n in (0, 1)]
            if child_transposed:
                c = [[c[0][0], c[1][0]], [c[0][1], c[1][1]]]
            a00, a01, a10, a11 = c[0][0], c[0][1], c[1][0], c[1][1]
            hg, gh, hh = a00 + a01 - a10 - a11, a00 - a01 + a10 - a11, a00 - a01 - a10 + a11
            if swap_bands:
                hg, gh = gh, hg
            if h_sign:
                hg, hh = -hg, -hh
            p = 1 << j
            num[p + kx, ky] += hg
            num[kx, p + ky] += gh
            num[p + kx, p + ky] += hh
            for n in (0, 1):
                for m in (0, 1):
                    stack.append((j + 1, 2 * kx + n, 2 * ky + m, c[n][m]))
    return poly


MUTANTS = {
    "area_edge_sign": ("intersection_area", _area_edge_sign),
    "area_height_from_top": ("intersection_area", _area_height_from_top),
    "scale_level_up": ("level_scale", _scale_level_up),
    "bands_swapped": ("_polygon", _make_poly(swap_bands=True)),
    "h_filter_sign": ("_polygon", _make_poly(h_sign=True)),
    "stops_a_level_early": ("_polygon", _make_poly(shallow=True)),
    "children_transposed": ("_polygon", _make_poly(child_transposed=True)),
}


def _run_pins():
    cs = haar_clips()
    return {"dht": max(pins.pin_haar_dht(c) for c in cs[:2]),
            "parseval": pins.pin_haar_parseval(cs[0]),
            "half": pins.pin_haar_half_tile(16, 4)}


def test_unmutated_oracle_passes_all_pins():
    assert max(_run_pins().values()) < 1e-12


def test_the_unmutated_polygon_recursion_is_the_oracle():
    c = haar_clips()[0]
    ref = haar.pcht(c.x, c.y, c.poly_offsets, c.T, 4)
    num = np.zeros((16, 16), dtype=np.int64)
    for m in range(c.n_polys):
        a, b = int(c.poly_offsets[m]), int(c.poly_offsets[m + 1])
        _make_poly()(haar.horizontal_edges(c.x[a:b], c.y[a:b]), c.T, 4, num)
    assert np.array_equal(num * haar.level_scale(4, c.T), ref)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, monkeypatch):
    attr, fn = MUTANTS[name]
    monkeypatch.setattr(haar, attr, fn)
    errs = _run_pins()
    assert max(errs.values()) > 1e-3, (name, errs)


def test_step_of_the_flow_figure():
    """Fig. sigflow prunes the 1-D Haar flow of f(t) = u(t - 3) on [0, 8) to the
    supports that straddle t = 3: [0, 8), [0, 4) and [2, 4).  On the tile its
    2-D extension [3, 8) x [0, 8) (N = 8, J = 3) is constant along y, so only
    the x-details (hg) of those supports are nonzero, at every ky.  From the
    definitions (areas of the children A_nm, n along x):
      <f, phi_000> = 40 / 8 = 5;
      j = 0: (2^0 / 8)((4 + 4) - (16 + 16)) = -3;
      j = 1, kx = 0 (children of side 2): (2 / 8)((0 + 0) - (2 + 2)) = -1;
      j = 2, kx = 1 (children of side 1): (4 / 8)((0 + 0) - (1 + 1)) = -1."""
    from synth import clip_from_rings, rect_ring
    c = clip_from_rings(8, [rect_ring(3, 0, 8, 8)])
    W = haar.pcht(c.x, c.y, c.poly_offsets, 8, 3)
    ref = np.zeros((8, 8))
    ref[0, 0] = 5.0
    ref[1, 0] = -3.0
    ref[2, 0] = ref[2, 1] = -1.0
    ref[4 + 1, 0:4] = -1.0
    assert np.array_equal(W, ref)
