"""The synthetic clips are valid Manhattan layouts (Sec. II-A.2)."""
import numpy as np
import pytest

from synth import (make_clip, config_clip, config4_target, batch_vertex_targets, draw_u64,
                   clip_from_rings, rect_ring, concat_clips, TEMPLATES)
from synth.layout import KINDS
from oracle.brute import rasterise


def test_splitmix64_published_vector():
    # First outputs of SplitMix64 seeded with 1234567 (Vigna's reference code).
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    got = [int(v) for v in draw_u64(1234567, np.arange(5))]
    assert got == want


def _ring_checks(clip):
    for m in range(clip.n_polys):
        rx, ry = clip.ring(m)
        n = rx.shape[0]
        assert n % 2 == 0 and 4 <= n <= 12
        nx, ny = np.roll(rx, -1), np.roll(ry, -1)
        horiz = ry == ny
        vert = rx == nx
        assert np.all(horiz ^ vert), "edges must be axis-parallel and non-degenerate"
        assert np.all(horiz[0::2]) and np.all(vert[1::2]), "edges alternate, first horizontal"
        shoelace = np.sum(rx * ny - nx * ry)
        assert shoelace < 0, "clockwise with y up"
        a, b = clip.poly_offsets[m], clip.poly_offsets[m + 1]
        s = clip.s[a:b].astype(np.int64)
        # the start corner of a horizontal edge is -1, its end corner +1
        assert np.all(s[0::2] == -1) and np.all(s[1::2] == 1)


@pytest.mark.parametrize("T,n,seed", [(64, 9, 1), (128, 30, 2), (256, 40, 3), (96, 16, 4)])
def test_clips_disjoint_and_simple(T, n, seed):
    clip = make_clip(T, n, seed, smin=4, smax=40, wmin=1, margin=1)
    _ring_checks(clip)
    occ = rasterise(clip.x, clip.y, clip.poly_offsets, T)
    assert occ.max() <= 1, "polygons overlap"
    for m in range(clip.n_polys):
        rx, ry = clip.ring(m)
        occ_m = rasterise(rx, ry, np.array([0, rx.shape[0]]), T)
        area = -np.sum(rx * np.roll(ry, -1) - np.roll(rx, -1) * ry) // 2
        assert occ_m.sum() == area
    assert np.all((clip.x >= 0) & (clip.x <= T) & (clip.y >= 0) & (clip.y <= T))


def test_templates_cover_shape_classes():
    counts = {name: sorted({k.ci.shape[0] for k in KINDS[name]}) for name in TEMPLATES}
    assert counts == {"rect": [4], "L": [6], "T": [8], "U": [8], "plus": [12], "stair": [8]}


@pytest.mark.parametrize("i", [1, 2, 4, 5])
def test_config_sizes(i):
    clip, K = config_clip(i)
    want_V = {1: 64, 2: 12000, 4: 30000, 5: 1_000_000}[i]
    assert abs(clip.V - want_V) <= 0.07 * want_V
    # every vertical line and every horizontal line carries signs summing to zero
    for coord in (clip.x, clip.y):
        acc = np.zeros(clip.T + 1, dtype=np.int64)
        np.add.at(acc, coord, clip.s.astype(np.int64))
        assert not acc.any()
    if i in (1, 2):
        _ring_checks(clip)


def test_config2_disjoint():
    clip, _ = config_clip(2)
    # polygons sit in disjoint grid cells: check each polygon stays in its cell
    c = clip.meta["cell"]
    n = int(np.ceil(np.sqrt(clip.n_polys)))
    for m in range(0, clip.n_polys, 7):
        rx, ry = clip.ring(m)
        cx, cy = (m % n) * c, (m // n) * c
        assert rx.min() >= cx + 1 and rx.max() <= cx + c - 1
        assert ry.min() >= cy + 1 and ry.max() <= cy + c - 1


def test_config4_jitter_keeps_validity():
    clip, _ = config_clip(4, scale=0.02)
    tgt, d = config4_target(clip)
    assert d.min() >= -2 and d.max() <= 2 and np.any(d != 0)
    _ring_checks_relaxed(tgt)
    occ = rasterise(tgt.x, tgt.y, tgt.poly_offsets, tgt.T)
    assert occ.max() <= 1


def _ring_checks_relaxed(clip):
    for m in range(clip.n_polys):
        rx, ry = clip.ring(m)
        nx, ny = np.roll(rx, -1), np.roll(ry, -1)
        assert np.all((rx == nx) ^ (ry == ny))
        assert np.sum(rx * ny - nx * ry) < 0


def test_batch_vertex_counts_log_uniform():
    v = batch_vertex_targets()
    assert v.shape == (512,) and v.min() >= 1000 and v.max() <= 100000
    lv = np.log10(v)
    assert abs(lv.mean() - 4.0) < 0.1  # log-uniform on [3, 5]


def test_determinism():
    a = make_clip(512, 50, 9)
    b = make_clip(512, 50, 9)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.y, b.y) and np.array_equal(a.s, b.s)


def test_clip_from_rings_and_concat():
    c = clip_from_rings(16, [rect_ring(1, 2, 5, 7), rect_ring(8, 8, 12, 10)])
    assert list(c.s) == [-1, 1, -1, 1, -1, 1, -1, 1]
    x, y, s, off = concat_clips([c, c])
    assert list(off) == [0, 8, 16] and x.shape == (16,)
