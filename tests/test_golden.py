"""The oracle still reproduces the values stored by tests/golden/make_golden.py."""
import json
import os

import numpy as np

import oracle
from synth import config_clip, clip_from_rings, rect_ring

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_samples.json")))


def _check(name, clip, T, K):
    g = GOLD[name]
    F = oracle.block(clip.x, clip.y, clip.s, T, K)
    assert oracle.area_exact(clip.x, clip.y, clip.s, T) == g["area"]
    for k, l, re, im in g["entries"]:
        assert abs(F[k + K, l + K] - complex(re, im)) <= 1e-12 * g["area"]


def test_golden_config1():
    clip, K = config_clip(1)
    _check("config1", clip, 256, K)


def test_golden_L_shape():
    L = clip_from_rings(16, [([2, 9, 9, 6, 6, 2], [11, 11, 3, 3, 7, 7])])
    _check("L_shape", L, 16, 4)


def test_golden_step():
    r = clip_from_rings(8, [rect_ring(3, 0, 8, 8)])
    _check("step_u_t_minus_3", r, 8, 2)
    # the k-axis of [3, 8) x [0, 8) is 8 * integral_3^8 e^{-j 2 pi k t / 8} dt and the
    # l-axis vanishes for l != 0 (full period in y)
    g = {(k, l): complex(re, im) for k, l, re, im in GOLD["step_u_t_minus_3"]["entries"]}
    assert abs(g[(0, 1)]) < 1e-12 and abs(g[(1, 1)]) < 1e-12
    assert abs(g[(0, 0)] - 40) < 1e-12


def test_golden_cosine():
    g = GOLD["cosine_config1"]
    clip, K = config_clip(1)
    C = oracle.cosine_block(clip.x, clip.y, clip.s, clip.T, K)
    assert C[0, 0] == g["area"]
    for k, l, v in g["entries"]:
        assert abs(C[k, l] - v) <= 1e-12 * g["area"]


def test_golden_haar():
    g = GOLD["haar_L_shape"]
    L = clip_from_rings(16, [([2, 9, 9, 6, 6, 2], [11, 11, 3, 3, 7, 7])])
    W = oracle.pcht(L.x, L.y, L.poly_offsets, 16, 4)
    assert np.array_equal(W.reshape(-1), np.array(g["square"]))   # exact dyadic values
    assert W[0, 0] * 16 == g["area"]
