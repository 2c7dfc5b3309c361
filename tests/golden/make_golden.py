"""Writes tests/golden/*.json from the oracles only (Fourier block, cosine
series, Haar transform).

The paper prints no numeric worked example for the Fourier series (its only
worked figure, the pruned Haar flow of u(t-3) on [0, 8), carries no values), so
the stored values here are oracle outputs on seeded clips.  They guard the
oracle against silent changes of its arithmetic; they are regenerated only by
this script, and a change to them must name the passage that justifies it.

Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from synth import config_clip, clip_from_rings, rect_ring  # noqa: E402


def sample(F, K, picks):
    return [[int(k), int(l), float(F[k + K, l + K].real), float(F[k + K, l + K].imag)]
            for k, l in picks]


def main():
    out = {}
    clip, K = config_clip(1)
    F = oracle.block(clip.x, clip.y, clip.s, clip.T, K)
    picks = [(0, 0), (1, 0), (0, 1), (1, 1), (-1, 1), (K, K), (-K, K), (7, -3), (-12, 25), (32, 0)]
    out["config1"] = dict(
        source="oracle.block on synth.config_clip(1): T=256, 16 rectangles, V=64, K=32",
        area=oracle.area_exact(clip.x, clip.y, clip.s, clip.T), entries=sample(F, K, picks))
    L = clip_from_rings(16, [([2, 9, 9, 6, 6, 2], [11, 11, 3, 3, 7, 7])])
    F = oracle.block(L.x, L.y, L.s, 16, 4)
    out["L_shape"] = dict(
        source="oracle.block on the L-shaped ring (2,11)(9,11)(9,3)(6,3)(6,7)(2,7), T=16, K=4",
        area=oracle.area_exact(L.x, L.y, L.s, 16),
        entries=sample(F, 4, [(0, 0), (1, 0), (0, -1), (1, 1), (2, -3), (4, 4)]))
    r = clip_from_rings(8, [rect_ring(3, 0, 8, 8)])
    F = oracle.block(r.x, r.y, r.s, 8, 2)
    out["step_u_t_minus_3"] = dict(
        source="oracle.block on [3, 8) x [0, 8), the 2-D extension of the step u(t-3) on [0, 8) "
               "used in the Haar flow figure (Fig. sigflow), T=8, K=2",
        area=oracle.area_exact(r.x, r.y, r.s, 8),
        entries=sample(F, 2, [(0, 0), (1, 0), (2, 0), (1, 1), (0, 1)]))
    clip, K = config_clip(1)
    C = oracle.cosine_block(clip.x, clip.y, clip.s, clip.T, K)
    out["cosine_config1"] = dict(
        source="oracle.cosine_block on synth.config_clip(1): T=256, 16 rectangles, V=64, K=32",
        area=oracle.area_exact(clip.x, clip.y, clip.s, clip.T),
        entries=[[int(k), int(l), float(C[k, l])] for k, l in
                 [(0, 0), (1, 0), (0, 1), (1, 1), (2, 5), (7, 3), (K, K), (K, 0), (13, 29)]])
    W = oracle.pcht(L.x, L.y, L.poly_offsets, 16, 4)
    out["haar_L_shape"] = dict(
        source="oracle.pcht on the L-shaped ring (2,11)(9,11)(9,3)(6,3)(6,7)(2,7), N=16, J=4 "
               "(the full 16 x 16 coefficient square, row-major)",
        area=oracle.area_exact(L.x, L.y, L.s, 16), square=[float(v) for v in W.reshape(-1)])
    with open(os.path.join(HERE, "oracle_samples.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
