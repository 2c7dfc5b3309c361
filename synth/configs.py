"""The five workloads of the FCFS block transform, as seeded synthetic clips.

Sizes follow the workloads the transform is measured on:

1. T=256, 16 rectangles (sides 4..40), V=64, K=32 (65x65 block).
2. T=4096, 2000 polygons (~12.6k vertices), K=256 (513x513 block).
3. a batch of 512 clips, T=2048, vertex counts log-uniform in [1e3, 1e5], K=128.
4. T=2048, 5000 polygons (~31k vertices), K=128; the target clip has every edge
   moved by U{-2..2}; the loss sums |F - F_target|^2 over the pupil disc
   k^2 + l^2 <= K^2.
5. T=65536, 150000 polygons (~0.95M vertices), K=1024 (2049x2049 block).

Polygons sit one per cell of a grid with side c = T // ceil(sqrt(M)); sides are
drawn in [min(20, c//4), min(200, c - 2*margin)] so that the requested number of
non-overlapping polygons always fits in the period.
"""
import math

import numpy as np

from .layout import RECT_ONLY, concat_clips, jitter_edges, make_clip
from .rng import draw_unit

MEAN_VERTICES = 6.3  # of the default shape mix

CONFIGS = {
    1: dict(T=256, K=32, n_polys=16, smin=4, smax=40, wmin=4, margin=1, mix=RECT_ONLY, seed=1001),
    2: dict(T=4096, K=256, n_polys=2000, smin=20, smax=200, wmin=4, margin=1, seed=1002),
    4: dict(T=2048, K=128, n_polys=5000, smin=20, smax=200, wmin=5, margin=3, seed=1004,
            jitter_seed=2004, jitter_amp=2),
    5: dict(T=65536, K=1024, n_polys=150000, smin=20, smax=200, wmin=4, margin=1, seed=1005),
}
BATCH = dict(T=2048, K=128, n_clips=512, v_min=1e3, v_max=1e5, seed=1003, clip_seed=3000)


def config_clip(i, scale=1.0):
    """Clip of workload ``i`` (1, 2, 4 or 5) and its cut-off K.

    ``scale`` < 1 shrinks the polygon count (same period and shapes) for quick tests.
    """
    c = dict(CONFIGS[i])
    K = c.pop("K")
    T = c.pop("T")
    c.pop("jitter_seed", None), c.pop("jitter_amp", None)
    n = max(1, int(round(c.pop("n_polys") * scale)))
    seed = c.pop("seed")
    return make_clip(T, n, seed, **c), K


def config4_target(clip):
    """The jittered target clip of workload 4 and the per-edge offsets."""
    c = CONFIGS[4]
    return jitter_edges(clip, c["jitter_seed"], c["jitter_amp"])


def batch_vertex_targets(n_clips=None):
    b = BATCH
    n = b["n_clips"] if n_clips is None else n_clips
    u = draw_unit(b["seed"], np.arange(n, dtype=np.int64))
    lo, hi = math.log(b["v_min"]), math.log(b["v_max"])
    return np.round(np.exp(lo + u * (hi - lo))).astype(np.int64)


def batch_clips(n_clips=None, vertex_scale=1.0):
    """Clips of the batch workload (log-uniform vertex counts)."""
    b = BATCH
    targets = batch_vertex_targets(n_clips)
    clips = []
    for c, vt in enumerate(targets):
        n_polys = max(1, int(round(vt * vertex_scale / MEAN_VERTICES)))
        clips.append(make_clip(b["T"], n_polys, b["clip_seed"] + c, smin=20, smax=200,
                               wmin=1, margin=1))
    return clips, b["K"]


def batch_arrays(n_clips=None, vertex_scale=1.0):
    clips, K = batch_clips(n_clips, vertex_scale)
    x, y, s, off = concat_clips(clips)
    return clips, x, y, s, off, K
