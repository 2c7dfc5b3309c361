"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

Nothing here evaluates the transform: it builds polygons, their signed corners
and their edges, and nothing else.
"""
from .rng import draw_u64, draw_unit, draw_int
from .layout import (Clip, make_clip, clip_from_rings, rect_ring, jitter_edges,
                     concat_clips, TEMPLATES, DEFAULT_MIX, RECT_ONLY)
from .configs import (CONFIGS, BATCH, config_clip, config4_target, batch_clips,
                      batch_arrays, batch_vertex_targets)
