"""Seeded synthetic Manhattan clips: disjoint rectilinear lattice polygons.

This module only builds inputs.  A clip is a square period [0, T) x [0, T)
holding disjoint simple rectilinear polygons whose vertices lie on the integer
lattice (Sec. II-A.2, Eq. polydef_R).  Each polygon is emitted three ways:

* as a clockwise vertex ring (y pointing up) whose first edge is horizontal,
  the form Alg. 2 and Prop. CFT consume;
* as signed vertices (x, y, s): s is the 2-D finite difference of the polygon's
  occupancy at the corner, i.e. +1 / -1 marks of the signed-corner encoding the
  transform library takes as input;
* as its ring edges (pairs of vertex indices plus the axis the edge is
  perpendicular to), so that per-vertex derivatives can be summed into per-edge
  derivatives.

Shapes are the classes of a VLSI metal layer (Sec. IV-A, Fig. layout):
rectangles, L-, T- and U-shapes and unions of up to four rectangles (plus and
staircase), 4 to 12 vertices each, built from small occupancy templates on a
compressed grid whose column widths and row heights are drawn at random.  The
polygons sit on a jittered grid, one per cell, with a margin that keeps them
disjoint; the paper's own layouts are proprietary and these clips stand in for
them.
"""
from dataclasses import dataclass, field
import math

import numpy as np

from .rng import draw_int, draw_unit

# Occupancy templates, rows listed from the bottom (small y) to the top.
TEMPLATES = {
    "rect": [[1]],
    "L": [[1, 1], [1, 0]],
    "T": [[0, 1, 0], [1, 1, 1]],
    "U": [[1, 1, 1], [1, 0, 1]],
    "plus": [[0, 1, 0], [1, 1, 1], [0, 1, 0]],
    "stair": [[1, 1, 1], [1, 1, 0], [1, 0, 0]],
}
# Shape mix of a metal layer: mean of about 6.3 vertices per polygon.
DEFAULT_MIX = (("rect", 0.35), ("L", 0.25), ("T", 0.15), ("U", 0.15),
               ("plus", 0.05), ("stair", 0.05))
RECT_ONLY = (("rect", 1.0),)


def _variants(grid):
    """The distinct images of an occupancy grid under the 8 symmetries of the square."""
    g = np.asarray(grid, dtype=np.int8)
    out, seen = [], set()
    for base in (g, np.fliplr(g)):
        for r in range(4):
            v = np.ascontiguousarray(np.rot90(base, r))
            key = (v.shape, v.tobytes())
            if key not in seen:
                seen.add(key)
                out.append(v)
    return out


def _trace(occ):
    """Clockwise corner ring of a one-piece occupancy grid, in breakpoint indices.

    Returns (ci, cj, cs): column/row breakpoint index and the finite-difference
    sign of each corner, ordered clockwise (y up) with a horizontal first edge.
    """
    nr, nc = occ.shape
    directed = {}
    for j in range(nr):
        for i in range(nc):
            if not occ[j, i]:
                continue
            # clockwise boundary of one cell when y points up
            pts = [(i, j), (i, j + 1), (i + 1, j + 1), (i + 1, j)]
            for a in range(4):
                p, q = pts[a], pts[(a + 1) % 4]
                if (q, p) in directed:
                    del directed[(q, p)]
                else:
                    directed[(p, q)] = True
    nxt = {}
    for p, q in directed:
        if p in nxt:
            raise ValueError("template has a pinch point")
        nxt[p] = q
    start = min(nxt)
    ring = [start]
    while True:
        q = nxt[ring[-1]]
        if q == start:
            break
        ring.append(q)
    if len(ring) != len(nxt):
        raise ValueError("template boundary is not one ring (hole or two pieces)")
    n = len(ring)
    corners = []
    for a in range(n):
        p0, p1, p2 = ring[a - 1], ring[a], ring[(a + 1) % n]
        d_in = (p1[0] - p0[0], p1[1] - p0[1])
        d_out = (p2[0] - p1[0], p2[1] - p1[1])
        if d_in != d_out:
            corners.append(p1)
    # rotate so that the edge corners[0] -> corners[1] is horizontal
    if corners[0][1] != corners[1][1]:
        corners = corners[1:] + corners[:1]

    def o(i, j):
        return int(occ[j, i]) if (0 <= i < nc and 0 <= j < nr) else 0

    ci = np.array([c[0] for c in corners], dtype=np.int64)
    cj = np.array([c[1] for c in corners], dtype=np.int64)
    cs = np.array([o(i, j) - o(i - 1, j) - o(i, j - 1) + o(i - 1, j - 1)
                   for i, j in corners], dtype=np.int8)
    if np.any(cs == 0):
        raise ValueError("corner with zero occupancy difference")
    return ci, cj, cs


@dataclass
class _Kind:
    name: str
    nr: int
    nc: int
    ci: np.ndarray
    cj: np.ndarray
    cs: np.ndarray


def _build_kinds():
    kinds = {}
    for name, grid in TEMPLATES.items():
        lst = []
        for v in _variants(grid):
            ci, cj, cs = _trace(v)
            lst.append(_Kind(name, v.shape[0], v.shape[1], ci, cj, cs))
        kinds[name] = lst
    return kinds


KINDS = _build_kinds()


@dataclass
class Clip:
    """One clip: signed vertices grouped per polygon in ring order, plus edges."""
    T: int
    x: np.ndarray              # int32 [V]
    y: np.ndarray              # int32 [V]
    s: np.ndarray              # int8  [V], +1 / -1
    poly_offsets: np.ndarray   # int64 [n_polys + 1]; polygon m owns vertices [off[m], off[m+1])
    ev0: np.ndarray            # int32 [E]; edge e runs from vertex ev0[e] to ev1[e] (ring order)
    ev1: np.ndarray            # int32 [E]
    eaxis: np.ndarray          # int8  [E]; 0: vertical edge (position is x), 1: horizontal (position is y)
    meta: dict = field(default_factory=dict)

    @property
    def V(self):
        return int(self.x.shape[0])

    @property
    def n_polys(self):
        return int(self.poly_offsets.shape[0] - 1)

    def ring(self, m):
        a, b = int(self.poly_offsets[m]), int(self.poly_offsets[m + 1])
        return self.x[a:b].astype(np.int64), self.y[a:b].astype(np.int64)

    def edge_positions(self):
        """Position of every edge: x of a vertical edge, y of a horizontal one."""
        return np.where(self.eaxis == 0, self.x[self.ev0], self.y[self.ev0]).astype(np.int64)


def _edges_from_offsets(x, y, offsets):
    n_v = np.diff(offsets)
    poly_of = np.repeat(np.arange(len(n_v)), n_v)
    idx = np.arange(len(x), dtype=np.int64)
    start = offsets[poly_of]
    nxt = start + (idx - start + 1) % n_v[poly_of]
    ev0 = idx.astype(np.int32)
    ev1 = nxt.astype(np.int32)
    eaxis = (y[ev0] == y[ev1]).astype(np.int8)
    return ev0, ev1, eaxis


def make_clip(T, n_polys, seed, smin=20, smax=200, wmin=1, margin=1, mix=DEFAULT_MIX):
    """A clip of ``n_polys`` polygons on a jittered grid (one polygon per cell).

    Bounding-box sides are drawn in [min(smin, c//4), min(smax, c - 2*margin)],
    c being the cell side, so that requested densities always fit; sub-widths of
    multi-column templates are at least ``wmin``.
    """
    n_polys = int(n_polys)
    n = max(1, int(math.ceil(math.sqrt(n_polys))))
    c = T // n
    s_lo = min(smin, max(1, c // 4))
    s_hi = min(smax, c - 2 * margin)
    if s_hi < 1:
        raise ValueError("cells too small for the requested polygon count")
    m = np.arange(n_polys, dtype=np.int64)
    ctr = m * 16

    names = [nm for nm, _ in mix]
    probs = np.array([p for _, p in mix], dtype=np.float64)
    cum = np.cumsum(probs / probs.sum())
    tsel = np.minimum(np.searchsorted(cum, draw_unit(seed, ctr + 0), side="right"), len(names) - 1)

    nv = np.zeros(n_polys, dtype=np.int64)
    groups = []
    for t, name in enumerate(names):
        mt = m[tsel == t]
        if mt.size == 0:
            continue
        variants = KINDS[name]
        vsel = draw_int(seed, mt * 16 + 1, 0, len(variants) - 1)
        for vi, kind in enumerate(variants):
            mk = mt[vsel == vi]
            if mk.size == 0:
                continue
            nv[mk] = kind.ci.shape[0]
            groups.append((kind, mk))
    offsets = np.zeros(n_polys + 1, dtype=np.int64)
    np.cumsum(nv, out=offsets[1:])
    V = int(offsets[-1])
    x = np.zeros(V, dtype=np.int32)
    y = np.zeros(V, dtype=np.int32)
    s = np.zeros(V, dtype=np.int8)

    for kind, mk in groups:
        k16 = mk * 16

        def split(total, parts, c_a, c_b):
            # ``parts`` widths >= wmin summing to ``total`` (breakpoint offsets returned)
            extra = total - parts * wmin
            cuts = []
            if parts >= 2:
                a = draw_int(seed, k16 + c_a, 0, extra)
                if parts == 3:
                    b = draw_int(seed, k16 + c_b, 0, extra)
                    cuts = [np.minimum(a, b), np.maximum(a, b)]
                else:
                    cuts = [a]
            bounds = [np.zeros_like(total)] + cuts + [extra]
            bp = [np.zeros_like(total)]
            for p in range(parts):
                bp.append(bp[-1] + (bounds[p + 1] - bounds[p]) + wmin)
            return np.stack(bp, axis=1)

        lo_w = min(max(s_lo, kind.nc * wmin), s_hi)
        lo_h = min(max(s_lo, kind.nr * wmin), s_hi)
        if s_hi < kind.nc * wmin or s_hi < kind.nr * wmin:
            raise ValueError("cells too small for template %s" % kind.name)
        W = draw_int(seed, k16 + 2, lo_w, s_hi)
        H = draw_int(seed, k16 + 3, lo_h, s_hi)
        bx = split(W, kind.nc, 4, 5)
        by = split(H, kind.nr, 6, 7)
        cx = (mk % n) * c
        cy = (mk // n) * c
        x0 = cx + margin + draw_int(seed, k16 + 8, 0, c - 2 * margin - W)
        y0 = cy + margin + draw_int(seed, k16 + 9, 0, c - 2 * margin - H)
        X = x0[:, None] + bx
        Y = y0[:, None] + by
        dst = offsets[mk][:, None] + np.arange(kind.ci.shape[0])[None, :]
        x[dst] = X[:, kind.ci]
        y[dst] = Y[:, kind.cj]
        s[dst] = kind.cs[None, :]

    ev0, ev1, eaxis = _edges_from_offsets(x, y, offsets)
    meta = dict(T=T, n_polys=n_polys, seed=seed, cell=c, side_range=(s_lo, s_hi),
                wmin=wmin, margin=margin)
    return Clip(T, x, y, s, offsets, ev0, ev1, eaxis, meta)


def clip_from_rings(T, rings):
    """A clip from explicit clockwise rings [(xs, ys), ...]; the first edge of each
    ring must be horizontal.  The sign of a corner is -1 at the start and +1 at the
    end of its horizontal edge (the finite difference of the occupancy)."""
    xs, ys, ss, offs = [], [], [], [0]
    for rx, ry in rings:
        rx = np.asarray(rx, dtype=np.int64)
        ry = np.asarray(ry, dtype=np.int64)
        n = rx.shape[0]
        if n % 2 or n < 4:
            raise ValueError("a rectilinear ring has an even number >= 4 of corners")
        if ry[0] != ry[1]:
            raise ValueError("first edge must be horizontal")
        sg = np.where(np.arange(n) % 2 == 0, -1, 1).astype(np.int8)
        xs.append(rx), ys.append(ry), ss.append(sg)
        offs.append(offs[-1] + n)
    x = np.concatenate(xs).astype(np.int32)
    y = np.concatenate(ys).astype(np.int32)
    s = np.concatenate(ss)
    offsets = np.array(offs, dtype=np.int64)
    ev0, ev1, eaxis = _edges_from_offsets(x, y, offsets)
    return Clip(T, x, y, s, offsets, ev0, ev1, eaxis, dict(T=T, n_polys=len(rings)))


def rect_ring(x1, y1, x2, y2):
    """Clockwise ring (y up) of the rectangle [x1, x2) x [y1, y2), horizontal edge first."""
    return [x1, x2, x2, x1], [y2, y2, y1, y1]


def jitter_edges(clip, seed, amp=2):
    """The same clip with every edge moved by an integer drawn from U{-amp..amp}.

    A vertex moves with its vertical edge in x and with its horizontal edge in y.
    Validity needs sub-widths >= 2*amp+1 and a cell margin >= amp+1.
    """
    d = draw_int(seed, np.arange(clip.ev0.shape[0], dtype=np.int64), -amp, amp)
    x = clip.x.astype(np.int64).copy()
    y = clip.y.astype(np.int64).copy()
    vert = clip.eaxis == 0
    for ends in (clip.ev0, clip.ev1):
        x[ends[vert]] += d[vert]
        y[ends[~vert]] += d[~vert]
    meta = dict(clip.meta, jitter_seed=seed, jitter_amp=amp)
    return Clip(clip.T, x.astype(np.int32), y.astype(np.int32), clip.s.copy(),
                clip.poly_offsets.copy(), clip.ev0.copy(), clip.ev1.copy(),
                clip.eaxis.copy(), meta), d


def concat_clips(clips):
    """Concatenated vertex arrays and int64 clip offsets [n+1] for a batch."""
    x = np.concatenate([c.x for c in clips])
    y = np.concatenate([c.y for c in clips])
    s = np.concatenate([c.s for c in clips])
    off = np.zeros(len(clips) + 1, dtype=np.int64)
    np.cumsum([c.V for c in clips], out=off[1:])
    return x, y, s, off
