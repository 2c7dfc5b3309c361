"""CPU oracle of the pruned continuous Haar transform (PCHT) of a Manhattan clip.

TEST INFRASTRUCTURE.  Only the tests, the smoke entry point and the bench's
CPU-baseline leg may import this module; the transform library never does, and
this module shares no code with it.

What it computes (Sec. II-C, Sec. III-B).  The 2-D Haar basis of the tile
[0, N) x [0, N) up to level J is the scaling function phi_{0,0,0} and, for
0 <= j < J and 0 <= kx, ky < 2^j, the three wavelets psi^(hg), psi^(gh),
psi^(hh) built from the scaling functions of level j + 1 with the Haar filters
g = (1, 1)/sqrt(2) and h = (1, -1)/sqrt(2) (the first letter acts along x).
phi_{j,kx,ky} is 2^j / N on the dyadic square S_{j,kx,ky} = [kx N/2^j, (kx+1) N/2^j)
x [ky N/2^j, (ky+1) N/2^j) and 0 elsewhere, so its inner product with a polygon's
indicator is 2^j / N times the intersection area (Lemma polyip's remark in
Sec. III-B).  With A_nm the areas of the four children S_{j+1, 2kx+n, 2ky+m}:

    <f, psi^(hg)_{j,kx,ky}> = (2^j / N) (A00 + A01 - A10 - A11)
    <f, psi^(gh)_{j,kx,ky}> = (2^j / N) (A00 - A01 + A10 - A11)
    <f, psi^(hh)_{j,kx,ky}> = (2^j / N) (A00 - A01 - A10 + A11)

The algorithm is the paper's: the transform is linear, so polygons are
transformed one at a time and summed; a polygon's transform is a recursion over
dyadic squares that stops where the square lies completely inside or outside
the polygon (every coefficient below it is zero), with the intersection areas
from Alg. 1 (IntersectionArea over the polygon's horizontal edges).

Areas are exact integers (integer corners, N / 2^J >= 1 an integer), and every
coefficient is an integer times 2^(j - log2 N), exact in FP64.

Output layout (a square of side 2^J, index [x-part, y-part]):
    W[0, 0]                    = <f, phi_{0,0,0}> = area / N
    W[2^j + kx, ky]            = <f, psi^(hg)_{j,kx,ky}>
    W[kx, 2^j + ky]            = <f, psi^(gh)_{j,kx,ky}>
    W[2^j + kx, 2^j + ky]      = <f, psi^(hh)_{j,kx,ky}>
"""
import numpy as np


def horizontal_edges(rx, ry):
    """The horizontal edges (x_i, y_i) -> (x_{i+1}, y_i) of one ring, as arrays."""
    rx = np.asarray(rx, dtype=np.int64)
    ry = np.asarray(ry, dtype=np.int64)
    nx, ny = np.roll(rx, -1), np.roll(ry, -1)
    h = ry == ny
    return rx[h], nx[h], ry[h]


def intersection_area(edges, a1, a2, b1, b2):
    """Alg. 1: area of the polygon inside [a1, a2) x [b1, b2), summed over its
    horizontal edges; an edge entering left to right counts +, right to left -,
    each weighted by the height of the part of the square below it."""
    x0, x1, ye = edges
    u = np.minimum(x0, x1)
    v = np.maximum(x0, x1)
    keep = ~((a2 <= u) | (v <= a1) | (ye <= b1))
    s = np.sign(x1 - x0)
    w = np.minimum(v, a2) - np.maximum(u, a1)
    h = np.minimum(ye, b2) - b1
    return int(np.sum((s * w * h)[keep]))


def _polygon(edges, N, J, num):
    """Add one polygon's coefficient numerators (integers, before the 2^j / N
    scale) into num; recursion over dyadic squares, pruned."""
    A0 = intersection_area(edges, 0, N, 0, N)
    num[0, 0] += A0   # the level-0 scaling numerator
    stack = [(0, 0, 0, A0)]
    while stack:
        j, kx, ky, A = stack.pop()
        side = N >> j
        if j >= J or A == 0 or A == side * side:
            continue   # outside, inside, or finest level: nothing below
        half = side >> 1
        x0, y0 = kx * side, ky * side
        c = [[intersection_area(edges, x0 + n * half, x0 + (n + 1) * half, y0 + m * half, y0 + (m + 1) * half)
              for m in (0, 1)] for n in (0, 1)]
        a00, a01, a10, a11 = c[0][0], c[0][1], c[1][0], c[1][1]
        p = 1 << j
        num[p + kx, ky] += a00 + a01 - a10 - a11
        num[kx, p + ky] += a00 - a01 + a10 - a11
        num[p + kx, p + ky] += a00 - a01 - a10 + a11
        for n in (0, 1):
            for m in (0, 1):
                stack.append((j + 1, 2 * kx + n, 2 * ky + m, c[n][m]))


def level_scale(J, N):
    """S[a, b] = 2^j / N, the scale of the coefficient stored at [a, b] (j = the
    level of that position; 0 for the scaling coefficient at [0, 0])."""
    idx = np.arange(1 << J)
    lev = np.zeros(1 << J, dtype=np.int64)
    lev[1:] = np.floor(np.log2(idx[1:])).astype(np.int64)
    j = np.maximum(lev[:, None], lev[None, :])
    return np.ldexp(1.0, (j - int(np.log2(N))).astype(np.int32))


def pcht(x, y, offsets, N, J):
    """Coefficients up to level J of the clip's polygons (rings in
    x[offsets[m]:offsets[m+1]], clockwise, y up), as the (2^J, 2^J) float64
    square described in the module docstring."""
    if J < 0 or (1 << J) > N:
        raise ValueError("need 0 <= J <= log2 N")
    x = np.asarray(x, dtype=np.int64)
    y = np.asarray(y, dtype=np.int64)
    num = np.zeros((1 << J, 1 << J), dtype=np.int64)
    for m in range(len(offsets) - 1):
        a, b = int(offsets[m]), int(offsets[m + 1])
        _polygon(horizontal_edges(x[a:b], y[a:b]), N, J, num)
    return num.astype(np.float64) * level_scale(J, N)
