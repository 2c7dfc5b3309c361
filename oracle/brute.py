"""O3: brute force over unit cells, for tiny periods only.

TEST INFRASTRUCTURE (see fcfs_oracle).  Uses neither the signed corners nor any
closed form of the transform:

* occupancy of each unit cell [i, i+1) x [j, j+1) from a point-in-polygon test
  of its centre against the clockwise rings (ray casting along +x; a centre has
  half-integer coordinates, so it never lies on an edge);
* the cell integral of the Fourier basis (Eq. inner_prod) by Gauss-Legendre
  quadrature on each unit interval, c_k(i) = integral_i^{i+1} e^{-j 2 pi k t / T} dt;
* F(k, l) = sum over occupied cells of c_k(i) c_l(j) (separability of the basis).

``cosine_block`` does the same with the cosine basis cos(pi k t / T) of the
continuous cosine series.
"""
import numpy as np

TWO_PI = 2.0 * np.pi


def rasterise(x, y, offsets, T):
    """occ[i, j] = number of rings whose interior holds the centre of cell (i, j)."""
    x = np.asarray(x, dtype=np.int64)
    y = np.asarray(y, dtype=np.int64)
    offsets = np.asarray(offsets, dtype=np.int64)
    occ = np.zeros((T, T), dtype=np.int64)
    cx = np.arange(T) + 0.5
    for m in range(offsets.shape[0] - 1):
        a, b = offsets[m], offsets[m + 1]
        rx, ry = x[a:b], y[a:b]
        inside = np.zeros((T, T), dtype=bool)
        n = b - a
        for t in range(n):
            xa, ya = rx[t], ry[t]
            xb, yb = rx[(t + 1) % n], ry[(t + 1) % n]
            if xa != xb:
                continue  # only vertical edges cross a horizontal ray
            lo, hi = min(ya, yb), max(ya, yb)
            rows = (cx > lo) & (cx < hi)          # cell centres j + 0.5 within the edge span
            cols = cx < xa                         # centres to the left of the edge
            inside ^= np.outer(cols, rows)
        occ += inside
    return occ


def cell_integrals(freq, T, nodes=32):
    """C[f, i] = integral_i^{i+1} exp(-j 2 pi f t / T) dt by Gauss-Legendre."""
    t, w = np.polynomial.legendre.leggauss(nodes)
    u = 0.5 * (t + 1.0)            # nodes on [0, 1]
    pos = np.arange(T)[:, None] + u[None, :]
    freq = np.asarray(freq, dtype=np.float64)
    ph = np.exp(-1j * TWO_PI * freq[:, None, None] * pos[None, :, :] / T)
    return np.sum(ph * (0.5 * w)[None, None, :], axis=2)


def block(x, y, offsets, T, K):
    occ = rasterise(x, y, offsets, T).astype(np.float64)
    f = np.arange(-K, K + 1)
    C = cell_integrals(f, T)
    return C @ occ @ C.T


def cell_integrals_cos(freq, T, nodes=32):
    """Cc[f, i] = integral_i^{i+1} cos(pi f t / T) dt by Gauss-Legendre."""
    t, w = np.polynomial.legendre.leggauss(nodes)
    u = 0.5 * (t + 1.0)
    pos = np.arange(T)[:, None] + u[None, :]
    freq = np.asarray(freq, dtype=np.float64)
    ph = np.cos(np.pi * freq[:, None, None] * pos[None, :, :] / T)
    return np.sum(ph * (0.5 * w)[None, None, :], axis=2)


def cosine_block(x, y, offsets, T, K):
    """C[k, l] = sum over occupied unit cells of Cc_k(i) Cc_l(j), 0 <= k, l <= K."""
    occ = rasterise(x, y, offsets, T).astype(np.float64)
    Cc = cell_integrals_cos(np.arange(0, K + 1), T)
    return Cc @ occ @ Cc.T
