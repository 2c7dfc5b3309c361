"""O2: the closed forms of Prop. CFT evaluated over clockwise vertex rings.

TEST INFRASTRUCTURE (see fcfs_oracle).  Independent of the signed-corner
encoding: it reads only the rings, in the paper's notation, where ring vertex
2i -> 2i+1 is a horizontal edge and 2i-1 -> 2i a vertical one (indices taken
modulo the ring length).  Coefficients are unnormalised, i.e. the paper's
alpha_{k,l} times T for a square period N_x = N_y = T:

    F(0,0) = sum_i y_{2i} (x_{2i+1} - x_{2i})                             (Eq. Fdc)
    F(k,0) = j T / (2 pi k) sum_i (y_{2i-1} - y_{2i}) e^{-j w k x_{2i}}      (Eq. Fk0)
    F(0,l) = j T / (2 pi l) sum_i (x_{2i+1} - x_{2i}) e^{-j w l y_{2i}}      (Eq. F0l)
    F(k,l) = -T^2 / (4 pi^2 k l) sum_i e^{-j w l y_{2i}}
                                   (e^{-j w k x_{2i+1}} - e^{-j w k x_{2i}})  (Eq. Fkl)

with w = 2 pi / T.  Linearity over disjoint polygons (Sec. III-C, multiple
polygons) sums the per-ring terms.
"""
import numpy as np

TWO_PI = 2.0 * np.pi


def _ring_triples(x, y, offsets):
    """Index arrays of ring vertices 2i-1, 2i, 2i+1 over all rings."""
    offsets = np.asarray(offsets, dtype=np.int64)
    n = np.diff(offsets)
    if np.any(n % 2):
        raise ValueError("rectilinear rings have an even number of vertices")
    half = n // 2
    ring = np.repeat(np.arange(n.shape[0]), half)
    i = np.arange(half.sum()) - np.repeat(np.cumsum(half) - half, half)
    base = offsets[ring]
    nr = n[ring]
    e = base + (2 * i) % nr
    o = base + (2 * i + 1) % nr
    p = base + (2 * i - 1) % nr
    return p, e, o


def _e(freq, coord, T):
    p = np.mod(np.multiply.outer(np.asarray(freq, dtype=np.int64),
                                 np.asarray(coord, dtype=np.int64)), T)
    return np.exp(-1j * TWO_PI * p.astype(np.float64) / T)


def block(x, y, offsets, T, K):
    """(2K+1) x (2K+1) block from rings (x, y in ring order, polygon offsets)."""
    x = np.asarray(x, dtype=np.int64)
    y = np.asarray(y, dtype=np.int64)
    p, e, o = _ring_triples(x, y, offsets)
    if np.any(y[e] != y[o]):
        raise ValueError("edge 2i -> 2i+1 must be horizontal in every ring")
    f = np.arange(-K, K + 1, dtype=np.int64)
    nz = f != 0
    F = np.zeros((2 * K + 1, 2 * K + 1), dtype=np.complex128)
    # Eq. Fkl
    Ey = _e(f[nz], y[e], T)                         # [l, i]
    Dx = _e(f[nz], x[o], T) - _e(f[nz], x[e], T)    # [k, i]
    kk = f[nz].astype(np.float64)
    alpha = -(T * T) / (4.0 * np.pi ** 2 * np.multiply.outer(kk, kk))
    F[np.ix_(nz, nz)] = alpha * (Dx @ Ey.T)
    # Eq. Fk0 (vertical edge lengths at x_{2i})
    F[nz, K] = (1j * T / (TWO_PI * kk)) * (_e(f[nz], x[e], T) @ (y[p] - y[e]).astype(np.float64))
    # Eq. F0l (horizontal edge lengths at y_{2i})
    F[K, nz] = (1j * T / (TWO_PI * kk)) * (_e(f[nz], y[e], T) @ (x[o] - x[e]).astype(np.float64))
    # Eq. Fdc
    F[K, K] = float(np.sum(y[e] * (x[o] - x[e])))
    return F
