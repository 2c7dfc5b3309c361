"""FP64 CPU oracle of the continuous cosine series of a Manhattan clip.

TEST INFRASTRUCTURE.  Only the tests, the smoke entry point and the bench's
CPU-baseline leg may import this module; the transform library never does, and
this module shares no code with it.

What it computes.  The concluding section names the continuous cosine series
as the direct extension of FCFS.  The paper prints no formula for it; the
reading taken here keeps the conventions of the Fourier block (inner product
with the basis, no basis normalisation, so C(0,0) is the area) and uses the
cosine basis of the interval [0, T] at half-period frequencies:

    C(k, l) = integral over the clip image of cos(pi k x / T) cos(pi l y / T) dx dy,
    0 <= k, l <= K.

The image is the same sum of polygon indicators as in Sec. III-A, Eq.
signal_model.  Lemma polyip holds for any primitive of the 1-D basis function
(the vertical edges cancel), so the tail primitive again turns each polygon
into signed upper-right quadrants [x_v, T] x [y_v, T] at its corners:

    C(k, l) = sum_v s_v Xc_k(x_v) Xc_l(y_v),   Xc_k(a) = integral_a^T cos(pi k t / T) dt,

with Xc_0(a) = T - a and, for k >= 1, Xc_k(a) = (T / (pi k)) (sin(pi k) - sin(pi k a / T))
= -(T / (pi k)) sin(pi k a / T).  This module evaluates exactly that sum with
the full tails (T - a included): it assumes nothing about the signs.  For
integer coordinates the phase k a is reduced modulo 2 T in integers before the
FP64 sine; the reduction is exact mathematics.

The block is a float64 array of shape (K + 1, K + 1), entry [k, l] = C(k, l).
"""
import numpy as np

_VBLOCK = 8192  # vertices per partial sum (bounds memory; the sum over v is order-free)


def _half_sin(freq, coord, T):
    """sin(pi f a / T) for every (f, a); the phase f a is reduced modulo 2T in
    integers when both are integers."""
    freq = np.asarray(freq)
    coord = np.asarray(coord)
    if np.issubdtype(coord.dtype, np.integer) and np.issubdtype(freq.dtype, np.integer):
        p = np.mod(np.multiply.outer(freq.astype(np.int64), coord.astype(np.int64)), 2 * T)
        ang = np.pi * p.astype(np.float64) / T
    else:
        ang = np.pi * np.multiply.outer(freq.astype(np.float64), coord.astype(np.float64)) / T
    return np.sin(ang)


def cos_tail(freq, coord, T):
    """Xc[f, v] = integral from coord[v] to T of cos(pi f t / T) dt (float64):
    T - a at f = 0, -(T / (pi f)) sin(pi f a / T) otherwise."""
    freq = np.asarray(freq)
    coord = np.asarray(coord)
    f = freq.astype(np.float64)
    nz = f != 0
    coef = np.zeros(f.shape, dtype=np.float64)
    coef[nz] = -T / (np.pi * f[nz])
    X = coef[:, None] * _half_sin(freq, coord, T)
    X[~nz, :] = T - coord.astype(np.float64)[None, :]
    return X


def cosine_freqs(K):
    return np.arange(0, K + 1, dtype=np.int64)


def cosine_entries(x, y, s, T, ks, ls):
    """C(k, l) for every k in ``ks`` and l in ``ls``: Xc diag(s) Yc^T, a library
    matmul summed over blocks of vertices."""
    ks = np.asarray(ks)
    ls = np.asarray(ls)
    s = np.asarray(s).astype(np.float64)
    V = s.shape[0]
    C = np.zeros((ks.shape[0], ls.shape[0]), dtype=np.float64)
    for a in range(0, V, _VBLOCK):
        b = min(V, a + _VBLOCK)
        X = cos_tail(ks, np.asarray(x)[a:b], T)
        Y = cos_tail(ls, np.asarray(y)[a:b], T)
        C += (X * s[None, a:b]) @ Y.T
    return C


def cosine_block(x, y, s, T, K):
    """The full (K + 1) x (K + 1) block, C[k, l] = C(k, l)."""
    f = cosine_freqs(K)
    return cosine_entries(x, y, s, T, f, f)
