"""O4: the four steps of FCFS (Sec. III-C.1, Alg. 2) with a library FFT.

TEST INFRASTRUCTURE (see fcfs_oracle).  Reads only the clockwise rings (edge
2i -> 2i+1 horizontal).  For a square period T and |k|, |l| <= K:

Step 1: F(0,0) = polygon area, sum over horizontal edges of y (x_end - x_start).
Step 2: f_x[n] = sum of vertical-edge lengths (y_start - y_end) of the edges at
        x = n mod T; F(k,0) = j T / (2 pi k) DFT_k{f_x}.
Step 3: f_y[n] = sum of horizontal-edge lengths (x_end - x_start) at y = n mod T;
        F(0,l) = j T / (2 pi l) DFT_l{f_y}.
Step 4: the sparse T x T image with +1 at (x_{2i+1}, y_{2i}) and -1 at
        (x_{2i}, y_{2i}); F(k,l) = -T^2 / (4 pi^2 k l) DFT2_{k mod T, l mod T}.

DFTs are numpy.fft (FP64); coefficients carry the unnormalised scale (alpha
times T).  Practical for T up to a few thousand (the image is T x T).
"""
import numpy as np

from .edge_form import _ring_triples

TWO_PI = 2.0 * np.pi


def block(x, y, offsets, T, K):
    x = np.asarray(x, dtype=np.int64)
    y = np.asarray(y, dtype=np.int64)
    p, e, o = _ring_triples(x, y, offsets)
    f = np.arange(-K, K + 1, dtype=np.int64)
    F = np.zeros((2 * K + 1, 2 * K + 1), dtype=np.complex128)
    # Step 4
    img = np.zeros((T, T), dtype=np.float64)
    np.add.at(img, (x[o] % T, y[e] % T), 1.0)
    np.add.at(img, (x[e] % T, y[e] % T), -1.0)
    D = np.fft.fft2(img)
    nz = f != 0
    kk = f[nz].astype(np.float64)
    alpha = -(T * T) / (4.0 * np.pi ** 2 * np.multiply.outer(kk, kk))
    F[np.ix_(nz, nz)] = alpha * D[np.ix_(f[nz] % T, f[nz] % T)]
    # Step 2: vertical edge 2i-1 -> 2i sits at x_{2i}
    fx = np.zeros(T)
    np.add.at(fx, x[e] % T, (y[p] - y[e]).astype(np.float64))
    F[nz, K] = (1j * T / (TWO_PI * kk)) * np.fft.fft(fx)[f[nz] % T]
    # Step 3: horizontal edge 2i -> 2i+1 sits at y_{2i}
    fy = np.zeros(T)
    np.add.at(fy, y[e] % T, (x[o] - x[e]).astype(np.float64))
    F[K, nz] = (1j * T / (TWO_PI * kk)) * np.fft.fft(fy)[f[nz] % T]
    # Step 1
    F[K, K] = float(np.sum(y[e] * (x[o] - x[e])))
    return F
