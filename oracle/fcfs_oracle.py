"""FP64 CPU oracle (O1) of the continuous Fourier-series block of a Manhattan clip.

TEST INFRASTRUCTURE.  Only the tests, the smoke entry point and the bench's
CPU-baseline leg may import this module; the transform library never does, and
this module shares no code with it.

What it computes.  The clip image is the sum of the indicators of disjoint
polygons (Sec. III-A, Eq. signal_model).  Its Fourier-series coefficient on the
period [0, T)^2 is the inner product with the Fourier basis (Eq. inner_prod,
Eq. fourier_basis), here without the basis normalisation, so F(0,0) is the area:

    F(k, l) = integral over the clip image of exp(-j 2 pi (k x + l y) / T) dx dy.

Derivation used (Prop. rect_union, Prop. poly_int, Lemma polyip).  Lemma polyip
holds for any primitive Omega of the 1-D basis function, because the vertical
edges cancel.  Taking the tail primitive Omega(x) = -integral_x^T phi turns each
horizontal edge's signed rectangle into signed upper-right quadrants
[x_v, T) x [y_v, T) at its two end corners (start corner -1, end corner +1 for a
clockwise ring), so that

    F(k, l) = sum_v s_v X_k(x_v) X_l(y_v),   X_k(a) = integral_a^T exp(-j 2 pi k t / T) dt,

with X_0(a) = T - a and X_k(a) = (j T / (2 pi k)) (1 - exp(-j 2 pi k a / T)) for
k != 0.  This module evaluates exactly that sum, with the FULL tail integrals
(constant parts and T - a included): it assumes nothing about the signs (no
balance), so comparing it with a reduced form checks the reduction.  For
integer coordinates the phase k*a is reduced modulo T in integers before the
FP64 exponential; the reduction is exact mathematics.

The block is returned as a complex128 array of shape (2K+1, 2K+1), entry
[k + K, l + K] holding F(k, l) for |k|, |l| <= K.
"""
import numpy as np

TWO_PI = 2.0 * np.pi
_VBLOCK = 8192  # vertices per partial sum (bounds memory; the sum over v is order-free)


def _phase_exp(freq, coord, T):
    """exp(-j 2 pi f a / T) for every (f, a); exact integer phase reduction when
    both are integers, direct FP64 angle otherwise."""
    freq = np.asarray(freq)
    coord = np.asarray(coord)
    if np.issubdtype(coord.dtype, np.integer) and np.issubdtype(freq.dtype, np.integer):
        p = np.mod(np.multiply.outer(freq.astype(np.int64), coord.astype(np.int64)), T)
        ang = TWO_PI * p.astype(np.float64) / T
    else:
        ang = TWO_PI * np.multiply.outer(freq.astype(np.float64), coord.astype(np.float64)) / T
    return np.exp(-1j * ang)


def tail_integral(freq, coord, T):
    """X[f, v] = integral from coord[v] to T of exp(-j 2 pi f t / T) dt (complex128).

    Closed form of the tail primitive in Lemma polyip for the Fourier basis
    (Eq. fourier_basis): T - a at f = 0, (j T / (2 pi f)) (1 - exp(-j 2 pi f a / T))
    otherwise.
    """
    freq = np.asarray(freq)
    coord = np.asarray(coord)
    E = _phase_exp(freq, coord, T)
    f = freq.astype(np.float64)
    nz = f != 0
    coef = np.zeros(f.shape, dtype=np.complex128)
    coef[nz] = 1j * T / (TWO_PI * f[nz])
    X = coef[:, None] * (1.0 - E)
    X[~nz, :] = T - coord.astype(np.float64)[None, :]
    return X


def freqs(K):
    return np.arange(-K, K + 1, dtype=np.int64)


def block_entries(x, y, s, T, ks, ls):
    """F(k, l) for every k in ``ks`` and l in ``ls`` (the direct vertex sum).

    F = X diag(s) Y^T with X[k, v] = tail_integral(k, x_v), Y[l, v] = tail_integral(l, y_v);
    the product is a library matmul, summed over blocks of vertices.
    """
    ks = np.asarray(ks)
    ls = np.asarray(ls)
    s = np.asarray(s).astype(np.float64)
    V = s.shape[0]
    F = np.zeros((ks.shape[0], ls.shape[0]), dtype=np.complex128)
    for a in range(0, V, _VBLOCK):
        b = min(V, a + _VBLOCK)
        X = tail_integral(ks, np.asarray(x)[a:b], T)
        Y = tail_integral(ls, np.asarray(y)[a:b], T)
        F += (X * s[None, a:b]) @ Y.T
    return F


def block(x, y, s, T, K):
    """The full (2K+1) x (2K+1) block, F[k + K, l + K] = F(k, l)."""
    f = freqs(K)
    return block_entries(x, y, s, T, f, f)


def area_exact(x, y, s, T):
    """F(0, 0) as an exact integer: sum_v s_v (T - x_v)(T - y_v) in int64."""
    x = np.asarray(x, dtype=np.int64)
    y = np.asarray(y, dtype=np.int64)
    s = np.asarray(s, dtype=np.int64)
    return int(np.sum(s * (T - x) * (T - y)))


def pupil_mask(K):
    """Pupil disc of the projection lens (Sec. I): k^2 + l^2 <= K^2."""
    f = freqs(K)
    return (f[:, None] ** 2 + f[None, :] ** 2) <= K * K


def pupil_loss(F, F_target, K):
    """L = sum over the pupil disc of |F - F_target|^2, and its cotangent
    Gbar = dL/dRe F + j dL/dIm F = 2 (F - F_target) on the disc, 0 elsewhere."""
    m = pupil_mask(K)
    D = (F - F_target) * m
    return float(np.sum(np.abs(D) ** 2)), 2.0 * D


def vertex_gradient(x, y, s, T, K, Gbar):
    """dL/dx_v and dL/dy_v for a real loss L with cotangent Gbar over the block.

    Differentiating F(k, l) = sum_v s_v X_k(x_v) X_l(y_v) (Lemma polyip with the
    tail primitive) and using dX_k(a)/da = -exp(-j 2 pi k a / T) for every k
    (including k = 0) gives

        dL/dx_v = -s_v Re sum_{k,l} conj(Gbar(k,l)) exp(-j 2 pi k x_v / T) X_l(y_v),
        dL/dy_v = -s_v Re sum_{k,l} conj(Gbar(k,l)) X_k(x_v) exp(-j 2 pi l y_v / T),

    with dL = Re sum conj(Gbar) dF.  Full tail integrals are used: per vertex,
    the constant parts do not cancel.
    """
    f = freqs(K)
    s = np.asarray(s).astype(np.float64)
    V = s.shape[0]
    Gc = np.conj(Gbar)
    gx = np.zeros(V)
    gy = np.zeros(V)
    for a in range(0, V, _VBLOCK):
        b = min(V, a + _VBLOCK)
        xa, ya = np.asarray(x)[a:b], np.asarray(y)[a:b]
        Ex = _phase_exp(f, xa, T)
        Ey = _phase_exp(f, ya, T)
        Xx = tail_integral(f, xa, T)
        Yy = tail_integral(f, ya, T)
        U = Gc @ Yy            # U[k, v] = sum_l conj(Gbar(k,l)) X_l(y_v)
        W = Gc.T @ Xx          # W[l, v] = sum_k conj(Gbar(k,l)) X_k(x_v)
        gx[a:b] = -s[a:b] * np.real(np.sum(Ex * U, axis=0))
        gy[a:b] = -s[a:b] * np.real(np.sum(Ey * W, axis=0))
    return gx, gy


def edge_gradient(gx, gy, ev0, ev1, eaxis):
    """Derivative w.r.t. each edge position: a vertical edge moves the x of both
    its corners, a horizontal edge the y of both its corners."""
    g_axis0 = np.asarray(gx)[ev0] + np.asarray(gx)[ev1]
    g_axis1 = np.asarray(gy)[ev0] + np.asarray(gy)[ev1]
    return np.where(np.asarray(eaxis) == 0, g_axis0, g_axis1)


def relative_error(F, F_ref, area):
    """max |F - F_ref| / area, the per-clip error measure of the block."""
    return float(np.max(np.abs(np.asarray(F) - np.asarray(F_ref)))) / float(area)
