"""Checks that pin the O1 oracle to facts outside itself.

Each function returns an error figure (0 when the fact holds exactly); the pin
tests assert them small, and the mutation tests assert that a planted mistake
in the oracle makes at least one of them large.  None of them re-types the
oracle's tail-integral formula.
"""
import numpy as np

import oracle
from oracle import brute, edge_form, sparse_fft
from synth import make_clip, clip_from_rings, rect_ring, RECT_ONLY

TWO_PI = 2.0 * np.pi


def _gl_integral(freq, a, b, T, nodes=64):
    """integral_a^b exp(-j 2 pi f t / T) dt by Gauss-Legendre (signed interval)."""
    t, w = np.polynomial.legendre.leggauss(nodes)
    mid, half = 0.5 * (a + b), 0.5 * (b - a)
    pts = mid + half * t
    freq = np.asarray(freq, dtype=np.float64)
    return half * np.sum(w[None, :] * np.exp(-1j * TWO_PI * freq[:, None] * pts[None, :] / T), axis=1)


def pin_area(clip, K=2):
    """F(0,0) equals the polygon area from the shoelace formula on the rings (Step 1)."""
    area = 0
    for m in range(clip.n_polys):
        rx, ry = clip.ring(m)
        area += -int(np.sum(rx * np.roll(ry, -1) - np.roll(rx, -1) * ry)) // 2
    F = oracle.block(clip.x, clip.y, clip.s, clip.T, K)
    e1 = abs(oracle.area_exact(clip.x, clip.y, clip.s, clip.T) - area)
    e2 = abs(F[K, K] - area) / max(area, 1)
    return max(e1, e2)


def pin_rectangle(T, x1, y1, x2, y2, K):
    """A rectangle's block is the outer product of two box transforms,
    (b - a) e^{-j pi f (a + b) / T} sinc(f (b - a) / T)."""
    c = clip_from_rings(T, [rect_ring(x1, y1, x2, y2)])
    F = oracle.block(c.x, c.y, c.s, T, K)
    f = np.arange(-K, K + 1)

    def box(a, b):
        return (b - a) * np.exp(-1j * np.pi * f * (a + b) / T) * np.sinc(f * (b - a) / T)

    ref = np.outer(box(x1, x2), box(y1, y2))
    return np.max(np.abs(F - ref)) / ((x2 - x1) * (y2 - y1))


def pin_single_quadrant(T, xv, yv, K):
    """One signed corner alone is the quadrant [x, T) x [y, T): compare with the
    sum of quadrature-integrated unit cells of that quadrant."""
    F = oracle.block(np.array([xv]), np.array([yv]), np.array([1], dtype=np.int8), T, K)
    f = np.arange(-K, K + 1)
    C = brute.cell_integrals(f, T)
    ref = np.outer(C[:, xv:].sum(axis=1), C[:, yv:].sum(axis=1))
    return np.max(np.abs(F - ref)) / ((T - xv) * (T - yv))


def pin_brute(clip, K):
    """O1 equals the unit-cell brute force (no signed corners, no closed form)."""
    F1 = oracle.block(clip.x, clip.y, clip.s, clip.T, K)
    F3 = brute.block(clip.x, clip.y, clip.poly_offsets, clip.T, K)
    return np.max(np.abs(F1 - F3)) / max(abs(F3[K, K]), 1)


def pin_edge_form(clip, K):
    F1 = oracle.block(clip.x, clip.y, clip.s, clip.T, K)
    F2 = edge_form.block(clip.x, clip.y, clip.poly_offsets, clip.T, K)
    return np.max(np.abs(F1 - F2)) / max(abs(F2[K, K]), 1)


def pin_sparse_fft(clip, K):
    F1 = oracle.block(clip.x, clip.y, clip.s, clip.T, K)
    F4 = sparse_fft.block(clip.x, clip.y, clip.poly_offsets, clip.T, K)
    return np.max(np.abs(F1 - F4)) / max(abs(F4[K, K]), 1)


def pin_hermitian(clip, K):
    """f is real, so F(-k,-l) = conj F(k,l)."""
    F = oracle.block(clip.x, clip.y, clip.s, clip.T, K)
    return np.max(np.abs(F[::-1, ::-1] - np.conj(F))) / max(abs(F[K, K]), 1)


def pin_merge(T, K):
    """Two rectangles sharing a side add up to the merged rectangle (Eq. signal_model:
    the half-open cells make them disjoint)."""
    a = clip_from_rings(T, [rect_ring(3, 5, 11, 14)])
    b = clip_from_rings(T, [rect_ring(11, 5, 20, 14)])
    u = clip_from_rings(T, [rect_ring(3, 5, 20, 14)])
    Fa = oracle.block(a.x, a.y, a.s, T, K)
    Fb = oracle.block(b.x, b.y, b.s, T, K)
    Fu = oracle.block(u.x, u.y, u.s, T, K)
    return np.max(np.abs(Fa + Fb - Fu)) / (17 * 9)


def pin_translation(clip, dx, dy, K):
    """Shifting the clip by (dx, dy) multiplies F(k,l) by e^{-j 2 pi (k dx + l dy) / T}."""
    T = clip.T
    F = oracle.block(clip.x, clip.y, clip.s, T, K)
    Fs = oracle.block(clip.x + dx, clip.y + dy, clip.s, T, K)
    f = np.arange(-K, K + 1)
    ramp = np.exp(-1j * TWO_PI * (f[:, None] * dx + f[None, :] * dy) / T)
    return np.max(np.abs(Fs - ramp * F)) / max(abs(F[K, K]), 1)


def _loss_at(xr, yr, s, T, K, Ft):
    F = oracle.block_entries(xr, yr, s, T, oracle.freqs(K), oracle.freqs(K))
    return oracle.pupil_loss(F, Ft, K)[0]


def pin_vertex_gradient_fd(clip, target, K, vertices, h=1e-4):
    """Analytic per-vertex gradient vs central differences of the loss, the vertex
    moved alone (F = sum_v s_v X(x_v) X(y_v) is smooth in each coordinate)."""
    T = clip.T
    Ft = oracle.block(target.x, target.y, target.s, T, K)
    F = oracle.block(clip.x, clip.y, clip.s, T, K)
    _, G = oracle.pupil_loss(F, Ft, K)
    gx, gy = oracle.vertex_gradient(clip.x, clip.y, clip.s, T, K, G)
    xr = clip.x.astype(np.float64)
    yr = clip.y.astype(np.float64)
    err, scale = 0.0, 0.0
    for v in vertices:
        for g, arr, other in ((gx, xr, yr), (gy, yr, xr)):
            keep = arr[v]
            arr[v] = keep + h
            lp = _loss_at(xr, yr, clip.s, T, K, Ft)
            arr[v] = keep - h
            lm = _loss_at(xr, yr, clip.s, T, K, Ft)
            arr[v] = keep
            fd = (lp - lm) / (2 * h)
            err = max(err, abs(fd - g[v]))
            scale = max(scale, abs(fd))
    return err / max(scale, 1e-300)


def pin_edge_gradient_boundary(clip, target, K):
    """dL/d(edge position) from the boundary integral of the moving edge.

    With y up and clockwise rings the interior lies right of the travel
    direction, so dF/da = -integral_{y_s}^{y_e} e^{-j w (k a + l y)} dy for a
    vertical edge at x = a, and dF/db = +integral_{x_s}^{x_e} e^{-j w (k x + l b)} dx
    for a horizontal edge at y = b (signed intervals, quadrature)."""
    T = clip.T
    f = oracle.freqs(K)
    Ft = oracle.block(target.x, target.y, target.s, T, K)
    F = oracle.block(clip.x, clip.y, clip.s, T, K)
    _, G = oracle.pupil_loss(F, Ft, K)
    gx, gy = oracle.vertex_gradient(clip.x, clip.y, clip.s, T, K, G)
    gE = oracle.edge_gradient(gx, gy, clip.ev0, clip.ev1, clip.eaxis)
    ref = np.zeros_like(gE)
    for e in range(clip.ev0.shape[0]):
        a, b = clip.ev0[e], clip.ev1[e]
        if clip.eaxis[e] == 0:
            pos = float(clip.x[a])
            Iy = _gl_integral(f, float(clip.y[a]), float(clip.y[b]), T)
            dF = -np.outer(np.exp(-1j * TWO_PI * f * pos / T), Iy)
        else:
            pos = float(clip.y[a])
            Ix = _gl_integral(f, float(clip.x[a]), float(clip.x[b]), T)
            dF = np.outer(Ix, np.exp(-1j * TWO_PI * f * pos / T))
        ref[e] = np.real(np.sum(np.conj(G) * dF))
    return np.max(np.abs(gE - ref)) / max(np.max(np.abs(ref)), 1e-300)


def tiny_clips():
    """Small clips for the brute-force pins (T <= 32)."""
    return [make_clip(16, 2, 11, smin=3, smax=6, wmin=1, margin=1),
            make_clip(24, 4, 12, smin=3, smax=9, wmin=1, margin=1),
            make_clip(32, 4, 13, smin=4, smax=14, wmin=1, margin=1),
            make_clip(32, 9, 14, smin=3, smax=8, wmin=1, margin=1, mix=RECT_ONLY)]


# ---------------------------------------------------------------------------
# Continuous cosine series, C(k, l) = integral of the image times
# cos(pi k x / T) cos(pi l y / T), 0 <= k, l <= K.
# ---------------------------------------------------------------------------
def _gl_cos_integral(freq, a, b, T, nodes=64):
    """integral_a^b cos(pi f t / T) dt by Gauss-Legendre."""
    t, w = np.polynomial.legendre.leggauss(nodes)
    mid, half = 0.5 * (a + b), 0.5 * (b - a)
    pts = mid + half * t
    freq = np.asarray(freq, dtype=np.float64)
    return half * np.sum(w[None, :] * np.cos(np.pi * freq[:, None] * pts[None, :] / T), axis=1)


def pin_cosine_brute(clip, K):
    """The cosine oracle equals unit-cell rasterisation plus quadrature."""
    C1 = oracle.cosine_block(clip.x, clip.y, clip.s, clip.T, K)
    C3 = brute.cosine_block(clip.x, clip.y, clip.poly_offsets, clip.T, K)
    return np.max(np.abs(C1 - C3)) / max(abs(C3[0, 0]), 1)


def pin_cosine_fourier(clip, K):
    """cos a cos b = (cos(a + b) + cos(a - b)) / 2, so with the Fourier block of
    period 2T (whose basis at (k, l) is exp(-j pi (k x + l y) / T)):
    C(k, l) = Re(F_2T(k, l) + F_2T(k, -l)) / 2."""
    C = oracle.cosine_block(clip.x, clip.y, clip.s, clip.T, K)
    F = oracle.block(clip.x, clip.y, clip.s, 2 * clip.T, K)
    ref = 0.5 * np.real(F[K:, K:] + F[K:, K::-1])
    return np.max(np.abs(C - ref)) / max(abs(ref[0, 0]), 1)


def pin_cosine_rectangle(T, x1, y1, x2, y2, K):
    """A rectangle's cosine block is the outer product of the two interval
    integrals of the 1-D cosines (quadrature, no closed form)."""
    c = clip_from_rings(T, [rect_ring(x1, y1, x2, y2)])
    C = oracle.cosine_block(c.x, c.y, c.s, T, K)
    f = np.arange(0, K + 1)
    ref = np.outer(_gl_cos_integral(f, x1, x2, T), _gl_cos_integral(f, y1, y2, T))
    return np.max(np.abs(C - ref)) / ((x2 - x1) * (y2 - y1))


def _reflect_rings(clip, how):
    """Rings of the clip reflected in x (x -> T - x) or across the diagonal
    (x <-> y), re-ordered so that each stays clockwise with a horizontal first edge."""
    rings = []
    for m in range(clip.n_polys):
        rx, ry = clip.ring(m)
        n = rx.shape[0]
        if how == "mirror_x":   # v1, v0, v_{n-1}, ..., v2: first edge = old edge 0, reversed
            order = np.concatenate([[1, 0], np.arange(n - 1, 1, -1)])
            rings.append((clip.T - rx[order], ry[order]))
        else:                   # v0, v_{n-1}, ..., v1: first edge = old last (vertical) edge
            order = np.concatenate([[0], np.arange(n - 1, 0, -1)])
            rings.append((ry[order], rx[order]))
    return clip_from_rings(clip.T, rings)


def pin_cosine_symmetry(clip, K):
    """cos(pi k (T - x) / T) = (-1)^k cos(pi k x / T): mirroring the clip in x
    multiplies row k by (-1)^k; swapping x and y transposes the block."""
    C = oracle.cosine_block(clip.x, clip.y, clip.s, clip.T, K)
    cm = _reflect_rings(clip, "mirror_x")
    ct = _reflect_rings(clip, "transpose")
    Cm = oracle.cosine_block(cm.x, cm.y, cm.s, clip.T, K)
    Ct = oracle.cosine_block(ct.x, ct.y, ct.s, clip.T, K)
    sgn = (-1.0) ** np.arange(K + 1)
    e1 = np.max(np.abs(Cm - sgn[:, None] * C))
    e2 = np.max(np.abs(Ct - C.T))
    return max(e1, e2) / max(abs(C[0, 0]), 1)


def pin_cosine_special(T, K):
    """Orthogonality on [0, T]: the full square has C = T^2 at (0, 0) and 0
    elsewhere; the strip [0, T] x [0, h] has C(k, l) = 0 for k >= 1 and
    C(0, l) = T integral_0^h cos(pi l y / T) dy."""
    sq = clip_from_rings(T, [rect_ring(0, 0, T, T)])
    C = oracle.cosine_block(sq.x, sq.y, sq.s, T, K)
    ref = np.zeros_like(C)
    ref[0, 0] = T * T
    e1 = np.max(np.abs(C - ref)) / (T * T)
    h = T // 2 + 1
    st = clip_from_rings(T, [rect_ring(0, 0, T, h)])
    C2 = oracle.cosine_block(st.x, st.y, st.s, T, K)
    ref2 = np.zeros_like(C2)
    ref2[0, :] = T * _gl_cos_integral(np.arange(0, K + 1), 0, h, T)
    e2 = np.max(np.abs(C2 - ref2)) / (T * h)
    return max(e1, e2)


def cosine_bessel_sum(clip, K):
    """(1/T^2) sum_{k,l <= K} w_k w_l C(k, l)^2 with w_0 = 1, w_k = 2: the squared
    norm of the image's projection on the first K + 1 cosines per axis
    (orthogonal basis with norms T and T/2), at most the area (Bessel) and
    tending to it as K grows (Parseval; the image is an indicator)."""
    C = oracle.cosine_block(clip.x, clip.y, clip.s, clip.T, K)
    w = np.full(K + 1, 2.0)
    w[0] = 1.0
    return float(np.sum(w[:, None] * w[None, :] * C * C)) / (clip.T * clip.T)


# ---------------------------------------------------------------------------
# Continuous Haar transform (PCHT), coefficients in the square layout of
# oracle.haar: W[0,0] scaling, level-j bands hg [2^j + kx, ky], gh [kx, 2^j + ky],
# hh [2^j + kx, 2^j + ky].
# ---------------------------------------------------------------------------
def dht_square(img):
    """Orthonormal 2-D discrete Haar transform of an N x N image (N = 2^n) by the
    textbook pyramid: at each level the 2 x 2 blocks (p00 p01; p10 p11), first
    index along x, give the scaling part (p00 + p01 + p10 + p11) / 2 and the
    details (p00 + p01 - p10 - p11) / 2 (x), (p00 - p01 + p10 - p11) / 2 (y),
    (p00 - p01 - p10 + p11) / 2 (both)."""
    a = np.asarray(img, dtype=np.float64)
    n = a.shape[0]
    W = np.zeros_like(a)
    while n > 1:
        h = n // 2
        p00, p01, p10, p11 = a[0::2, 0::2], a[0::2, 1::2], a[1::2, 0::2], a[1::2, 1::2]
        W[h:n, 0:h] = (p00 + p01 - p10 - p11) / 2
        W[0:h, h:n] = (p00 - p01 + p10 - p11) / 2
        W[h:n, h:n] = (p00 - p01 - p10 + p11) / 2
        a = (p00 + p01 + p10 + p11) / 2
        n = h
    W[0, 0] = a[0, 0]
    return W


def pin_haar_dht(clip, J=None):
    """The CHT and DHT coefficients coincide for lattice polygons (Sec. II-C): the
    PCHT to level J equals the top-left 2^J square of the DHT of the unit-cell
    rasterisation (point-in-polygon, no corners, no Alg. 1).  Exact."""
    from oracle import haar
    N = clip.T
    n = int(np.log2(N))
    J = n if J is None else J
    W = haar.pcht(clip.x, clip.y, clip.poly_offsets, N, J)
    D = dht_square(brute.rasterise(clip.x, clip.y, clip.poly_offsets, N))
    return float(np.max(np.abs(W - D[:1 << J, :1 << J])))


def pin_haar_parseval(clip):
    """Orthonormal and complete for unit-cell images at J = log2 N: the squared
    coefficients sum to the integral of f^2 = the area (disjoint polygons)."""
    from oracle import haar
    N = clip.T
    W = haar.pcht(clip.x, clip.y, clip.poly_offsets, N, int(np.log2(N)))
    A = oracle.area_exact(clip.x, clip.y, clip.s, N)
    return abs(float(np.sum(W * W)) - A) / A


def pin_haar_half_tile(N, J):
    """f = indicator of [0, N/2) x [0, N): <f, phi_000> = (N^2/2)/N = N/2, the
    level-0 x-detail (2^0/N)(A00 + A01 - A10 - A11) = (N^2/2)/N = N/2, all else 0."""
    from oracle import haar
    c = clip_from_rings(N, [rect_ring(0, 0, N // 2, N)])
    W = haar.pcht(c.x, c.y, c.poly_offsets, N, J)
    ref = np.zeros_like(W)
    ref[0, 0] = N / 2
    if J > 0:
        ref[1, 0] = N / 2
    return float(np.max(np.abs(W - ref))) / N


def _r2(n):
    """Representations of n as a^2 + b^2 over ordered signed pairs, by Jacobi's
    two-square theorem: r2(0) = 1, r2(n) = 4 (d1(n) - d3(n)) with d_i the number
    of divisors of n congruent to i mod 4.  Number theory only: no disc test."""
    if n == 0:
        return 1
    d1 = d3 = 0
    i = 1
    while i * i <= n:
        if n % i == 0:
            for d in {i, n // i}:
                if d % 4 == 1:
                    d1 += 1
                elif d % 4 == 3:
                    d3 += 1
        i += 1
    return 4 * (d1 - d3)


def pin_pupil(Ks=(0, 1, 2, 3, 5, 8, 13, 32)):
    """The pupil disc of Sec. I, k^2 + l^2 <= K^2 on the (2K+1)^2 block, against
    facts fixed by arithmetic: its size is the Gauss circle count sum_{n <= K^2}
    r2(n) (1, 5, 13, 29, 81, 197, 529, 3209 for the Ks above), it is symmetric
    under k -> -k, l -> -l and transposition, and the rim points (+-K, 0),
    (0, +-K) belong to it while (K, 1) does not.  Returns the number of
    violated facts (0 when all hold)."""
    bad = 0
    for K in Ks:
        m = np.asarray(oracle.pupil_mask(K), dtype=bool)
        if m.shape != (2 * K + 1, 2 * K + 1):
            bad += 1
            continue
        if int(m.sum()) != sum(_r2(n) for n in range(K * K + 1)):
            bad += 1
        if not (np.array_equal(m, m[::-1, :]) and np.array_equal(m, m[:, ::-1]) and np.array_equal(m, m.T)):
            bad += 1
        if K >= 1:
            c = K   # index of frequency 0
            if not (m[c + K, c] and m[c - K, c] and m[c, c + K] and m[c, c - K]) or m[c + K, c + 1]:
                bad += 1
    return bad
