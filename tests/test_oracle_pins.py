"""The FP64 oracle against what the paper and the mathematics fix."""
import numpy as np
import pytest

import oracle
import pins
from synth import config_clip, make_clip, config4_target

TOL = 1e-12


@pytest.mark.parametrize("clip", pins.tiny_clips(), ids=lambda c: "T%d_V%d" % (c.T, c.V))
def test_brute_force_unit_cells(clip):
    assert pins.pin_brute(clip, K=min(8, clip.T // 2)) < TOL


@pytest.mark.parametrize("clip", pins.tiny_clips()[:2], ids=lambda c: "T%d" % c.T)
def test_brute_force_beyond_nyquist(clip):
    # the continuous transform has no aliasing: check K > T/2 too (Sec. II-C)
    assert pins.pin_brute(clip, K=clip.T) < TOL


@pytest.mark.parametrize("rect,T,K", [((3, 5, 11, 14), 32, 10), ((0, 0, 7, 3), 16, 20),
                                      ((100, 2000, 3000, 4096), 4096, 64), ((5, 9, 6, 10), 64, 33)])
def test_rectangle_closed_form(rect, T, K):
    assert pins.pin_rectangle(T, *rect, K) < TOL


@pytest.mark.parametrize("xv,yv,T", [(3, 7, 16), (0, 0, 12), (15, 2, 16), (16, 5, 16)])
def test_single_quadrant(xv, yv, T):
    if xv == T:
        # an empty quadrant (corner on the right border of the period)
        F = oracle.block(np.array([xv]), np.array([yv]), np.array([1], dtype=np.int8), T, 4)
        assert np.max(np.abs(F)) < 1e-12
    else:
        assert pins.pin_single_quadrant(T, xv, yv, 6) < TOL


@pytest.mark.parametrize("i", [1, 2])
def test_area_equals_shoelace(i):
    clip, _ = config_clip(i)
    assert pins.pin_area(clip) == 0 or pins.pin_area(clip) < 1e-15


def test_area_larger_configs():
    clip, _ = config_clip(5, scale=0.05)
    assert pins.pin_area(clip, K=1) < 1e-15


@pytest.mark.parametrize("i,scale,K", [(1, 1.0, 32), (2, 0.1, 64), (4, 0.05, 40)])
def test_edge_form_prop_cft(i, scale, K):
    clip, _ = config_clip(i, scale)
    assert pins.pin_edge_form(clip, K) < TOL


@pytest.mark.parametrize("i,scale,K", [(1, 1.0, 32), (2, 0.1, 64), (4, 0.05, 128)])
def test_sparse_dft_steps(i, scale, K):
    clip, _ = config_clip(i, scale)
    assert pins.pin_sparse_fft(clip, K) < TOL


def test_hermitian():
    clip, K = config_clip(1)
    assert pins.pin_hermitian(clip, K) < 1e-13


def test_merge_adjacent_rectangles():
    assert pins.pin_merge(32, 12) < TOL


def test_translation_phase_ramp():
    clip, K = config_clip(1)
    dx = int(256 - clip.x.max()) // 2
    dy = -int(clip.y.min()) // 2
    assert pins.pin_translation(clip, dx, dy, K) < 1e-12


def test_disjoint_additivity():
    a = make_clip(64, 4, 21, smin=4, smax=12)
    b = make_clip(64, 4, 22, smin=4, smax=12)
    b_x = b.x + 0  # b lives in the same period; shift b's polygons into free space
    # place each clip in one half of a 128 period so they are disjoint
    T, K = 128, 9
    Fa = oracle.block(a.x, a.y, a.s, T, K)
    Fb = oracle.block(b_x + 64, b.y, b.s, T, K)
    Fu = oracle.block(np.concatenate([a.x, b_x + 64]), np.concatenate([a.y, b.y]),
                      np.concatenate([a.s, b.s]), T, K)
    assert np.max(np.abs(Fa + Fb - Fu)) / abs(Fu[K, K]) < TOL


def _grad_clip():
    clip, _ = config_clip(4, scale=0.002)   # a few polygons, T = 2048
    target, _ = config4_target(clip)
    return clip, target


def test_vertex_gradient_finite_differences():
    clip, target = _grad_clip()
    vs = list(range(0, clip.V, max(1, clip.V // 6)))
    assert pins.pin_vertex_gradient_fd(clip, target, 10, vs) < 1e-6


def test_edge_gradient_boundary_integral():
    clip, target = _grad_clip()
    assert pins.pin_edge_gradient_boundary(clip, target, 10) < 1e-10


def test_edge_gradient_finite_differences_on_polygon():
    """Moving a whole edge keeps a valid polygon: FD of the loss matches the chained gradient."""
    clip, target = _grad_clip()
    T, K = clip.T, 10
    Ft = oracle.block(target.x, target.y, target.s, T, K)
    F = oracle.block(clip.x, clip.y, clip.s, T, K)
    _, G = oracle.pupil_loss(F, Ft, K)
    gx, gy = oracle.vertex_gradient(clip.x, clip.y, clip.s, T, K, G)
    gE = oracle.edge_gradient(gx, gy, clip.ev0, clip.ev1, clip.eaxis)
    h = 1e-4
    worst = 0.0
    for e in range(0, clip.ev0.shape[0], 3):
        xr = clip.x.astype(np.float64)
        yr = clip.y.astype(np.float64)
        arr = xr if clip.eaxis[e] == 0 else yr
        ends = [clip.ev0[e], clip.ev1[e]]
        arr[ends] += h
        lp = pins._loss_at(xr, yr, clip.s, T, K, Ft)
        arr[ends] -= 2 * h
        lm = pins._loss_at(xr, yr, clip.s, T, K, Ft)
        fd = (lp - lm) / (2 * h)
        worst = max(worst, abs(fd - gE[e]) / max(abs(gE).max(), 1e-300))
    assert worst < 1e-6


def test_bessel_bound_and_parseval_convergence():
    """The Fourier basis of the period is orthogonal with squared norm T^2, so
    (1/T^2) sum over |k|,|l| <= K of |F(k,l)|^2 is the squared norm of the image's
    projection: never above the integral of f^2 = the area (Bessel), increasing
    in K and tending to the area (Parseval; the image is an indicator)."""
    for c in pins.tiny_clips()[:2]:
        A = oracle.area_exact(c.x, c.y, c.s, c.T)
        sums = []
        for K in (4, 16, 64, 256):
            F = oracle.block(c.x, c.y, c.s, c.T, K)
            sums.append(float(np.sum(np.abs(F) ** 2)) / (c.T * c.T) / A)
        assert all(v <= 1.0 + 1e-12 for v in sums), sums
        assert all(b > a for a, b in zip(sums, sums[1:])), sums
        assert sums[-1] > 0.99, sums


def test_pupil_disc_lattice_count():
    """The pupil mask of Sec. I against the Gauss circle count from Jacobi's
    two-square theorem, its symmetries and its rim points."""
    assert pins.pin_pupil() == 0
