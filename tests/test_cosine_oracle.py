"""The continuous cosine series oracle against facts outside itself, and planted
mistakes in it that those facts must catch (CPU only).

C(k, l) = integral of the clip image times cos(pi k x / T) cos(pi l y / T),
0 <= k, l <= K (the cosine extension named in the concluding section).
"""
import numpy as np
import pytest

import oracle
from oracle import cosine as co
import pins
from synth import config_clip

_orig_sin = co._half_sin
_orig_tail = co.cos_tail
_orig_entries = co.cosine_entries


def test_brute_force_unit_cells():
    for c in pins.tiny_clips():
        assert pins.pin_cosine_brute(c, 10) < 1e-12


def test_brute_force_beyond_the_period():
    """Frequencies up to 4T (several periods of the half-period cosine)."""
    c = pins.tiny_clips()[0]
    assert pins.pin_cosine_brute(c, 4 * c.T) < 1e-11


def test_fourier_identity_period_2T():
    for c in pins.tiny_clips():
        assert pins.pin_cosine_fourier(c, 10) < 1e-12
    clip, _ = config_clip(2, scale=0.05)
    assert pins.pin_cosine_fourier(clip, 24) < 1e-12


@pytest.mark.parametrize("rect,T,K", [((3, 5, 11, 14), 32, 12), ((0, 0, 7, 3), 16, 9), ((10, 2, 64, 61), 64, 16)])
def test_rectangle_quadrature(rect, T, K):
    assert pins.pin_cosine_rectangle(T, *rect, K) < 1e-12


def test_mirror_and_transpose():
    for c in pins.tiny_clips():
        assert pins.pin_cosine_symmetry(c, 9) < 1e-12


@pytest.mark.parametrize("T,K", [(16, 20), (32, 9), (4, 6)])
def test_orthogonality_special_cases(T, K):
    assert pins.pin_cosine_special(T, K) < 1e-12


def test_area_at_origin():
    for c in pins.tiny_clips():
        C = oracle.cosine_block(c.x, c.y, c.s, c.T, 2)
        assert C[0, 0] == oracle.area_exact(c.x, c.y, c.s, c.T)


def test_bessel_bound_and_convergence():
    """The projection's squared norm never exceeds the area and approaches it."""
    for c in pins.tiny_clips()[:2]:
        A = oracle.area_exact(c.x, c.y, c.s, c.T)
        sums = [pins.cosine_bessel_sum(c, K) / A for K in (4, 16, 64, 256)]
        assert all(b <= 1.0 + 1e-12 for b in sums), sums
        assert all(b2 > b1 for b1, b2 in zip(sums, sums[1:])), sums
        assert sums[-1] > 0.98, sums


# ---------------------------------------------------------------------------
# Planted mistakes
# ---------------------------------------------------------------------------
def _sin_period_T(freq, coord, T):       # phase reduced as if the period were T
    return _orig_sin(freq, coord, T / 2)


def _tail_k0_uses_a(freq, coord, T):
    X = _orig_tail(freq, coord, T)
    X[np.asarray(freq) == 0, :] = np.asarray(coord, dtype=np.float64)[None, :]
    return X


def _tail_sign(freq, coord, T):
    X = _orig_tail(freq, coord, T)
    X[np.asarray(freq) != 0, :] *= -1.0
    return X


def _tail_cos_for_sin(freq, coord, T):
    f = np.asarray(freq, dtype=np.float64)
    X = _orig_tail(freq, coord, T)
    nz = f != 0
    ang = np.pi * np.multiply.outer(f, np.asarray(coord, dtype=np.float64)) / T
    X[nz] = (-T / (np.pi * f[nz]))[:, None] * np.cos(ang[nz])
    return X


def _entries_transposed(x, y, s, T, ks, ls):
    return _orig_entries(y, x, s, T, ks, ls)


def _entries_unsigned(x, y, s, T, ks, ls):
    return _orig_entries(x, y, np.abs(np.asarray(s)), T, ks, ls)


def _freqs_from_one(K):
    return np.arange(1, K + 2, dtype=np.int64)


MUTANTS = {
    "sin_period_T": ("_half_sin", _sin_period_T),
    "tail_k0_uses_a": ("cos_tail", _tail_k0_uses_a),
    "tail_sign": ("cos_tail", _tail_sign),
    "tail_cos_for_sin": ("cos_tail", _tail_cos_for_sin),
    "entries_transposed": ("cosine_entries", _entries_transposed),
    "entries_unsigned": ("cosine_entries", _entries_unsigned),
    "freqs_from_one": ("cosine_freqs", _freqs_from_one),
}


def _run_pins():
    tiny = pins.tiny_clips()
    return {
        "brute": max(pins.pin_cosine_brute(c, 8) for c in tiny[:2]),
        "fourier": pins.pin_cosine_fourier(tiny[1], 8),
        "rect": pins.pin_cosine_rectangle(32, 3, 5, 11, 14, 8),
        "special": pins.pin_cosine_special(16, 6),
    }


def test_unmutated_oracle_passes_all_pins():
    errs = _run_pins()
    assert max(errs.values()) < 1e-10, errs


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, monkeypatch):
    attr, fn = MUTANTS[name]
    monkeypatch.setattr(co, attr, fn)
    if hasattr(oracle, attr):
        monkeypatch.setattr(oracle, attr, fn)
    errs = _run_pins()
    assert max(errs.values()) > 1e-3, (name, errs)
