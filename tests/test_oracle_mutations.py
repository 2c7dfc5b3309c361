"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin fails.

Each mutant replaces one oracle function with a subtly wrong version: a dropped
term, a wrong sign, a transposed operand, an index shift.  The pin suite must
flag every one of them.
"""
import numpy as np
import pytest

import oracle
from oracle import fcfs_oracle as fo
import pins
from synth import config_clip, config4_target

_orig_tail = fo.tail_integral
_orig_phase = fo._phase_exp
_orig_entries = fo.block_entries
_orig_vgrad = fo.vertex_gradient
_orig_pupil = fo.pupil_mask


def _tail_no_constant(freq, coord, T):
    X = _orig_tail(freq, coord, T)
    f = np.asarray(freq, dtype=np.float64)
    nz = f != 0
    X[nz] -= (1j * T / (2 * np.pi * f[nz]))[:, None]
    return X


def _tail_k0_wrong(freq, coord, T):
    X = _orig_tail(freq, coord, T)
    X[np.asarray(freq) == 0, :] = np.asarray(coord, dtype=np.float64)[None, :]
    return X


def _tail_half_angle(freq, coord, T):
    return _orig_tail(freq, coord, 2 * T) / 2.0


def _phase_conj(freq, coord, T):
    return np.conj(_orig_phase(freq, coord, T))


def _entries_transposed(x, y, s, T, ks, ls):
    return _orig_entries(y, x, s, T, ks, ls)


def _entries_unsigned(x, y, s, T, ks, ls):
    return _orig_entries(x, y, np.abs(np.asarray(s)), T, ks, ls)


def _freqs_shifted(K):
    return np.arange(-K + 1, K + 2, dtype=np.int64)


def _vgrad_sign(x, y, s, T, K, G):
    gx, gy = _orig_vgrad(x, y, s, T, K, G)
    return -gx, -gy


def _vgrad_swapped(x, y, s, T, K, G):
    gx, gy = _orig_vgrad(x, y, s, T, K, G)
    return gy, gx


def _vgrad_conj_cotangent(x, y, s, T, K, G):
    return _orig_vgrad(x, y, s, T, K, np.conj(G))


def _pupil_strict(K):
    f = np.arange(-K, K + 1)
    return (f[:, None] ** 2 + f[None, :] ** 2) < K * K


def _pupil_half_radius(K):
    f = np.arange(-K, K + 1)
    return (f[:, None] ** 2 + f[None, :] ** 2) <= (K // 2) ** 2


def _pupil_square(K):
    return np.ones((2 * K + 1, 2 * K + 1), dtype=bool)


MUTANTS = {
    "tail_no_constant": ("tail_integral", _tail_no_constant),
    "tail_k0_uses_a": ("tail_integral", _tail_k0_wrong),
    "tail_half_angle": ("tail_integral", _tail_half_angle),
    "phase_sign": ("_phase_exp", _phase_conj),
    "entries_transposed": ("block_entries", _entries_transposed),
    "entries_unsigned": ("block_entries", _entries_unsigned),
    "freqs_shifted": ("freqs", _freqs_shifted),
    "grad_sign": ("vertex_gradient", _vgrad_sign),
    "grad_swapped": ("vertex_gradient", _vgrad_swapped),
    "grad_conj_cotangent": ("vertex_gradient", _vgrad_conj_cotangent),
    "pupil_strict": ("pupil_mask", _pupil_strict),
    "pupil_half_radius": ("pupil_mask", _pupil_half_radius),
    "pupil_square": ("pupil_mask", _pupil_square),
}


def _run_pins():
    errs = {}
    tiny = pins.tiny_clips()
    errs["brute"] = max(pins.pin_brute(c, 6) for c in tiny[:2])
    errs["rect"] = pins.pin_rectangle(32, 3, 5, 11, 14, 8)
    errs["quadrant"] = pins.pin_single_quadrant(16, 3, 7, 5)
    errs["area"] = pins.pin_area(tiny[1])
    errs["hermitian"] = pins.pin_hermitian(tiny[1], 6)
    errs["merge"] = pins.pin_merge(32, 8)
    clip, _ = config_clip(4, scale=0.002)
    target, _ = config4_target(clip)
    errs["edge_grad"] = pins.pin_edge_gradient_boundary(clip, target, 6)
    errs["vertex_fd"] = pins.pin_vertex_gradient_fd(clip, target, 6, [0, 5])
    errs["pupil"] = float(pins.pin_pupil())
    return errs


def test_unmutated_oracle_passes_all_pins():
    errs = _run_pins()
    assert max(errs.values()) < 1e-6, errs


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, monkeypatch):
    attr, fn = MUTANTS[name]
    monkeypatch.setattr(fo, attr, fn)
    if hasattr(oracle, attr):
        monkeypatch.setattr(oracle, attr, fn)
    errs = _run_pins()
    assert max(errs.values()) > 1e-3, (name, errs)
