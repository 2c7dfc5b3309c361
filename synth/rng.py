"""Counter-based SplitMix64 draws, vectorised over numpy uint64 arrays.

SplitMix64 is the generator published by Steele, Lea and Flood (OOPSLA 2014):
the n-th output of a stream with state ``seed`` is the 64-bit finaliser applied
to ``seed + n * 0x9E3779B97F4A7C15`` (n = 1, 2, ...).  Because the n-th output
depends only on (seed, n), every draw here is addressed by a counter, which lets
whole arrays of polygons be generated at once and makes every draw reproducible
on any machine.
"""
import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def _finalise(z):
    z = (z ^ (z >> np.uint64(30))) * _MIX1
    z = (z ^ (z >> np.uint64(27))) * _MIX2
    return z ^ (z >> np.uint64(31))


def draw_u64(seed, counter):
    """The ``counter``-th (0-based) SplitMix64 output of stream ``seed``."""
    with np.errstate(over="ignore"):
        c = np.asarray(counter, dtype=np.uint64)
        z = np.uint64(seed) + (c + np.uint64(1)) * _GAMMA
        return _finalise(z)


def draw_unit(seed, counter):
    """Uniform doubles in [0, 1) with 53 random bits."""
    u = draw_u64(seed, counter)
    return (u >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def draw_int(seed, counter, lo, hi):
    """Uniform integers in the closed range [lo, hi] (arrays broadcast)."""
    lo = np.asarray(lo, dtype=np.int64)
    hi = np.asarray(hi, dtype=np.int64)
    span = (hi - lo + 1).astype(np.float64)
    v = lo + np.floor(draw_unit(seed, counter) * span).astype(np.int64)
    return np.minimum(v, hi)
