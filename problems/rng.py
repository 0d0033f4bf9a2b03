"""Counter-based random numbers: SplitMix64 and Box-Muller, vectorised in numpy.

Every draw is a pure function of (seed, stream, index), so a problem instance
is the same on any machine and numpy version (numpy's own Generator streams are
not guaranteed stable across versions).

SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): state_k = seed + (k+1) * 0x9E3779B97F4A7C15, then the
published three-step xor-shift-multiply finaliser.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def stream_seed(seed: int, stream: int) -> np.uint64:
    """Derive an independent 64-bit seed for sub-stream `stream` of `seed`."""
    with np.errstate(over="ignore"):
        s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ _mix(np.uint64(stream + 1) * _GOLDEN)
        return _mix(s)


def raw_u64(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    s = stream_seed(seed, stream)
    k = np.arange(offset, offset + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(s + (k + np.uint64(1)) * _GOLDEN)


def uniform01(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each SplitMix64 word."""
    z = raw_u64(seed, stream, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, count: int) -> np.ndarray:
    """Standard normals by the Box-Muller transform on pairs of uniforms."""
    m = (count + 1) // 2
    u = uniform01(seed, stream, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    rad = np.sqrt(-2.0 * np.log1p(-u1))  # 1-u1 in (0, 1]
    out = np.empty(2 * m)
    out[0::2] = rad * np.cos(2.0 * np.pi * u2)
    out[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return out[:count]


def integers(seed: int, stream: int, count: int, lo: int, hi: int) -> np.ndarray:
    """Integers uniform in [lo, hi] (inclusive), by scaling a uniform double."""
    u = uniform01(seed, stream, count)
    return lo + np.minimum((u * (hi - lo + 1)).astype(np.int64), hi - lo)
