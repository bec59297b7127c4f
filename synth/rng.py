"""Counter-based SplitMix64 streams (Steele, Lea & Flood, OOPSLA 2014).

Element ``i`` of stream ``(seed, stream)`` is ``mix64(key + (i + 1) * GOLDEN)`` with
``key = mix64(seed + (stream + 1) * GOLDEN)``; ``mix64`` is the SplitMix64 output
finaliser.  Every value is a pure function of (seed, stream, i), so any slice of a
stream can be produced independently and in any order.
"""
import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_S30, _S27, _S31 = np.uint64(30), np.uint64(27), np.uint64(31)


def mix64(z):
    """SplitMix64 finaliser on a uint64 array (wrap-around arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    z = (z ^ (z >> _S30)) * _M1
    z = (z ^ (z >> _S27)) * _M2
    return z ^ (z >> _S31)


def _key(seed, stream):
    return int(mix64(np.array([(int(seed) + (int(stream) + 1) * GOLDEN) & MASK64],
                              dtype=np.uint64))[0])


def u64_stream(seed, stream, count, offset=0):
    """``count`` raw 64-bit values of stream (seed, stream), starting at element ``offset``."""
    key = np.uint64(_key(seed, stream))
    i = np.arange(offset + 1, offset + 1 + count, dtype=np.uint64)
    return mix64(key + i * np.uint64(GOLDEN))


def uniform(seed, stream, count, offset=0):
    """Doubles in [0, 1): the top 53 bits of each raw value times 2^-53."""
    return (u64_stream(seed, stream, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed, stream, count, offset=0):
    """Doubles in [-1, 1)."""
    return 2.0 * uniform(seed, stream, count, offset) - 1.0


def normal(seed, stream, count, offset=0):
    """Standard normals by Box-Muller, one normal per pair of uniforms (cosine branch)."""
    u = uniform(seed, stream, 2 * count, 2 * offset)
    u1 = 1.0 - u[0::2]          # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
