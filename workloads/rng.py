"""Counter-based SplitMix64 streams (vectorised with numpy uint64 arithmetic)."""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def raw64(seed, count, offset=0):
    """Draws ``offset .. offset+count-1`` of the SplitMix64 stream ``seed``."""
    i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GAMMA
        return _mix(state)


def uniform01(seed, count, offset=0):
    """Uniforms in [0, 1) with 53 random bits each."""
    return (raw64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform(seed, count, lo, hi, offset=0):
    return lo + (hi - lo) * uniform01(seed, count, offset)


def normal(seed, count, offset=0):
    """Standard normals by Box-Muller; uses 2*ceil(count/2) uniforms."""
    pairs = (count + 1) // 2
    u = uniform01(seed, 2 * pairs, 2 * offset)
    u1 = 1.0 - u[0::2]          # in (0, 1], keeps log finite
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * pairs)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]


def complex_normal(seed, count):
    """Complex normals with i.i.d. N(0, 1/2) real and imaginary parts (E|z|^2 = 1)."""
    z = normal(seed, 2 * count)
    return (z[0::2] + 1j * z[1::2]) / np.sqrt(2.0)
