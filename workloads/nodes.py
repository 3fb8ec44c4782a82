"""Node families x_j in [-1/2, 1/2) used by the paper's experiments (Sec. 3.1, Ex. 3.3
jittered nodes eq:jittered_nodes; Remark on cond(A), Chebyshev nodes eq:tschebyscheff_nodes)."""
import numpy as np
from .rng import uniform


def wrap_half(x):
    """Maps reals onto the torus representative in [-1/2, 1/2)."""
    y = np.asarray(x, dtype=np.float64)
    y = y - np.floor(y + 0.5)
    # floor(y + 0.5) can round so that y lands exactly on +1/2; fold it back
    y[y >= 0.5] -= 1.0
    return y


def equispaced(n):
    """x_j = j/n, j = -n/2 .. n/2-1 (the equispaced case of Sec. 3.2)."""
    return (np.arange(n, dtype=np.float64) - n // 2) / n


def jittered(seed, n, jitter=None):
    """x_j = (j - n/2)/n + U(-jitter, jitter), j = 0..n-1, wrapped.

    Default jitter 1/(4n): the scale of eq:jittered_nodes, centred on the
    equispaced grid as in the large-scale workload."""
    if jitter is None:
        jitter = 1.0 / (4.0 * n)
    base = (np.arange(n, dtype=np.float64) - n / 2.0) / n
    return wrap_half(base + uniform(seed, n, -jitter, jitter))


def iid_uniform(seed, n):
    return wrap_half(uniform(seed, n, -0.5, 0.5))


def chebyshev_jittered(seed, n, rel_jitter=1e-3):
    """x_j = cos(pi (j - 1/2)/n)/2 + U(-rel_jitter/n, rel_jitter/n), j = 1..n, wrapped."""
    j = np.arange(1, n + 1, dtype=np.float64)
    base = 0.5 * np.cos(np.pi * (j - 0.5) / n)
    return wrap_half(base + uniform(seed, n, -rel_jitter / n, rel_jitter / n))
