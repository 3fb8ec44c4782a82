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


def radial(seed, spokes, samples, jitter=1e-4):
    """Radial trajectory in [-1/2, 1/2)^2 (the 2-D workload): spoke s at angle
    theta_s = pi s / spokes (s = 0 .. spokes-1), samples at radii
    r_i = -1/2 + i / samples (i = 0 .. samples-1), each coordinate perturbed by
    U(-jitter, jitter) and wrapped.  Node j = s * samples + i; returns (N, 2)."""
    s = np.arange(spokes, dtype=np.float64)
    r = -0.5 + np.arange(samples, dtype=np.float64) / samples
    th = np.pi * s / spokes
    n = spokes * samples
    x = np.empty((n, 2))
    x[:, 0] = (np.cos(th)[:, None] * r[None, :]).ravel()
    x[:, 1] = (np.sin(th)[:, None] * r[None, :]).ravel()
    jit = uniform(seed, 2 * n, -jitter, jitter).reshape(n, 2)
    return wrap_half(x + jit).reshape(n, 2)
