"""The synthetic workloads (sizes, node families, data) and the test-data generator.

Seeds: stream ``CONFIG_SEED_BASE + c`` for workload ``c``; sub-streams are
derived by adding fixed offsets (nodes, coefficients, noise).
"""
from dataclasses import dataclass
import numpy as np

from .rng import complex_normal, uniform
from .nodes import iid_uniform, jittered, chebyshev_jittered, radial

CONFIG_SEED_BASE = 1811053350
_NODES, _COEF, _NOISE = 1, 2, 3


def trig_poly_eval(x, fhat, block=256):
    """f_j = sum_{k=-M/2}^{M/2-1} fhat_k exp(2 pi i k x_j)  (eq:trig_polynomial).

    Evaluated in fp64 with the frequency split k = -M/2 + block*q + r so the sum
    becomes one complex matrix product; every exponential is formed directly
    from its own argument, reduced modulo 1 without loss: x is split as
    x_hi + x_lo with x_hi of 26 significant bits (Veltkamp's splitting), so that
    x_hi * K is exact for every integer |K| < 2^26 and its integer part is removed
    exactly, and the small x_lo * K is added afterwards.  Accuracy is ~1e-15
    relative at M = 2^16 (an unsplit product x * K loses ~1e-12 of the angle).
    This is input generation, not part of the inversion method."""
    x = np.asarray(x, dtype=np.float64)
    fhat = np.asarray(fhat, dtype=np.complex128)
    M = fhat.shape[0]
    if M % block != 0:
        block = M
    Q = M // block
    r = np.arange(block, dtype=np.float64)
    q = np.arange(Q, dtype=np.float64)
    t = 134217729.0 * x                     # 2^27 + 1
    x_hi = t - (t - x)
    x_lo = x - x_hi
    out = np.empty(x.shape[0], dtype=np.complex128)
    F = fhat.reshape(Q, block)              # F[q, r] = fhat at k = -M/2 + block q + r

    def phase(s, K):
        a = np.outer(x_hi[s:s + 8192], K)
        a -= np.round(a)
        a += np.outer(x_lo[s:s + 8192], K)
        return np.exp(2j * np.pi * a)

    for s in range(0, x.shape[0], 8192):
        E1 = phase(s, r)                                # (n, block)
        E2 = phase(s, block * q - M / 2)                # (n, Q)
        T = E1 @ F.T                                    # (n, Q): sum over r
        out[s:s + 8192] = np.sum(E2 * T, axis=1)
    return out


@dataclass
class Problem:
    name: str
    M: int
    N: int
    sigma: float
    m: int
    x: np.ndarray
    fhat: np.ndarray
    f: np.ndarray


def make_problem(config, m=None, M=None, N=None, with_data=True, noise_rel=None, seed=None):
    """Workload ``config`` in {1, 2, 5} (1-D single-problem forms).

    1: M=64, N=128, i.i.d. uniform nodes, exact data, sigma=2, m=4.
    2: M=2^16, N=2^18 jittered nodes, data plus 1e-8 relative complex noise, sigma=2, m in {4,6,8}.
    5: M=2^14, N=2^16 i.i.d. uniform nodes, exact data, sigma=2, m=4.
    M, N override the sizes (same recipe, smaller problem for fast tests)."""
    seed = CONFIG_SEED_BASE + config if seed is None else seed
    if config == 1:
        M = M or 64; N = N or 128; m = m or 4
        x = iid_uniform(seed * 16 + _NODES, N)
        noise_rel = 0.0 if noise_rel is None else noise_rel
    elif config == 2:
        M = M or 2 ** 16; N = N or 2 ** 18; m = m or 4
        x = jittered(seed * 16 + _NODES, N)
        noise_rel = 1e-8 if noise_rel is None else noise_rel
    elif config == 5:
        M = M or 2 ** 14; N = N or 2 ** 16; m = m or 4
        x = iid_uniform(seed * 16 + _NODES, N)
        noise_rel = 0.0 if noise_rel is None else noise_rel
    elif config == "cheb":
        M = M or 1024; N = N or 3 * 1024; m = m or 6
        x = chebyshev_jittered(seed * 16 + _NODES, N)
        noise_rel = 0.0 if noise_rel is None else noise_rel
    else:
        raise ValueError(f"unknown workload {config!r}")
    fhat = complex_normal(seed * 16 + _COEF, M)
    f = None
    if with_data:
        f = trig_poly_eval(x, fhat)
        if noise_rel:
            eta = complex_normal(seed * 16 + _NOISE, N)
            eta *= noise_rel * np.linalg.norm(f) / np.linalg.norm(eta)
            f = f + eta
    return Problem(f"config{config}", M, N, 2.0, m, x, fhat, f)


@dataclass
class BatchWorkload:
    name: str
    M: np.ndarray        # (P,) even coefficient counts
    N: np.ndarray        # (P,) node counts
    m: int
    x: list              # P node arrays
    seed: int

    @property
    def x_all(self):
        return np.concatenate(self.x)


_SIZES, _RATIOS = 4, 5


def make_batch(P=4096, seed=None, M_range=(256, 8192), r_range=(2.0, 4.0), m=6, nodes="chebyshev"):
    """Workload 3: P independent problems.

    M_p = 2 round(exp(U(ln(M_lo/2), ln(M_hi/2)))) (even, log-uniform in M_range),
    N_p = round(r_p M_p) with r_p ~ U(r_range), and per problem the Chebyshev-
    clustered nodes x_j = cos(pi (j - 1/2)/N_p)/2 + U(-1e-3/N_p, 1e-3/N_p), wrapped
    ("jittered" and "uniform" give the other node families).  sigma = 2, m = 6."""
    seed = CONFIG_SEED_BASE + 3 if seed is None else seed
    lo, hi = np.log(M_range[0] / 2.0), np.log(M_range[1] / 2.0)
    M = 2 * np.round(np.exp(uniform(seed * 16 + _SIZES, P, lo, hi))).astype(np.int64)
    r = uniform(seed * 16 + _RATIOS, P, r_range[0], r_range[1])
    N = np.maximum(np.round(r * M).astype(np.int64), 1)
    xs = []
    for p in range(P):
        s = seed * 16 * 65536 + 16 * p + _NODES
        if nodes == "chebyshev":
            xs.append(chebyshev_jittered(s, int(N[p])))
        elif nodes == "jittered":
            xs.append(jittered(s, int(N[p])))
        else:
            xs.append(iid_uniform(s, int(N[p])))
    return BatchWorkload("config3", M, N, m, xs, seed)


def trig_poly_eval_2d(x, fhat):
    """f_j = sum_{k1, k2} fhat[k1, k2] exp(2 pi i (k1 x_j1 + k2 x_j2)), k_t = -M_t/2 .. M_t/2-1
    (eq:trig_polynomial on the 2-D torus), in fp64.  The sum over k2 is one complex
    matrix product per block of nodes; every exponential is formed from its own
    argument reduced modulo 1.  Input generation, not part of the inversion method."""
    x = np.asarray(x, dtype=np.float64)
    fhat = np.asarray(fhat, dtype=np.complex128)
    M1, M2 = fhat.shape
    k1 = np.arange(-(M1 // 2), M1 // 2, dtype=np.float64)
    k2 = np.arange(-(M2 // 2), M2 // 2, dtype=np.float64)
    out = np.empty(x.shape[0], dtype=np.complex128)
    for s in range(0, x.shape[0], 8192):
        xs = x[s:s + 8192]
        a1 = np.outer(xs[:, 0], k1)
        a1 -= np.round(a1)
        a2 = np.outer(xs[:, 1], k2)
        a2 -= np.round(a2)
        T = np.exp(2j * np.pi * a2) @ fhat.T            # (n, M1): sum over k2
        out[s:s + 8192] = np.sum(np.exp(2j * np.pi * a1) * T, axis=1)
    return out


@dataclass
class Workload2D:
    name: str
    M1: int
    M2: int
    m: int
    x: np.ndarray        # (N, 2) nodes in [-1/2, 1/2)^2
    seed: int

    @property
    def N(self):
        return self.x.shape[0]


def make_2d(spokes=512, samples=512, M=(256, 256), m=4, jitter=1e-4, seed=None):
    """Workload 4: the 2-D tensor-product form on a radial trajectory: spokes at
    angles pi s / spokes, equispaced radii -1/2 + i / samples, U(-jitter, jitter)
    per coordinate; M = M1 x M2 coefficients, sigma = 2 per dimension, m = 4."""
    seed = CONFIG_SEED_BASE + 4 if seed is None else seed
    x = radial(seed * 16 + _NODES, spokes, samples, jitter)
    return Workload2D("config4", int(M[0]), int(M[1]), m, x, seed)
