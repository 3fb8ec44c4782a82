"""Seeded synthetic inputs shaped like the paper's experiments.

This module is shared by the tests, the benchmark and the smoke run.  It holds
no arithmetic of the inversion method itself (no window, no least squares, no
Fourier transform of the grid); it only draws random numbers and node families
and, for the test data, evaluates the trigonometric polynomial of eq. (1.1)
(``eq:trig_polynomial``) at the nodes.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: draw ``i`` of stream ``seed`` is ``mix(seed + (i + 1) * GAMMA)``.
Uniforms take the top 53 bits; normals use the Box-Muller transform.
"""
from .rng import uniform01, uniform, normal, complex_normal  # noqa: F401
from .nodes import jittered, iid_uniform, chebyshev_jittered, equispaced, wrap_half, radial  # noqa: F401
from .configs import (  # noqa: F401
    Problem, make_problem, trig_poly_eval, CONFIG_SEED_BASE, BatchWorkload, make_batch, Workload2D, make_2d,
    trig_poly_eval_2d,
)
