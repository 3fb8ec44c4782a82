"""Pins for oracle.kernel: the Dirichlet choice of Remark remark:Dirichlet_ansatz2."""
import numpy as np
import pytest

from oracle import kernel
from workloads import uniform


def test_golden_values(golden):
    for M, t, full, sym in golden("dirichlet_values.txt"):
        M = int(M)
        # M_sigma = 1 makes kappa the bare exponential sum
        assert abs(kernel.re_kappa_closed(t, M, 1, "full") - full) < 1e-12
        assert abs(kernel.re_kappa_closed(t, M, 1, "sym") - sym) < 1e-12
        assert abs(kernel.kappa_sum(t, M, 1, "full").real - full) < 1e-12
        assert abs(kernel.kappa_sum(t, M, 1, "sym").real - sym) < 1e-12


@pytest.mark.parametrize("M,Ms", [(4, 8), (16, 32), (64, 128), (10, 15), (256, 256)])
@pytest.mark.parametrize("kind", ["full", "sym"])
def test_closed_form_equals_sum(M, Ms, kind):
    t = np.concatenate([uniform(M, 200, -1.0, 1.0), uniform(M + 1, 50, -1e-6, 1e-6), [0.0, 0.5, -0.5]])
    want = kernel.kappa_sum(t, M, Ms, kind).real
    got = kernel.re_kappa_closed(t, M, Ms, kind)
    np.testing.assert_allclose(got, want, atol=1e-13 * M / Ms + 1e-15)


def test_sym_is_the_real_dirichlet_kernel():
    """The sym sum is real: D_{M/2-1}(t) = sin((M-1) pi t)/sin(pi t) (eq:kernel_Dirichlet)."""
    t = uniform(3, 100, -0.5, 0.5)
    k = kernel.kappa_sum(t, 12, 1, "sym")
    assert np.abs(k.imag).max() < 1e-12
    np.testing.assert_allclose(k.real, np.sin(11 * np.pi * t) / np.sin(np.pi * t), rtol=1e-12, atol=1e-12)


def test_full_minus_sym_identity():
    """cos(x) sin(Mx)/sin(x) = sin((M-1)x)/sin(x) + cos(Mx): full = sym + the k = -M/2 term."""
    M, Ms = 20, 40
    t = uniform(5, 100, -0.5, 0.5)
    lhs = kernel.re_kappa_closed(t, M, Ms, "full")
    rhs = kernel.re_kappa_closed(t, M, Ms, "sym") + np.cos(np.pi * M * t) / Ms
    np.testing.assert_allclose(lhs, rhs, atol=1e-14)


def test_periodic_and_even():
    M, Ms = 16, 32
    t = uniform(8, 100, -0.5, 0.5)
    for kind in ("full", "sym"):
        a = kernel.re_kappa_closed(t, M, Ms, kind)
        np.testing.assert_allclose(kernel.re_kappa_closed(t + 1.0, M, Ms, kind), a, atol=1e-13)
        np.testing.assert_allclose(kernel.re_kappa_closed(-t, M, Ms, kind), a, atol=1e-13)


def test_diag_D_and_gram_diag():
    assert np.all(kernel.diag_D(8, 16, "full") == 1 / 16)
    d = kernel.diag_D(8, 16, "sym")
    assert d[0] == 0 and np.all(d[1:] == 1 / 16)
    assert kernel.gram_diag(8, 16, "full") == 0.5
    assert kernel.gram_diag(8, 16, "sym") == 7 / 16


def test_torus_diff_exact_rational():
    """torus_diff returns the representative in [-1/2, 1/2] of a - b mod 1, correctly
    rounded (checked in exact rational arithmetic), including pairs straddling the seam."""
    from fractions import Fraction
    rng = np.random.default_rng(3)
    a = np.concatenate([uniform(1, 300, -0.5, 0.5), 0.5 - rng.uniform(0, 1e-4, 100), [np.nextafter(0.5, 0)]])
    b = np.concatenate([uniform(2, 300, -0.5, 0.5), -0.5 + rng.uniform(0, 1e-4, 100), [-0.5]])
    for ai, bi in [(a, b), (b, a)]:
        d = kernel.torus_diff(ai, bi)
        for x, y, got in zip(ai, bi, d):
            ex = Fraction(float(x)) - Fraction(float(y))
            while ex > Fraction(1, 2):
                ex -= 1
            while ex < Fraction(-1, 2):
                ex += 1
            assert float(ex) == got, (x, y)


def test_torus_diff_seam_precision():
    """Nodes 2e-7 apart across the seam: torus_diff keeps full relative precision,
    where subtracting first and wrapping afterwards is off by ~1e-17 (1e-11 relative)."""
    from fractions import Fraction
    a, b = 0.4999999123456789, -0.4999998765432101
    exact = Fraction(a) - Fraction(b) - 1
    assert abs(Fraction(float(kernel.torus_diff(a, b))) - exact) < Fraction(1, 10 ** 21)
    assert abs(Fraction(float(kernel.torus_diff(b, a))) + exact) < Fraction(1, 10 ** 21)
    naive = (a - b) - 1.0
    assert abs(Fraction(naive) - exact) > Fraction(1, 10 ** 18)
