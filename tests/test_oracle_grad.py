"""Pins for oracle.grad: the kernel derivative and the gradients of the reconstruction loss."""
import numpy as np
import pytest

from oracle import grad, kernel, bopt, infft
from workloads import make_problem, uniform, complex_normal


@pytest.mark.parametrize("M,Ms", [(64, 128), (256, 512), (1000, 2000)])
@pytest.mark.parametrize("kind", ["full", "sym"])
def test_kappa_prime_equals_derivative_of_sum(M, Ms, kind):
    """Closed form and small-t series against d/dt of the defining sum, term by term."""
    t = np.concatenate([uniform(M, 100, -0.5, 0.5), uniform(M + 1, 50, -0.2 / M, 0.2 / M),
                        uniform(M + 2, 20, -1e-7, 1e-7), [0.1 / M, -0.1 / M, 0.0]])
    want = grad.kappa_prime_sum(t, M, Ms, kind)
    got = grad.kappa_prime(t, M, Ms, kind)
    scale = np.pi * M * M / Ms
    np.testing.assert_allclose(got, want, atol=1e-12 * scale)


def test_kappa_prime_matches_finite_difference_of_kappa():
    M, Ms = 128, 256
    t = uniform(9, 200, -0.45, 0.45)
    h = 1e-7
    fd = (kernel.re_kappa_closed(t + h, M, Ms, "full") - kernel.re_kappa_closed(t - h, M, Ms, "full")) / (2 * h)
    np.testing.assert_allclose(grad.kappa_prime(t, M, Ms, "full"), fd, atol=1e-6 * np.pi * M * M / Ms)


def test_grad_f_is_exact_for_the_quadratic_loss():
    """L is quadratic in f: central differences on Re f_j and Im f_j are exact up to rounding."""
    p = make_problem(5, M=32, N=128, m=3)
    L, B = grad.loss(p.x, p.f, p.fhat, p.M, 2.0, 3)
    w = 2 * (infft.infft_apply(B, p.f) - p.fhat)
    g = grad.grad_f(B, w)
    h = 1e-4
    for j in (0, 17, 90):
        for unit in (1.0, 1j):
            fp, fm = p.f.copy(), p.f.copy()
            fp[j] += h * unit
            fm[j] -= h * unit
            r1 = infft.infft_apply(B, fp) - p.fhat
            r2 = infft.infft_apply(B, fm) - p.fhat
            fd = (np.vdot(r1, r1).real - np.vdot(r2, r2).real) / (2 * h)
            want = g[j].real if unit == 1.0 else g[j].imag
            assert abs(fd - want) <= 1e-7 * (abs(want) + 1.0)


def test_fd_helper_equals_full_recomputation():
    """The incremental central difference equals recomputing the whole loss at x +- h."""
    p = make_problem(5, M=32, N=96, m=3)
    L, B = grad.loss(p.x, p.f, p.fhat, p.M, 2.0, 3)
    nodes = grad.safe_nodes(B, p.x, 1e-5, 4)
    h = 1e-5
    inc = grad.fd_grad_x(B, p.x, p.f, p.fhat, nodes, h)
    full = []
    for j in nodes:
        xp, xm = p.x.copy(), p.x.copy()
        xp[j] += h
        xm[j] -= h
        full.append((grad.loss(xp, p.f, p.fhat, p.M, 2.0, 3)[0] - grad.loss(xm, p.f, p.fhat, p.M, 2.0, 3)[0]) / (2 * h))
    np.testing.assert_allclose(inc, full, rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("kind", ["full", "sym"])
def test_grad_x_matches_finite_differences(kind):
    """Implicit differentiation against Richardson-extrapolated central differences; the
    loss is smooth in x only on small scales (the regularised solves are ill-conditioned),
    so the steps are 1e-7 and 5e-8 here."""
    p = make_problem(5, M=256, N=1024, m=4)
    B = bopt.bopt_closed(p.x, p.M, 2.0, 4, kind)
    w = 2 * (infft.infft_apply(B, p.f) - p.fhat)
    g = grad.grad_x(B, p.x, p.f, w)
    nodes = grad.safe_nodes(B, p.x, 1e-7, 12, seed=1)
    d1 = grad.fd_grad_x(B, p.x, p.f, p.fhat, nodes, 1e-7)
    d2 = grad.fd_grad_x(B, p.x, p.f, p.fhat, nodes, 5e-8)
    rich = d2 + (d2 - d1) / 3
    assert np.linalg.norm(rich - g[nodes]) <= 2e-3 * np.linalg.norm(rich)


def test_grad_x_zero_when_loss_is_zero():
    """w = 0 (loss at a stationary point) gives a zero node gradient."""
    p = make_problem(5, M=32, N=128, m=3)
    B = bopt.bopt_closed(p.x, p.M, 2.0, 3)
    assert np.all(grad.grad_x(B, p.x, p.f, np.zeros(p.M)) == 0.0)
