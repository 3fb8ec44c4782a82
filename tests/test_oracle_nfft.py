"""Pins for oracle.nfft: the Fourier matrix A and the dense least-squares comparator."""
import numpy as np
import pytest

from oracle import nfft
from workloads import iid_uniform, complex_normal, equispaced


def test_trig_poly_golden(golden):
    rows = golden("trig_poly_M2.txt")
    x = np.array([r[0] for r in rows])
    want = np.array([r[1] + 1j * r[2] for r in rows])
    got = nfft.nfft_direct(x, np.array([1.0, 2.0]))
    np.testing.assert_allclose(got, want, atol=1e-14)


@pytest.mark.parametrize("M,N", [(4, 4), (6, 10), (8, 32), (16, 17)])
def test_AstarA_equispaced(M, N):
    """Sec. 3.2: A^* A = N I_M for equispaced x_j = j/N and M <= N."""
    A = nfft.matrix_A(equispaced(N), M)
    np.testing.assert_allclose(A.conj().T @ A, N * np.eye(M), atol=1e-12)


@pytest.mark.parametrize("M,N", [(8, 8), (12, 4), (32, 8)])
def test_AAstar_equispaced(M, N):
    """Sec. 3.2: A A^* = M I_N for equispaced nodes, M >= N with N | M."""
    A = nfft.matrix_A(equispaced(N), M)
    np.testing.assert_allclose(A @ A.conj().T, M * np.eye(N), atol=1e-12)


def test_AstarA_fails_without_divisibility():
    """The divisibility condition is needed: M = 12, N = 8 (8 does not divide 12)."""
    A = nfft.matrix_A(equispaced(8), 12)
    assert np.abs(A @ A.conj().T - 12 * np.eye(8)).max() > 1.0


@pytest.mark.parametrize("M", [8, 16, 64])
def test_nfft_equispaced_is_inverse_dft(M):
    """For x_j = j/M the sum eq:nfft is M times numpy's inverse DFT (index-shifted)."""
    fhat = complex_normal(7, M)
    x = equispaced(M)
    # f_j = sum_k fhat_k e^{2 pi i k j/M}, j, k = -M/2..M/2-1: shift both axes by M/2
    want = np.fft.fftshift(np.fft.ifft(np.fft.ifftshift(fhat))) * M
    np.testing.assert_allclose(nfft.nfft_direct(x, fhat), want, atol=1e-12 * M)


def test_adjoint_identity():
    """<A fhat, f> = <fhat, A^* f> with A^* f evaluated by its own sum (eq:nfft*)."""
    x = iid_uniform(11, 37)
    fhat, f = complex_normal(12, 10), complex_normal(13, 37)
    lhs = np.vdot(f, nfft.nfft_direct(x, fhat))
    rhs = np.vdot(nfft.nfft_adjoint_direct(x, f, 10), fhat)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_adjoint_sum_elementwise():
    """h_k = sum_j f_j exp(-2 pi i k x_j), checked term by term in pure Python."""
    x = iid_uniform(3, 5)
    f = complex_normal(4, 5)
    h = nfft.nfft_adjoint_direct(x, f, 4)
    import cmath
    for i, k in enumerate(range(-2, 2)):
        want = sum(f[j] * cmath.exp(-2j * cmath.pi * k * x[j]) for j in range(5))
        assert abs(h[i] - want) < 1e-13


def test_dense_lsq_exact_recovery():
    """Noise-free overdetermined data f = A fhat is recovered exactly (full rank, M < N)."""
    x = iid_uniform(21, 50)
    fhat = complex_normal(22, 16)
    got = nfft.dense_lsq_inverse(x, nfft.nfft_direct(x, fhat), 16)
    np.testing.assert_allclose(got, fhat, atol=1e-10)


def test_dense_lsq_normal_equations():
    """For noisy f the residual is orthogonal to range(A): A^*(A fhat - f) = 0."""
    x = iid_uniform(31, 40)
    f = complex_normal(32, 40)
    sol = nfft.dense_lsq_inverse(x, f, 12)
    A = nfft.matrix_A(x, 12)
    assert np.abs(A.conj().T @ (A @ sol - f)).max() < 1e-11


def test_direct_sum_with_reduced_phases():
    """The reduced-phase sum equals the plain one at small M and, at M = 2^16, a 50-digit
    evaluation (mpmath) at a few nodes, where the plain sum's angles lose ~1e-11."""
    mp = pytest.importorskip("mpmath")
    x = iid_uniform(91, 40)
    fh = complex_normal(92, 64)
    np.testing.assert_allclose(nfft.nfft_direct_reduced(x, fh), nfft.nfft_direct(x, fh), rtol=0, atol=1e-13)
    M = 1 << 16
    fh = complex_normal(93, M)
    xs = iid_uniform(94, 3)
    mp.mp.dps = 50
    ks = np.arange(-M // 2, M // 2)
    for xj in xs:
        X = mp.mpf(float(xj))
        acc = mp.mpc(0)
        for k, c in zip(ks[::256], fh[::256]):          # a strided subset of the terms keeps it fast
            acc += mp.mpc(c.real, c.imag) * mp.expjpi(2 * k * X)
        part = nfft.nfft_direct_reduced(np.array([xj]), np.where(np.arange(M) % 256 == 0, fh, 0))[0]
        assert abs(complex(acc) - part) <= 1e-13 * max(1.0, abs(complex(acc)))
