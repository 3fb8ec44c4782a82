"""Nonequispaced Fourier matrix and direct sums (Sec. 1-2, eq:matrix_A, eq:nfft, eq:nfft*)."""
import numpy as np


def freqs(M):
    """k = -M/2 .. M/2-1 (M even, eq:trig_polynomial)."""
    return np.arange(-(M // 2), M // 2)


def matrix_A(x, M):
    """A = (exp(2 pi i k x_j))_{j, k}  in C^{N x M}  (eq:matrix_A)."""
    return np.exp(2j * np.pi * np.outer(np.asarray(x, np.float64), freqs(M)))


def nfft_direct(x, fhat):
    """f_j = sum_k fhat_k exp(2 pi i k x_j)  (eq:nfft), O(NM)."""
    return matrix_A(x, len(fhat)) @ np.asarray(fhat, np.complex128)


def nfft_adjoint_direct(x, f, M):
    """h_k = sum_j f_j exp(-2 pi i k x_j)  (eq:nfft*), O(NM)."""
    return matrix_A(x, M).conj().T @ np.asarray(f, np.complex128)


def dense_lsq_inverse(x, f, M):
    """Least-squares solution of A fhat = f (eq:problem_infft) by LAPACK's
    SVD-based solver: the exact comparator for small overdetermined problems."""
    sol, *_ = np.linalg.lstsq(matrix_A(x, M), np.asarray(f, np.complex128), rcond=None)
    return sol


def nfft_direct_reduced(x, fhat):
    """f_j = sum_k fhat_k exp(2 pi i k x_j) (eq:nfft) with every phase k x_j reduced modulo 1
    exactly before the exponential, so that large M loses no accuracy in the angle: x is split
    as x_hi + x_lo with x_hi of 26 significant bits (Veltkamp's splitting), k x_hi is then exact
    in fp64 for |k| < 2^26 and its integer part is removed exactly; k x_lo (below 2^-10) is
    added afterwards."""
    x = np.asarray(x, np.float64)
    fhat = np.asarray(fhat, np.complex128)
    k = freqs(len(fhat)).astype(np.float64)
    t = 134217729.0 * x                      # 2^27 + 1
    x_hi = t - (t - x)
    x_lo = x - x_hi
    out = np.empty(len(x), np.complex128)
    for s in range(0, len(x), 64):
        a = np.multiply.outer(x_hi[s:s + 64], k)
        a -= np.round(a)
        a += np.multiply.outer(x_lo[s:s + 64], k)
        out[s:s + 64] = np.exp(2j * np.pi * a) @ fhat
    return out
