"""The modified adjoint NFFT and its adjoint (Sec. 3.2.2 eq:approx_ansatz2,
Remark remark:ansatz2_adj), the Frobenius objective (eq:matrixnorm_opt_ansatz2)
and the error measures (eq:errors_per_node_lagrange)."""
import numpy as np

from .nfft import matrix_A, nfft_direct
from .kernel import diag_D
from .bopt import BOpt, bopt_closed, bopt_naive, matrix_F


def spread(B: BOpt, f):
    """g~ = B_opt^* f, g~_l = sum_{j in I(l)} b_{l,j} f_j  (B real, Sec. 3.2.2)."""
    f = np.asarray(f, dtype=np.complex128)
    g = np.zeros(B.Ms, dtype=np.complex128)
    col = np.repeat(np.arange(B.Ms), np.diff(B.ptr))
    np.add.at(g, col, B.b * f[B.idx])
    return g


def interpolate(B: BOpt, g):
    """f_j = sum_{l in I(x_j)} b_{l,j} g_l  (B_opt applied to a grid vector)."""
    g = np.asarray(g, dtype=np.complex128)
    f = np.zeros(B.N, dtype=np.complex128)
    col = np.repeat(np.arange(B.Ms), np.diff(B.ptr))
    np.add.at(f, B.idx, B.b * g[col])
    return f


def F_adjoint(g, M, Ms, method="fft"):
    """h_k = sum_{l=-M_sigma/2}^{M_sigma/2-1} g_l exp(-2 pi i k l / M_sigma), k = -M/2 .. M/2-1 (F^*, eq:matrix_F).

    "direct" multiplies by the explicit matrix F^*; "fft" uses numpy's FFT over
    p = l + M_sigma/2, where exp(-2 pi i k l/M_sigma) = (-1)^k exp(-2 pi i k p/M_sigma)."""
    g = np.asarray(g, dtype=np.complex128)
    if method == "direct":
        return matrix_F(M, Ms).conj().T @ g
    k = np.arange(-(M // 2), M // 2)
    G = np.fft.fft(g)
    return np.where(k % 2 == 0, 1.0, -1.0) * G[k % Ms]


def F_apply(c, M, Ms, method="fft"):
    """g_l = sum_k c_k exp(2 pi i k l / M_sigma), l = -M_sigma/2 .. M_sigma/2-1 (F, eq:matrix_F)."""
    c = np.asarray(c, dtype=np.complex128)
    if method == "direct":
        return matrix_F(M, Ms) @ c
    k = np.arange(-(M // 2), M // 2)
    C = np.zeros(Ms, dtype=np.complex128)
    C[k % Ms] = np.where(k % 2 == 0, 1.0, -1.0) * c
    return np.fft.ifft(C) * Ms


def infft_apply(B: BOpt, f, method="fft"):
    """fhat ~ h~ = D^* F^* B_opt^* f  (eq:approx_ansatz2); D is real for the Dirichlet choice."""
    d = diag_D(B.M, B.Ms, B.kernel)
    return np.conj(d) * F_adjoint(spread(B, f), B.M, B.Ms, method)


def nfft_apply(B: BOpt, fhat, method="fft"):
    """f ~ B_opt F D fhat, the exact adjoint of infft_apply (Remark remark:ansatz2_adj)."""
    d = diag_D(B.M, B.Ms, B.kernel)
    return interpolate(B, F_apply(d * np.asarray(fhat, np.complex128), B.M, B.Ms, method))


def infft(x, f, M, sigma=2.0, m=4, kernel="full", tau=1e-12, tier="closed"):
    """Precompute B_opt (Sec. 3.2.2) and return (fhat_check, B_opt)."""
    B = (bopt_closed if tier == "closed" else bopt_naive)(x, M, sigma, m, kernel, tau)
    return infft_apply(B, f, "fft" if tier == "closed" else "direct"), B


def frobenius_objective(B: BOpt):
    """||F D A^* B_opt - I_{M_sigma}||_F^2 = sum_l ||L_l b_l - e_l||^2 (separable form, Sec. 3.2.2)."""
    return float(np.sum(B.J))


def frobenius_objective_dense(x, Bdense, M, Ms, kernel):
    """||F D A^* B - I_{M_sigma}||_F^2 from the explicit matrices (eq:matrixnorm_opt_ansatz2 squared)."""
    A = matrix_A(x, M)
    K_star = matrix_F(M, Ms) @ (diag_D(M, Ms, kernel)[:, None] * A.conj().T)
    return float(np.linalg.norm(K_star @ Bdense - np.eye(Ms)) ** 2)


def errors_per_node(fhat, fcheck, N):
    """e_r^abs/N and e_r^rel/N for r in {2, inf} (eq:errors_per_node_lagrange)."""
    out = {}
    for r, ordr in (("2", 2), ("inf", np.inf)):
        e = np.linalg.norm(np.asarray(fhat) - np.asarray(fcheck), ordr)
        out["abs_" + r] = e / N
        out["rel_" + r] = e / (N * np.linalg.norm(fhat, ordr))
    return out


def rel_l2(a, b):
    """||a - b||_2 / ||b||_2."""
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def refine(B: BOpt, x, f, fhat, sweeps=1):
    """Residual correction of an inverse-NFFT estimate, `sweeps` times:

        fhat <- fhat + D^* F^* B_opt^* (f - A fhat),   A fhat by its direct sum (eq:nfft).

    The modified adjoint NFFT (eq:approx_ansatz2) serves as an approximate left inverse of A
    in a Richardson iteration for A fhat = f (eq:problem_infft; Sec. 1 surveys iterative
    solvers of this system).  For data f = A fhat_true each sweep maps the error e to
    (I - D^* F^* B_opt^* A) e."""
    f = np.asarray(f, np.complex128)
    fhat = np.asarray(fhat, np.complex128).copy()
    for _ in range(sweeps):
        fhat = fhat + infft_apply(B, f - nfft_direct(x, fhat))
    return fhat
