"""Optimisation of the sparse matrix B, overdetermined case (Sec. 3.2.2).

The Frobenius problem eq:opt_ansatz2, min ||K^* B - I_{M_sigma}||_F^2 over
(2m+1)-sparse real B, splits into one problem per grid point l:

    min_{b real}  ||L_l b - e_l||_2^2,   L_l = F D H_l  (eq:matrix_Ll),

whose full-rank solution is eq:solution_ansatz2.  Readings (the paper assumes
full rank and prints the complex formula): b is real, so the normal equations
are Re(G_l) b = Re(r_l) with G_l = L_l^* L_l and r_l = L_l^* e_l; rank
deficiency is handled by Tikhonov regularisation with
mu = tau * (diagonal of Re G_l) (tau = 1e-12 by default):

    b_l = argmin ||L_l b - e_l||^2 + mu ||b||^2.

Two tiers compute the same b_l:

* ``bopt_naive``  forms L_l = F D H_l explicitly (M_sigma x |I(l)|) and solves
  the stacked real least-squares problem [Re L; Im L; sqrt(mu) I] b = [e_l; 0; 0]
  with LAPACK (SVD based).  O(M_sigma M |I(l)|) per column: small sizes only.
* ``bopt_closed`` uses F^* F = M_sigma I_M (|k - k'| < M <= M_sigma), so
  G_l = M_sigma H_l^* D^* D H_l, whose real part has the closed form
  Re G_{jj'} = Re kappa(x_j - x_j'), and Re r_j = Re kappa(l/M_sigma - x_j)
  (oracle.kernel, differences taken on the torus by torus_diff); then
  (Re G_l + mu I) b = Re r_l by LAPACK LU.

Both return the column structure (ptr, idx): I(l) = idx[ptr[p]:ptr[p+1]] with
p = l + M_sigma/2, the coefficients b (aligned with idx) and the column
objectives J_l = ||L_l b_l - e_l||^2 (without the mu term).
"""
from dataclasses import dataclass
import numpy as np

from .nfft import freqs
from .pattern import index_sets_l, index_sets_l_fast
from .kernel import diag_D, re_kappa_closed, gram_diag, torus_diff

TAU_DEFAULT = 1e-12


@dataclass
class BOpt:
    M: int
    Ms: int
    N: int
    m: int
    kernel: str
    tau: float
    ptr: np.ndarray      # (Ms+1,) column pointers, column p <-> l = p - Ms/2
    idx: np.ndarray      # (nnz,) node index j of each stored entry
    b: np.ndarray        # (nnz,) real coefficients of B_opt
    J: np.ndarray        # (Ms,) column objectives ||L_l b_l - e_l||^2

    def dense(self):
        """B_opt as a dense real N x M_sigma matrix (eq:matrix_B layout)."""
        B = np.zeros((self.N, self.Ms))
        for p in range(self.Ms):
            s, e = self.ptr[p], self.ptr[p + 1]
            B[self.idx[s:e], p] = self.b[s:e]
        return B


def oversampled_size(M, sigma):
    """M_sigma = sigma M, required to be an even integer (grid l = -M_sigma/2 .. M_sigma/2-1)."""
    Ms = sigma * M
    if Ms != int(round(Ms)) or int(round(Ms)) % 2:
        raise ValueError("sigma * M must be an even integer")
    return int(round(Ms))


def matrix_F(M, Ms):
    """F = (exp(2 pi i k s / M_sigma))_{s, k}, s = -M_sigma/2 .. M_sigma/2-1 (eq:matrix_F)."""
    s = np.arange(-(Ms // 2), Ms // 2)
    return np.exp(2j * np.pi * np.outer(s, freqs(M)) / Ms)


def matrix_H(xI, M):
    """H_l = (exp(-2 pi i k x_j))_{k, j in I(l)} (Sec. 3.2.2)."""
    return np.exp(-2j * np.pi * np.outer(freqs(M), xI))


def matrix_L(xI, M, Ms, kernel):
    """L_l = F D H_l  (eq:matrix_Ll), formed explicitly."""
    return matrix_F(M, Ms) @ (diag_D(M, Ms, kernel)[:, None] * matrix_H(xI, M))


def solve_column_naive(L, p, mu):
    """argmin over real b of ||L b - e_p||^2 + mu ||b||^2 via the stacked real system."""
    Ms, n = L.shape
    e = np.zeros(Ms)
    e[p] = 1.0
    A = np.vstack([L.real, L.imag, np.sqrt(mu) * np.eye(n)])
    rhs = np.concatenate([e, np.zeros(Ms), np.zeros(n)])
    b, *_ = np.linalg.lstsq(A, rhs, rcond=None)
    J = np.linalg.norm(L @ b - e) ** 2
    return b, J


def bopt_naive(x, M, sigma, m, kernel="full", tau=TAU_DEFAULT):
    Ms = oversampled_size(M, sigma)
    x = np.asarray(x, dtype=np.float64)
    cols = index_sets_l(x, Ms, m)
    mu = tau * gram_diag(M, Ms, kernel)
    ptr = np.zeros(Ms + 1, dtype=np.int64)
    idx, bs, J = [], [], np.ones(Ms)
    for p, I in enumerate(cols):
        ptr[p + 1] = ptr[p] + len(I)
        if len(I) == 0:
            continue                     # empty column: b_l empty, J_l = ||e_l||^2 = 1
        L = matrix_L(x[I], M, Ms, kernel)
        b, J[p] = solve_column_naive(L, p, mu)
        idx.append(I)
        bs.append(b)
    idx = np.concatenate(idx) if idx else np.zeros(0, np.int64)
    bs = np.concatenate(bs) if bs else np.zeros(0)
    return BOpt(M, Ms, len(x), m, kernel, tau, ptr, idx, bs, J)


def column_system_closed(x, I, l, M, Ms, kernel, mu):
    """Re G_l + mu I and Re r_l for one column in closed form."""
    xI = x[I]
    G = re_kappa_closed(torus_diff(xI[:, None], xI[None, :]), M, Ms, kernel) + mu * np.eye(len(I))
    r = re_kappa_closed(torus_diff(l / Ms, xI), M, Ms, kernel)
    return G, r


def bopt_closed(x, M, sigma, m, kernel="full", tau=TAU_DEFAULT, chunk=8192):
    """Closed-form tier; the per-column solves are batched over columns of equal
    size (a batched LAPACK call, no change to any column's arithmetic)."""
    Ms = oversampled_size(M, sigma)
    x = np.asarray(x, dtype=np.float64)
    ptr, idx = index_sets_l_fast(x, Ms, m)
    mu = tau * gram_diag(M, Ms, kernel)
    b = np.zeros(len(idx))
    J = np.ones(Ms)
    counts = np.diff(ptr)
    for n in np.unique(counts):
        if n == 0:
            continue
        ps = np.nonzero(counts == n)[0]
        for c0 in range(0, len(ps), chunk):
            pc = ps[c0:c0 + chunk]
            I = idx[ptr[pc][:, None] + np.arange(n)[None, :]]          # (C, n)
            xI = x[I]
            l = (pc - Ms // 2).astype(np.float64)
            Gre = re_kappa_closed(torus_diff(xI[:, :, None], xI[:, None, :]), M, Ms, kernel)
            r = re_kappa_closed(torus_diff(l[:, None] / Ms, xI), M, Ms, kernel)
            bc = np.linalg.solve(Gre + mu * np.eye(n)[None], r[:, :, None])[:, :, 0]
            b[ptr[pc][:, None] + np.arange(n)[None, :]] = bc
            # J_l = ||L b - e_l||^2 = b^T Re G b - 2 Re r . b + 1  (b real)
            J[pc] = np.einsum("ci,cij,cj->c", bc, Gre, bc) - 2 * np.sum(r * bc, axis=1) + 1.0
    return BOpt(M, Ms, len(x), m, kernel, tau, ptr, idx, b, J)
