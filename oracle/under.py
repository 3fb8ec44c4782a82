"""Optimisation of B, underdetermined case (Sec. 3.2.1, "ansatz 1").

TEST INFRASTRUCTURE ONLY (see the package docstring).

The estimate is f_check = (1/M) D^* F^* B_opt^* f (eq:approx_ansatz1), and
B_opt minimises ||A D^* F^* B^* - M I_N||_F^2 over (2m+1)-sparse real B
(eq:min_norm_ansatz1).  The Frobenius norm splits over the N columns of B^*
(eq:min_decomp_ansatz1), one problem per node x_j:

    min_{b real}  ||K_j b - M e_j||_2^2,   K_j = A D^* T_j  (eq:matrix_Kj),

with (K_j)_{h,l} = kappa(x_h - l/M_sigma) for h = 1..N and l in I(x_j)
(eq:set_xj); with the Dirichlet choice (Remark remark:Dirichlet_ansatz1) kappa
is the kernel of oracle.kernel (D = diag(c_k)/M_sigma, eq:matrix_K).  The
full-rank solution is eq:solution_ansatz1.  Readings, as in Sec. 3.2.2: b is
real, so the normal equations are Re(K_j^* K_j) b = M Re(K_j^* e_j); rank
deficiency is handled by Tikhonov regularisation with
mu_j = tau * (mean diagonal entry of Re K_j^* K_j):

    b_j = argmin ||K_j b - M e_j||^2 + mu_j ||b||^2.

Two tiers, both from the explicit N x |I(x_j)| matrix K_j:

* ``bopt_under_naive`` solves the stacked real least-squares problem
  [Re K_j; Im K_j; sqrt(mu_j) I] b = [M e_j; 0; 0] with LAPACK (SVD based);
* ``bopt_under`` forms Re(K_j^* K_j) + mu_j I and Re(K_j^* e_j) and solves the
  normal equations with LAPACK LU, nodes batched by |I(x_j)|.

Both return the column layout of B_opt (ptr, idx, b as in oracle.bopt.BOpt, so
oracle.infft.spread / interpolate apply unchanged) and the node objectives
J_j = ||K_j b_j - M e_j||^2 (without the mu term).
"""
from dataclasses import dataclass
import numpy as np

from .nfft import matrix_A
from .pattern import grid_lo_hi, reduce_l, index_sets_l_fast
from .kernel import kappa_closed, torus_diff, diag_D
from .bopt import BOpt, oversampled_size, matrix_F, TAU_DEFAULT
from .infft import spread, interpolate, F_adjoint, F_apply


@dataclass
class BOptUnder:
    B: BOpt              # column layout of B_opt (B.J unused: all ones)
    Jn: np.ndarray       # (N,) node objectives ||K_j b_j - M e_j||^2
    mu: np.ndarray       # (N,) the Tikhonov weight used for each node


def node_grid_points(x, Ms, m):
    """I(x_j) per node as the increasing integer run ceil(u_j) - m .. floor(u_j) + m
    (eq:set_xj before reduction; u_j = fl(M_sigma x_j)).  Runs longer than
    M_sigma (tiny grids) are not supported by this tier."""
    lo, hi = grid_lo_hi(x, Ms, m)
    if np.any(hi - lo + 1 > Ms):
        raise ValueError("2m + 1 > M_sigma")
    return lo, hi


def matrix_K_j(x, l, M, Ms, kernel):
    """K_j = (kappa(x_h - l/M_sigma))_{h, l in I(x_j)} in C^{N x |I(x_j)|} (eq:matrix_Kj)."""
    return kappa_closed(torus_diff(np.asarray(x, np.float64)[:, None], reduce_l(l, Ms)[None, :] / Ms),
                        M, Ms, kernel)


def node_system(x, j, l, M, Ms, kernel, tau=TAU_DEFAULT):
    """Re(K_j^* K_j) + mu_j I, M Re(K_j^* e_j) and mu_j for node j (normal equations of eq:opt_ansatz1)."""
    K = matrix_K_j(x, l, M, Ms, kernel)
    G = (K.conj().T @ K).real
    mu = tau * float(np.mean(np.diag(G)))
    r = M * K[j].conj().real
    return G + mu * np.eye(len(l)), r, mu


def _assemble(x, M, Ms, m, kernel, tau, lo, b_nodes, Jn, mu):
    """Column layout of B_opt^* from the per-node coefficients b_j on l = lo_j + 0 .. n_j - 1."""
    N = len(x)
    ptr, idx = index_sets_l_fast(x, Ms, m)
    b = np.zeros(len(idx))
    for p in range(Ms):
        s, e = ptr[p], ptr[p + 1]
        l = p - Ms // 2
        for q in range(s, e):
            j = idx[q]
            a = (l - lo[j]) % Ms          # position of l in the run of node j
            b[q] = b_nodes[j][a]
    B = BOpt(M, Ms, N, m, kernel, tau, ptr, idx, b, np.ones(Ms))
    return BOptUnder(B, np.asarray(Jn), np.asarray(mu))


def bopt_under_naive(x, M, sigma, m, kernel="full", tau=TAU_DEFAULT):
    Ms = oversampled_size(M, sigma)
    x = np.asarray(x, np.float64)
    N = len(x)
    lo, hi = node_grid_points(x, Ms, m)
    bs, Jn, mus = [], np.zeros(N), np.zeros(N)
    for j in range(N):
        l = np.arange(lo[j], hi[j] + 1)
        K = matrix_K_j(x, l, M, Ms, kernel)
        mu = tau * float(np.mean(np.sum(np.abs(K) ** 2, axis=0)))
        e = np.zeros(N)
        e[j] = M
        A = np.vstack([K.real, K.imag, np.sqrt(mu) * np.eye(len(l))])
        rhs = np.concatenate([e, np.zeros(N), np.zeros(len(l))])
        b, *_ = np.linalg.lstsq(A, rhs, rcond=None)
        bs.append(b)
        Jn[j] = np.linalg.norm(K @ b - e) ** 2
        mus[j] = mu
    return _assemble(x, M, Ms, m, kernel, tau, lo, bs, Jn, mus)


def bopt_under(x, M, sigma, m, kernel="full", tau=TAU_DEFAULT, chunk=64):
    """Normal-equation tier; nodes with equal |I(x_j)| are solved in batches
    (a batched LAPACK call, no change to any node's arithmetic)."""
    Ms = oversampled_size(M, sigma)
    x = np.asarray(x, np.float64)
    N = len(x)
    lo, hi = node_grid_points(x, Ms, m)
    width = hi - lo + 1
    bs = [None] * N
    Jn, mus = np.zeros(N), np.zeros(N)
    for n in np.unique(width):
        js = np.nonzero(width == n)[0]
        for c0 in range(0, len(js), chunk):
            jj = js[c0:c0 + chunk]
            l = lo[jj][:, None] + np.arange(n)[None, :]
            K = kappa_closed(torus_diff(x[None, :, None], reduce_l(l, Ms)[:, None, :] / Ms), M, Ms, kernel)
            G = np.einsum("chi,chk->cik", K.conj(), K).real
            mu = tau * np.einsum("cii->c", G) / n
            r = M * K[np.arange(len(jj)), jj, :].conj().real
            b = np.linalg.solve(G + mu[:, None, None] * np.eye(n)[None], r[:, :, None])[:, :, 0]
            E = np.einsum("chi,ci->ch", K, b)
            E[np.arange(len(jj)), jj] -= M
            Jn[jj] = np.sum(np.abs(E) ** 2, axis=1)
            mus[jj] = mu
            for q, j in enumerate(jj):
                bs[j] = b[q]
    return _assemble(x, M, Ms, m, kernel, tau, lo, bs, Jn, mus)


def infft_apply_under(U: BOptUnder, f, method="fft"):
    """f_check = (1/M) D^* F^* B_opt^* f  (eq:approx_ansatz1)."""
    B = U.B
    d = diag_D(B.M, B.Ms, B.kernel)
    return np.conj(d) * F_adjoint(spread(B, f), B.M, B.Ms, method) / B.M


def adjoint_inverse_apply_under(U: BOptUnder, h, method="fft"):
    """f_tilde = (1/M) B_opt F D h, the estimate of f from h = A^* f (Remark
    remark:ansatz1_adj, Example ex:trig_poly_ansatz1_adj); the adjoint of
    infft_apply_under."""
    B = U.B
    d = diag_D(B.M, B.Ms, B.kernel)
    return interpolate(B, F_apply(d * np.asarray(h, np.complex128), B.M, B.Ms, method)) / B.M


def frobenius_objective_under_dense(x, Bdense, M, Ms, kernel):
    """||A D^* F^* B^* - M I_N||_F^2 from the explicit matrices (eq:norm_frobenius); Bdense is N x M_sigma."""
    A = matrix_A(x, M)
    K = A @ (diag_D(M, Ms, kernel)[:, None] * matrix_F(M, Ms).conj().T)
    return float(np.linalg.norm(K @ Bdense.T - M * np.eye(len(x))) ** 2)
