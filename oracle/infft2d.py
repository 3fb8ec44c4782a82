"""Two-dimensional tensor-product form of the modified adjoint NFFT (a reading
of Sec. 3.2.2 for d = 2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper treats d = 1; its conclusion leaves higher dimensions open, and
Remark remark:toeplitz_approach notes that the exact Toeplitz approach has no
counterpart for d > 1.  The reading used here takes every object of Sec. 3.2.2
as the tensor product of its 1-D counterpart:

* frequencies k = (k1, k2), k_t = -M_t/2 .. M_t/2-1; nodes x_j in [-1/2, 1/2)^2;
  A = (exp(2 pi i k.x_j))_{j,k} (eq:matrix_A with k x_j -> k.x_j);
* grid points l = (l1, l2), l_t = -Ms_t/2 .. Ms_t/2-1, Ms_t = sigma M_t;
  F = (exp(2 pi i (k1 l1/Ms1 + k2 l2/Ms2)))_{l,k} (eq:matrix_F per dimension);
* D = diag(c1_{k1} c2_{k2} / (Ms1 Ms2)), c_t the 1-D Dirichlet choice (full / sym,
  oracle.kernel.kept) in each dimension;
* the pattern (eq:set_xj per dimension): l is in I(x_j) iff l_t is in the 1-D
  set of x_jt for t = 1 and t = 2 -- a box of (2m or 2m+1)^2 grid points;
* L_l = F D H_l with H_l = (exp(-2 pi i k.x_j))_{k, j in I(l)} (eq:matrix_Ll).
  Because F^* F = Ms1 Ms2 I on the kept frequencies, G_l = L_l^* L_l has entries
  kappa(x_j - x_j') and r_l = L_l^* e_l has entries conj(kappa(l/Ms - x_j)), with
  kappa(t) = kappa_1(t_1) kappa_2(t_2) the product of the complex 1-D kernels
  (oracle.kernel.kappa_closed; for the full kernel Re kappa is not the product of
  the 1-D real parts);
* the same real, Tikhonov-regularised column problems as d = 1
  (eq:opt_ansatz2 .. eq:solution_ansatz2): (Re G_l + mu I) b = Re r_l,
  mu = tau * Re kappa(0).

Storage: column p = (l1 + Ms1/2) Ms2 + (l2 + Ms2/2); fhat[k1 + M1/2, k2 + M2/2];
nodes x[j] = (x_j1, x_j2).
"""
from dataclasses import dataclass
import numpy as np

from .nfft import freqs
from .kernel import kept, kappa_closed, kappa_sum, torus_diff
from .pattern import grid_lo_hi, reduce_l
from .bopt import oversampled_size, solve_column_naive

TAU_DEFAULT = 1e-12


@dataclass
class BOpt2:
    M1: int
    M2: int
    Ms1: int
    Ms2: int
    N: int
    m: int
    kernel: str
    tau: float
    ptr: np.ndarray      # (Ms1 Ms2 + 1,) column pointers
    idx: np.ndarray      # (nnz,) node index j of each entry (increasing within a column)
    b: np.ndarray        # (nnz,) real coefficients
    J: np.ndarray        # (Ms1 Ms2,) column objectives ||L_l b_l - e_l||^2


# ---- the nonequispaced Fourier matrix in two dimensions ---------------------

def matrix_A2(x, M1, M2):
    """A = (exp(2 pi i (k1 x_j1 + k2 x_j2)))_{j, (k1, k2)}, column (k1 + M1/2) M2 + k2 + M2/2."""
    x = np.asarray(x, np.float64)
    e1 = np.exp(2j * np.pi * np.outer(x[:, 0], freqs(M1)))
    e2 = np.exp(2j * np.pi * np.outer(x[:, 1], freqs(M2)))
    return (e1[:, :, None] * e2[:, None, :]).reshape(len(x), M1 * M2)


def nfft2_direct(x, fhat):
    """f_j = sum_k fhat_k exp(2 pi i k.x_j)  (eq:nfft in 2-D), O(N M1 M2)."""
    M1, M2 = fhat.shape
    return matrix_A2(x, M1, M2) @ np.asarray(fhat, np.complex128).ravel()


def nfft2_adjoint_direct(x, f, M1, M2):
    """h_k = sum_j f_j exp(-2 pi i k.x_j)  (eq:nfft* in 2-D), as an (M1, M2) array."""
    return (matrix_A2(x, M1, M2).conj().T @ np.asarray(f, np.complex128)).reshape(M1, M2)


def dense_lsq_inverse2(x, f, M1, M2):
    """Least-squares solution of A fhat = f (eq:problem_infft in 2-D) by LAPACK's SVD solver."""
    sol, *_ = np.linalg.lstsq(matrix_A2(x, M1, M2), np.asarray(f, np.complex128), rcond=None)
    return sol.reshape(M1, M2)


# ---- D, F and the kernel ----------------------------------------------------

def diag_D2(M1, M2, Ms1, Ms2, kernel):
    """Diagonal of D as an (M1, M2) array: c1_{k1} c2_{k2} / (Ms1 Ms2)."""
    return np.outer(kept(M1, kernel), kept(M2, kernel)) / (Ms1 * Ms2)


def kappa2(t1, t2, M1, M2, Ms1, Ms2, kernel):
    """kappa(t) = sum_k d_k exp(2 pi i k.t) = kappa_1(t1) kappa_2(t2) (complex)."""
    return kappa_closed(t1, M1, Ms1, kernel) * kappa_closed(t2, M2, Ms2, kernel)


def kappa2_sum(t1, t2, M1, M2, Ms1, Ms2, kernel):
    """kappa(t) by its defining double sum over the kept frequencies."""
    return kappa_sum(t1, M1, Ms1, kernel) * kappa_sum(t2, M2, Ms2, kernel)


def gram_diag2(M1, M2, Ms1, Ms2, kernel):
    """Re kappa(0): (#kept k1)(#kept k2)/(Ms1 Ms2)."""
    return kept(M1, kernel).sum() * kept(M2, kernel).sum() / (Ms1 * Ms2)


def matrix_F2(M1, M2, Ms1, Ms2):
    """F: rows l (p order), columns k ((k1 + M1/2) M2 + k2 + M2/2)."""
    l1 = np.arange(-(Ms1 // 2), Ms1 // 2)
    l2 = np.arange(-(Ms2 // 2), Ms2 // 2)
    f1 = np.exp(2j * np.pi * np.outer(l1, freqs(M1)) / Ms1)
    f2 = np.exp(2j * np.pi * np.outer(l2, freqs(M2)) / Ms2)
    return np.einsum("ak,bq->abkq", f1, f2).reshape(Ms1 * Ms2, M1 * M2)


def matrix_L2(xI, M1, M2, Ms1, Ms2, kernel):
    """L_l = F D H_l, formed explicitly (small sizes only)."""
    H = matrix_A2(xI, M1, M2).conj().T                      # (M1 M2, n)
    d = diag_D2(M1, M2, Ms1, Ms2, kernel).ravel()
    return matrix_F2(M1, M2, Ms1, Ms2) @ (d[:, None] * H)


# ---- the pattern ------------------------------------------------------------

def node_boxes(x, Ms1, Ms2, m):
    """Per node the integer intervals [lo_t, hi_t] of eq:set_xj in each dimension."""
    x = np.asarray(x, np.float64)
    lo1, hi1 = grid_lo_hi(x[:, 0], Ms1, m)
    lo2, hi2 = grid_lo_hi(x[:, 1], Ms2, m)
    return lo1, hi1, lo2, hi2


def index_sets_l2(x, Ms1, Ms2, m):
    """I(l) for every grid point, column p = (l1 + Ms1/2) Ms2 + l2 + Ms2/2, built
    node by node from the box of each node (increasing node indices)."""
    lo1, hi1, lo2, hi2 = node_boxes(x, Ms1, Ms2, m)
    cols = [[] for _ in range(Ms1 * Ms2)]
    for j in range(len(lo1)):
        a1 = np.unique(reduce_l(np.arange(lo1[j], hi1[j] + 1), Ms1)) + Ms1 // 2
        a2 = np.unique(reduce_l(np.arange(lo2[j], hi2[j] + 1), Ms2)) + Ms2 // 2
        for p1 in a1:
            for p2 in a2:
                cols[int(p1) * Ms2 + int(p2)].append(j)
    return [np.asarray(c, dtype=np.int64) for c in cols]


def index_sets_l2_fast(x, Ms1, Ms2, m):
    """The same sets as index_sets_l2, vectorised: (ptr, idx)."""
    lo1, hi1, lo2, hi2 = node_boxes(x, Ms1, Ms2, m)
    N = len(lo1)
    w1, w2 = hi1 - lo1 + 1, hi2 - lo2 + 1
    cnt = w1 * w2
    nodes = np.repeat(np.arange(N, dtype=np.int64), cnt)
    off = np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    W2 = np.repeat(w2, cnt)
    a1 = reduce_l(np.repeat(lo1, cnt) + off // W2, Ms1) + Ms1 // 2
    a2 = reduce_l(np.repeat(lo2, cnt) + off % W2, Ms2) + Ms2 // 2
    p = a1 * Ms2 + a2
    order = np.lexsort((nodes, p))
    p, nodes = p[order], nodes[order]
    ptr = np.zeros(Ms1 * Ms2 + 1, dtype=np.int64)
    np.add.at(ptr, p + 1, 1)
    return np.cumsum(ptr), nodes


def column_l(p, Ms1, Ms2):
    """Grid point (l1, l2) of column p."""
    return p // Ms2 - Ms1 // 2, p % Ms2 - Ms2 // 2


# ---- B_opt -------------------------------------------------------------------

def column_system2(x, I, p, M1, M2, Ms1, Ms2, kernel, mu):
    """Re G_l + mu I and Re r_l of column p in closed form."""
    xI = np.asarray(x, np.float64)[I]
    l1, l2 = column_l(p, Ms1, Ms2)
    d1 = torus_diff(xI[:, None, 0], xI[None, :, 0])
    d2 = torus_diff(xI[:, None, 1], xI[None, :, 1])
    G = kappa2(d1, d2, M1, M2, Ms1, Ms2, kernel).real + mu * np.eye(len(I))
    r = kappa2(torus_diff(l1 / Ms1, xI[:, 0]), torus_diff(l2 / Ms2, xI[:, 1]), M1, M2, Ms1, Ms2, kernel).real
    return G, r


def solve_column2(x, I, p, M1, M2, Ms1, Ms2, kernel, tau=TAU_DEFAULT):
    """b_l and J_l = b^T Re G b - 2 Re r.b + 1 of one column (LAPACK LU)."""
    if len(I) == 0:
        return np.zeros(0), 1.0
    mu = tau * gram_diag2(M1, M2, Ms1, Ms2, kernel)
    Gm, r = column_system2(x, I, p, M1, M2, Ms1, Ms2, kernel, mu)
    b = np.linalg.solve(Gm, r)
    G = Gm - mu * np.eye(len(I))
    return b, float(b @ G @ b - 2.0 * r @ b + 1.0)


def bopt2_closed(x, M1, M2, sigma=2.0, m=4, kernel="full", tau=TAU_DEFAULT, chunk=4096):
    """Closed-form B_opt for every column; columns of equal size are solved in
    batched LAPACK calls (no change to any column's arithmetic)."""
    Ms1, Ms2 = oversampled_size(M1, sigma), oversampled_size(M2, sigma)
    x = np.asarray(x, np.float64)
    ptr, idx = index_sets_l2_fast(x, Ms1, Ms2, m)
    mu = tau * gram_diag2(M1, M2, Ms1, Ms2, kernel)
    b = np.zeros(len(idx))
    J = np.ones(Ms1 * Ms2)
    counts = np.diff(ptr)
    for n in np.unique(counts):
        if n == 0:
            continue
        ps = np.nonzero(counts == n)[0]
        for c0 in range(0, len(ps), chunk):
            pc = ps[c0:c0 + chunk]
            I = idx[ptr[pc][:, None] + np.arange(n)[None, :]]
            xI = x[I]                                               # (C, n, 2)
            l1, l2 = column_l(pc, Ms1, Ms2)
            d1 = torus_diff(xI[:, :, None, 0], xI[:, None, :, 0])
            d2 = torus_diff(xI[:, :, None, 1], xI[:, None, :, 1])
            G = kappa2(d1, d2, M1, M2, Ms1, Ms2, kernel).real
            r = kappa2(torus_diff(l1[:, None] / Ms1, xI[:, :, 0]), torus_diff(l2[:, None] / Ms2, xI[:, :, 1]),
                       M1, M2, Ms1, Ms2, kernel).real
            bc = np.linalg.solve(G + mu * np.eye(n)[None], r[:, :, None])[:, :, 0]
            b[ptr[pc][:, None] + np.arange(n)[None, :]] = bc
            J[pc] = np.einsum("ci,cij,cj->c", bc, G, bc) - 2 * np.sum(r * bc, axis=1) + 1.0
    return BOpt2(M1, M2, Ms1, Ms2, len(x), m, kernel, tau, ptr, idx, b, J)


def bopt2_naive(x, M1, M2, sigma=2.0, m=1, kernel="full", tau=TAU_DEFAULT):
    """Naive tier: L_l = F D H_l formed explicitly and the stacked real problem
    [Re L; Im L; sqrt(mu) I] b = [e_l; 0; 0] solved by LAPACK (tiny sizes only)."""
    Ms1, Ms2 = oversampled_size(M1, sigma), oversampled_size(M2, sigma)
    x = np.asarray(x, np.float64)
    cols = index_sets_l2(x, Ms1, Ms2, m)
    mu = tau * gram_diag2(M1, M2, Ms1, Ms2, kernel)
    P = Ms1 * Ms2
    ptr = np.zeros(P + 1, dtype=np.int64)
    idx, bs, J = [], [], np.ones(P)
    for p, I in enumerate(cols):
        ptr[p + 1] = ptr[p] + len(I)
        if len(I) == 0:
            continue
        L = matrix_L2(x[I], M1, M2, Ms1, Ms2, kernel)
        b, J[p] = solve_column_naive(L, p, mu)
        idx.append(I)
        bs.append(b)
    idx = np.concatenate(idx) if idx else np.zeros(0, np.int64)
    bs = np.concatenate(bs) if bs else np.zeros(0)
    return BOpt2(M1, M2, Ms1, Ms2, len(x), m, kernel, tau, ptr, idx, bs, J)


# ---- the modified adjoint NFFT ------------------------------------------------

def spread2(B: BOpt2, f):
    """g~_l = sum_{j in I(l)} b_{l,j} f_j on the (Ms1, Ms2) grid."""
    f = np.asarray(f, np.complex128)
    g = np.zeros(B.Ms1 * B.Ms2, np.complex128)
    col = np.repeat(np.arange(B.Ms1 * B.Ms2), np.diff(B.ptr))
    np.add.at(g, col, B.b * f[B.idx])
    return g.reshape(B.Ms1, B.Ms2)


def F2_adjoint(g, M1, M2, method="fft"):
    """h_k = sum_l g_l exp(-2 pi i (k1 l1/Ms1 + k2 l2/Ms2)) for the kept k (F^*).
    "direct" multiplies by the explicit matrix; "fft" uses numpy's 2-D FFT over
    p_t = l_t + Ms_t/2, exp(-2 pi i k l/Ms) = (-1)^k exp(-2 pi i k p/Ms)."""
    g = np.asarray(g, np.complex128)
    Ms1, Ms2 = g.shape
    if method == "direct":
        return (matrix_F2(M1, M2, Ms1, Ms2).conj().T @ g.ravel()).reshape(M1, M2)
    k1, k2 = freqs(M1), freqs(M2)
    G = np.fft.fft2(g)[np.ix_(k1 % Ms1, k2 % Ms2)]
    s1 = np.where(k1 % 2 == 0, 1.0, -1.0)
    s2 = np.where(k2 % 2 == 0, 1.0, -1.0)
    return np.outer(s1, s2) * G


def infft2_apply(B: BOpt2, f, method="fft"):
    """fhat ~ D^* F^* B_opt^* f (eq:approx_ansatz2 in 2-D), an (M1, M2) array."""
    d = diag_D2(B.M1, B.M2, B.Ms1, B.Ms2, B.kernel)
    return np.conj(d) * F2_adjoint(spread2(B, f), B.M1, B.M2, method)


def infft2_apply_impulse(x, j, M1, M2, sigma=2.0, m=4, kernel="full", tau=TAU_DEFAULT):
    """fhat for the data f = e_j (one node): only the columns l in I(x_j) contribute,
    fhat_k = conj(d_k) sum_{l in I(x_j)} b_{l,j} exp(-2 pi i k.l/Ms).  Solves just
    those columns (each through its full I(l)), so it runs at any problem size."""
    Ms1, Ms2 = oversampled_size(M1, sigma), oversampled_size(M2, sigma)
    x = np.asarray(x, np.float64)
    lo1, hi1, lo2, hi2 = node_boxes(x[j:j + 1], Ms1, Ms2, m)
    a1 = np.unique(reduce_l(np.arange(lo1[0], hi1[0] + 1), Ms1)) + Ms1 // 2
    a2 = np.unique(reduce_l(np.arange(lo2[0], hi2[0] + 1), Ms2)) + Ms2 // 2
    LO1, HI1, LO2, HI2 = node_boxes(x, Ms1, Ms2, m)
    g = {}
    for p1 in a1:
        for p2 in a2:
            p = int(p1) * Ms2 + int(p2)
            l1, l2 = column_l(p, Ms1, Ms2)
            I = np.nonzero(_covers(LO1, HI1, l1, Ms1) & _covers(LO2, HI2, l2, Ms2))[0]
            b, _ = solve_column2(x, I, p, M1, M2, Ms1, Ms2, kernel, tau)
            g[(l1, l2)] = b[np.searchsorted(I, j)]
    k1, k2 = freqs(M1), freqs(M2)
    h = np.zeros((M1, M2), np.complex128)
    for (l1, l2), v in g.items():
        h += v * np.outer(np.exp(-2j * np.pi * k1 * l1 / Ms1), np.exp(-2j * np.pi * k2 * l2 / Ms2))
    return np.conj(diag_D2(M1, M2, Ms1, Ms2, kernel)) * h


def _covers(lo, hi, l, Ms):
    """Nodes whose interval [lo, hi] (eq:set_xj) contains l modulo Ms."""
    return ((l - lo) % Ms) <= (hi - lo)


def column_nodes2(x, p, Ms1, Ms2, m):
    """I(l) of one column p (increasing node indices), at any problem size."""
    LO1, HI1, LO2, HI2 = node_boxes(x, Ms1, Ms2, m)
    l1, l2 = column_l(p, Ms1, Ms2)
    return np.nonzero(_covers(LO1, HI1, l1, Ms1) & _covers(LO2, HI2, l2, Ms2))[0]
