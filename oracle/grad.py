"""Gradients of a reconstruction loss through the inverse NFFT (differentiable form).

Loss L(f, x) = || fhat(f; x) - t ||_2^2 with fhat = D^* F^* B_opt(x)^* f (eq:approx_ansatz2)
and B_opt(x) from the regularised column problems of Sec. 3.2.2.  Gradients use the
convention of complex autograd: for a complex input z, grad = dL/dRe z + i dL/dIm z; w is
that gradient with respect to fhat (here w = 2 (fhat - t)).

* d/df: fhat is linear in f, so grad_f = (D^* F^* B_opt^*)^* w = B_opt F D w
  (Remark remark:ansatz2_adj: the modified NFFT is the exact adjoint).
* d/dx: implicit differentiation of every column's normal equations
  A_l b_l = r_l, A_l = Re G_l + mu I (the pattern I(l) is piecewise constant in x and held
  fixed).  With gamma = F D w on the grid and beta_{l,i} = Re(conj(gamma_l) f_i) = dL/db_{l,i},
  lambda_l = A_l^{-1} beta_l, and kappa' the derivative of Re kappa (odd, kappa'(0) = 0):
     dL/dx_j = sum_{l : j in I(l)} [ -lambda_{l,j} kappa'(l/M_sigma - x_j)
                                     - lambda_{l,j} sum_k kappa'(x_j - x_k) b_{l,k}
                                     - b_{l,j} sum_i kappa'(x_j - x_i) lambda_{l,i} ].
"""
import numpy as np

from .kernel import kept, gram_diag, re_kappa_closed, torus_diff
from .bopt import BOpt, oversampled_size, TAU_DEFAULT
from .infft import F_apply, infft_apply, nfft_apply
from .pattern import index_sets_l_fast


def kappa_prime_sum(t, M, Ms, kernel):
    """d/dt Re kappa(t) = -(2 pi / M_sigma) sum_k c_k k sin(2 pi k t), by its defining sum."""
    t = np.asarray(t, dtype=np.float64)
    k = np.arange(-(M // 2), M // 2)
    c = kept(M, kernel)
    return -(2 * np.pi / Ms) * (np.sin(2 * np.pi * np.multiply.outer(t, k)) @ (c * k))


def kappa_prime(t, M, Ms, kernel):
    """d/dt Re kappa(t) in closed form (t wrapped to [-1/2, 1/2)):

    full: (pi / M_sigma) [M cot(pi t) cos(pi M t) - sin(pi M t) / sin^2(pi t)]
    sym : (pi / M_sigma) [(M-1) cos((M-1) pi t) / sin(pi t) - sin((M-1) pi t) cos(pi t) / sin^2(pi t)]
    For |M t| < 0.1, where the closed form cancels, the Taylor series of the defining sum:
    -(1/M_sigma) sum_p (-1)^p (2 pi)^{2p+2} S_{2p+2} t^{2p+1} / (2p+1)!,  S_q = sum_k c_k k^q."""
    t = np.asarray(t, dtype=np.float64)
    t = t - np.floor(t + 0.5)
    out = np.empty_like(t)
    small = np.abs(M * t) < 0.1
    ts = t[small]
    k = np.arange(-(M // 2), M // 2, dtype=np.float64)
    c = kept(M, kernel)
    acc = np.zeros_like(ts)
    fact = 1.0
    for p in range(10):
        if p > 0:
            fact *= (2 * p) * (2 * p + 1)
        S = float(np.sum(c * k ** (2 * p + 2)))
        acc += (-1) ** p * (2 * np.pi) ** (2 * p + 2) * S * ts ** (2 * p + 1) / fact
    out[small] = -acc / Ms
    tb = t[~small]
    u = np.pi * tb
    s, co = np.sin(u), np.cos(u)
    if kernel == "full":
        val = M * (co / s) * np.cos(M * u) - np.sin(M * u) / s ** 2
    else:
        val = (M - 1) * np.cos((M - 1) * u) / s - np.sin((M - 1) * u) * co / s ** 2
    out[~small] = np.pi / Ms * val
    return out


def loss(x, f, target, M, sigma, m, kernel="full", tau=TAU_DEFAULT):
    """L = || D^* F^* B_opt(x)^* f - target ||^2 with B_opt from the closed-form tier."""
    from .bopt import bopt_closed
    B = bopt_closed(x, M, sigma, m, kernel, tau)
    r = infft_apply(B, f) - target
    return float(np.vdot(r, r).real), B


def grad_f(B: BOpt, w):
    """dL/dRe f + i dL/dIm f = B_opt F D w."""
    return nfft_apply(B, w)


def grad_x(B: BOpt, x, f, w, chunk=4096):
    """dL/dx_j by implicit differentiation of the column normal equations (module
    docstring).  Columns of equal size are processed together (batched LAPACK solves);
    each column's arithmetic is the formula above."""
    M, Ms, kernel = B.M, B.Ms, B.kernel
    x = np.asarray(x, dtype=np.float64)
    f = np.asarray(f, dtype=np.complex128)
    d = kept(M, kernel) / Ms
    gamma = F_apply(d * np.asarray(w, np.complex128), M, Ms)
    mu = B.tau * gram_diag(M, Ms, kernel)
    g = np.zeros(len(x))
    counts = np.diff(B.ptr)
    for n in np.unique(counts):
        if n == 0:
            continue
        ps = np.nonzero(counts == n)[0]
        for c0 in range(0, len(ps), chunk):
            pc = ps[c0:c0 + chunk]
            ent = B.ptr[pc][:, None] + np.arange(n)[None, :]
            I = B.idx[ent]
            b = B.b[ent]
            xI = x[I]
            D = torus_diff(xI[:, :, None], xI[:, None, :])
            A = re_kappa_closed(D, M, Ms, kernel) + mu * np.eye(n)[None]
            beta = (np.conj(gamma[pc])[:, None] * f[I]).real
            lam = np.linalg.solve(A, beta[:, :, None])[:, :, 0]
            Kp = kappa_prime(D, M, Ms, kernel)                       # K'_{jk} = kappa'(x_j - x_k)
            Kp[:, np.arange(n), np.arange(n)] = 0.0
            tl = kappa_prime(torus_diff(((pc - Ms // 2) / Ms)[:, None], xI), M, Ms, kernel)
            contrib = (-lam * tl - lam * np.einsum("cjk,ck->cj", Kp, b)
                       - b * np.einsum("cjk,ck->cj", Kp, lam))
            np.add.at(g, I.ravel(), contrib.ravel())
    return g


def fd_grad_x(B: BOpt, x, f, target, nodes, h):
    """Central finite differences (L(x + h e_j) - L(x - h e_j)) / (2h) for the given nodes.

    Only the columns l with j in I(l) change when x_j moves (the pattern is held fixed:
    nodes must lie more than h M_sigma from a pattern boundary), so each side is
    evaluated exactly from the base residual r = fhat - target:
    L(x') - L(x) = 2 Re <r, dfhat> + ||dfhat||^2 with dfhat = D^* F^* dg and dg supported
    on those columns (a direct sum over them)."""
    from .bopt import column_system_closed
    M, Ms, kernel = B.M, B.Ms, B.kernel
    x = np.asarray(x, dtype=np.float64)
    f = np.asarray(f, dtype=np.complex128)
    r = infft_apply(B, f) - np.asarray(target, np.complex128)
    mu = B.tau * gram_diag(M, Ms, kernel)
    d = kept(M, kernel) / Ms
    k = np.arange(-(M // 2), M // 2)
    col_of = np.repeat(np.arange(Ms), np.diff(B.ptr))
    out = []
    for j in nodes:
        cols = np.unique(col_of[B.idx == j])
        side = []
        for sgn in (1.0, -1.0):
            xp = x.copy()
            xp[j] = x[j] + sgn * h
            dfh = np.zeros(M, dtype=np.complex128)
            for p in cols:
                s, e = B.ptr[p], B.ptr[p + 1]
                I = B.idx[s:e]
                G, rr = column_system_closed(xp, I, p - Ms // 2, M, Ms, kernel, mu)
                db = np.linalg.solve(G, rr) - B.b[s:e]
                dg = np.dot(db, f[I])
                dfh += d * dg * np.exp(-2j * np.pi * k * (p - Ms // 2) / Ms)
            side.append(2 * np.vdot(r, dfh).real + np.vdot(dfh, dfh).real)
        out.append((side[0] - side[1]) / (2 * h))
    return np.array(out)


def safe_nodes(B: BOpt, x, h, count, seed=0, margin=1e-3):
    """`count` random nodes whose u = M_sigma x is farther than 2 h M_sigma + margin cells from
    an integer (so the pattern does not change under x +- h)."""
    u = B.Ms * np.asarray(x, np.float64)
    dist = np.abs(u - np.round(u))
    ok = np.nonzero(dist > 2 * h * B.Ms + margin)[0]
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(ok, size=min(count, len(ok)), replace=False))
