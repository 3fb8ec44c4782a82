"""The Dirichlet choice of the window (Remark remark:Dirichlet_ansatz2, eq:kernel_Dirichlet).

With w_hat(k) = 1 on the kept frequencies, D = diag(c_k / M_sigma) (eq:matrix_D,
the 1/M_sigma lives in D) and the entries of L_l = F D H_l (eq:matrix_Ll) are
kappa(s/M_sigma - x_j) with

    kappa(t) = (1/M_sigma) * sum_k c_k exp(2 pi i k t).

kernel "full": c_k = 1 for k = -M/2 .. M/2-1;
kernel "sym" : c_k = 1 for k = -M/2+1 .. M/2-1 and c_{-M/2} = 0 (the remark's
               "last nonzero entry of D^* is set to zero"; the remark's sum
               index runs -M/2+1 .. M/2-1, so the dropped entry is k = -M/2).
"""
import numpy as np
from .nfft import freqs

KERNELS = ("full", "sym")


def kept(M, kernel):
    """c_k in {0, 1} for k = -M/2 .. M/2-1."""
    c = np.ones(M)
    if kernel == "sym":
        c[0] = 0.0
    elif kernel != "full":
        raise ValueError(kernel)
    return c


def diag_D(M, Ms, kernel):
    """Diagonal of D (eq:matrix_D with the Dirichlet choice): c_k / M_sigma."""
    return kept(M, kernel) / Ms


def kappa_sum(t, M, Ms, kernel):
    """kappa(t) by its defining sum over k (complex)."""
    t = np.asarray(t, dtype=np.float64)
    c = kept(M, kernel)
    return (np.exp(2j * np.pi * np.multiply.outer(t, freqs(M))) @ c) / Ms


def torus_diff(a, b):
    """a - b as the representative in [-1/2, 1/2] of the difference on the torus
    R/Z ("observing the periodicity", Sec. 3.2.2).  When a - b leaves [-1/2, 1/2]
    the +-1/2 shifts are applied to each operand first, so two nodes that are
    close across the seam x = +-1/2 get their small difference to full relative
    precision (a plain a - b near +-1 loses it before the wrap)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    d = a - b
    d = np.where(d > 0.5, (a - 0.5) - (b + 0.5), d)
    d = np.where(d < -0.5, (a + 0.5) - (b - 0.5), d)
    return d


def _wrap(t):
    t = np.asarray(t, dtype=np.float64)
    return t - np.floor(t + 0.5)


def re_kappa_closed(t, M, Ms, kernel):
    """Re kappa(t) in closed form (geometric sums; both kernels are 1-periodic):

    full: (1/M_sigma) cos(pi t) sin(pi M t) / sin(pi t),  value M/M_sigma at t = 0;
    sym : (1/M_sigma) sin(pi (M-1) t) / sin(pi t)  (the Dirichlet kernel
          D_{M/2-1}, eq:kernel_Dirichlet), value (M-1)/M_sigma at t = 0."""
    t = _wrap(t)
    s = np.sin(np.pi * t)
    zero = (t == 0.0)
    safe = np.where(zero, 1.0, s)
    if kernel == "full":
        v = np.cos(np.pi * t) * np.sin(np.pi * M * t) / safe
        v = np.where(zero, float(M), v)
    elif kernel == "sym":
        v = np.sin(np.pi * (M - 1) * t) / safe
        v = np.where(zero, float(M - 1), v)
    else:
        raise ValueError(kernel)
    return v / Ms


def kappa_closed(t, M, Ms, kernel):
    """kappa(t) (complex) in closed form, the geometric sum over the kept k:

    full: (1/M_sigma) exp(-i pi t) sin(pi M t) / sin(pi t), value M/M_sigma at t = 0;
    sym : the real Dirichlet kernel (1/M_sigma) sin(pi (M-1) t) / sin(pi t)
          (eq:kernel_Dirichlet; Remark remark:Dirichlet_ansatz1 uses it for K_j)."""
    t = _wrap(t)
    if kernel == "sym":
        return re_kappa_closed(t, M, Ms, kernel).astype(np.complex128)
    if kernel != "full":
        raise ValueError(kernel)
    s = np.sin(np.pi * t)
    zero = (t == 0.0)
    v = np.sin(np.pi * M * t) / np.where(zero, 1.0, s)
    v = np.where(zero, float(M), v)
    return np.exp(-1j * np.pi * t) * v / Ms


def gram_diag(M, Ms, kernel):
    """Diagonal entry of Re G_l = Re(L_l^* L_l): (#kept frequencies)/M_sigma."""
    return kept(M, kernel).sum() / Ms
