"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI and
compare it with the FP64 oracle on the same seeded inputs."""
import numpy as np

import oracle
from oracle.kernel import re_kappa_closed, gram_diag, torus_diff

EPS = np.finfo(np.float64).eps


def run_gpu(x, f, M, sigma, m, kernel="full", tau=1e-12, fhat_in=None, z=False):
    """Plan, precompute, apply (and the adjoint when fhat_in is given) on cuda:0."""
    import torch
    import paper_1811_05335_gb300 as g
    dev = torch.device("cuda:0")
    plan = g.infft_plan_create(M, len(x), sigma, m, kernel=kernel, tau=tau)
    g.infft_set_nodes(plan, torch.tensor(x, dtype=torch.float64, device=dev))
    g.infft_precompute(plan)
    ct = torch.complex128 if z else torch.complex64
    fd = torch.tensor(np.asarray(f), dtype=ct, device=dev)
    apply, nfft = (g.infft_apply_z, g.nfft_apply_z) if z else (g.infft_apply, g.nfft_apply)
    fhat = apply(plan, fd)
    back = None
    if fhat_in is not None:
        back = nfft(plan, torch.tensor(np.asarray(fhat_in), dtype=ct, device=dev)).cpu().numpy()
    torch.cuda.synchronize()
    data = g.infft_copy_plan_data(plan)
    info = g.infft_get_info(plan)
    return plan, fhat.cpu().numpy().astype(np.complex128), back, data, info


def gpu_columns(data, N):
    """(column id, node index, weight) of every stored entry, in storage order."""
    count = data["col_count"].astype(np.int64)
    start = data["col_start"].astype(np.int64)
    off = data["col_offset"].astype(np.int64)
    nnz = int(off[-1])
    col = np.repeat(np.arange(len(count)), count)
    pos = (np.repeat(start, count) + np.arange(nnz) - np.repeat(off[:-1], count)) % N
    return col, data["perm"].astype(np.int64)[pos], data["weights"][:nnz] if "weights" in data else None


def assert_pattern_equal(data, B):
    """Bit-exact: the GPU's I(l) equals the oracle's for every l (as sets)."""
    col, node, _ = gpu_columns(data, B.N)
    assert np.array_equal(data["col_count"], np.diff(B.ptr)), "column sizes differ"
    order = np.lexsort((node, col))
    assert np.array_equal(node[order], B.idx), "column node sets differ"


def regularised_excess(data, x, M, Ms, kernel, tau, cols=None):
    """For each checked column: Phi(b_gpu) - Phi(b_oracle) and its rounding tolerance.

    Phi(b) = ||L_l b - e_l||^2 + mu ||b||^2 = b^T (Re G + mu I) b - 2 Re r . b + 1 is the
    regularised column objective; its minimum is unique, so the GPU's b must attain it.
    The tolerance is 1e-12 relative plus the rounding of evaluating Phi at b."""
    col, node, w = gpu_columns(data, len(x))
    off = data["col_offset"].astype(np.int64)
    counts = data["col_count"].astype(np.int64)
    mu = tau * gram_diag(M, Ms, kernel)
    cols = np.arange(Ms) if cols is None else np.asarray(cols)
    excess, tol, Jdiff = [], [], []
    for n in np.unique(counts[cols]):
        if n == 0:
            continue
        ps = cols[counts[cols] == n]
        ent = off[ps][:, None] + np.arange(n)[None, :]
        xI = x[node[ent]]
        b = w[ent]
        l = (ps - Ms // 2).astype(np.float64)
        G = re_kappa_closed(torus_diff(xI[:, :, None], xI[:, None, :]), M, Ms, kernel)
        r = re_kappa_closed(torus_diff(l[:, None] / Ms, xI), M, Ms, kernel)
        Greg = G + mu * np.eye(n)[None]
        bo = np.linalg.solve(Greg, r[:, :, None])[:, :, 0]
        phi = lambda c: np.einsum("ci,cij,cj->c", c, Greg, c) - 2 * np.sum(r * c, axis=1) + 1.0
        pg, po = phi(b), phi(bo)
        scale = np.einsum("ci,cij,cj->c", np.abs(b), np.abs(Greg), np.abs(b)) + 2 * np.sum(np.abs(r * b), 1) + 1
        excess.append(pg - po)
        tol.append(1e-12 * np.abs(po) + 256 * EPS * scale)
        Jg = data["objective"][ps]
        Jo = np.einsum("ci,cij,cj->c", b, G, b) - 2 * np.sum(r * b, axis=1) + 1.0
        # J_gpu = 1 - r.b - mu|b|^2 assumes (G + mu I) b = r; a backward-stable solve leaves a
        # residual of order n eps |G||b|, so the two forms differ by up to b . residual
        Jdiff.append(np.abs(Jg - Jo) / (64 * n * EPS * scale + 1e-13))
    return np.concatenate(excess), np.concatenate(tol), np.concatenate(Jdiff)
