"""Index sets of the truncated window (Sec. 3.2.1 eq:set_xj, Sec. 3.2.2 eq:set_l).

I(x_j) = { l : exists z in Z, -m <= M_sigma x_j - l + M_sigma z <= m }  and
I(l)   = { j : same relation }.  The relation is decided exactly on the real
number u_j = fl(M_sigma * x_j) (one rounded fp64 product): since m and l are
integers, |u - l + M_sigma z| <= m  iff  ceil(u) - m <= l - M_sigma z <= floor(u) + m.
"""
import numpy as np


def grid_u(x, Ms):
    """u_j = fl(M_sigma * x_j), a single rounded fp64 multiply."""
    return np.float64(Ms) * np.asarray(x, dtype=np.float64)


def grid_lo_hi(x, Ms, m):
    """Per node the integer interval [ceil(u_j) - m, floor(u_j) + m] of grid
    points l (before reduction mod M_sigma), eq:set_xj."""
    u = grid_u(x, Ms)
    return np.ceil(u).astype(np.int64) - m, np.floor(u).astype(np.int64) + m


def reduce_l(l, Ms):
    """Representative of l mod M_sigma in [-M_sigma/2, M_sigma/2)."""
    return (np.asarray(l) + Ms // 2) % Ms - Ms // 2


def index_sets_x(x, Ms, m):
    """I(x_j) for every node j as a sorted array of grid indices l (eq:set_xj)."""
    lo, hi = grid_lo_hi(x, Ms, m)
    return [np.unique(reduce_l(np.arange(a, b + 1), Ms)) for a, b in zip(lo, hi)]


def index_sets_l(x, Ms, m):
    """I(l) for l = -M_sigma/2 .. M_sigma/2-1 (list index p = l + M_sigma/2),
    each an increasing array of node indices j (eq:set_l), built by inverting
    eq:set_xj node by node."""
    lo, hi = grid_lo_hi(x, Ms, m)
    cols = [[] for _ in range(Ms)]
    for j, (a, b) in enumerate(zip(lo, hi)):
        for l in np.unique(reduce_l(np.arange(a, b + 1), Ms)):
            cols[int(l) + Ms // 2].append(j)
    return [np.asarray(c, dtype=np.int64) for c in cols]


def index_sets_l_fast(x, Ms, m):
    """Same sets as index_sets_l, vectorised (CSC-like arrays): returns
    (ptr, idx) with I(l) = idx[ptr[p]:ptr[p+1]], nodes increasing."""
    lo, hi = grid_lo_hi(x, Ms, m)
    width = hi - lo + 1                       # 2m or 2m+1
    N = len(lo)
    nodes = np.repeat(np.arange(N, dtype=np.int64), width)
    offs = np.arange(width.sum()) - np.repeat(np.cumsum(width) - width, width)
    ls = reduce_l(np.repeat(lo, width) + offs, Ms) + Ms // 2
    order = np.lexsort((nodes, ls))
    ls, nodes = ls[order], nodes[order]
    ptr = np.zeros(Ms + 1, dtype=np.int64)
    np.add.at(ptr, ls + 1, 1)
    return np.cumsum(ptr), nodes
