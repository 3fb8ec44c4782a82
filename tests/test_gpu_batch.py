"""Parity of the batched form (many problems of uneven size in one plan, through the
C ABI) with the FP64 oracle, problem by problem.

Each problem of a batch must give what the oracle gives for it alone: bit-exact
index sets I(l), every column's b at the regularised minimum (as in
test_gpu_infft.py, including the columns of more than 224 nodes that the
large-column solver takes), and fhat within the fp32 tolerance 1e-5 (rel l2).
The batch mixes node families and sizes: M not a power of two (the chirp
convolution of the batched FFT), M = 8 and 10 (chirp lengths 16 and 32), M = 8190
(chirp length 16384), and Chebyshev-clustered nodes whose columns near x = +-1/2 hold up to
338 nodes.  The full-size workload (4096 problems) is checked on sampled
problems whose data is evaluated exactly.
"""
import numpy as np
import pytest

import oracle
from workloads import (chebyshev_jittered, jittered, iid_uniform, complex_normal, trig_poly_eval,
                       make_batch)
from gpu_support import assert_pattern_equal, regularised_excess

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5

# (M, N, node family, seed)
SPECS = [(1000, 3500, "cheb", 21), (1536, 6000, "cheb", 22), (8, 30, "unif", 23), (34, 100, "jit", 24),
         (100, 300, "cheb", 25), (256, 1024, "jit", 26), (258, 700, "unif", 27), (1022, 2100, "unif", 28),
         (10, 25, "unif", 29), (8190, 16400, "jit", 30)]


def nodes(fam, seed, n):
    return {"cheb": chebyshev_jittered, "jit": jittered, "unif": iid_uniform}[fam](seed, n)


def c64(a):
    return np.asarray(a, np.complex64).astype(np.complex128)


_cache = {}


def batch_run(kernel="full", m=6):
    key = (kernel, m)
    if key in _cache:
        return _cache[key]
    import torch
    import paper_1811_05335_gb300 as g
    dev = torch.device("cuda:0")
    Ms = [s[0] for s in SPECS]
    Ns = [s[1] for s in SPECS]
    xs = [nodes(fam, sd, n) for (M, n, fam, sd) in SPECS]
    fh = [complex_normal(100 + sd, M) for (M, n, fam, sd) in SPECS]
    fs = [trig_poly_eval(x, c) for x, c in zip(xs, fh)]
    b = g.infft_batch_create(Ms, Ns, 2.0, m, kernel=kernel)
    g.infft_batch_set_nodes(b, torch.tensor(np.concatenate(xs), dtype=torch.float64, device=dev))
    g.infft_batch_precompute(b)
    f = torch.tensor(np.concatenate(fs), dtype=torch.complex64, device=dev)
    out = g.infft_batch_apply(b, f)
    torch.cuda.synchronize()
    info = g.infft_batch_get_info(b)
    data = [g.infft_batch_copy_problem(b, p) for p in range(len(SPECS))]
    fhat = out.cpu().numpy().astype(np.complex128)
    res = dict(batch=b, xs=xs, fs=fs, info=info, data=data, fhat=fhat, Ms=Ms, Ns=Ns, m=m, kernel=kernel,
               B=[oracle.bopt.bopt_closed(x, M, 2.0, m, kernel) for x, M in zip(xs, Ms)])
    _cache[key] = res
    return res


def test_batch_info_sums():
    r = batch_run()
    info = r["info"]
    assert info["P"] == len(SPECS)
    assert info["nnz"] == sum(len(B.idx) for B in r["B"])
    assert info["max_column"] == max(int(np.diff(B.ptr).max()) for B in r["B"])
    assert info["bad_nodes"] == 0
    assert info["fallback_columns"] == 0 and info["unsupported_columns"] == 0
    assert info["large_columns"] == sum(int((np.diff(B.ptr) > 224).sum()) for B in r["B"]) > 0
    J = sum(B.J.sum() for B in r["B"])
    assert abs(info["objective"] - J) <= 1e-9 * J + 1e-9


@pytest.mark.parametrize("p", range(len(SPECS)))
def test_batch_pattern_bit_exact(p):
    r = batch_run()
    assert_pattern_equal(r["data"][p], r["B"][p])


@pytest.mark.parametrize("p", range(len(SPECS)))
def test_batch_bopt_attains_regularised_minimum(p):
    r = batch_run()
    M, x, data = r["Ms"][p], r["xs"][p], r["data"][p]
    excess, tol, jdiff = regularised_excess(data, x, M, 2 * M, r["kernel"], 1e-12)
    assert np.all(np.abs(excess) <= tol), f"max |excess|/tol {np.max(np.abs(excess) / tol):.3g}"
    assert np.all(jdiff <= 1.0), f"max J mismatch / tol {jdiff.max():.3g}"


@pytest.mark.parametrize("p", range(len(SPECS)))
def test_batch_apply_fp32(p):
    r = batch_run()
    a, b = int(np.sum(r["Ms"][:p])), int(np.sum(r["Ms"][:p + 1]))
    want = oracle.infft.infft_apply(r["B"][p], c64(r["fs"][p]))
    err = oracle.infft.rel_l2(r["fhat"][a:b], want)
    assert err <= FP32_TOL, f"problem {p} (M={r['Ms'][p]}): rel l2 {err:.3e}"


def test_batch_sym_kernel():
    """Kernel sym: d_{-M/2} = 0 in every problem's deconvolution."""
    r = batch_run(kernel="sym", m=4)
    for p in range(len(SPECS)):
        a, b = int(np.sum(r["Ms"][:p])), int(np.sum(r["Ms"][:p + 1]))
        want = oracle.infft.infft_apply(r["B"][p], c64(r["fs"][p]))
        assert r["fhat"][a] == 0
        assert oracle.infft.rel_l2(r["fhat"][a:b], want) <= FP32_TOL


def test_batch_matches_single_plan():
    """A power-of-two problem gives the same fhat in the batch as in a plan of its own
    (same pattern and B_opt; only the FFT differs: chirp convolution vs four-step)."""
    import torch
    import paper_1811_05335_gb300 as g
    r = batch_run()
    p = 5                                    # M = 256, jittered
    M, x, f = r["Ms"][p], r["xs"][p], r["fs"][p]
    dev = torch.device("cuda:0")
    plan = g.infft_plan_create(M, len(x), 2.0, r["m"])
    g.infft_set_nodes(plan, torch.tensor(x, dtype=torch.float64, device=dev))
    g.infft_precompute(plan)
    one = g.infft_apply(plan, torch.tensor(f, dtype=torch.complex64, device=dev)).cpu().numpy()
    a = int(np.sum(r["Ms"][:p]))
    assert oracle.infft.rel_l2(r["fhat"][a:a + M], one) <= 2e-6
    single = g.infft_copy_plan_data(plan)
    assert np.array_equal(single["col_count"], r["data"][p]["col_count"])
    assert np.array_equal(single["perm"], r["data"][p]["perm"])


def test_batch_host_buffers():
    """Host f and fhat go through the batch's staging buffers (synchronous result)."""
    r = batch_run()
    import paper_1811_05335_gb300 as g
    f = np.concatenate(r["fs"]).astype(np.complex64)
    out = np.empty(int(np.sum(r["Ms"])), np.complex64)
    g.infft_batch_apply(r["batch"], f, out=out)
    assert np.max(np.abs(out - r["fhat"])) <= 1e-6 * np.max(np.abs(r["fhat"]))


def test_batch_argument_errors():
    import paper_1811_05335_gb300 as g
    with pytest.raises(g.InfftError):
        g.infft_batch_create([10, 7], [20, 20])          # odd M
    with pytest.raises(g.InfftError):
        g.infft_batch_create([10, 8194], [20, 20])       # M above 8192
    with pytest.raises(g.InfftError):
        g.infft_batch_create([10], [20], sigma=1.5)      # sigma must be 2
    b = g.infft_batch_create([10], [20])
    with pytest.raises(g.InfftError):
        g.infft_batch_precompute(b)                      # before set_nodes
    with pytest.raises(g.InfftError):
        g.infft_batch_set_nodes(b, np.full(20, 0.5))     # node outside [-1/2, 1/2)
    b.close()


def test_batch_full_workload_sampled():
    """The full batched workload (4096 problems, M log-uniform in [256, 8192], N = 2-4 M,
    Chebyshev-clustered nodes, m = 6): sampled small problems get exact trigonometric-
    polynomial data and must match the oracle; every column is solved."""
    import torch
    import paper_1811_05335_gb300 as g
    w = make_batch()
    dev = torch.device("cuda:0")
    b = g.infft_batch_create(w.M, w.N, 2.0, w.m)
    g.infft_batch_set_nodes(b, torch.tensor(w.x_all, dtype=torch.float64, device=dev))
    g.infft_batch_precompute(b)
    order = np.argsort(w.M)
    sample = [int(order[0]), int(order[1]), int(order[len(order) // 8])]
    rng = np.random.default_rng(5)
    f = (rng.standard_normal(int(w.N.sum())) + 1j * rng.standard_normal(int(w.N.sum()))).astype(np.complex64)
    fh_true = {}
    for p in sample:
        fh_true[p] = complex_normal(500 + p, int(w.M[p]))
        a = int(w.N[:p].sum())
        f[a:a + int(w.N[p])] = trig_poly_eval(w.x[p], fh_true[p]).astype(np.complex64)
    out = g.infft_batch_apply(b, torch.tensor(f, device=dev)).cpu().numpy().astype(np.complex128)
    info = g.infft_batch_get_info(b)
    assert info["unsupported_columns"] == 0 and info["fallback_columns"] == 0
    assert info["large_columns"] > 0
    for p in sample:
        M, a, fa = int(w.M[p]), int(w.M[:p].sum()), int(w.N[:p].sum())
        B = oracle.bopt.bopt_closed(w.x[p], M, 2.0, w.m)
        want = oracle.infft.infft_apply(B, c64(f[fa:fa + int(w.N[p])]))
        assert oracle.infft.rel_l2(out[a:a + M], want) <= FP32_TOL
    assert np.all(np.isfinite(out))
    b.close()
