"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances:
* pattern (integer work): bit-exact sets I(l);
* B_opt (fp64): every column's b attains the oracle's unique minimum of the regularised
  objective Phi_l within 1e-12 relative (plus evaluation rounding); b itself is not
  compared, because the normal matrix has condition ~ 1/tau and b is ill-determined
  along near-null directions of L_l that do not affect fhat for data in range(A);
* fhat, fp32 path: rel l2 <= 1e-5 against the oracle's fp64 fhat on the same complex64
  input values (the fp32 path's input is complex64; rounding the data itself moves
  fhat by up to ~2e-5 on i.i.d. uniform nodes, where ||b_l||_1 reaches 1e4);
* fhat, fp64 path: rel l2 <= 1e-9, the bound that the fp64 solve supports:
  eps / (2 sqrt(mu)) ~ 7e-11 with mu = tau/sigma, tau = 1e-12 (times a margin); on
  i.i.d. uniform nodes with N = 2M, 4x the disagreement of the oracle's two tiers;
* nfft_apply (B_opt F D): adjoint identity with infft_apply on random probes (1e-5 fp32,
  1e-11 fp64), element-wise oracle parity where B_opt is well determined (sigma = 1
  equispaced), and fp32 = fp64 on the same B_opt.
"""
import numpy as np
import pytest

import oracle
from workloads import make_problem, jittered, iid_uniform, chebyshev_jittered, complex_normal, trig_poly_eval
from gpu_support import run_gpu, assert_pattern_equal, regularised_excess

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
FP64_TOL = 1e-9


def problem(name):
    if name == "cfg1":
        p = make_problem(1)
        return p.x, p.f, p.M, 2.0, p.m, "full"
    if name == "jit_small":          # M_sigma = 2048: single-CTA FFT
        p = make_problem(2, M=1024, N=4096, m=4)
        return p.x, p.f, p.M, 2.0, 4, "full"
    if name == "jit_fourstep":       # M_sigma = 8192: four-step FFT; |I(l)| = 25: group tier
        p = make_problem(2, M=4096, N=16384, m=6)
        return p.x, p.f, p.M, 2.0, 6, "full"
    if name == "jit_m8":             # |I(l)| = 33: group tier, 4 lanes per column
        p = make_problem(2, M=2048, N=8192, m=8)
        return p.x, p.f, p.M, 2.0, 8, "full"
    if name == "unif_m4":            # i.i.d. uniform nodes: column sizes mixed within tiles, every tier
        p = make_problem(5, M=2048, N=8192, m=4)
        return p.x, p.f, p.M, 2.0, 4, "full"
    if name == "cheb":               # |I(l)| up to ~86: CTA tier
        x = chebyshev_jittered(11, 768)
        fh = complex_normal(12, 256)
        return x, trig_poly_eval(x, fh), 256, 2.0, 4, "full"
    if name == "cheb_big":           # |I(l)| up to ~212: CTA tier, packed storage
        x = chebyshev_jittered(13, 3072)
        fh = complex_normal(14, 1024)
        return x, trig_poly_eval(x, fh), 1024, 2.0, 6, "full"
    if name == "ragged":             # N = 3001: two sort tiles and a ragged tail
        x = iid_uniform(15, 3001)
        fh = complex_normal(16, 512)
        return x, trig_poly_eval(x, fh), 512, 2.0, 3, "full"
    if name == "sigma1":             # M_sigma = M
        x = jittered(17, 1024)
        fh = complex_normal(18, 256)
        return x, trig_poly_eval(x, fh), 256, 1.0, 2, "full"
    if name == "sym":
        p = make_problem(2, M=512, N=2048, m=4)
        return p.x, p.f, p.M, 2.0, 4, "sym"
    raise KeyError(name)


CASES = ["cfg1", "jit_small", "jit_fourstep", "jit_m8", "unif_m4", "cheb", "cheb_big", "ragged", "sigma1", "sym"]
_cache = {}


def c64(a):
    """The complex64 values the fp32 path receives, as exact complex128."""
    return np.asarray(a, np.complex64).astype(np.complex128)


def solved(name):
    if name not in _cache:
        x, f, M, sigma, m, kernel = problem(name)
        B = oracle.bopt.bopt_closed(x, M, sigma, m, kernel)
        ghat = complex_normal(99, M)
        gpu = run_gpu(x, f, M, sigma, m, kernel, fhat_in=ghat)
        _cache[name] = (x, f, M, sigma, m, kernel, B, ghat, gpu)
    return _cache[name]


@pytest.mark.parametrize("name", CASES)
def test_pattern_bit_exact(name):
    x, f, M, sigma, m, kernel, B, ghat, (plan, fhat, back, data, info) = solved(name)
    assert_pattern_equal(data, B)
    assert info["nnz"] == len(B.idx)
    assert info["max_column"] == int(np.diff(B.ptr).max())
    assert info["empty_columns"] == int((np.diff(B.ptr) == 0).sum())
    assert info["bad_nodes"] == 0


@pytest.mark.parametrize("name", CASES)
def test_bopt_attains_regularised_minimum(name):
    x, f, M, sigma, m, kernel, B, ghat, (plan, fhat, back, data, info) = solved(name)
    assert info["fallback_columns"] == 0 and info["unsupported_columns"] == 0
    excess, tol, jdiff = regularised_excess(data, x, M, B.Ms, kernel, 1e-12)
    assert np.all(excess <= tol), f"max excess/tol {np.max(excess / tol):.3g}"
    assert np.all(excess >= -tol)
    assert np.all(jdiff <= 1.0), f"max J mismatch / tol {jdiff.max():.3g}"
    assert abs(info["objective"] - B.J.sum()) <= 1e-9 * B.J.sum() + 1e-9


@pytest.mark.parametrize("name", CASES)
def test_infft_apply_fp32(name):
    x, f, M, sigma, m, kernel, B, ghat, (plan, fhat, back, data, info) = solved(name)
    want = oracle.infft.infft_apply(B, c64(f))
    err = oracle.infft.rel_l2(fhat, want)
    assert err <= FP32_TOL, f"{name}: rel l2 {err:.3e}"


def run_probes(name, z, k=6):
    """Adjoint-identity probes: <infft_apply(f_r), g_r> vs <f_r, nfft_apply(g_r)> on the GPU."""
    import torch
    import paper_1811_05335_gb300 as g
    x, f, M, sigma, m, kernel, B, ghat, _ = solved(name)
    dev = torch.device("cuda:0")
    ct = torch.complex128 if z else torch.complex64
    plan = g.infft_plan_create(M, len(x), sigma, m, kernel=kernel)
    g.infft_set_nodes(plan, torch.tensor(x, dtype=torch.float64, device=dev))
    g.infft_precompute(plan)
    apply, nfft = (g.infft_apply_z, g.nfft_apply_z) if z else (g.infft_apply, g.nfft_apply)
    errs = []
    for r in range(k):
        fr = torch.tensor(complex_normal(1000 + r, len(x)), dtype=ct, device=dev)
        gr = torch.tensor(complex_normal(2000 + r, M), dtype=ct, device=dev)
        a = torch.vdot(gr, apply(plan, fr)).item()
        b = torch.vdot(nfft(plan, gr), fr).item()
        scale = (torch.linalg.vector_norm(apply(plan, fr)) * torch.linalg.vector_norm(gr)).item()
        errs.append(abs(a - b) / scale)
    plan.close()
    return max(errs)


@pytest.mark.parametrize("name", CASES)
def test_nfft_apply_is_adjoint_fp32(name):
    """B_opt F D is the exact adjoint of D^* F^* B_opt^* (Remark remark:ansatz2_adj), probed
    with random vectors.  nfft_apply is not compared element by element with the oracle:
    it applies the weights b_l directly, and b_l is determined only to ~eps/mu along
    near-null directions of L_l (see test_bopt_attains_regularised_minimum), which
    infft_apply never sees for data in range(A) but nfft_apply does."""
    assert run_probes(name, z=False) <= 1e-5


@pytest.mark.parametrize("name", ["cfg1", "jit_small", "jit_fourstep", "cheb", "sym"])
def test_nfft_apply_is_adjoint_fp64(name):
    assert run_probes(name, z=True) <= 1e-11


@pytest.mark.parametrize("M,z", [(256, False), (256, True), (4096, False), (4096, True)])
def test_nfft_apply_equispaced_elementwise(M, z):
    """sigma = 1, M = N, x_j = j/M: Re G_l = I, so B_opt is well determined (= I/(1+tau))
    and nfft_apply matches the oracle element by element."""
    from workloads import equispaced
    x = equispaced(M)
    ghat = complex_normal(31, M)
    B = oracle.bopt.bopt_closed(x, M, 1.0, 2)
    _, _, back, _, info = run_gpu(x, complex_normal(32, M), M, 1.0, 2, fhat_in=ghat, z=z)
    want = oracle.infft.nfft_apply(B, ghat if z else c64(ghat))
    assert oracle.infft.rel_l2(back, want) <= (FP64_TOL if z else FP32_TOL)


@pytest.mark.parametrize("name", ["cfg1", "jit_small", "cheb"])
def test_nfft_fp32_matches_fp64(name):
    """Same (deterministic) B_opt: the fp32 adjoint equals the fp64 adjoint to fp32 rounding."""
    x, f, M, sigma, m, kernel, B, ghat, (plan, fhat, back, data, info) = solved(name)
    _, _, back64, _, _ = run_gpu(x, f, M, sigma, m, kernel, fhat_in=c64(ghat), z=True)
    assert oracle.infft.rel_l2(back, back64) <= FP32_TOL


@pytest.mark.parametrize("name", ["cfg1", "jit_small", "jit_fourstep", "sym"])
def test_adjoint_identity_gpu(name):
    """<infft_apply(f), g> = <f, nfft_apply(g)> with both sides computed on the GPU."""
    x, f, M, sigma, m, kernel, B, ghat, (plan, fhat, back, data, info) = solved(name)
    lhs = np.vdot(c64(ghat), fhat)
    rhs = np.vdot(back, c64(f))
    # fp32 rounding of an inner product is bounded by the norms of its factors, not by
    # the (possibly much smaller) result; on i.i.d. uniform nodes the weights cancel
    scale = np.linalg.norm(ghat) * np.linalg.norm(fhat) + np.linalg.norm(back) * np.linalg.norm(f)
    assert abs(lhs - rhs) <= 1e-5 * scale


@pytest.mark.parametrize("name", ["cfg1", "jit_small", "jit_fourstep", "cheb", "sym"])
def test_fp64_apply(name):
    x, f, M, sigma, m, kernel, B, ghat, _ = solved(name)
    plan, fhat, back, data, info = run_gpu(x, f, M, sigma, m, kernel, fhat_in=ghat, z=True)
    err = oracle.infft.rel_l2(fhat, oracle.infft.infft_apply(B, f))
    tol = FP64_TOL
    if name == "cfg1":
        # i.i.d. uniform nodes with N = 2M: columns are much worse conditioned
        # (||b_l||_1 up to 2.5e4); the bound is the oracle's own ambiguity, the
        # disagreement of its two exact tiers, times a margin of 4
        Bn = oracle.bopt.bopt_naive(x, M, sigma, m, kernel)
        amb = oracle.infft.rel_l2(oracle.infft.infft_apply(Bn, f, "direct"), oracle.infft.infft_apply(B, f))
        tol = max(tol, 4 * amb)
    print(f"{name}: fp64 fhat rel l2 {err:.3e} (tolerance {tol:.1e})")
    assert err <= tol


def test_host_pointers_match_device():
    """The e2e path (host arrays through the C ABI) gives the device path's bits."""
    import torch
    import paper_1811_05335_gb300 as g
    x, f, M, sigma, m, kernel, B, ghat, (plan, fhat, back, data, info) = solved("jit_small")
    plan2 = g.infft_plan(M, len(x), np.asarray(x), sigma, m)
    g.infft_precompute(plan2)
    out = g.infft_apply(plan2, np.asarray(f, dtype=np.complex64))
    assert isinstance(out, np.ndarray)
    assert np.array_equal(out.astype(np.complex128), fhat)
    plan2.close()


def test_deterministic():
    x, f, M, sigma, m, kernel, B, ghat, (plan, fhat, back, data, info) = solved("ragged")
    _, fhat2, back2, data2, _ = run_gpu(x, f, M, sigma, m, kernel, fhat_in=ghat)
    assert np.array_equal(fhat, fhat2) and np.array_equal(back, back2)
    assert np.array_equal(data["weights"], data2["weights"])


def test_reconstruction_quality_reported():
    """Ex. ex:trig_poly_ansatz2 setting: the GPU result is as close to the true
    coefficients as the oracle's (the paper prints no numbers to match)."""
    p = make_problem(2, M=1024, N=4096, m=4, noise_rel=0.0)
    B = oracle.bopt.bopt_closed(p.x, p.M, 2.0, 4)
    want = oracle.infft.infft_apply(B, p.f)
    _, fhat, _, _, _ = run_gpu(p.x, p.f, p.M, 2.0, 4)
    e_orc = oracle.infft.rel_l2(want, p.fhat)
    e_gpu = oracle.infft.rel_l2(fhat, p.fhat)
    print(f"rel l2 vs truth: oracle {e_orc:.3e}, gpu {e_gpu:.3e}")
    assert e_gpu <= e_orc + 2e-6


def test_empty_columns_and_duplicates():
    """Clustered nodes leave empty columns (J_l = 1); duplicated nodes make Re G_l
    singular, which the regularisation absorbs without fallback."""
    x = np.concatenate([np.full(8, 0.1), jittered(21, 64) * 0.2])
    x = np.where(x >= 0.5, x - 1, x)
    fh = complex_normal(22, 32)
    f = trig_poly_eval(x, fh)
    B = oracle.bopt.bopt_closed(x, 32, 2.0, 3)
    plan, fhat, back, data, info = run_gpu(x, f, 32, 2.0, 3)
    assert_pattern_equal(data, B)
    assert info["empty_columns"] > 0 and info["fallback_columns"] == 0
    assert np.all(data["objective"][data["col_count"] == 0] == 1.0)
    assert oracle.infft.rel_l2(fhat, oracle.infft.infft_apply(B, c64(f))) <= FP32_TOL


def test_boundary_nodes():
    """Nodes at -1/2, on grid points and one ulp beside them (pattern decided exactly)."""
    Ms = 64
    xs = [-0.5, np.nextafter(0.5, 0), 0.0]
    for l in (-31, -5, 1, 30):
        xs += [l / Ms, np.nextafter(l / Ms, 1), np.nextafter(l / Ms, -1)]
    x = np.concatenate([np.array(xs), iid_uniform(23, 100)])
    fh = complex_normal(24, 32)
    f = trig_poly_eval(x, fh)
    B = oracle.bopt.bopt_closed(x, 32, 2.0, 4)
    plan, fhat, back, data, info = run_gpu(x, f, 32, 2.0, 4)
    assert_pattern_equal(data, B)
    assert oracle.infft.rel_l2(fhat, oracle.infft.infft_apply(B, c64(f))) <= FP32_TOL


def test_single_node_and_smallest_sizes():
    x = np.array([0.123])
    plan, fhat, back, data, info = run_gpu(x, np.array([1 + 2j]), 2, 2.0, 1)
    B = oracle.bopt.bopt_closed(x, 2, 2.0, 1)
    assert_pattern_equal(data, B)
    assert oracle.infft.rel_l2(fhat, oracle.infft.infft_apply(B, np.array([1 + 2j]))) <= FP32_TOL


def test_errors_on_device():
    import torch
    import paper_1811_05335_gb300 as g
    plan = g.infft_plan_create(64, 16, 2.0, 2)
    f = torch.zeros(16, dtype=torch.complex64, device="cuda:0")
    with pytest.raises(g.InfftError) as ei:
        g.infft_apply(plan, f)
    assert ei.value.code == 4                     # ENOTREADY
    with pytest.raises(g.InfftError) as ei:
        g.infft_set_nodes(plan, np.full(16, 0.7))  # host nodes outside [-1/2, 1/2)
    assert ei.value.code == 1
    bad = torch.full((16,), float("nan"), dtype=torch.float64, device="cuda:0")
    g.infft_set_nodes(plan, bad)                   # device nodes: counted, not fatal
    assert g.infft_get_info(plan)["bad_nodes"] == 16
    plan.close()


@pytest.mark.slow
@pytest.mark.parametrize("m", [4, 6, 8])
def test_full_size_config2(m):
    """M = 2^16, N = 2^18 jittered nodes, 1e-8 noise, sigma = 2 (the benchmark's workload)."""
    p = make_problem(2, m=m)
    B = oracle.bopt.bopt_closed(p.x, p.M, 2.0, m)
    plan, fhat, back, data, info = run_gpu(p.x, p.f, p.M, 2.0, m)
    assert_pattern_equal(data, B)
    assert info["fallback_columns"] == 0 and info["unsupported_columns"] == 0
    rng = np.random.default_rng(m)
    cols = rng.choice(B.Ms, 4096, replace=False)
    excess, tol, jdiff = regularised_excess(data, p.x, p.M, B.Ms, "full", 1e-12, cols)
    assert np.all(np.abs(excess) <= tol) and np.all(jdiff <= 1.0)
    want = oracle.infft.infft_apply(B, c64(p.f))
    err = oracle.infft.rel_l2(fhat, want)
    print(f"config2 m={m}: fp32 rel l2 vs oracle {err:.3e}; vs truth {oracle.infft.rel_l2(fhat, p.fhat):.3e}")
    assert err <= FP32_TOL


def test_apply_many_equals_single_applies():
    """K data vectors in one call give, vector by vector, what infft_apply gives (to fp32
    rounding: spreading tiles and FFT split differ), and match the oracle."""
    import torch
    import paper_1811_05335_gb300 as g
    p = make_problem(2, M=4096, N=16384, m=4, with_data=False)
    dev = torch.device("cuda:0")
    plan = g.infft_plan_create(p.M, p.N, 2.0, 4)
    g.infft_set_nodes(plan, torch.tensor(p.x, dtype=torch.float64, device=dev))
    g.infft_precompute(plan)
    K = 5
    fs = np.stack([trig_poly_eval(p.x, complex_normal(200 + k, p.M)) for k in range(K)]).astype(np.complex64)
    ft = torch.tensor(fs, device=dev)
    many = g.infft_apply_many(plan, ft).cpu().numpy()
    B = oracle.bopt.bopt_closed(p.x, p.M, 2.0, 4)
    for k in range(K):
        one = g.infft_apply(plan, ft[k].contiguous()).cpu().numpy()
        assert np.linalg.norm(many[k] - one) <= 1e-6 * np.linalg.norm(one)
        assert oracle.infft.rel_l2(many[k].astype(np.complex128), oracle.infft.infft_apply(B, c64(fs[k]))) <= FP32_TOL
    with pytest.raises(g.InfftError):     # workspace too small
        g.infft_apply_many(plan, ft, workspace=torch.empty(16, dtype=torch.uint8, device=dev))
    small = g.infft_plan_create(64, 128, 2.0, 4)
    g.infft_set_nodes(small, torch.tensor(make_problem(1).x, dtype=torch.float64, device=dev))
    g.infft_precompute(small)
    with pytest.raises(g.InfftError):     # M_sigma <= 2048
        g.infft_apply_many(small, torch.zeros((2, 128), dtype=torch.complex64, device=dev))
    plan.close()
    small.close()
