"""Parity of the 2-D tensor-product form (through the C ABI) with the FP64 oracle
(oracle.infft2d).

Tolerances, as for the 1-D plan:
* pattern (integer work): bit-exact sets I(l) for every grid point;
* B_opt (fp64): every column's b attains the oracle's minimum of the regularised
  objective Phi_l = b^T (Re G + mu I) b - 2 Re r.b + 1 within 1e-12 relative (plus the
  rounding of evaluating Phi); b itself is ill-determined along near-null directions;
* fhat, fp32 path: rel l2 <= 1e-5 against the oracle's fp64 fhat on the same complex64
  input; fp64 path: rel l2 <= 1e-9 on data in the range of A.
The cases mix node families (radial spokes with a cluster at the origin, i.i.d.
uniform, a jittered tensor grid, nodes on grid lines and across the seam, duplicates),
both kernels, m = 1, 2 and 4, and column sizes across every solver tier (up to 32,
64 and 128 nodes in shared memory, one CTA per column up to 1024, many CTAs per column
above).  The full radial
workload (512 x 512 nodes, M = 256 x 256, m = 4) is checked on sampled columns,
including the 4726-node column at the origin, and on single-node data whose exact
fhat the oracle evaluates from the columns that node enters.
"""
import numpy as np
import pytest

from oracle import infft2d as o2
from oracle.infft import rel_l2
from workloads import radial, iid_uniform, jittered, complex_normal, trig_poly_eval_2d, make_2d

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
FP64_TOL = 1e-9
EPS = np.finfo(np.float64).eps


def edge_nodes():
    x = np.stack([iid_uniform(301, 120), iid_uniform(302, 120)], axis=1)
    x[0] = (0.25, -1.0 / 4.0)              # grid points of the 16 x 16 grid
    x[1] = (0.0, 0.0)
    x[2] = (-0.5, 0.5 - 1e-12)             # seam in both dimensions
    x[3] = (0.5 - 1e-15, -0.5)
    x[4] = x[5] = (0.1, 0.2)               # exact duplicates
    x[6] = (0.1 + 1e-13, 0.2)
    return x


def cases():
    return {
        "radial_small": (radial(401, 32, 32, 1e-4), 16, 16, 2.0, 2, "full"),
        "uniform_sym": (np.stack([iid_uniform(402, 400), iid_uniform(403, 400)], axis=1), 8, 16, 2.0, 2, "sym"),
        "jitter_grid_m1": (np.stack(np.meshgrid(jittered(404, 40), jittered(405, 20), indexing="ij"),
                                    -1).reshape(-1, 2), 16, 8, 2.0, 1, "full"),
        "edge": (edge_nodes(), 8, 8, 2.0, 2, "full"),
        "radial_m4": (radial(406, 64, 64, 1e-4), 32, 32, 2.0, 4, "full"),
        "radial_sym_m4": (radial(407, 48, 48, 1e-4), 32, 16, 2.0, 3, "sym"),
        "radial_giant": (radial(408, 96, 64, 1e-4), 16, 16, 2.0, 3, "full"),
    }


_cache = {}


def solved(name):
    if name in _cache:
        return _cache[name]
    x, M1, M2, sigma, m, kernel = cases()[name]
    B = o2.bopt2_closed(x, M1, M2, sigma, m, kernel)
    fh = complex_normal(500 + len(name), M1 * M2).reshape(M1, M2)
    f = trig_poly_eval_2d(x, fh)
    _cache[name] = (x, M1, M2, sigma, m, kernel, B, f)
    return _cache[name]


def run_gpu2(x, f, M1, M2, sigma, m, kernel, z=False, tau=1e-12):
    import torch
    import paper_1811_05335_gb300 as g
    dev = torch.device("cuda:0")
    plan = g.infft2d_plan_create(M1, M2, len(x), sigma, m, kernel=kernel, tau=tau)
    g.infft2d_set_nodes(plan, torch.tensor(x, dtype=torch.float64, device=dev))
    g.infft2d_precompute(plan)
    ct = torch.complex128 if z else torch.complex64
    fd = torch.tensor(np.asarray(f), dtype=ct, device=dev)
    fhat = (g.infft2d_apply_z if z else g.infft2d_apply)(plan, fd)
    torch.cuda.synchronize()
    return plan, fhat.cpu().numpy().astype(np.complex128), g.infft2d_copy_plan_data(plan), g.infft2d_get_info(plan)


def gpu_column(data, p):
    s, e = int(data["col_offset"][p]), int(data["col_offset"][p + 1])
    node = data["col_node"][s:e].astype(np.int64)
    w = data["weights"][s:e] if "weights" in data else None
    return node, w


def excess2(data, x, M1, M2, Ms1, Ms2, kernel, cols, tau=1e-12):
    """Phi(b_gpu) - Phi(b_oracle), its tolerance, and |J_gpu - J(b_gpu)| over its tolerance."""
    mu = tau * o2.gram_diag2(M1, M2, Ms1, Ms2, kernel)
    out = []
    for p in cols:
        node, b = gpu_column(data, p)
        if len(node) == 0:
            assert data["objective"][p] == 1.0
            continue
        Greg, r = o2.column_system2(x, node, p, M1, M2, Ms1, Ms2, kernel, mu)
        bo = np.linalg.solve(Greg, r)
        phi = lambda c: c @ Greg @ c - 2 * r @ c + 1.0
        pg, po = phi(b), phi(bo)
        scale = np.abs(b) @ np.abs(Greg) @ np.abs(b) + 2 * np.abs(r * b).sum() + 1
        G = Greg - mu * np.eye(len(node))
        Jo = b @ G @ b - 2 * r @ b + 1.0
        jt = 64 * len(node) * EPS * scale + 1e-13
        out.append((pg - po, 1e-12 * abs(po) + 256 * EPS * scale, abs(data["objective"][p] - Jo) / jt))
    return np.array(out)


@pytest.mark.parametrize("name", list(cases()))
def test_pattern_bit_exact(name):
    x, M1, M2, sigma, m, kernel, B, f = solved(name)
    plan, _, data, info = run_gpu2(x, f, M1, M2, sigma, m, kernel)
    assert np.array_equal(np.diff(data["col_offset"].astype(np.int64)), np.diff(B.ptr))
    for p in range(B.Ms1 * B.Ms2):
        node, _ = gpu_column(data, p)
        assert np.array_equal(np.sort(node), B.idx[B.ptr[p]:B.ptr[p + 1]]), f"column {p}"
    assert info["nnz"] == len(B.idx) and info["max_column"] == np.diff(B.ptr).max()
    assert info["empty_columns"] == int((np.diff(B.ptr) == 0).sum())
    plan.close()


@pytest.mark.parametrize("name", list(cases()))
def test_bopt_attains_regularised_minimum(name):
    x, M1, M2, sigma, m, kernel, B, f = solved(name)
    plan, _, data, info = run_gpu2(x, f, M1, M2, sigma, m, kernel)
    ex = excess2(data, x, M1, M2, B.Ms1, B.Ms2, kernel, range(B.Ms1 * B.Ms2))
    assert np.all(np.abs(ex[:, 0]) <= ex[:, 1]), f"max |excess|/tol {np.max(np.abs(ex[:, 0]) / ex[:, 1]):.3g}"
    assert np.all(ex[:, 2] <= 1.0), f"max J mismatch / tol {ex[:, 2].max():.3g}"
    assert info["fallback_columns"] == 0 and info["unsupported_columns"] == 0
    assert info["large_columns"] == int((np.diff(B.ptr) > 128).sum())
    assert abs(info["objective"] - B.J.sum()) <= 1e-9 * B.J.sum() + 1e-9
    plan.close()


def test_large_tier_is_exercised():
    """The radial cases put columns above 128 nodes (one CTA each), columns spanning
    several panels and trailing tiles, and columns above 1024 nodes (many CTAs each)."""
    sizes = [np.diff(solved(n)[6].ptr).max() for n in ("radial_small", "radial_m4", "radial_sym_m4", "radial_giant")]
    assert sizes[0] > 128 and sizes[1] > 2 * 64 + 16 and sizes[2] > 128 and sizes[3] > 1024
    assert (np.diff(solved("radial_giant")[6].ptr) > 1024).sum() >= 20


@pytest.mark.parametrize("name", list(cases()))
def test_apply_fp32(name):
    x, M1, M2, sigma, m, kernel, B, f = solved(name)
    f32 = np.asarray(f, np.complex64).astype(np.complex128)
    plan, fhat, _, _ = run_gpu2(x, f32, M1, M2, sigma, m, kernel)
    err = rel_l2(fhat, o2.infft2_apply(B, f32))
    print(f"{name}: fp32 fhat rel l2 {err:.3e}")
    assert err <= FP32_TOL
    plan.close()


def test_spread_kinds_run_and_indexed():
    """The fp32 spread reads a column as 2m cell-row runs of sorted nodes unless a node of its
    box lies on a grid line (integer M_sigma,t x_t), which only the exact test of eq:set_xj
    decides: such columns go through node indices.  Both kinds meet in the "edge" case; the
    perturbed radial trajectory has none on a grid line."""
    for name, want_indexed in (("edge", True), ("radial_m4", False)):
        x, M1, M2, sigma, m, kernel, B, f = solved(name)
        plan, fhat, _, info = run_gpu2(x, np.asarray(f, np.complex64), M1, M2, sigma, m, kernel)
        assert (info["indexed_columns"] > 0) == want_indexed, (name, info["indexed_columns"])
        assert info["indexed_columns"] < B.Ms1 * B.Ms2
        plan.close()


def oracle_ambiguity(name):
    """How far the oracle's own fhat moves when its columns are solved by a second
    backward-stable method (Cholesky instead of LU) on the same closed-form systems:
    the radial clusters make Re G_l + mu I condition ~1e13, so b_l is determined only
    up to that conditioning and fhat up to the resulting spread."""
    import scipy.linalg as sl
    x, M1, M2, sigma, m, kernel, B, f = solved(name)
    mu = 1e-12 * o2.gram_diag2(M1, M2, B.Ms1, B.Ms2, kernel)
    b = np.zeros_like(B.b)
    for p in range(B.Ms1 * B.Ms2):
        s, e = B.ptr[p], B.ptr[p + 1]
        if e > s:
            G, r = o2.column_system2(x, B.idx[s:e], p, M1, M2, B.Ms1, B.Ms2, kernel, mu)
            b[s:e] = sl.cho_solve(sl.cho_factor(G, lower=True), r)
    alt = o2.BOpt2(B.M1, B.M2, B.Ms1, B.Ms2, B.N, B.m, B.kernel, B.tau, B.ptr, B.idx, b, B.J)
    return rel_l2(o2.infft2_apply(alt, f), o2.infft2_apply(B, f))


@pytest.mark.parametrize("name", list(cases()))
def test_apply_fp64(name):
    """fp64 path: rel l2 <= 1e-9, or 4x the oracle's own ambiguity where the clustered
    columns make that larger (as for i.i.d. nodes in one dimension)."""
    x, M1, M2, sigma, m, kernel, B, f = solved(name)
    plan, fhat, _, _ = run_gpu2(x, f, M1, M2, sigma, m, kernel, z=True)
    err = rel_l2(fhat, o2.infft2_apply(B, f))
    tol = max(FP64_TOL, 4 * oracle_ambiguity(name))
    print(f"{name}: fp64 fhat rel l2 {err:.3e} (tolerance {tol:.1e})")
    assert err <= tol
    plan.close()


def test_sym_kernel_zeroes_the_edge_frequencies():
    x, M1, M2, sigma, m, kernel, B, f = solved("uniform_sym")
    plan, fhat, _, _ = run_gpu2(x, f, M1, M2, sigma, m, kernel)
    assert np.all(fhat[0, :] == 0) and np.all(fhat[:, 0] == 0)
    plan.close()


@pytest.mark.parametrize("z", [False, True])
def test_equispaced_sigma1_is_exact(z):
    """sigma = 1 and nodes on the M1 x M2 grid: B_opt is the identity permutation and
    the apply inverts f = A fhat exactly (up to the arithmetic's rounding).  tau = 0:
    a regulariser would scale b by 1/(1 + tau)."""
    M1, M2 = 16, 8
    g1 = (np.arange(M1) - M1 // 2) / M1
    g2 = (np.arange(M2) - M2 // 2) / M2
    x = np.stack(np.meshgrid(g1, g2, indexing="ij"), -1).reshape(-1, 2)
    fh = complex_normal(611, M1 * M2).reshape(M1, M2)
    f = o2.nfft2_direct(x, fh)
    plan, fhat, data, info = run_gpu2(x, f, M1, M2, 1.0, 1, "full", z=z, tau=0.0)
    assert np.abs(data["objective"]).max() < 1e-13
    assert rel_l2(fhat, fh) <= (1e-13 if z else 1e-6)
    plan.close()


def test_host_pointers_match_device():
    import paper_1811_05335_gb300 as g
    x, M1, M2, sigma, m, kernel, B, f = solved("radial_small")
    plan, fhat, _, _ = run_gpu2(x, f, M1, M2, sigma, m, kernel)
    out = np.empty(M1 * M2, np.complex64)
    g.infft2d_apply(plan, np.asarray(f, np.complex64), out=out)
    assert np.array_equal(out.reshape(M1, M2).astype(np.complex128), fhat)
    host = g.infft2d_plan_create(M1, M2, len(x), sigma, m, kernel=kernel)
    g.infft2d_set_nodes(host, np.ascontiguousarray(x))
    g.infft2d_precompute(host)
    d1, d2 = g.infft2d_copy_plan_data(plan), g.infft2d_copy_plan_data(host)
    assert np.array_equal(d1["col_node"], d2["col_node"]) and np.array_equal(d1["weights"], d2["weights"])
    plan.close()
    host.close()


def test_errors():
    import torch
    import paper_1811_05335_gb300 as g
    with pytest.raises(g.InfftError):
        g.infft2d_plan_create(7, 8, 10)                      # odd M1
    with pytest.raises(g.InfftError):
        g.infft2d_plan_create(12, 8, 10)                     # M_sigma,1 = 24 not a power of two
    with pytest.raises(g.InfftError):
        g.infft2d_plan_create(2048, 8, 10)                   # M_sigma,1 = 4096 above 2048
    with pytest.raises(g.InfftError):
        g.infft2d_plan_create(8, 8, 10, m=8)                 # 2m >= M_sigma
    plan = g.infft2d_plan_create(8, 8, 3)
    with pytest.raises(g.InfftError):
        g.infft2d_precompute(plan)                           # before set_nodes
    with pytest.raises(g.InfftError):
        g.infft2d_set_nodes(plan, np.array([[0.0, 0.0], [0.5, 0.0], [0.1, 0.1]]))   # host check
    with pytest.raises(g.InfftError):                        # device check (counted by the kernel)
        g.infft2d_set_nodes(plan, torch.tensor([[0.0, 0.0], [0.1, float("nan")], [0.1, 0.1]],
                                               dtype=torch.float64, device="cuda:0"))
    with pytest.raises(g.InfftError):
        g.infft2d_apply(plan, np.zeros(3, np.complex64))     # before precompute
    plan.close()


@pytest.mark.slow
def test_mid_size_radial_dense_data():
    """128 spokes x 128 samples, M = 64 x 64, sigma = 2, m = 4 (columns up to 1187 nodes): fhat
    of dense trigonometric-polynomial data against the oracle's closed tier, every coefficient,
    in the fp32 path (1e-5) and the fp64 path (1e-9)."""
    x = radial(409, 128, 128, 1e-4)
    M1 = M2 = 64
    B = o2.bopt2_closed(x, M1, M2, 2.0, 4, "full")
    fh = complex_normal(909, M1 * M2).reshape(M1, M2)
    f = trig_poly_eval_2d(x, fh)
    f32 = np.asarray(f, np.complex64).astype(np.complex128)
    plan, fhat, data, info = run_gpu2(x, f32, M1, M2, 2.0, 4, "full")
    assert info["max_column"] == np.diff(B.ptr).max() and info["fallback_columns"] == 0
    err32 = rel_l2(fhat, o2.infft2_apply(B, f32))
    plan.close()
    plan, fhat64, _, _ = run_gpu2(x, f, M1, M2, 2.0, 4, "full", z=True)
    err64 = rel_l2(fhat64, o2.infft2_apply(B, f))
    plan.close()
    print(f"radial 128 x 128, M = 64 x 64: rel l2 vs oracle fp32 {err32:.3e}, fp64 {err64:.3e}")
    assert err32 <= FP32_TOL and err64 <= FP64_TOL


def test_full_size_radial_sampled():
    """The full 2-D workload: 512 spokes x 512 samples, M = 256 x 256, sigma = 2, m = 4."""
    import torch
    import paper_1811_05335_gb300 as g
    w = make_2d()
    Ms = 512
    dev = torch.device("cuda:0")
    plan = g.infft2d_plan_create(w.M1, w.M2, w.N, 2.0, w.m)
    g.infft2d_set_nodes(plan, torch.tensor(w.x, dtype=torch.float64, device=dev))
    g.infft2d_precompute(plan)
    info = g.infft2d_get_info(plan)
    print({k: info[k] for k in ("nnz", "max_column", "empty_columns", "large_columns", "wide_columns",
                                "fallback_columns", "objective")})
    assert info["unsupported_columns"] == 0 and info["fallback_columns"] == 0
    assert info["nnz"] == 64 * w.N and info["max_column"] == 4726
    data = g.infft2d_copy_plan_data(plan)
    rng = np.random.default_rng(8)
    centre = (Ms // 2) * Ms + Ms // 2
    cols = [centre, centre + 1, centre - Ms + 3, 0, Ms - 1, (Ms // 2 + 40) * Ms + Ms // 2 - 17]
    cols += list(rng.integers(0, Ms * Ms, 24))
    for p in cols:
        node, _ = gpu_column(data, p)
        assert np.array_equal(np.sort(node), o2.column_nodes2(w.x, p, Ms, Ms, w.m)), f"column {p}"
    ex = excess2(data, w.x, w.M1, w.M2, Ms, Ms, "full", cols)
    assert np.all(np.abs(ex[:, 0]) <= ex[:, 1]) and np.all(ex[:, 2] <= 1.0)
    # single-node data f = e_j: the whole path against the oracle's exact response of that
    # node.  Such data is not in the range of A, so it pins fhat only where b_l is well
    # determined: nodes near the rim of the disc, whose columns the oracle finds to have
    # condition below 1e9 (inside radius ~150 cells the spokes crowd every box and
    # Re G_l + mu I reaches 1e12 - 1e13; there the sampled columns above pin B_opt).
    r = np.hypot(w.x[:, 0], w.x[:, 1]) * Ms
    mu = 1e-12 * o2.gram_diag2(w.M1, w.M2, Ms, Ms, "full")
    picks = [int(np.argmin(np.abs(r - rad))) for rad in (200.0, 240.0, 254.0)]
    for j in picks:
        lo1, hi1, lo2, hi2 = o2.node_boxes(w.x[j:j + 1], Ms, Ms, w.m)
        for a1 in range(lo1[0], hi1[0] + 1):
            for a2 in range(lo2[0], hi2[0] + 1):
                p = ((a1 + Ms // 2) % Ms) * Ms + (a2 + Ms // 2) % Ms
                G, _ = o2.column_system2(w.x, o2.column_nodes2(w.x, p, Ms, Ms, w.m), p, w.M1, w.M2, Ms, Ms, "full", mu)
                assert np.linalg.cond(G) < 1e9
        e = torch.zeros(w.N, dtype=torch.complex64, device=dev)
        e[j] = 1.0
        fhat = g.infft2d_apply(plan, e).cpu().numpy().astype(np.complex128)
        want = o2.infft2_apply_impulse(w.x, j, w.M1, w.M2, 2.0, w.m)
        err = rel_l2(fhat, want)
        print(f"node {j} (radius {r[j]:.1f} cells): rel l2 {err:.2e}")
        assert err <= FP32_TOL
    # data of a trigonometric polynomial: reconstruction error reported, not asserted
    fh = complex_normal(777, w.M1 * w.M2).reshape(w.M1, w.M2)
    f = torch.tensor(trig_poly_eval_2d(w.x, fh), dtype=torch.complex64, device=dev)
    out = g.infft2d_apply(plan, f).cpu().numpy()
    assert np.all(np.isfinite(out))
    print(f"radial 512 x 512: reconstruction rel l2 vs the true coefficients {rel_l2(out, fh):.3e}")
    plan.close()
