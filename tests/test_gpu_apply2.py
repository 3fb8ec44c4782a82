"""The two-launch fp32 apply (spreading fused with pass A of the four-step FFT, then pass B
with D^*, eq:approx_ansatz2) through the C ABI, against the FP64 oracle.

* every tile shape valid at the plan's M_sigma: fhat within rel l2 1e-5 of the oracle's on
  the same complex64 input (the shapes differ only in the FFT split, so in rounding);
* node families whose tiles do not fit the staging buffers (clustered Chebyshev nodes) and
  columns that spread in float-float (||b_l||_1 > 32): the same tolerance;
* samples given in sorted node order (infft_apply_sorted, infft_sort_values): the same bits
  as infft_apply;
* the early reads of plan data (before the wait on the previous kernel): applies on two
  plans back to back, and an apply right after a new set_nodes + precompute of the same
  plan, give the bits of isolated applies;
* the tuner (infft_tune_apply) picks a valid shape and leaves the result within tolerance.
"""
import numpy as np
import pytest

import oracle
from workloads import make_problem, iid_uniform, chebyshev_jittered, complex_normal, trig_poly_eval

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


def c64(a):
    return np.asarray(a, np.complex64).astype(np.complex128)


def make_plan(x, M, m, sigma=2.0, kernel="full"):
    import torch
    import paper_1811_05335_gb300 as g
    plan = g.infft_plan_create(M, len(x), sigma, m, kernel=kernel)
    g.infft_set_nodes(plan, torch.tensor(x, dtype=torch.float64, device="cuda:0"))
    g.infft_precompute(plan)
    return plan


def cases():
    out = {}
    p = make_problem(2, M=4096, N=16384, m=4)
    out["jit_m4"] = (p.x, p.f, p.M, 4, 2.0, "full")                  # M_sigma = 8192
    p = make_problem(2, M=8192, N=32768, m=6)
    out["jit_m6_sym"] = (p.x, p.f, p.M, 6, 2.0, "sym")                # M_sigma = 16384
    p = make_problem(2, M=2048, N=8192, m=8)
    out["jit_m8"] = (p.x, p.f, p.M, 8, 2.0, "full")                   # M_sigma = 4096, 256-point tiles
    p = make_problem(5, M=4096, N=16384, m=4)
    out["iid_m4"] = (p.x, p.f, p.M, 4, 2.0, "full")                   # mixed column sizes
    x = chebyshev_jittered(21, 6144)
    out["cheb"] = (x, trig_poly_eval(x, complex_normal(22, 2048)), 2048, 3, 2.0, "full")  # clustered ends
    p = make_problem(5, M=4096, N=8192, m=4)
    out["iid_wide"] = (p.x, p.f, p.M, 4, 2.0, "full")                  # N = 2M: ~2000 wide columns
    x = iid_uniform(26, 32768)                                          # sigma = 1, 8 nodes per cell: the
    out["dense_sigma1"] = (x, trig_poly_eval(x, complex_normal(27, 4096)), 4096, 2, 1.0, "full")  # tiles overflow
    x = iid_uniform(23, 9001)
    out["ragged"] = (x, trig_poly_eval(x, complex_normal(24, 4096)), 4096, 3, 2.0, "full")  # N ragged
    return out


_cache = {}


def solved(name):
    if name not in _cache:
        x, f, M, m, sigma, kernel = cases()[name]
        B = oracle.bopt.bopt_closed(x, M, sigma, m, kernel)
        _cache[name] = (x, f, M, m, sigma, kernel, B, oracle.infft.infft_apply(B, c64(f)))
    return _cache[name]


@pytest.mark.parametrize("name", list(cases()))
def test_every_tile_shape_matches_oracle(name):
    import torch
    import paper_1811_05335_gb300 as g
    x, f, M, m, sigma, kernel, B, want = solved(name)
    plan = make_plan(x, M, m, sigma, kernel)
    info = g.infft_get_info(plan)
    assert info["fallback_columns"] == 0 and info["unsupported_columns"] == 0
    assert g.infft_get_apply_config(plan) >= 0
    fd = torch.tensor(np.asarray(f, np.complex64), device="cuda:0")
    tried = 0
    for cid, shape in enumerate(g.infft_apply_configs()):
        log1, C = shape
        log2 = plan.M_sigma.bit_length() - 1 - log1
        if not (6 <= log2 <= 12 and (1 << log2) >= C):
            with pytest.raises(g.InfftError):
                g.infft_set_apply_config(plan, cid)
            continue
        g.infft_set_apply_config(plan, cid)
        assert g.infft_get_apply_config(plan) == cid
        got = g.infft_apply(plan, fd).cpu().numpy().astype(np.complex128)
        err = oracle.infft.rel_l2(got, want)
        print(f"{name}: shape {shape}: rel l2 {err:.3e}")
        assert err <= FP32_TOL, f"{name} shape {shape}: {err:.3e}"
        tried += 1
    assert tried >= 2
    plan.close()


def test_float_float_and_overflow_cases_are_exercised():
    """The i.i.d. N = 2M case has wide columns (spread in float-float; ||b_l||_1 reaches 1e5),
    and the sigma = 1 case's tiles exceed the staging buffers (every column by direct loads)."""
    B = solved("iid_wide")[6]
    l1 = np.add.reduceat(np.abs(B.b), B.ptr[:-1][np.diff(B.ptr) > 0])
    assert (l1 > 32).sum() > 1000
    B = solved("dense_sigma1")[6]
    assert len(B.idx) / (B.Ms / 512) > 8192     # weights per 512-point tile above the staging size


def test_sorted_input_gives_the_same_bits():
    import torch
    import paper_1811_05335_gb300 as g
    for name in ("jit_m4", "iid_wide", "dense_sigma1"):
        x, f, M, m, sigma, kernel, B, want = solved(name)
        plan = make_plan(x, M, m, sigma, kernel)
        fd = torch.tensor(np.asarray(f, np.complex64), device="cuda:0")
        one = g.infft_apply(plan, fd)
        fs = g.infft_sort_values(plan, fd)
        perm = g.infft_copy_plan_data(plan, weights=False)["perm"].astype(np.int64)
        assert np.array_equal(fs.cpu().numpy(), np.asarray(f, np.complex64)[perm])
        two = g.infft_apply_sorted(plan, fs)
        assert torch.equal(one, two), name
        plan.close()


def test_back_to_back_applies_and_replanning():
    """Applies alternate between two plans without synchronisation, and one plan gets new
    nodes and a new B_opt between applies: every result equals the isolated apply's."""
    import torch
    import paper_1811_05335_gb300 as g
    xa, fa, M, m = solved("jit_m4")[:4]
    xb, fb = solved("iid_m4")[:2]
    pa, pb = make_plan(xa, M, m), make_plan(xb, M, m)
    ta = torch.tensor(np.asarray(fa, np.complex64), device="cuda:0")
    tb = torch.tensor(np.asarray(fb, np.complex64), device="cuda:0")
    ref_a = g.infft_apply(pa, ta).clone()
    ref_b = g.infft_apply(pb, tb).clone()
    torch.cuda.synchronize()
    outs = []
    for _ in range(5):
        outs.append(g.infft_apply(pa, ta))
        outs.append(g.infft_apply(pb, tb))
    torch.cuda.synchronize()
    for i, o in enumerate(outs):
        assert torch.equal(o, ref_a if i % 2 == 0 else ref_b)
    # replan pa onto pb's nodes in the stream right behind an apply: the next apply must see
    # the new B_opt
    g.infft_apply(pa, ta)
    g.infft_set_nodes(pa, torch.tensor(xb, dtype=torch.float64, device="cuda:0"))
    g.infft_precompute(pa)
    got = g.infft_apply(pa, tb)
    torch.cuda.synchronize()
    assert torch.equal(got, ref_b)
    pa.close()
    pb.close()


def test_tuner_picks_a_valid_shape():
    import torch
    import paper_1811_05335_gb300 as g
    x, f, M, m, sigma, kernel, B, want = solved("jit_m4")
    plan = make_plan(x, M, m)
    best, ms = g.infft_tune_apply(plan, repeats=5)
    print("tile shape times (ms):", ms, "best", best)
    assert best >= 0 and ms[best] > 0 and ms[best] == min(t for t in ms if t > 0)
    assert g.infft_get_apply_config(plan) == best
    got = g.infft_apply(plan, torch.tensor(np.asarray(f, np.complex64), device="cuda:0"))
    assert oracle.infft.rel_l2(got.cpu().numpy().astype(np.complex128), want) <= FP32_TOL
    plan.close()
