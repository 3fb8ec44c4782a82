"""Single-problem plans whose oversampled grid M_sigma = 2M is not a power of two (Sec. 2.1
allows any even sigma M): the plan runs as a batch of one problem, the FFT a chirp convolution of
power-of-two length.  Through the C ABI against the FP64 oracle on the same seeded inputs:

* pattern (integer work): bit-exact index sets I(l);
* B_opt: every column at the oracle's minimum of the regularised objective (the single-problem
  tolerance);
* fhat, fp32 path: rel l2 <= 1e-5 against the oracle's fp64 fhat on the same complex64 input,
  from device and from host buffers;
* the calls such a plan lacks return INFFT_EUNSUPPORTED, and so do sizes it cannot take."""
import numpy as np
import pytest

import oracle
from workloads import jittered, iid_uniform, chebyshev_jittered, complex_normal, trig_poly_eval
from gpu_support import run_gpu, assert_pattern_equal, regularised_excess

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


def c64(a):
    return np.asarray(a, np.complex64).astype(np.complex128)


def cases():
    return {
        "jit_M3000": (jittered(61, 12000), 3000, 4, "full"),        # M_sigma = 6000
        "iid_M1500_sym": (iid_uniform(62, 4500), 1500, 3, "sym"),    # M_sigma = 3000
        "cheb_M8190": (chebyshev_jittered(63, 20000), 8190, 4, "full"),   # the largest M, two FFT halves
        "tiny_M6": (iid_uniform(64, 20), 6, 2, "full"),              # M_sigma = 12
    }


@pytest.mark.parametrize("name", list(cases()))
def test_nonpow2_plan_matches_oracle(name):
    x, M, m, kernel = cases()[name]
    f = trig_poly_eval(x, complex_normal(65, M))
    B = oracle.bopt.bopt_closed(x, M, 2.0, m, kernel)
    assert B.Ms & (B.Ms - 1) != 0
    plan, fhat, _, data, info = run_gpu(x, f, M, 2.0, m, kernel)
    assert plan.M_sigma == 2 * M
    assert_pattern_equal(data, B)
    assert info["fallback_columns"] == 0 and info["unsupported_columns"] == 0
    excess, tol, jdiff = regularised_excess(data, x, M, B.Ms, kernel, 1e-12)
    assert np.all(np.abs(excess) <= tol) and np.all(jdiff <= 1.0)
    want = oracle.infft.infft_apply(B, c64(f))
    err = oracle.infft.rel_l2(fhat, want)
    print(f"{name}: M_sigma = {B.Ms}: rel l2 vs oracle {err:.3e}")
    assert err <= FP32_TOL
    plan.close()


def test_nonpow2_host_buffers_and_unsupported_calls():
    import torch
    import paper_1811_05335_gb300 as g
    x, M, m, kernel = cases()["jit_M3000"]
    f = np.asarray(trig_poly_eval(x, complex_normal(66, M)), np.complex64)
    plan = g.infft_plan(M, len(x), np.asarray(x), 2.0, m)        # host nodes
    g.infft_precompute(plan)
    out_host = g.infft_apply(plan, f)                              # host data and result
    out_dev = g.infft_apply(plan, torch.tensor(f, device="cuda:0")).cpu().numpy()
    assert np.array_equal(out_host, out_dev)
    dev = torch.zeros(len(x), dtype=torch.complex64, device="cuda:0")
    for call in (lambda: g.infft_apply_z(plan, dev.to(torch.complex128)),
                 lambda: g.nfft_apply(plan, torch.zeros(M, dtype=torch.complex64, device="cuda:0")),
                 lambda: g.infft_tune_apply(plan),
                 lambda: g.infft_grad_nodes(plan, dev, torch.zeros(M, dtype=torch.complex64, device="cuda:0"))):
        with pytest.raises(g.InfftError) as ei:
            call()
        assert ei.value.code == 5
    assert g.infft_get_apply_config(plan) == -1
    plan.close()
    with pytest.raises(g.InfftError) as ei:                       # sigma != 2 with a non-power-of-two grid
        g.infft_plan_create(1000, 4000, 1.5, 4)
    assert ei.value.code == 5
    with pytest.raises(g.InfftError) as ei:                       # M above the chirp FFT's 8192
        g.infft_plan_create(8194, 20000, 2.0, 4)
    assert ei.value.code == 5
