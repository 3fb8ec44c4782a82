"""The fp64 direct sum f = A fhat (infft_ndft_z) and the residual-correction sweep
fhat <- fhat + D^* F^* B_opt^* (f - A fhat) (infft_refine_z) against the oracle
(oracle.nfft.nfft_direct, oracle.infft.refine).

Tolerances: the direct sum is exact up to fp64 rounding (rel l2 <= 1e-13; the rotation
restarts every 32 frequencies); so is the windowed NFFT that the sweep uses for sigma >= 2
(Kaiser-Bessel, 25 grid points: truncation error far below rounding; rel l2 <= 1e-13).  The sweep's result is compared through its error against
the true coefficients, which is what the iteration fixes: on jittered nodes (N = 4M) both the
GPU and the oracle reach ~1e-14 after one sweep; on i.i.d. nodes (N = 2M, a slow contraction)
the GPU's error tracks the oracle's to 1e-6 (the fp64 apply's ambiguity is 1e-9).
"""
import numpy as np
import pytest

import oracle
from workloads import jittered, iid_uniform, complex_normal, trig_poly_eval

pytestmark = pytest.mark.gpu


def plan_for(x, M, m=4, ansatz="over"):
    import torch
    import paper_1811_05335_gb300 as g
    p = g.infft_plan_create_ansatz(M, len(x), 2.0, m, ansatz=ansatz)
    g.infft_set_nodes(p, torch.tensor(x, dtype=torch.float64, device="cuda:0"))
    g.infft_precompute(p)
    return p


@pytest.mark.parametrize("M,N,fam", [(64, 128, "unif"), (1024, 4096, "jit"), (32, 100, "unif")])
def test_ndft_matches_direct_sum(M, N, fam):
    import torch
    import paper_1811_05335_gb300 as g
    x = iid_uniform(701, N) if fam == "unif" else jittered(701, N)
    fh = complex_normal(702, M)
    p = plan_for(x, M, m=2)
    f = g.infft_ndft_z(p, torch.tensor(fh, dtype=torch.complex128, device="cuda:0")).cpu().numpy()
    err = oracle.infft.rel_l2(f, oracle.nfft.nfft_direct(x, fh))
    print(f"ndft M={M} N={N}: rel l2 {err:.2e}")
    assert err <= 1e-13
    p.close()


def test_ndft_large_sampled():
    """M = 2^14, N = 2^16: 256 sampled nodes against the oracle's sum at those nodes (phases
    reduced exactly: the plain sum's angles k x lose ~1e-11 at this M)."""
    import torch
    import paper_1811_05335_gb300 as g
    M, N = 1 << 14, 1 << 16
    x = iid_uniform(703, N)
    fh = complex_normal(704, M)
    p = plan_for(x, M, m=2)
    f = g.infft_ndft_z(p, torch.tensor(fh, dtype=torch.complex128, device="cuda:0")).cpu().numpy()
    idx = np.random.default_rng(5).choice(N, 256, replace=False)
    want = oracle.nfft.nfft_direct_reduced(x[idx], fh)
    assert oracle.infft.rel_l2(f[idx], want) <= 1e-13
    p.close()


@pytest.mark.parametrize("M,N,fam", [(64, 128, "unif"), (1024, 4096, "jit"), (512, 700, "unif")])
def test_nfft_kb_matches_direct_sum(M, N, fam):
    """The windowed NFFT (Sec. 2.1, Kaiser-Bessel, 25 grid points per node) within 1e-13 of the sum."""
    import torch
    import paper_1811_05335_gb300 as g
    x = iid_uniform(721, N) if fam == "unif" else jittered(721, N)
    fh = complex_normal(722, M)
    p = plan_for(x, M, m=2)
    f = g.infft_nfft_kb_z(p, torch.tensor(fh, dtype=torch.complex128, device="cuda:0")).cpu().numpy()
    err = oracle.infft.rel_l2(f, oracle.nfft.nfft_direct(x, fh))
    print(f"nfft_kb M={M} N={N}: rel l2 {err:.2e}")
    assert err <= 1e-13
    p.close()


def test_nfft_kb_large_sampled_and_unsupported():
    import torch
    import paper_1811_05335_gb300 as g
    M, N = 1 << 16, 1 << 18
    x = jittered(723, N)
    fh = complex_normal(724, M)
    p = plan_for(x, M, m=2)
    f = g.infft_nfft_kb_z(p, torch.tensor(fh, dtype=torch.complex128, device="cuda:0")).cpu().numpy()
    idx = np.random.default_rng(6).choice(N, 128, replace=False)
    assert oracle.infft.rel_l2(f[idx], oracle.nfft.nfft_direct_reduced(x[idx], fh)) <= 1e-13
    p.close()
    q = g.infft_plan_create(64, 64, 1.0, 2)                 # sigma = 1: the window needs oversampling
    g.infft_set_nodes(q, torch.tensor(jittered(725, 64), dtype=torch.float64, device="cuda:0"))
    with pytest.raises(g.InfftError):
        g.infft_nfft_kb_z(q, torch.zeros(64, dtype=torch.complex128, device="cuda:0"))
    q.close()


def test_refine_reaches_fp64_on_jittered_nodes():
    import torch
    import paper_1811_05335_gb300 as g
    M, N = 256, 1024
    x = jittered(705, N)
    fh = complex_normal(706, M)
    f = oracle.nfft.nfft_direct(x, fh)
    p = plan_for(x, M)
    fd = torch.tensor(f, dtype=torch.complex128, device="cuda:0")
    est = g.infft_apply_z(p, fd)
    e = [oracle.infft.rel_l2(est.cpu().numpy(), fh)]
    for _ in range(2):
        g.infft_refine_z(p, fd, est, 1)
        e.append(oracle.infft.rel_l2(est.cpu().numpy(), fh))
    B = oracle.bopt.bopt_closed(x, M, 2.0, 4)
    eo = [oracle.infft.rel_l2(oracle.infft.refine(B, x, f, oracle.infft.infft_apply(B, f), k), fh) for k in range(3)]
    print("GPU errors", e, "oracle errors", eo)
    assert 1e-9 < e[0] < 1e-5
    assert e[1] <= 10 * eo[1] + 1e-13 and e[1] < 1e-12
    assert e[2] <= 1e-13          # the floor: the windowed NFFT's and the apply's fp64 rounding


def test_refine_tracks_the_oracle_on_iid_nodes():
    """Configuration-1 nodes (i.i.d., N = 2M): a slow contraction; the GPU's error after each
    sweep equals the oracle's."""
    import torch
    import paper_1811_05335_gb300 as g
    M, N = 64, 128
    x = iid_uniform(707, N)
    fh = complex_normal(708, M)
    f = oracle.nfft.nfft_direct(x, fh)
    p = plan_for(x, M)
    fd = torch.tensor(f, dtype=torch.complex128, device="cuda:0")
    est = g.infft_apply_z(p, fd)
    B = oracle.bopt.bopt_closed(x, M, 2.0, 4)
    f0 = oracle.infft.infft_apply(B, f)
    for k in (1, 2, 3):
        g.infft_refine_z(p, fd, est, 1)
        eg = oracle.infft.rel_l2(est.cpu().numpy(), fh)
        eo = oracle.infft.rel_l2(oracle.infft.refine(B, x, f, f0, k), fh)
        print(k, eg, eo)
        assert abs(eg - eo) <= 1e-6 * eo + 1e-12


def test_refine_mid_size():
    """M = 2^12, N = 2^14 jittered nodes, m = 4: one sweep from ~1e-7 to below 1e-12."""
    import torch
    import paper_1811_05335_gb300 as g
    M, N = 1 << 12, 1 << 14
    x = jittered(709, N)
    fh = complex_normal(710, M)
    f = trig_poly_eval(x, fh)
    p = plan_for(x, M)
    fd = torch.tensor(f, dtype=torch.complex128, device="cuda:0")
    est = g.infft_apply_z(p, fd)
    e0 = oracle.infft.rel_l2(est.cpu().numpy(), fh)
    g.infft_refine_z(p, fd, est, 2)
    e2 = oracle.infft.rel_l2(est.cpu().numpy(), fh)
    print(f"M=2^12: {e0:.2e} -> {e2:.2e}")
    assert e0 > 1e-9 and e2 < 1e-12


def test_refine_underdetermined_reduces_the_residual():
    """Underdetermined plan (M = 4N): the sweep lowers ||f - A fhat|| in data space."""
    import torch
    import paper_1811_05335_gb300 as g
    N, M = 256, 1024
    x = jittered(711, N)
    fh = complex_normal(712, M)
    f = oracle.nfft.nfft_direct(x, fh)
    p = plan_for(x, M, ansatz="under")
    fd = torch.tensor(f, dtype=torch.complex128, device="cuda:0")
    est = g.infft_apply_z(p, fd)
    r0 = np.linalg.norm(f - oracle.nfft.nfft_direct(x, est.cpu().numpy()))
    g.infft_refine_z(p, fd, est, 2)
    r2 = np.linalg.norm(f - oracle.nfft.nfft_direct(x, est.cpu().numpy()))
    print(f"underdetermined residual {r0:.2e} -> {r2:.2e}")
    assert r2 < 0.5 * r0


def test_refine_argument_errors():
    import torch
    import paper_1811_05335_gb300 as g
    x = jittered(713, 64)
    p = plan_for(x, 16)
    f = torch.zeros(64, dtype=torch.complex128, device="cuda:0")
    fh = torch.zeros(16, dtype=torch.complex128, device="cuda:0")
    with pytest.raises(g.InfftError):
        g.infft_refine_z(p, f, fh, -1)
    with pytest.raises(g.InfftError):
        g.infft_refine_z(p, np.zeros(64, np.complex128), fh, 1)      # host f
    g.infft_refine_z(p, f, fh, 0)                                     # zero sweeps: nothing to do
    p.close()
