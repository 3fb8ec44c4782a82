"""The allocation-free entry point infft_fft_deconv_noalloc, for callers that cannot
allocate device memory when they call (their device memory belongs to their own pool
allocator, or they must not call cudaMalloc while other work is being recorded).

It is checked two ways, each on two calls in a row with different data:
* against the FP64 oracle on the same grid: fhat = conj(d) F^* g, numpy's FFT with the
  (-1)^k phase and D (1/M_sigma, and 0 at k = -M/2 for kernel sym) applied on the host,
  at rel l2 <= 1e-5; sizes cover the single-CTA transform, the four-step transform at the
  largest scratch size M_sigma = 2^20, kernel sym and M = M_sigma;
* against the existing entry point infft_apply: on a plan, the grid g = B_opt^* f formed on
  the host from the plan's exported weights, transformed here, reproduces infft_apply(f).
This file runs last so that a run stopping at the first failure has already run every
other test."""
import numpy as np
import pytest

import oracle
from workloads import complex_normal

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


def host_grid(data, f, Ms, N):
    """g_l = sum_{j in I(l)} b_{l,j} f_j from the plan's exported pattern and fp64 weights."""
    count = data["col_count"].astype(np.int64)
    start = data["col_start"].astype(np.int64)
    off = data["col_offset"].astype(np.int64)
    nnz = int(off[-1])
    col = np.repeat(np.arange(Ms), count)
    pos = (np.repeat(start, count) + np.arange(nnz) - np.repeat(off[:-1], count)) % N
    g = np.zeros(Ms, np.complex128)
    np.add.at(g, col, data["weights"][:nnz] * f[data["perm"].astype(np.int64)[pos]])
    return g


@pytest.mark.parametrize("M,Ms,kernel", [
    (512, 1024, "full"),          # single-CTA transform
    (1024, 1024, "sym"),          # M = M_sigma, kernel sym
    (6000, 16384, "full"),        # four-step, M not a power of two
    (4096, 8192, "sym"),
    (1 << 19, 1 << 20, "full"),   # the largest M_sigma the static scratch holds
    (1 << 20, 1 << 20, "sym"),
])
def test_fft_deconv_noalloc_matches_oracle(M, Ms, kernel):
    import torch
    import paper_1811_05335_gb300 as g
    d = oracle.kernel.diag_D(M, Ms, kernel)
    for call in range(2):                         # two calls in a row, different data
        grid = complex_normal(1000 + 7 * call + Ms % 97, Ms).astype(np.complex64)
        want = np.conj(d) * oracle.infft.F_adjoint(grid.astype(np.complex128), M, Ms)
        got = g.infft_fft_deconv_noalloc(torch.tensor(grid, device="cuda:0"), M, kernel=kernel)
        got = got.cpu().numpy().astype(np.complex128)
        err = oracle.infft.rel_l2(got, want)
        assert err <= FP32_TOL, f"call {call}: rel l2 {err:.3e}"
        if kernel == "sym":
            assert got[0] == 0


@pytest.mark.parametrize("M,N,m", [(4096, 16384, 4), (512, 2048, 3)])   # four-step and single-CTA paths
def test_fft_deconv_noalloc_matches_infft_apply(M, N, m):
    import torch
    import paper_1811_05335_gb300 as g
    from workloads import make_problem
    dev = torch.device("cuda:0")
    p = make_problem(2, M=M, N=N, m=m)
    plan = g.infft_plan_create(M, N, 2.0, m)
    g.infft_set_nodes(plan, torch.tensor(p.x, dtype=torch.float64, device=dev))
    g.infft_precompute(plan)
    data = g.infft_copy_plan_data(plan)
    Ms = plan.M_sigma
    for call in range(2):                         # two calls in a row, different data
        f = np.asarray(p.f * (1.0 + 0.5j * call), np.complex64)
        want = g.infft_apply(plan, torch.tensor(f, device=dev)).cpu().numpy().astype(np.complex128)
        grid = torch.tensor(host_grid(data, f.astype(np.complex128), Ms, N).astype(np.complex64), device=dev)
        got = g.infft_fft_deconv_noalloc(grid, M).cpu().numpy().astype(np.complex128)
        err = np.linalg.norm(got - want) / np.linalg.norm(want)
        assert err <= FP32_TOL, f"call {call}: rel l2 {err:.3e}"
    plan.close()


def test_fft_deconv_noalloc_rejects_sizes():
    import torch
    import paper_1811_05335_gb300 as g
    lib = g.library()
    grid = torch.zeros(8, dtype=torch.complex64, device="cuda:0")
    out = torch.zeros(8, dtype=torch.complex64, device="cuda:0")
    # M_sigma above the static scratch (2^20): refused before any GPU work
    assert lib.infft_fft_deconv_noalloc(grid.data_ptr(), 8, 1 << 21, 0, out.data_ptr(), None) == 5
    assert b"exceeds" in lib.infft_last_error()
    assert lib.infft_fft_deconv_noalloc(grid.data_ptr(), 8, 12, 0, out.data_ptr(), None) == 1   # not a power of 2
    host = np.zeros(8, np.complex64)
    assert lib.infft_fft_deconv_noalloc(host.ctypes.data, 8, 8, 0, out.data_ptr(), None) == 1  # host pointer
