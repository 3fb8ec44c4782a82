"""Pins of the underdetermined-case oracle (Sec. 3.2.1) against what the paper and the
mathematics fix: the closed-form kernel against its defining sum, the equispaced case
with N | M where A A^* = M I_N (Sec. 3.2 opening), a brute-force joint Frobenius fit on a
tiny grid (the split eq:min_decomp_ansatz1), optimality of every node's solution, the
Frobenius decomposition itself and the adjoint pair of Remark remark:ansatz1_adj."""
import numpy as np
import pytest

from oracle import under, kernel, nfft, pattern
from oracle.under import bopt_under, bopt_under_naive, infft_apply_under, adjoint_inverse_apply_under
from workloads import jittered, iid_uniform, complex_normal, trig_poly_eval


@pytest.mark.parametrize("kern", ["full", "sym"])
def test_kappa_closed_matches_defining_sum(kern):
    M, Ms = 32, 64
    rng = np.random.default_rng(1)
    t = np.concatenate([rng.uniform(-0.5, 0.5, 200), [0.0, 1e-9, -1e-9, 0.4999999, -0.5, 1.0 / Ms]])
    want = kernel.kappa_sum(t, M, Ms, kern)
    got = kernel.kappa_closed(t, M, Ms, kern)
    assert np.max(np.abs(got - want)) <= 1e-14 * M / Ms
    assert np.allclose(got.real, kernel.re_kappa_closed(t, M, Ms, kern), atol=1e-15)


@pytest.mark.parametrize("N,M,m", [(16, 32, 1), (16, 64, 2), (32, 64, 3)])
def test_equispaced_n_divides_m_is_exact(N, M, m):
    """x_j = j/N, sigma = 1, N | M: A A^* = M I_N, so b_j = M e_{l_j} (l_j = M x_j) reaches
    J_j = 0 and f_check = (1/M) A^* f solves A f_check = f exactly."""
    x = np.arange(-(N // 2), N // 2) / N
    U = bopt_under(x, M, 1.0, m)
    assert np.all(U.Jn <= 1e-18 * M ** 2)
    Bd = U.B.dense()
    lj = np.rint(M * x).astype(int) + M // 2
    want = np.zeros_like(Bd)
    want[np.arange(N), lj] = M
    assert np.max(np.abs(Bd - want)) <= 1e-9 * M
    f = complex_normal(5, N)
    fc = infft_apply_under(U, f)
    A = nfft.matrix_A(x, M)
    assert np.allclose(fc, A.conj().T @ f / M, rtol=0, atol=1e-12 * np.abs(f).max())
    assert np.linalg.norm(A @ fc - f) <= 1e-11 * np.linalg.norm(f)


@pytest.mark.parametrize("kern", ["full", "sym"])
def test_joint_frobenius_fit_equals_per_node_solutions(kern):
    """One least-squares fit over all nonzeros of B^* at once (the Frobenius problem
    eq:min_norm_ansatz1 with each node's Tikhonov rows) equals the per-node solutions."""
    N, M, sigma, m = 6, 16, 2.0, 1
    Ms = 32
    x = iid_uniform(7, N)
    U = bopt_under_naive(x, M, sigma, m, kern)
    K = nfft.matrix_A(x, M) @ (kernel.diag_D(M, Ms, kern)[:, None] *
                               np.exp(-2j * np.pi * np.outer(np.arange(-(M // 2), M // 2),
                                                             np.arange(-(Ms // 2), Ms // 2)) / Ms))
    lo, hi = pattern.grid_lo_hi(x, Ms, m)
    unknowns = [(j, int(l)) for j in range(N) for l in pattern.reduce_l(np.arange(lo[j], hi[j] + 1), Ms)]
    rows_re, rows_im, rhs = [], [], []
    for h in range(N):
        for j in range(N):                      # entry (h, j) of K B^* - M I
            row = np.zeros(len(unknowns), complex)
            for q, (jj, l) in enumerate(unknowns):
                if jj == j:
                    row[q] = K[h, l + Ms // 2]
            rows_re.append(row.real)
            rows_im.append(row.imag)
            rhs.append(M if h == j else 0.0)
    A = np.vstack([np.array(rows_re), np.array(rows_im)])
    b_rhs = np.concatenate([rhs, np.zeros(N * N)])
    reg = np.zeros((len(unknowns), len(unknowns)))
    for q, (jj, l) in enumerate(unknowns):
        reg[q, q] = np.sqrt(U.mu[jj])
    sol, *_ = np.linalg.lstsq(np.vstack([A, reg]), np.concatenate([b_rhs, np.zeros(len(unknowns))]), rcond=None)
    Bd = U.B.dense()
    for q, (j, l) in enumerate(unknowns):
        assert abs(sol[q] - Bd[j, l + Ms // 2]) <= 1e-8 * max(1.0, abs(sol[q]))


@pytest.mark.parametrize("kern", ["full", "sym"])
def test_node_solutions_are_optimal(kern):
    N, M, m = 48, 192, 2
    x = jittered(9, N)
    U = bopt_under(x, M, 2.0, m, kern)
    lo, hi = pattern.grid_lo_hi(x, 2 * M, m)
    rng = np.random.default_rng(2)
    Bd = U.B.dense()
    for j in range(0, N, 5):
        l = np.arange(lo[j], hi[j] + 1)
        G, r, mu = under.node_system(x, j, l, M, 2 * M, kern)
        b = Bd[j, pattern.reduce_l(l, 2 * M) + M]
        assert np.linalg.norm(G @ b - r) <= 1e-10 * np.linalg.norm(r)
        phi = lambda c: c @ G @ c - 2 * r @ c + M ** 2
        assert phi(b) <= M ** 2 * (1 + 1e-12)                  # no worse than b = 0
        for _ in range(5):
            d = rng.standard_normal(len(b)) * 1e-3 * (1 + np.abs(b))
            assert phi(b) <= phi(b + d) + 1e-9 * M ** 2
        assert U.Jn[j] <= M ** 2


@pytest.mark.parametrize("kern", ["full", "sym"])
def test_naive_and_normal_equation_tiers_agree(kern):
    N, M, m = 40, 160, 2
    x = iid_uniform(11, N)
    U1 = bopt_under_naive(x, M, 2.0, m, kern)
    U2 = bopt_under(x, M, 2.0, m, kern)
    assert np.array_equal(U1.B.ptr, U2.B.ptr) and np.array_equal(U1.B.idx, U2.B.idx)
    assert np.allclose(U1.Jn, U2.Jn, rtol=1e-8, atol=1e-10 * M ** 2)
    assert np.max(np.abs(U1.B.b - U2.B.b)) <= 1e-7 * np.max(np.abs(U2.B.b))


def test_frobenius_objective_splits_over_nodes():
    """sum_j J_j = ||A D^* F^* B_opt^* - M I_N||_F^2 (eq:min_decomp_ansatz1), from the dense matrices."""
    N, M, m = 24, 96, 2
    x = jittered(12, N)
    for kern in ("full", "sym"):
        U = bopt_under(x, M, 2.0, m, kern)
        dense = under.frobenius_objective_under_dense(x, U.B.dense(), M, 2 * M, kern)
        assert abs(U.Jn.sum() - dense) <= 1e-9 * max(1.0, dense)


def test_adjoint_pair():
    """<f_check(f), g> = <f, (1/M) B_opt F D g>: the inverse adjoint estimate of Remark
    remark:ansatz1_adj uses the adjoint of the same operator."""
    N, M, m = 40, 160, 2
    x = jittered(13, N)
    U = bopt_under(x, M, 2.0, m)
    f = complex_normal(14, N)
    g = complex_normal(15, M)
    lhs = np.vdot(g, infft_apply_under(U, f))
    rhs = np.vdot(adjoint_inverse_apply_under(U, g), f)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_underdetermined_reconstruction_improves_with_m():
    """Reported quality (the paper gives figures only): for jittered nodes, M = 4N, sigma = 2,
    the reconstruction residual ||A f_check - f|| / ||f|| is small and m = 4 beats b = B_opt at m = 1."""
    N, M = 128, 512
    x = jittered(16, N)
    fh = complex_normal(17, M)
    f = trig_poly_eval(x, fh)
    A = nfft.matrix_A(x, M)
    res = {}
    for m in (1, 4):
        U = bopt_under(x, M, 2.0, m)
        res[m] = np.linalg.norm(A @ infft_apply_under(U, f) - f) / np.linalg.norm(f)
    assert res[4] < res[1] and res[4] < 0.05
