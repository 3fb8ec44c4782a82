"""Pins for oracle.infft: the modified adjoint NFFT D^* F^* B_opt^* f and its adjoint."""
import numpy as np
import pytest

from oracle import infft, bopt, kernel, nfft
from workloads import iid_uniform, jittered, complex_normal, equispaced, make_problem


@pytest.mark.parametrize("M,Ms", [(8, 16), (6, 18), (16, 16), (4, 12)])
def test_F_fft_equals_direct(M, Ms):
    g = complex_normal(M * Ms, Ms)
    c = complex_normal(M + Ms, M)
    np.testing.assert_allclose(infft.F_adjoint(g, M, Ms, "fft"), infft.F_adjoint(g, M, Ms, "direct"), atol=1e-12)
    np.testing.assert_allclose(infft.F_apply(c, M, Ms, "fft"), infft.F_apply(c, M, Ms, "direct"), atol=1e-12)


@pytest.mark.parametrize("kind", ["full", "sym"])
def test_apply_equals_dense_product(kind):
    """D^* F^* B^* f with the explicit matrices (eq:approx_ansatz2)."""
    x = jittered(5, 40)
    B = bopt.bopt_closed(x, 10, 2.0, 3, kind)
    f = complex_normal(6, 40)
    d = kernel.diag_D(10, 20, kind)
    want = np.diag(d).conj().T @ bopt.matrix_F(10, 20).conj().T @ B.dense().T @ f
    np.testing.assert_allclose(infft.infft_apply(B, f), want, atol=1e-12)
    wantf = B.dense() @ bopt.matrix_F(10, 20) @ (d * complex_normal(7, 10))
    np.testing.assert_allclose(infft.nfft_apply(B, complex_normal(7, 10)), wantf, atol=1e-12)


def test_adjoint_pair():
    """<infft_apply(f), g> = <f, nfft_apply(g)> (Remark remark:ansatz2_adj: B F D is the adjoint of D^* F^* B^*)."""
    x = iid_uniform(8, 70)
    B = bopt.bopt_closed(x, 16, 2.0, 4)
    f, g = complex_normal(9, 70), complex_normal(10, 16)
    lhs = np.vdot(g, infft.infft_apply(B, f))
    rhs = np.vdot(infft.nfft_apply(B, g), f)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("M", [8, 32])
def test_equispaced_sigma1_exact_inverse(M):
    """sigma = 1, M = N, x_j = j/M, kernel full: fhat_check = fhat / (1 + tau) exactly."""
    x = equispaced(M)
    fhat = complex_normal(M, M)
    f = nfft.nfft_direct(x, fhat)
    got, _ = infft.infft(x, f, M, 1.0, 2, "full", 1e-12)
    np.testing.assert_allclose(got, fhat / (1 + 1e-12), atol=1e-12)


def test_sym_loses_only_the_nyquist_coefficient():
    """kernel sym: D's k = -M/2 entry is 0, so that coefficient is never recovered."""
    x = equispaced(16)
    fhat = complex_normal(3, 16)
    got, _ = infft.infft(x, nfft.nfft_direct(x, fhat), 16, 1.0, 2, "sym", 0.0)
    assert got[0] == 0
    assert np.abs(got[1:] - fhat[1:]).max() < 0.2      # O(1/M) leakage of the dropped term


def test_jittered_reconstruction_and_error_measures():
    """Ex. ex:trig_poly_ansatz2 setting (Dirichlet, sigma = 2, jittered, N = 4M, m = 4):
    reconstruction is accurate; the paper's values are figures only, so this asserts
    properties, not its numbers."""
    errs = []
    for M in (32, 256):
        p = make_problem(2, M=M, N=4 * M, m=4, noise_rel=0.0)
        got, _ = infft.infft(p.x, p.f, M, 2.0, 4)
        errs.append(infft.rel_l2(got, p.fhat))
        e = infft.errors_per_node(p.fhat, got, p.N)
        assert e["rel_2"] <= e["abs_2"] / np.linalg.norm(p.fhat) * 1.0000001
    assert errs[1] < 1e-5
    assert errs[1] < errs[0]          # "errors ... decrease for large sizes of M"


def test_errors_per_node_golden(golden):
    """Hand-worked values of eq:errors_per_node_lagrange (tests/golden/errors_per_node.txt):
    a wrong divisor (N or the norm of fhat), a swapped norm or a squared norm fails them."""
    rows = golden("errors_per_node.txt")
    assert len(rows) % 3 == 0
    for c in range(0, len(rows), 3):
        N = int(rows[c][0])
        fh = np.array(rows[c][1::2]) + 1j * np.array(rows[c][2::2])
        fc = np.array(rows[c + 1][0::2]) + 1j * np.array(rows[c + 1][1::2])
        want = dict(zip(("abs_2", "rel_2", "abs_inf", "rel_inf"), rows[c + 2]))
        got = infft.errors_per_node(fh, fc, N)
        for key, val in want.items():
            assert abs(got[key] - val) <= 1e-15 * abs(val), (c // 3, key, got[key], val)


def test_refine_is_the_residual_error_map():
    """One sweep maps the error e of noiseless data to (I - D^* F^* B_opt^* A) e, with every
    matrix formed explicitly (eq:matrix_A, eq:matrix_F, eq:matrix_D, eq:matrix_B)."""
    x = jittered(31, 64)
    M, Ms = 16, 32
    B = bopt.bopt_closed(x, M, 2.0, 3)
    fh = complex_normal(32, M)
    f = nfft.nfft_direct(x, fh)
    Bt = np.diag(kernel.diag_D(M, Ms, "full")).conj().T @ bopt.matrix_F(M, Ms).conj().T @ B.dense().T
    A = nfft.matrix_A(x, M)
    start = infft.infft_apply(B, f) + 1e-3 * complex_normal(33, M)       # any starting estimate
    e1 = infft.refine(B, x, f, start, 1) - fh
    np.testing.assert_allclose(e1, (np.eye(M) - Bt @ A) @ (start - fh), atol=1e-13)
    assert np.array_equal(infft.refine(B, x, f, start, 0), start)


def test_refine_converges_on_jittered_nodes():
    """Jittered nodes, N = 4M, m = 4: the inverse NFFT is accurate to ~1e-7, so each sweep
    shrinks the error about 1e7-fold until fp64 rounding."""
    x = jittered(34, 256)
    fh = complex_normal(35, 64)
    f = nfft.nfft_direct(x, fh)
    B = bopt.bopt_closed(x, 64, 2.0, 4)
    f0 = infft.infft_apply(B, f)
    e = [infft.rel_l2(infft.refine(B, x, f, f0, k), fh) for k in range(3)]
    assert 1e-9 < e[0] < 1e-5 and e[1] < 1e-12 and e[2] < 1e-14


def test_refine_keeps_an_exact_inverse():
    """sigma = 1, M = N equispaced, kernel full: the estimate fhat/(1 + tau) is corrected to
    fhat up to tau^2."""
    x = equispaced(32)
    fh = complex_normal(36, 32)
    f = nfft.nfft_direct(x, fh)
    B = bopt.bopt_closed(x, 32, 1.0, 2, "full", 1e-12)
    np.testing.assert_allclose(infft.refine(B, x, f, infft.infft_apply(B, f), 1), fh, atol=1e-14)
