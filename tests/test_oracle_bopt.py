"""Pins for oracle.bopt: the per-grid-point least-squares problems of Sec. 3.2.2."""
import numpy as np
import pytest

from oracle import bopt, kernel, pattern, infft, nfft
from workloads import iid_uniform, jittered, equispaced, chebyshev_jittered


def test_FstarF_is_Ms_identity():
    """F^* F = M_sigma I_M since |k - k'| < M <= M_sigma (eq:matrix_F); the closed form rests on it."""
    for M, Ms in [(8, 8), (8, 16), (6, 9 * 2)]:
        F = bopt.matrix_F(M, Ms)
        np.testing.assert_allclose(F.conj().T @ F, Ms * np.eye(M), atol=1e-11)


@pytest.mark.parametrize("kind", ["full", "sym"])
def test_closed_gram_equals_explicit(kind):
    """Re(L_l^* L_l) and Re(L_l^* e_l) from the explicit L_l = F D H_l (eq:matrix_Ll)
    equal the closed forms used by the scalable tier."""
    M, sigma, m = 16, 2.0, 3
    Ms = 32
    x = iid_uniform(41, 60)
    ptr, idx = pattern.index_sets_l_fast(x, Ms, m)
    for p in (0, 5, 17, 31):
        I = idx[ptr[p]:ptr[p + 1]]
        if len(I) == 0:
            continue
        L = bopt.matrix_L(x[I], M, Ms, kind)
        G, r = bopt.column_system_closed(x, I, p - Ms // 2, M, Ms, kind, 0.0)
        np.testing.assert_allclose((L.conj().T @ L).real, G, atol=1e-14)
        np.testing.assert_allclose(L[p].real, r, atol=1e-14)     # (L^* e_l)_j = conj(L_{l,j})
        if kind == "sym":
            assert np.abs(L.imag).max() < 1e-14                  # the remark's L_l is real


@pytest.mark.parametrize("kind", ["full", "sym"])
def test_tiers_agree(kind):
    """Both tiers minimise the same regularised objective; compare what is unique
    (the minimum value) rather than b, which is ill-determined along near-null
    directions of L_l."""
    x = iid_uniform(51, 96)
    M, sigma, m = 32, 2.0, 3
    A = bopt.bopt_naive(x, M, sigma, m, kind)
    B = bopt.bopt_closed(x, M, sigma, m, kind)
    assert np.array_equal(A.ptr, B.ptr) and np.array_equal(A.idx, B.idx)
    mu = 1e-12 * kernel.gram_diag(M, A.Ms, kind)
    for p in range(A.Ms):
        s, e = A.ptr[p], A.ptr[p + 1]
        if e == s:
            continue
        L = bopt.matrix_L(x[A.idx[s:e]], M, A.Ms, kind)
        ep = np.zeros(A.Ms)
        ep[p] = 1.0
        phi = [np.linalg.norm(L @ c.b[s:e] - ep) ** 2 + mu * c.b[s:e] @ c.b[s:e] for c in (A, B)]
        assert abs(phi[0] - phi[1]) <= 1e-11 * phi[0]
    f = nfft.nfft_direct(x, np.exp(1j * np.arange(M)))
    assert infft.rel_l2(infft.infft_apply(B, f), infft.infft_apply(A, f, "direct")) < 1e-6


def test_naive_column_is_a_minimiser():
    """Random real perturbations never lower the regularised column objective."""
    x = jittered(61, 48)
    M, Ms, m = 12, 24, 3
    rng = np.random.default_rng(0)
    mu = 1e-12 * kernel.gram_diag(M, Ms, "full")
    cols = pattern.index_sets_l(x, Ms, m)
    for p in (0, 7, 23):
        I = cols[p]
        L = bopt.matrix_L(x[I], M, Ms, "full")
        b, J = bopt.solve_column_naive(L, p, mu)
        ep = np.zeros(Ms)
        ep[p] = 1.0
        phi = lambda c: np.linalg.norm(L @ c - ep) ** 2 + mu * c @ c
        assert abs(J - np.linalg.norm(L @ b - ep) ** 2) < 1e-14
        for _ in range(20):
            assert phi(b + 1e-3 * rng.standard_normal(len(b))) >= phi(b)
        assert phi(b) <= phi(np.zeros(len(b)))       # b = 0 gives ||e_l||^2 = 1


def test_closed_normal_equation_residual():
    x = chebyshev_jittered(71, 200)
    B = bopt.bopt_closed(x, 64, 2.0, 4)
    mu = 1e-12 * kernel.gram_diag(64, 128, "full")
    for p in range(0, 128, 9):
        s, e = B.ptr[p], B.ptr[p + 1]
        if e == s:
            continue
        G, r = bopt.column_system_closed(x, B.idx[s:e], p - 64, 64, 128, "full", mu)
        assert np.linalg.norm(G @ B.b[s:e] - r) <= 1e-9 * (np.linalg.norm(r) + 1e-300) + 1e-15


def test_separability_brute_force():
    """eq:opt_ansatz2 over all (2m+1)-sparse real B, regularised by mu ||B||_F^2, solved as ONE
    least-squares problem in all pattern entries, equals the column-by-column solutions."""
    M, Ms, m = 6, 12, 2
    x = iid_uniform(81, 10)
    B = bopt.bopt_naive(x, M, Ms / M, m)
    mu = 1e-12 * kernel.gram_diag(M, Ms, "full")
    A = nfft.matrix_A(x, M)
    Kstar = bopt.matrix_F(M, Ms) @ (kernel.diag_D(M, Ms, "full")[:, None] * A.conj().T)
    # unknowns: the pattern entries (j, p); residual vec(K^* B - I) (real and imaginary parts)
    ents = [(j, p) for p in range(Ms) for j in B.idx[B.ptr[p]:B.ptr[p + 1]]]
    rows = []
    for (j, p) in ents:
        col = np.zeros((Ms, Ms), dtype=complex)
        col[:, p] = Kstar[:, j]
        rows.append(col.ravel())
    Z = np.array(rows).T                                  # (Ms*Ms, nunk)
    target = np.eye(Ms).ravel()
    S = np.vstack([Z.real, Z.imag, np.sqrt(mu) * np.eye(len(ents))])
    rhs = np.concatenate([target, np.zeros(Ms * Ms), np.zeros(len(ents))])
    joint, *_ = np.linalg.lstsq(S, rhs, rcond=None)
    Bj = np.zeros((len(x), Ms))
    for v, (j, p) in zip(joint, ents):
        Bj[j, p] = v
    Bd = B.dense()
    obj = lambda Bm: np.linalg.norm(Kstar @ Bm - np.eye(Ms)) ** 2 + mu * np.sum(Bm ** 2)
    assert abs(obj(Bd) - obj(Bj)) <= 1e-10 * obj(Bj)
    # and sum_l J_l is the unregularised Frobenius objective
    assert abs(infft.frobenius_objective(B) - np.linalg.norm(Kstar @ Bd - np.eye(Ms)) ** 2) < 1e-10


def test_equispaced_sigma1_is_identity(golden):
    """Sec. 3.2 equispaced case: B_opt is the (scaled) identity pattern, J_l = (tau/(1+tau))^2."""
    for N, m, tau, bdiag, Jwant in golden("equispaced_identity.txt"):
        N, m = int(N), int(m)
        x = equispaced(N)
        for tier in (bopt.bopt_closed, bopt.bopt_naive):
            B = tier(x, N, 1.0, m, "full", tau)
            Bd = B.dense()
            np.testing.assert_allclose(Bd, bdiag * np.eye(N), atol=1e-12)
            np.testing.assert_allclose(B.J, Jwant, atol=1e-13)


def test_objective_lower_bound_and_reduction():
    """J_l >= 1 - 1/sigma (distance of e_l to range(F), dim M in C^{M_sigma});
    the optimised objective is below that of B = 0 and of perturbed B (Ex. ex:matrixnorm_ansatz2)."""
    x = jittered(91, 256)
    B = bopt.bopt_closed(x, 64, 2.0, 4)
    assert B.J.min() >= 0.5 - 1e-12
    base = infft.frobenius_objective_dense(x, B.dense(), 64, 128, "full")
    assert abs(base - infft.frobenius_objective(B)) < 1e-8 * base
    assert base < 128.0
    rng = np.random.default_rng(1)
    Bd = B.dense()
    mask = Bd != 0
    for _ in range(3):
        P = Bd + 1e-2 * rng.standard_normal(Bd.shape) * mask
        assert infft.frobenius_objective_dense(x, P, 64, 128, "full") > base


def test_sigma1_beats_sigma2_for_overdetermined():
    """Ex. ex:matrixnorm_ansatz2: with sigma = 1 and N >> M the optimisation drives the
    objective towards 0, while sigma = 2 stays at the floor M_sigma (1 - 1/sigma)."""
    x = jittered(93, 1024)
    B1 = bopt.bopt_closed(x, 64, 1.0, 2)
    B2 = bopt.bopt_closed(x, 64, 2.0, 2)
    assert infft.frobenius_objective(B1) / 64 < 1e-3
    assert infft.frobenius_objective(B2) / 128 > 0.5 - 1e-9


def test_empty_columns():
    """Grid points with no node within m cells give empty b_l and J_l = 1."""
    x = np.array([-0.3, -0.29, 0.1])
    B = bopt.bopt_closed(x, 32, 2.0, 2)
    empty = np.diff(B.ptr) == 0
    assert empty.sum() > 0 and np.all(B.J[empty] == 1.0)
