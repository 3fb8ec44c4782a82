"""Pins for oracle.infft2d, the 2-D tensor-product reading of Sec. 3.2.2.

Each pin ties a part of the 2-D oracle to something outside it: the defining
double sum of the kernel, the explicit matrices F, D, H, the pattern's
definition checked by brute force over the periodic images, the 1-D oracle
(itself pinned) through the Kronecker structure of tensor-grid nodes, exact
inversion in the equispaced sigma = 1 case, and the orthogonality of A on a
tensor grid.
"""
import numpy as np
import pytest

from oracle import infft2d as o2, bopt, nfft
from workloads import iid_uniform, jittered, radial, complex_normal, trig_poly_eval_2d


def rand_nodes(seed, n):
    return np.stack([iid_uniform(seed, n), iid_uniform(seed + 1, n)], axis=1)


@pytest.mark.parametrize("kernel", ["full", "sym"])
def test_kappa2_is_the_double_sum(kernel):
    """kappa(t) = sum_{k1, k2} d_k exp(2 pi i k.t), written out term by term."""
    M1, M2, Ms1, Ms2 = 6, 8, 12, 16
    rng = np.random.default_rng(3)
    t = rng.uniform(-0.5, 0.5, (20, 2))
    t[0] = 0.0
    t[1] = (0.0, 0.25)
    d = o2.diag_D2(M1, M2, Ms1, Ms2, kernel)
    for (t1, t2) in t:
        want = 0j
        for a, k1 in enumerate(range(-M1 // 2, M1 // 2)):
            for b, k2 in enumerate(range(-M2 // 2, M2 // 2)):
                want += d[a, b] * np.exp(2j * np.pi * (k1 * t1 + k2 * t2))
        got = o2.kappa2(np.float64(t1), np.float64(t2), M1, M2, Ms1, Ms2, kernel)
        assert abs(got - want) <= 1e-15 * 16
    # the full kernel's real part is not the product of the 1-D real parts
    if kernel == "full":
        g = o2.kappa2(np.float64(0.1), np.float64(0.2), M1, M2, Ms1, Ms2, kernel)
        from oracle.kernel import re_kappa_closed
        sep = re_kappa_closed(0.1, M1, Ms1, kernel) * re_kappa_closed(0.2, M2, Ms2, kernel)
        assert abs(g.real - sep) > 1e-4


def test_F2_columns_orthogonal():
    """F^* F = Ms1 Ms2 I on the kept frequencies, and one entry by its definition."""
    M1, M2, Ms1, Ms2 = 4, 6, 8, 12
    F = o2.matrix_F2(M1, M2, Ms1, Ms2)
    np.testing.assert_allclose(F.conj().T @ F, Ms1 * Ms2 * np.eye(M1 * M2), atol=1e-11)
    l1, l2, k1, k2 = -3, 5, 1, -2
    p = (l1 + Ms1 // 2) * Ms2 + l2 + Ms2 // 2
    q = (k1 + M1 // 2) * M2 + k2 + M2 // 2
    assert abs(F[p, q] - np.exp(2j * np.pi * (k1 * l1 / Ms1 + k2 * l2 / Ms2))) < 1e-14


@pytest.mark.parametrize("kernel", ["full", "sym"])
def test_closed_gram_equals_explicit(kernel):
    """Re(L^* L) and Re(L^* e_l) from the explicit L_l = F D H_l equal the closed form."""
    M1, M2 = 4, 6
    Ms1, Ms2 = 8, 12
    x = rand_nodes(11, 30)
    ptr, idx = o2.index_sets_l2_fast(x, Ms1, Ms2, 1)
    checked = 0
    for p in range(0, Ms1 * Ms2, 7):
        I = idx[ptr[p]:ptr[p + 1]]
        if len(I) == 0:
            continue
        L = o2.matrix_L2(x[I], M1, M2, Ms1, Ms2, kernel)
        G, r = o2.column_system2(x, I, p, M1, M2, Ms1, Ms2, kernel, 0.0)
        np.testing.assert_allclose((L.conj().T @ L).real, G, atol=1e-15)
        np.testing.assert_allclose(L[p].real, r, atol=1e-15)
        checked += 1
    assert checked >= 5


def brute_pattern(x, Ms1, Ms2, m):
    """j in I(l) iff for t = 1, 2 some z in {-1, 0, 1} gives |Ms_t x_jt - l_t + Ms_t z| <= m."""
    P = Ms1 * Ms2
    cols = [[] for _ in range(P)]
    for j, (x1, x2) in enumerate(x):
        for p in range(P):
            l1, l2 = p // Ms2 - Ms1 // 2, p % Ms2 - Ms2 // 2
            ok1 = any(abs(Ms1 * x1 - l1 + Ms1 * z) <= m for z in (-1, 0, 1))
            ok2 = any(abs(Ms2 * x2 - l2 + Ms2 * z) <= m for z in (-1, 0, 1))
            if ok1 and ok2:
                cols[p].append(j)
    return cols


@pytest.mark.parametrize("m", [1, 2])
def test_pattern_brute_force(m):
    """Both pattern builders equal the definition, including nodes on grid points
    (the closed inequality admits 2m + 1 points) and nodes next to the seam."""
    Ms1, Ms2 = 8, 12
    x = rand_nodes(21, 25)
    x[0] = (0.25, -1.0 / 3.0)            # on a grid line in dimension 1 (u = 2)
    x[1] = (-0.5, 0.5 - 1e-9)            # seam in both dimensions
    x[2] = (3.0 / 8.0, 5.0 / 12.0 - 1e-17)
    x[3] = (0.0, 0.0)                    # a grid point in both dimensions
    want = brute_pattern(x, Ms1, Ms2, m)
    slow = o2.index_sets_l2(x, Ms1, Ms2, m)
    ptr, idx = o2.index_sets_l2_fast(x, Ms1, Ms2, m)
    for p in range(Ms1 * Ms2):
        assert list(slow[p]) == want[p]
        assert list(idx[ptr[p]:ptr[p + 1]]) == want[p]
        assert list(o2.column_nodes2(x, p, Ms1, Ms2, m)) == want[p]
    counts = np.diff(ptr)
    assert counts.sum() == sum((2 * m + (Ms1 * a == np.floor(Ms1 * a))) * (2 * m + (Ms2 * b == np.floor(Ms2 * b)))
                               for a, b in x)


@pytest.mark.parametrize("kernel", ["full", "sym"])
def test_tiers_agree(kernel):
    """Naive (explicit L, SVD least squares) and closed-form tiers reach the same
    regularised minimum in every column, and give the same fhat."""
    M1, M2, sigma, m = 4, 6, 2.0, 1
    x = rand_nodes(31, 40)
    A = o2.bopt2_naive(x, M1, M2, sigma, m, kernel)
    B = o2.bopt2_closed(x, M1, M2, sigma, m, kernel)
    assert np.array_equal(A.ptr, B.ptr) and np.array_equal(A.idx, B.idx)
    mu = 1e-12 * o2.gram_diag2(M1, M2, A.Ms1, A.Ms2, kernel)
    for p in range(A.Ms1 * A.Ms2):
        s, e = A.ptr[p], A.ptr[p + 1]
        if e == s:
            continue
        L = o2.matrix_L2(x[A.idx[s:e]], M1, M2, A.Ms1, A.Ms2, kernel)
        ep = np.zeros(L.shape[0])
        ep[p] = 1.0
        phi = [np.linalg.norm(L @ c.b[s:e] - ep) ** 2 + mu * c.b[s:e] @ c.b[s:e] for c in (A, B)]
        assert abs(phi[0] - phi[1]) <= 1e-10 * phi[0] + 1e-14
        assert abs(np.linalg.norm(L @ B.b[s:e] - ep) ** 2 - B.J[p]) <= 1e-10
    f = complex_normal(5, len(x))
    np.testing.assert_allclose(o2.infft2_apply(B, f), o2.infft2_apply(A, f, "direct"), atol=1e-8, rtol=0)


def test_closed_column_is_the_regularised_minimiser():
    """Random perturbations of b never lower ||L b - e_l||^2 + mu ||b||^2 (explicit L)."""
    M1, M2 = 6, 4
    x = rand_nodes(41, 50)
    B = o2.bopt2_closed(x, M1, M2, 2.0, 2, "full")
    mu = 1e-12 * o2.gram_diag2(M1, M2, B.Ms1, B.Ms2, "full")
    rng = np.random.default_rng(1)
    for p in (3, 20, 47, 70):
        s, e = B.ptr[p], B.ptr[p + 1]
        L = o2.matrix_L2(x[B.idx[s:e]], M1, M2, B.Ms1, B.Ms2, "full")
        ep = np.zeros(L.shape[0])
        ep[p] = 1.0

        def phi(b):
            return np.linalg.norm(L @ b - ep) ** 2 + mu * b @ b
        base = phi(B.b[s:e])
        for _ in range(20):
            assert phi(B.b[s:e] + 1e-3 * rng.standard_normal(e - s)) >= base - 1e-15
        assert base <= 1.0                  # b = 0 gives 1
    assert np.all(B.J <= 1.0 + 1e-12)


def test_sym_tensor_grid_is_kronecker_of_1d():
    """Kernel sym on a tensor grid of nodes: L_l = L1 (x) L2 (a real product
    kernel and a box pattern), so without regularisation every 2-D column is the
    Kronecker product of the 1-D oracle's columns and J = 1 - (1 - J1)(1 - J2)."""
    M1, M2, m = 8, 6, 2
    x1, x2 = jittered(61, 13), jittered(62, 9)
    x = np.stack(np.meshgrid(x1, x2, indexing="ij"), axis=-1).reshape(-1, 2)    # j = i1 * 9 + i2
    B = o2.bopt2_closed(x, M1, M2, 2.0, m, "sym", tau=0.0)
    B1 = bopt.bopt_closed(x1, M1, 2.0, m, "sym", tau=0.0)
    B2 = bopt.bopt_closed(x2, M2, 2.0, m, "sym", tau=0.0)
    for p in range(B.Ms1 * B.Ms2):
        p1, p2 = p // B.Ms2, p % B.Ms2
        I1 = B1.idx[B1.ptr[p1]:B1.ptr[p1 + 1]]
        I2 = B2.idx[B2.ptr[p2]:B2.ptr[p2 + 1]]
        I = B.idx[B.ptr[p]:B.ptr[p + 1]]
        assert np.array_equal(I, (I1[:, None] * len(x2) + I2[None, :]).ravel())
        if len(I) == 0:
            continue
        b = np.kron(B1.b[B1.ptr[p1]:B1.ptr[p1 + 1]], B2.b[B2.ptr[p2]:B2.ptr[p2 + 1]])
        np.testing.assert_allclose(B.b[B.ptr[p]:B.ptr[p + 1]], b, atol=1e-9 * max(1.0, np.abs(b).max()))
        assert abs(B.J[p] - (1 - (1 - B1.J[p1]) * (1 - B2.J[p2]))) < 1e-9


def test_equispaced_sigma1_inverts_exactly():
    """sigma = 1, nodes on the M1 x M2 grid: Re G = I, B_opt is the identity
    permutation (all J = 0) and D^* F^* B^* f is the exact inverse of f = A fhat."""
    M1, M2 = 8, 6
    g1 = (np.arange(M1) - M1 // 2) / M1
    g2 = (np.arange(M2) - M2 // 2) / M2
    x = np.stack(np.meshgrid(g1, g2, indexing="ij"), axis=-1).reshape(-1, 2)
    fh = complex_normal(71, M1 * M2).reshape(M1, M2)
    f = o2.nfft2_direct(x, fh)
    for m in (1, 2):
        B = o2.bopt2_closed(x, M1, M2, 1.0, m, "full")
        assert np.abs(B.J).max() < 1e-13
        D = np.zeros((len(x), M1 * M2))
        for p in range(M1 * M2):
            s, e = B.ptr[p], B.ptr[p + 1]
            D[B.idx[s:e], p] = B.b[s:e]
        np.testing.assert_allclose(D, np.eye(M1 * M2), atol=1e-12)
        np.testing.assert_allclose(o2.infft2_apply(B, f), fh, atol=1e-12)


def test_A2_adjoint_and_orthogonality():
    """<A fhat, f> = <fhat, A^* f>; A^* A = N I on an n1 x n2 tensor grid with M_t <= n_t."""
    M1, M2 = 4, 6
    x = rand_nodes(81, 17)
    fh = complex_normal(82, M1 * M2).reshape(M1, M2)
    f = complex_normal(83, 17)
    lhs = np.vdot(f, o2.nfft2_direct(x, fh))
    rhs = np.vdot(o2.nfft2_adjoint_direct(x, f, M1, M2).ravel(), fh.ravel())
    assert abs(lhs - rhs) < 1e-12
    g = np.stack(np.meshgrid(np.arange(8) / 8 - 0.5, np.arange(6) / 6 - 0.5, indexing="ij"), -1).reshape(-1, 2)
    A = o2.matrix_A2(g, M1, M2)
    np.testing.assert_allclose(A.conj().T @ A, 48 * np.eye(M1 * M2), atol=1e-11)
    # the dense least-squares comparator recovers noiseless data exactly
    y = rand_nodes(84, 60)
    np.testing.assert_allclose(o2.dense_lsq_inverse2(y, o2.nfft2_direct(y, fh), M1, M2), fh, atol=1e-10)


def test_F2_adjoint_fft_matches_direct():
    g = (complex_normal(91, 8 * 12)).reshape(8, 12)
    np.testing.assert_allclose(o2.F2_adjoint(g, 4, 6, "fft"), o2.F2_adjoint(g, 4, 6, "direct"), atol=1e-12)


@pytest.mark.parametrize("kernel", ["full", "sym"])
def test_impulse_response_matches_full_apply(kernel):
    """The one-node helper used on the full-size workload gives the same fhat as
    the full oracle applied to f = e_j."""
    M1, M2, m = 8, 8, 2
    x = radial(95, 12, 16, 1e-4)
    B = o2.bopt2_closed(x, M1, M2, 2.0, m, kernel)
    for j in (0, 7, 100, len(x) - 1):
        e = np.zeros(len(x), np.complex128)
        e[j] = 1.0
        np.testing.assert_allclose(o2.infft2_apply_impulse(x, j, M1, M2, 2.0, m, kernel), o2.infft2_apply(B, e),
                                   atol=1e-12)


def test_trig_poly_eval_2d_is_the_direct_sum():
    x = rand_nodes(97, 40)
    fh = complex_normal(98, 8 * 6).reshape(8, 6)
    np.testing.assert_allclose(trig_poly_eval_2d(x, fh), o2.nfft2_direct(x, fh), atol=1e-12)


def test_radial_trajectory_shape():
    """Spoke s, sample i at r_i (cos, sin)(pi s / spokes) within the jitter, wrapped into [-1/2, 1/2)^2."""
    x = radial(7, 8, 16, 1e-4)
    assert x.shape == (128, 2) and np.all(x >= -0.5) and np.all(x < 0.5)
    s, i = 3, 5
    r = -0.5 + i / 16
    want = (r * np.cos(np.pi * s / 8), r * np.sin(np.pi * s / 8))
    assert np.abs(x[s * 16 + i] - want).max() <= 1e-4
