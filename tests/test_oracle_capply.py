"""The C apply of the oracle (oracle/capply.c: gather, radix-2 FFT, D in plain C) against the
numpy apply of the oracle and against the explicit matrices: two independent evaluations of
D^* F^* B_opt^* f (eq:approx_ansatz2) must agree to fp64 rounding.  A mistake in either
FFT (a sign, a twiddle index, the (-1)^k of the grid offset) or in the D entries fails here."""
import numpy as np
import pytest

from oracle import bopt, infft, kernel, capply
from workloads import jittered, iid_uniform, complex_normal


@pytest.mark.parametrize("M,sigma,m,kind,nodes", [
    (16, 2.0, 3, "full", "jit"), (64, 2.0, 4, "sym", "iid"), (32, 1.0, 2, "full", "jit"),
    (256, 2.0, 4, "full", "iid"), (8, 4.0, 2, "sym", "jit")])
def test_c_apply_equals_numpy_apply(M, sigma, m, kind, nodes):
    N = 3 * M
    x = jittered(40 + M, N) if nodes == "jit" else iid_uniform(40 + M, N)
    B = bopt.bopt_closed(x, M, sigma, m, kind)
    f = complex_normal(41 + M, N)
    want = infft.infft_apply(B, f)
    got = capply.CApply(B, "f64")(f)
    assert infft.rel_l2(got, want) <= 1e-13
    got32 = capply.CApply(B, "f32")(f.astype(np.complex64))
    assert infft.rel_l2(got32.astype(np.complex128), want) <= 1e-4 * max(1.0, np.abs(B.b).sum() / B.Ms)


def test_c_fft_equals_the_explicit_matrix():
    """With B = identity (one node per grid point) the C apply is D^* F^* f, compared with
    the explicit F (eq:matrix_F) and D (eq:matrix_D)."""
    M, Ms = 12, 32
    x = (np.arange(Ms) - Ms // 2) / Ms
    B = bopt.BOpt(M=M, Ms=Ms, N=Ms, m=1, kernel="full", tau=0.0, ptr=np.arange(Ms + 1),
                  idx=np.arange(Ms), b=np.ones(Ms), J=np.zeros(Ms))
    f = complex_normal(42, Ms)
    want = np.conj(kernel.diag_D(M, Ms, "full")) * (bopt.matrix_F(M, Ms).conj().T @ f)
    assert np.abs(capply.CApply(B, "f64")(f) - want).max() <= 1e-13 * np.abs(want).max()
    assert capply.threads() >= 1
