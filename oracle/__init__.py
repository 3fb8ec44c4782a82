"""Plain, slow FP64 CPU oracle for the direct inverse NFFT (Kircheis & Potts,
"Direct inversion of the nonequispaced fast Fourier transform").

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never imports, links or calls it, and it imports
nothing from the CUDA path.  It shares no code with the CUDA path; the only
common module is ``workloads`` (seeded random inputs), which holds none of the
method's arithmetic.

Layout (each function cites the passage it follows):

* ``nfft``     -- the nonequispaced Fourier matrix A (eq:matrix_A), direct
                  sums f = A fhat (eq:nfft) and h = A^* f (eq:nfft*), and the
                  dense least-squares inverse used as the exact comparator.
* ``pattern``  -- the index sets I(x_j) (eq:set_xj) and I(l) (eq:set_l).
* ``kernel``   -- the Dirichlet choice of Remark remark:Dirichlet_ansatz2:
                  the diagonal D (eq:matrix_D) and the kernel entries of L_l.
* ``bopt``     -- the per-grid-point least-squares problems of Sec. 3.2.2
                  (eq:opt_ansatz2 .. eq:solution_ansatz2): a naive tier that
                  forms L_l = F D H_l explicitly (eq:matrix_Ll) and a closed-form
                  tier that forms Re(L_l^* L_l) directly.
* ``infft``    -- the modified adjoint NFFT fhat ~ D^* F^* B_opt^* f
                  (eq:approx_ansatz2), its adjoint B_opt F D (Remark
                  remark:ansatz2_adj), the Frobenius objective, the
                  per-node error measures (eq:errors_per_node_lagrange) and
                  the residual correction fhat += D^* F^* B_opt^* (f - A fhat).
* ``infft2d``  -- the 2-D tensor-product reading of Sec. 3.2.2 (box pattern,
                  product kernel, 2-D F and D), naive and closed-form tiers.
* ``under``    -- the underdetermined case of Sec. 3.2.1: one least-squares
                  problem per node with the explicit matrix K_j (eq:matrix_Kj),
                  f_check = (1/M) D^* F^* B_opt^* f (eq:approx_ansatz1) and the
                  inverse adjoint estimate (1/M) B_opt F D h.

Readings of the paper that are not fixed by its text (all shared by both tiers):

* kernel "full": the Dirichlet choice with all M frequencies kept, D = I/M_sigma;
  kernel "sym": the remark's literal choice, D's k = -M/2 entry set to 0.
* the coefficient vector b_l is real (eq:opt_ansatz2 takes B real), so the
  normal equations are Re(G_l) b = Re(r_l), G_l = L_l^* L_l, r_l = L_l^* e_l.
* rank deficiency (the paper assumes full rank): Tikhonov regularisation
  (Re G_l + mu I) b = Re r_l with mu = tau * (diagonal of Re G_l), tau = 1e-12.
* the pattern is decided exactly on u_j = fl(M_sigma * x_j): l is in I(x_j)
  iff ceil(u_j) - m <= l <= floor(u_j) + m (mod M_sigma).
* grid index l = -M_sigma/2 .. M_sigma/2-1 is stored at p = l + M_sigma/2 and
  frequency k = -M/2 .. M/2-1 at k + M/2.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
(tests/test_oracle_*.py) except the reconstruction quality of the whole method
against the true coefficients, whose values the paper prints only as figures
("parity unpinned" for that comparison; it is reported, not asserted).
"""
from . import nfft, pattern, kernel, bopt, infft, under, infft2d  # noqa: F401
