"""Pins of the oracle's diagonal Schur approximation S_D (Section 4.1):
S_D = M - 2 delta K + delta K M_D^{-1} K with M_D = diag(M), and the preconditioner
P(S_D) whose step (3) runs a fixed number of Jacobi-PCG iterations (Table 2: 20).

* Lemma 1: each eigenvalue of S_D^{-1} S is the scalar ratio of its proof, written
  out through M^(1/2) from an independent eigendecomposition; where its first-order
  part is non-negative it lies within the bounds that the eigenvalues mu of
  M_D^{-1} M (from the generalised eigenproblem (M, M_D)) give.  Reading: the proof
  writes k^2 where y.Khat^2 y = |Khat y|^2 >= k^2 belongs, and the bound needs
  1 - 2 delta k >= 0 (outside it the ratio is not confined to [1, 1/d]).
* With exact inner solves, FGMRES preconditioned by P(S_D) reaches the dense
  solution of the stage system; with PCG inner solves it does too.
* rtol = 0 runs exactly the requested number of PCG iterations.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle.mesh import structured_mesh
from oracle.rosenbrock import PFCProblem
from oracle.solvers import PCH, fgmres, pcg_jacobi


@pytest.mark.parametrize("dim,side", [(2, 3), (3, 2)])
def test_lemma1_identity_and_bounds(dim, side):
    """Each eigenpair (lam, x) of S x = lam S_D x satisfies, with y = M^(1/2) x / |.|,
    Khat = M^(-1/2) K M^(-1/2), Dhat = M^(1/2) M_D^(-1) M^(1/2), k = y.Khat y, q = |Khat y|^2
    and d = (Khat y).Dhat (Khat y) / q:
        lam = (1 - 2 delta k + delta q) / (1 - 2 delta k + delta q d),
    the scalar form used in the proof of Lemma 1 (with q in place of k^2).  Where
    1 - 2 delta k >= 0, lam lies between 1 and 1/d, hence inside
    [min(1, 1/mu_max), max(1, 1/mu_min)] for mu the eigenvalues of M_D^(-1) M."""
    prob = PFCProblem(structured_mesh(dim, side, float(side)), -0.35)
    M, K = prob.M.toarray(), prob.K.toarray()
    w, V = np.linalg.eigh(M)
    Mh, Mhi = V @ np.diag(np.sqrt(w)) @ V.T, V @ np.diag(1 / np.sqrt(w)) @ V.T
    Kh = Mhi @ K @ Mhi
    Dh = Mh @ np.diag(1 / np.diag(M)) @ Mh
    mu = sla.eigh(M, np.diag(np.diag(M)), eigvals_only=True)
    lo, hi = min(1.0, 1.0 / mu.max()), max(1.0, 1.0 / mu.min())
    for tau in (0.01, 0.1):
        delta = np.sqrt(tau)
        S = M - 2 * delta * K + delta * K @ np.linalg.solve(M, K)
        SD = PCH(prob.M, prob.K, tau, 1.0, schur="sd").SD.toarray()
        lam, X = sla.eigh(S, SD)
        checked = 0
        for j in range(len(lam)):
            y = Mh @ X[:, j]
            y /= np.linalg.norm(y)
            ky = Kh @ y
            k, q = float(y @ ky), float(ky @ ky)
            d = float(ky @ Dh @ ky) / q if q > 0 else 1.0
            assert lam[j] == pytest.approx((1 - 2 * delta * k + delta * q) / (1 - 2 * delta * k + delta * q * d),
                                           rel=1e-8, abs=1e-10)
            if 1 - 2 * delta * k >= 0:
                assert lo - 1e-10 <= lam[j] <= hi + 1e-10
                checked += 1
        assert checked > 0


def test_pcg_fixed_iterations():
    prob = PFCProblem(structured_mesh(2, 4, 4.0), -0.35)
    b = synth.random_vector(prob.n, 3)
    res = pcg_jacobi(prob.M, b, 0.0, 20)
    assert res.iterations == 20 and not res.converged


@pytest.mark.parametrize("inner", ["exact", "pcg"])
def test_psd_preconditioned_stage_solve_matches_dense(inner):
    prob = PFCProblem(structured_mesh(2, 4, 8.0), -0.35)
    x = prob.consistent_state(synth.initial_psi(2, 4, -0.35, 0.1, 4))
    n = prob.n
    tau, gamma = 0.1, 0.78867513459481287
    A = prob.stage_matrix(x[n:2 * n], tau)
    b = prob.stage_rhs(x, [], [], tau)
    pc = PCH(prob.M, prob.K, tau, gamma, inner=inner, schur="sd")
    y, st = fgmres(lambda v: A @ v, b, pc.apply, 1e-13, 30, 2000)
    yd = np.linalg.solve(A.toarray(), b)
    assert st.converged and np.linalg.norm(y - yd) <= 1e-10 * np.linalg.norm(yd)
    if inner == "pcg":
        # steps (1), (2), (3), (5): four inner solves per application, step (3) with 20 iterations
        assert pc.log.calls == 4 * st.outer_iterations
        assert pc.log.per_call[2] == 20
