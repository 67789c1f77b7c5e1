"""Pins of the oracle's solvers and preconditioner (oracle/solvers.py).

* Jacobi-PCG and FGMRES against direct solves (library LU).
* The full stage solve (FGMRES(30) + P_CH + PCG inner) against a dense LU of A^R
  on tiny meshes, to 1e-12.
* The discrete form of the spectral statement of Section 6 (Eq. 6.9): for a
  constant psi_bar and exact inner solves the preconditioned stage operator has
  the eigenvalue 1 (2n times) and q_CH(mu_j) for the generalised eigenvalues mu_j
  of (K, M), with tau replaced by tau_e = gamma tau.
* Lemma 2: the eigenvalues of S_CH^{-1} S lie in [(1 - sqrt(delta))/2, 1].
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import analysis, assembly
from oracle.mesh import structured_mesh
from oracle.rosenbrock import ROS3PW, PFCProblem
from oracle.solvers import PCH, fgmres, pcg_jacobi


def test_pcg_jacobi_reaches_tolerance_and_solution():
    mesh = structured_mesh(2, 6, 6.0)
    M = assembly.mass_matrix(mesh)
    K = assembly.stiffness_matrix(mesh)
    A = (M + 0.3 * K).tocsr()
    b = synth.random_vector(mesh.n, 3)
    res = pcg_jacobi(A, b, 1e-12, 1000)
    assert res.converged and res.iterations < mesh.n
    xd = spla.spsolve(A.tocsc(), b)
    assert np.linalg.norm(res.x - xd) / np.linalg.norm(xd) < 1e-10
    loose = pcg_jacobi(A, b, 1e-3, 1000)
    assert np.linalg.norm(b - A @ loose.x) <= 1e-3 * np.linalg.norm(b)
    assert loose.iterations < res.iterations
    assert pcg_jacobi(A, np.zeros(mesh.n), 1e-3, 10).iterations == 0


def test_fgmres_identity_preconditioner_nonsymmetric():
    n = 80
    rng = np.random.default_rng(0)
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) / math.sqrt(n)
    b = rng.standard_normal(n)
    x, st = fgmres(lambda v: A @ v, b, lambda v: v, 1e-12, restart=10, max_outer=2000)
    assert st.converged and st.restarts > 1
    assert np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-10 * np.linalg.norm(x)


TINY = [(2, 2, 4.0), (2, 3, 3.0), (2, 4, 8.0), (3, 1, 2.0), (3, 2, 4.0)]


@pytest.mark.parametrize("dim,side,L", TINY, ids=[f"{d}d-s{s}" for d, s, _ in TINY])
@pytest.mark.parametrize("tau", [0.1, 1.0])
def test_stage_solve_matches_dense_lu(dim, side, L, tau):
    prob = PFCProblem(structured_mesh(dim, side, L), -0.4)
    x = np.concatenate([synth.random_vector(prob.n, 21), synth.initial_psi(dim, side, -0.3, 0.1, 22),
                        synth.random_vector(prob.n, 23)])
    psi = x[prob.n:2 * prob.n]
    A = prob.stage_matrix(psi, tau)
    b = prob.stage_rhs(x, [synth.random_vector(prob.n, 24)], [ROS3PW.c21], tau)
    y, st = prob.stage_solve(A, b, tau, tol=1e-13)
    yd = np.linalg.solve(A.toarray(), b)
    assert st.converged
    assert np.linalg.norm(y - yd) / np.linalg.norm(yd) < 1e-12


def _dense_pinv(pc, n3):
    return np.column_stack([pc.apply(e) for e in np.eye(n3)])


@pytest.mark.parametrize("dim,side,L,tau,psi_bar,r", [
    (2, 3, 6.0, 0.1, -0.3, -0.4),
    (2, 3, 3.0, 1.0, -0.35, -0.35),
    (3, 1, 2.0, 0.5, -0.34, -0.3),
])
def test_spectrum_of_preconditioned_stage_operator(dim, side, L, tau, psi_bar, r):
    prob = PFCProblem(structured_mesh(dim, side, L), r)
    n = prob.n
    A = prob.stage_matrix(np.full(n, psi_bar), tau).toarray()
    pc = PCH(prob.M, prob.K, tau, ROS3PW.gamma, inner="exact")
    ev = np.linalg.eigvals(A @ _dense_pinv(pc, 3 * n))
    assert np.abs(ev.imag).max() < 1e-5
    mus = sla.eigh(prob.K.toarray(), prob.M.toarray(), eigvals_only=True)
    mus = np.maximum(mus, 0.0)
    tau_e = ROS3PW.gamma * tau
    want = np.concatenate([np.ones(2 * n), [analysis.qch_eigenvalue(m, tau_e, r, psi_bar) for m in mus]])
    got = np.sort(ev.real)
    want = np.sort(want)
    assert np.abs(got - want).max() < 1e-5 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("delta", [0.05, 0.3, 0.9])
def test_lemma2_schur_approximation_bounds(delta):
    prob = PFCProblem(structured_mesh(2, 4, 4.0), -0.4)
    M, K = prob.M.toarray(), prob.K.toarray()
    KMK = K @ np.linalg.solve(M, K)
    S = M - 2 * delta * K + delta * KMK
    Sch = M + 2 * math.sqrt(delta) * K + delta * KMK
    lam = np.sort(sla.eigvals(S, Sch).real)
    lo, hi = analysis.lemma2_bounds(delta)
    assert lam.min() >= lo - 1e-10 and lam.max() <= hi + 1e-10
    # the closed form lambda(mu) over the eigenvalues mu of M^{-1}K
    mus = sla.eigh(K, M, eigvals_only=True)
    assert np.allclose(np.sort([analysis.lemma2_lambda(m, delta) for m in mus]), lam, atol=1e-9)
    # (3.1) + (3.2) with exact solves apply S_CH^{-1} M
    pc = PCH(prob.M, prob.K, delta ** 2 / ROS3PW.gamma, ROS3PW.gamma, inner="exact")
    y1 = synth.random_vector(prob.n, 5)
    w = pc._solve(pc.MsK, prob.M @ y1)
    x1 = pc._solve(pc.MsK, prob.M @ w)
    assert np.allclose(x1, np.linalg.solve(Sch, M @ y1), rtol=1e-10, atol=1e-12)


def test_inner_pcg_counts_are_logged():
    prob = PFCProblem(structured_mesh(2, 8, 8.0), -0.4)
    pc = PCH(prob.M, prob.K, 0.1, ROS3PW.gamma)
    pc.apply(synth.random_vector(3 * prob.n, 9))
    assert pc.log.calls == 5 and all(k > 0 for k in pc.log.per_call)
