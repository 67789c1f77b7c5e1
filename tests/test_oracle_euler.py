"""Pins of the oracle's linearised semi-implicit Euler step (Section 3, Eq. 3.3-3.4)."""
import numpy as np
import pytest

import synth
from oracle import assembly
from oracle.mesh import structured_mesh
from oracle.rosenbrock import PFCProblem, euler_matrix, euler_rhs, euler_step


@pytest.fixture(scope="module")
def prob():
    return PFCProblem(structured_mesh(2, 4, 8.0), -0.35)


def test_euler_step_matches_dense_solve(prob):
    x0 = prob.consistent_state(synth.initial_psi(2, 4, -0.35, 0.1, 3))
    x1, st = euler_step(prob, x0, 0.1)
    A = euler_matrix(prob, x0[prob.n:2 * prob.n], 0.1).toarray()
    xd = np.linalg.solve(A, euler_rhs(prob, x0[prob.n:2 * prob.n]))
    assert st.converged and np.linalg.norm(x1 - xd) <= 1e-12 * np.linalg.norm(xd)


def test_euler_step_solves_the_weak_form(prob):
    """The three rows of Eq. (3.4) hold for the new state, written out independently:
    (mu - (1+r) psi - 3 psi_k^2 psi, th) + (2 grad psi + grad om, grad th) = (-2 psi_k^3, th);
    (psi, th') + tau (grad mu, grad th') = (psi_k, th');  (om, th'') + (grad psi, grad th'') = 0."""
    n = prob.n
    x0 = prob.consistent_state(synth.initial_psi(2, 4, -0.35, 0.1, 4))
    tau = 0.3
    x1, _ = euler_step(prob, x0, tau)
    mu, psi, om = x1[:n], x1[n:2 * n], x1[2 * n:]
    psik = x0[n:2 * n]
    M, K = prob.M, prob.K
    N = assembly.nonlinear_mass(prob.mesh, psik, prob.ref)      # (-3 psi_k^2 phi_j, phi_i)
    r0 = M @ mu - (1 + prob.r) * (M @ psi) + N @ psi + 2 * (K @ psi) + K @ om \
        + 2 * assembly.load_cubed(prob.mesh, psik, prob.ref)
    r1 = M @ psi + tau * (K @ mu) - M @ psik
    r2 = M @ om + K @ psi
    scale = np.linalg.norm(M @ psik)
    for rr in (r0, r1, r2):
        assert np.linalg.norm(rr) <= 1e-11 * scale


def test_euler_conserves_mass(prob):
    x0 = prob.consistent_state(synth.initial_psi(2, 4, -0.35, 0.1, 5))
    x1, _ = euler_step(prob, x0, 1.0)
    assert prob.mass(x1) == pytest.approx(prob.mass(x0), rel=1e-11)
