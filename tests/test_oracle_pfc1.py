"""Pins of the oracle's PFC1 (mobility) parts: the Wasserstein flow of Eq. 2.3 with
psi^+ = psi - psi_min, the matrices K_+(psi) and F(mu) of Eq. 3.10 and the stage and
Euler systems built from them.

Each pin checks against something other than the formula it tests:
* K_+ at constant mobility c is c K (the assembled stiffness matrix);
* K_+ is symmetric, annihilates constants, and reproduces a closed-form integral for
  polynomials that P2 represents exactly;
* F(mu) is the derivative of the directly integrated load (psi^+ grad mu, grad phi_i)
  in psi (central differences are exact: the load is affine in psi);
* the PFC1 stage system's second block row is the Jacobian of that load;
* a PFC1 stage solve agrees with a dense solve, and a PFC1 Ros3Pw step conserves mass.
"""
import numpy as np
import pytest

import synth
from oracle import assembly
from oracle.mesh import structured_mesh
from oracle.rosenbrock import PFCProblem, StepControl, euler_matrix, euler_rhs, euler_step, pfc_step


@pytest.fixture(scope="module")
def mesh2():
    return structured_mesh(2, 4, 4.0)


def lattice_coords(mesh):
    """Coordinates of the P2 dofs (lexicographic half-spacing lattice, x fastest)."""
    dim, side, L = mesh.dim, mesh.side, mesh.length
    lat = 2 * side + 1
    idx = np.arange(mesh.n)
    return [((idx // lat ** k) % lat) * (L / (2 * side)) for k in range(dim)]


def test_kplus_at_constant_mobility_is_scaled_stiffness(mesh2):
    K = assembly.stiffness_matrix(mesh2)
    for c in (0.3, 1.0, 2.7):
        Kp = assembly.mobility_stiffness(mesh2, np.full(mesh2.n, c))
        assert abs(Kp - c * K).max() <= 1e-13 * abs(K).max()


def test_kplus_symmetric_and_annihilates_constants(mesh2):
    psi_plus = 1.0 + 0.5 * synth.random_vector(mesh2.n, 3)
    Kp = assembly.mobility_stiffness(mesh2, psi_plus)
    assert abs(Kp - Kp.T).max() <= 1e-14 * abs(Kp).max()
    assert np.abs(Kp @ np.ones(mesh2.n)).max() <= 1e-13 * abs(Kp).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_kplus_closed_form(dim):
    """v = x, mu = x^2, psi^+ = x + 1 on [0, L]^dim: v^T K_+ mu = int (x + 1) 2x dx = L^(dim-1) (2 L^3/3 + L^2)."""
    L = 3.0
    mesh = structured_mesh(dim, 3, L)
    x = lattice_coords(mesh)[0]
    Kp = assembly.mobility_stiffness(mesh, x + 1.0)
    want = L ** (dim - 1) * (2.0 * L ** 3 / 3.0 + L ** 2)
    assert float(x @ (Kp @ x ** 2)) == pytest.approx(want, rel=1e-12)


def test_mobility_load_is_kplus_times_mu(mesh2):
    psi_plus = 1.2 + 0.3 * synth.random_vector(mesh2.n, 4)
    mu = synth.random_vector(mesh2.n, 5)
    direct = assembly.mobility_load(mesh2, psi_plus, mu)
    Kp = assembly.mobility_stiffness(mesh2, psi_plus)
    assert np.abs(direct - Kp @ mu).max() <= 1e-13 * np.abs(direct).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_F_is_the_psi_derivative_of_the_mobility_load(dim):
    mesh = structured_mesh(dim, 2, 2.0)
    psi_plus = 1.1 + 0.2 * synth.random_vector(mesh.n, 6)
    mu = synth.random_vector(mesh.n, 7)
    d = synth.random_vector(mesh.n, 8)
    eps = 0.25
    fd = (assembly.mobility_load(mesh, psi_plus + eps * d, mu)
          - assembly.mobility_load(mesh, psi_plus - eps * d, mu)) / (2 * eps)
    F = assembly.mobility_derivative(mesh, mu)
    assert np.abs(F @ d - fd).max() <= 1e-12 * np.abs(fd).max()
    assert abs(assembly.mobility_derivative(mesh, np.full(mesh.n, 3.0))).max() <= 1e-13


def test_stage_row_is_the_jacobian_of_the_flux():
    """Second block row of A^R / tau minus the M / (gamma tau) part equals the derivative
    of (mu, psi) -> (psi^+ grad mu, grad phi_i), taken by central differences."""
    mesh = structured_mesh(2, 3, 3.0)
    prob = PFCProblem(mesh, -0.35, model=1)
    n = prob.n
    mu = synth.random_vector(n, 9)
    psi = -0.3 + 0.2 * synth.random_vector(n, 10)
    tau, gamma = 0.4, 0.78867513459481287
    A = prob.stage_matrix(psi, tau, mu_k=mu).tocsr()
    row = A[n:2 * n, :2 * n] - __import__("scipy.sparse", fromlist=["hstack"]).hstack(
        [0 * prob.M, prob.M / gamma]).tocsr()
    dmu, dpsi = synth.random_vector(n, 11), synth.random_vector(n, 12)
    eps = 0.1
    flux = lambda m, p: assembly.mobility_load(mesh, p - prob.psi_min, m)
    fd = (flux(mu + eps * dmu, psi + eps * dpsi) - flux(mu - eps * dmu, psi - eps * dpsi)) / (2 * eps)
    got = row @ np.concatenate([dmu, dpsi]) / tau
    assert np.abs(got - fd).max() <= 1e-12 * np.abs(fd).max()


def test_pfc1_reduces_to_pfc2_pieces():
    """With model 2 the mobility matrices are K and 0; model 1 differs from it."""
    mesh = structured_mesh(2, 2, 2.0)
    p2 = PFCProblem(mesh, -0.35)
    p1 = PFCProblem(mesh, -0.35, M=p2.M, K=p2.K, model=1)
    psi = np.full(p2.n, -0.5)            # psi^+ = 1 everywhere
    assert abs(p1.kplus(psi) - p2.K).max() <= 1e-13 * abs(p2.K).max()
    assert p1.m0(psi) == pytest.approx(1.0, rel=1e-13)


def test_pfc1_stage_solve_matches_dense():
    mesh = structured_mesh(2, 3, 3.0)
    prob = PFCProblem(mesh, -0.35, model=1)
    x = prob.consistent_state(synth.initial_psi(2, 3, -0.35, 0.1, 13))
    mu, psi, _ = prob.split(x)
    tau = 0.5
    A = prob.stage_matrix(psi, tau, mu_k=mu)
    b = prob.stage_rhs(x, [], [], tau)
    y, st = prob.stage_solve(A, b, tau, tol=1e-13, m0=prob.m0(psi))
    yd = np.linalg.solve(A.toarray(), b)
    # the F(mu) block makes A^R far from normal here (|grad mu| of a noisy start is large),
    # so a 1e-13 residual bounds the error less tightly than for PFC2
    assert st.converged and np.linalg.norm(y - yd) <= 1e-9 * np.linalg.norm(yd)


def test_pfc1_step_conserves_mass_and_euler_matches_dense():
    mesh = structured_mesh(2, 4, 8.0)
    prob = PFCProblem(mesh, -0.35, model=1)
    x0 = prob.consistent_state(synth.initial_psi(2, 4, -0.35, 0.1, 14))
    # a noisy start has a large grad mu, so the mobility term moves psi fast: small step
    res = pfc_step(prob, x0, 0.01, StepControl(atol=1e-2, rtol=1e-2))
    assert res.accepted
    assert prob.mass(res.x_new) == pytest.approx(prob.mass(x0), rel=1e-11)
    x1, st = euler_step(prob, x0, 0.3)
    psi_k = x0[prob.n:2 * prob.n]
    xd = np.linalg.solve(euler_matrix(prob, psi_k, 0.3).toarray(), euler_rhs(prob, psi_k))
    assert st.converged and np.linalg.norm(x1 - xd) <= 1e-11 * np.linalg.norm(xd)
