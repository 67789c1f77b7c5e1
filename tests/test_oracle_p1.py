"""Pins of the oracle's P1 discretisation (Lagrange degree p = 1, Section 3; the
paper's solver tables report P1 beside P2): structured meshes with the dofs on the
vertices, the P1 basis lambda_k, and the matrices and systems built from them."""
import numpy as np
import pytest

import synth
from oracle import assembly
from oracle.mesh import structured_mesh
from oracle.rosenbrock import PFCProblem, euler_matrix, euler_rhs, euler_step


@pytest.mark.parametrize("dim,side,L", [(2, 4, 3.0), (3, 3, 2.0)])
def test_p1_reproduces_linear_integrals(dim, side, L):
    """p = 1 + 2x - y: int p^2 and int |grad p|^2 over [0, L]^dim in closed form."""
    mesh = structured_mesh(dim, side, L, degree=1)
    assert mesh.n == (side + 1) ** dim
    x, y = mesh.coords[:, 0], mesh.coords[:, 1]
    p = 1.0 + 2.0 * x - y
    M, K = assembly.mass_matrix(mesh), assembly.stiffness_matrix(mesh)
    # int over [0,L]^2 of (1 + 2x - y)^2, times L^(dim-2) for the extra axis
    ix = lambda k: L ** (k + 1) / (k + 1)
    i2 = (L * L + 4 * ix(2) * L + ix(2) * L + 2 * 2 * ix(1) * L - 2 * ix(1) * L - 2 * 2 * ix(1) * ix(1))
    assert float(p @ (M @ p)) == pytest.approx(i2 * L ** (dim - 2), rel=1e-12)
    assert float(p @ (K @ p)) == pytest.approx(5.0 * L ** dim, rel=1e-12)
    assert float(np.ones(mesh.n) @ (M @ np.ones(mesh.n))) == pytest.approx(L ** dim, rel=1e-12)
    assert np.abs(K @ np.ones(mesh.n)).max() <= 1e-12


@pytest.mark.parametrize("side", [1, 2, 5])
def test_p1_pattern_nnz_2d(side):
    """Vertices plus both directions of every edge (horizontal, vertical, diagonal)."""
    mesh = structured_mesh(2, side, 1.0, degree=1)
    edges = 2 * side * (side + 1) + side * side
    assert assembly.pattern_nnz(mesh) == (side + 1) ** 2 + 2 * edges


def test_p1_nonlinear_terms_at_constant_psi():
    mesh = structured_mesh(2, 3, 2.0, degree=1)
    M = assembly.mass_matrix(mesh)
    c = 0.7
    N = assembly.nonlinear_mass(mesh, np.full(mesh.n, c))
    assert abs(N + 3 * c * c * M).max() <= 1e-13
    lc = assembly.load_cubed(mesh, np.full(mesh.n, c))
    assert np.abs(lc - c ** 3 * (M @ np.ones(mesh.n))).max() <= 1e-13


def test_p1_stage_and_euler_solves_match_dense():
    mesh = structured_mesh(2, 6, 6.0, degree=1)
    prob = PFCProblem(mesh, -0.35)
    x = prob.consistent_state(synth.initial_psi(2, 6, -0.35, 0.1, 8, degree=1))
    n = prob.n
    tau = 0.2
    A = prob.stage_matrix(x[n:2 * n], tau)
    b = prob.stage_rhs(x, [], [], tau)
    y, st = prob.stage_solve(A, b, tau, tol=1e-13)
    yd = np.linalg.solve(A.toarray(), b)
    assert st.converged and np.linalg.norm(y - yd) <= 1e-10 * np.linalg.norm(yd)
    x1, st = euler_step(prob, x, tau)
    xd = np.linalg.solve(euler_matrix(prob, x[n:2 * n], tau).toarray(), euler_rhs(prob, x[n:2 * n]))
    assert st.converged and np.linalg.norm(x1 - xd) <= 1e-10 * np.linalg.norm(xd)
