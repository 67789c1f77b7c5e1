"""Planted mistakes in the oracle must fail a pin (mistakes are planted on the CPU only)."""
import numpy as np
import pytest

import synth
from oracle import assembly, p2
from oracle.mesh import structured_mesh
from oracle.rosenbrock import ROS3PW, PFCProblem


def test_wrong_edge_basis_breaks_quadratic_reproduction(monkeypatch):
    good = p2.basis

    def bad(xi):
        v, g = good(xi)
        v = v.copy()
        v[:, 3:] *= 0.5          # 2 lambda_a lambda_b instead of 4 lambda_a lambda_b
        return v, g

    monkeypatch.setattr(p2, "basis", bad)
    mesh = structured_mesh(2, 2, 2.0)
    M = assembly.mass_matrix(mesh, assembly.Reference(2))
    one = np.ones(mesh.n)
    assert abs(one @ (M @ one) - 4.0) > 1e-3


def test_transposed_inverse_jacobian_breaks_stiffness(monkeypatch):
    good = assembly._geometry

    def bad(verts):
        det, inv = good(verts)
        return det, np.transpose(inv, (0, 2, 1))

    monkeypatch.setattr(assembly, "_geometry", bad)
    mesh = structured_mesh(2, 2, 2.0)
    K = assembly.stiffness_matrix(mesh)
    u = mesh.coords[:, 0] * mesh.coords[:, 1] + mesh.coords[:, 0]
    # int over [0,2]^2 of |grad (xy + x)|^2 = int (y+1)^2 + x^2 = 52/3 + 16/3 = 68/3
    assert abs(u @ (K @ u) - 68.0 / 3.0) > 1e-3


def test_sign_error_in_stage_rhs_breaks_consistency(monkeypatch):
    prob = PFCProblem(structured_mesh(2, 3, 6.0), -0.4)
    x0 = prob.consistent_state(synth.initial_psi(2, 3, -0.3, 0.1, 1))
    good = prob.stage_rhs

    def bad(x_i, dpsi, c_row, tau):
        b = good(x_i, dpsi, c_row, tau)
        n = prob.n
        b[2 * n:] += 2.0 * (prob.K @ x_i[n:2 * n])      # -M omega + K psi
        return b

    n = prob.n
    b = bad(x0, [], [], 0.1)
    assert np.linalg.norm(b[2 * n:]) > 1e-3 * np.linalg.norm(b[n:2 * n])
