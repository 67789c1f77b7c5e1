"""Pins of the oracle FGMRES's solution-error stop (oracle/solvers.py, ``err_tol``).

The stage solution is the exact solution of A^R y = b (Eq. 3.10); the library
and the oracle must reach it to a relative error, and near the critical width
of Lemma 3 the relative residual understates that error by four orders of
magnitude.  These tests check the rule against things other than itself:

* sigma, the smallest singular value of the cycles' Hessenberg matrices, equals
  the smallest singular value of A P^{-1} (dense SVD) once the Krylov space is
  the whole space, and never lies below it;
* with err_tol = 1e-9 the stage solve is within 1e-9 of a sparse direct solve
  (library LU) of the same system, for tau from 0.1 up to 0.9 of the critical
  width, on a mesh with the spacing of the 2D 512^2 workload (h = 0.5), where a
  plain 1e-11 residual stop misses 1e-8 by an order of magnitude;
* the estimate E is not below the true error by more than a small factor and
  not above it by more than a small factor.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle.mesh import structured_mesh
from oracle.rosenbrock import ROS3PW, PFCProblem
from oracle.solvers import fgmres


def test_sigma_is_smallest_singular_value_of_preconditioned_operator():
    n = 24
    rng = np.random.default_rng(7)
    A = np.eye(n) * 3 + rng.standard_normal((n, n)) / math.sqrt(n)
    A[0, 0] = 0.05                           # one small singular value
    d = 1.0 + rng.random(n)                  # a fixed diagonal preconditioner
    b = rng.standard_normal(n)
    smin = np.linalg.svd(A / d[None, :], compute_uv=False)[-1]
    # a Krylov space of dimension n (one cycle, no early stop) spans everything; the
    # agreement is limited by modified Gram-Schmidt, whose basis loses orthogonality
    # as the residual reaches rounding level (here ~1e-15 at k = n)
    _, st = fgmres(lambda v: A @ v, b, lambda v: v / d, 1e-300, restart=n, max_outer=n)
    assert st.sigma == pytest.approx(smin, rel=1e-4)
    # shorter cycles only see part of the space: never below the operator's value
    _, st = fgmres(lambda v: A @ v, b, lambda v: v / d, 1e-12, restart=5, max_outer=400)
    assert st.sigma >= smin * (1 - 1e-12)


_PROB = {}


def _problem():
    if "p" not in _PROB:
        w = synth.C2_2D_LARGE
        side = 24
        prob = PFCProblem(structured_mesh(2, side, side * w.length / w.side), w.r)
        x0 = prob.consistent_state(synth.initial_psi(2, side, w.psi_mean, w.amp, w.seed))
        _PROB["p"] = (prob, x0)
    return _PROB["p"]


# gamma tau = 0.08, 3.6 and 6.7 = 0.9 tau*(r = -0.4, psi_bar = -0.3)
@pytest.mark.parametrize("tau", [0.1, 4.57, 8.5])
def test_error_stop_meets_tolerance_against_direct_solve(tau):
    prob, x0 = _problem()
    n = prob.n
    A = prob.stage_matrix(x0[n:2 * n], tau)
    b = prob.stage_rhs(x0, [], [], tau)
    y_ex = spla.splu(A.tocsc()).solve(b)
    y, st = prob.stage_solve(A, b, tau, tol=1e-10, err_tol=1e-9)
    assert st.converged
    err = np.linalg.norm(y - y_ex) / np.linalg.norm(y_ex)
    assert err <= 1e-9
    assert err / 1.5 <= st.err_estimate <= 6.0 * max(err, 1e-13)
    assert st.rel_residual <= 1e-10


def test_plain_residual_stop_is_not_enough_near_critical_width():
    # the reason for the rule: at 0.9 tau* a 1e-11 residual leaves an error above 1e-8
    prob, x0 = _problem()
    n = prob.n
    tau = 8.5
    A = prob.stage_matrix(x0[n:2 * n], tau)
    b = prob.stage_rhs(x0, [], [], tau)
    y_ex = spla.splu(A.tocsc()).solve(b)
    y, st = prob.stage_solve(A, b, tau, tol=1e-11)
    assert st.converged
    assert np.linalg.norm(y - y_ex) / np.linalg.norm(y_ex) > 1e-8
