"""Pins of the oracle's Ros3Pw step (oracle/rosenbrock.py).

* Table 1 as printed (golden file) equals the oracle's coefficient set.
* Order conditions: R(z) - e^z = O(z^4) on y' = lambda y;
  |R(z)| <= 1 on the left half plane and |R(-inf)| < 1 (strong A-stability, Section 3.1).
* Global order 3 (main) / 2 (embedded) on a nonlinear ODE, against a library integrator.
* PFC system: consistent start makes the algebraic rows of stage 1 vanish;
  1^T M psi is conserved (1^T K = 0); temporal order ~3 on a tiny mesh; the
  energy of Eq. (2.1) decreases over accepted steps (checked, not guaranteed).
"""
import math
import os
import warnings

import numpy as np
import pytest
from scipy.integrate import solve_ivp

import synth
from oracle.mesh import structured_mesh
from oracle.rosenbrock import (ROS3PW, PFCProblem, Ros3Pw, StepControl, next_tau, pfc_step,
                               rosenbrock_ode_step, step_error)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_table1_golden():
    vals = {}
    for line in open(os.path.join(GOLDEN, "ros3pw_table1.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    c = ROS3PW
    assert vals["gamma"] == c.gamma
    assert (vals["a21"], vals["a31"]) == (c.a21, c.a31)
    assert (vals["c21"], vals["c31"], vals["c32"]) == (c.c21, c.c31, c.c32)
    assert tuple(vals[f"m{i}"] for i in (1, 2, 3)) == c.m
    assert tuple(vals[f"mhat{i}"] for i in (1, 2, 3)) == c.mhat


def _R(z, coef=ROS3PW):
    xn, xh = rosenbrock_ode_step(lambda x: z * x, lambda x: np.array([[z]]), np.array([1.0]), 1.0, coef)
    return xn[0], xh[0]


def test_linear_order_conditions():
    zs = [-0.05, -0.025, -0.0125, -0.00625]
    e = [abs(_R(z)[0] - math.exp(z)) for z in zs]
    for a, b in zip(e, e[1:]):
        assert 14.5 < a / b < 17.0          # local error O(z^4) (ratio -> 16)


def test_strong_a_stability():
    r_inf = _R(-1e12)[0]
    assert abs(r_inf) < 1.0
    for x in np.linspace(-50, -1e-3, 60):
        for y in np.linspace(-50, 50, 31):
            z = complex(x, y)
            xn, _ = rosenbrock_ode_step(lambda v: z * v, lambda v: np.array([[z]]), np.array([1.0 + 0j]), 1.0)
            assert abs(xn[0]) <= 1.0 + 1e-12


def test_a_plausible_coefficient_mistake_breaks_the_order():
    bad = Ros3Pw(c21=-ROS3PW.c21)
    zs = [-0.1, -0.05]
    e = [abs(_R(z, bad)[0] - math.exp(z)) for z in zs]
    assert e[0] / e[1] < 12.0


def _brusselator(x):
    return np.array([1.0 + x[0] ** 2 * x[1] - 4.0 * x[0], 3.0 * x[0] - x[0] ** 2 * x[1]])


def _brusselator_jac(x):
    return np.array([[2 * x[0] * x[1] - 4.0, x[0] ** 2], [3.0 - 2 * x[0] * x[1], -x[0] ** 2]])


def test_global_order_on_nonlinear_ode():
    x0, T = np.array([1.5, 3.0]), 1.0
    ref = solve_ivp(lambda t, x: _brusselator(x), (0, T), x0, method="DOP853", rtol=1e-13, atol=1e-13).y[:, -1]
    errs = []
    for nsteps in (20, 40, 80):
        x = x0.copy()
        tau = T / nsteps
        for _ in range(nsteps):
            x, _ = rosenbrock_ode_step(_brusselator, _brusselator_jac, x, tau)
        errs.append(np.linalg.norm(x - ref))
    ords = [math.log2(a / b) for a, b in zip(errs, errs[1:])]
    assert all(2.7 < o < 3.3 for o in ords), ords
    # embedded solution: local error O(tau^3) -> one-step error ratio ~8
    le = []
    lm = []
    for tau in (0.01, 0.005, 0.0025):
        xn, xh = rosenbrock_ode_step(_brusselator, _brusselator_jac, x0, tau)
        exact = solve_ivp(lambda t, v: _brusselator(v), (0, tau), x0, method="DOP853", rtol=1e-13, atol=1e-15).y[:, -1]
        le.append(np.linalg.norm(xh - exact))
        lm.append(np.linalg.norm(xn - exact))
    assert all(7.5 < a / b < 9.0 for a, b in zip(le, le[1:])), le     # embedded: O(tau^3) local
    assert all(15.0 < a / b < 17.0 for a, b in zip(lm, lm[1:])), lm   # main: O(tau^4) local


@pytest.fixture(scope="module")
def small_pfc():
    prob = PFCProblem(structured_mesh(2, 4, 8.0), -0.4)
    x0 = prob.consistent_state(synth.initial_psi(2, 4, -0.3, 0.1, 1))
    return prob, x0


def test_consistent_start_zeroes_algebraic_rows(small_pfc):
    prob, x0 = small_pfc
    n = prob.n
    b = prob.stage_rhs(x0, [], [], 0.1)
    scale = np.linalg.norm(b[n:2 * n])
    assert np.linalg.norm(b[:n]) < 1e-12 * scale
    assert np.linalg.norm(b[2 * n:]) < 1e-12 * scale
    assert abs(b[n:2 * n].sum()) < 1e-12 * scale


def test_consistent_start_by_pcg_matches_lu():
    """The PCG route of the consistent start (used on the benchmark mesh, where the LU
    of M is slow) gives the LU route's state, and so zeroes the algebraic rows too."""
    prob = PFCProblem(structured_mesh(2, 12, 6.0), -0.4)
    psi0 = synth.initial_psi(2, 12, -0.3, 0.1, 7)
    x_lu = prob.consistent_state(psi0)
    x_cg = prob.consistent_state(psi0, tol=1e-15, solver="pcg")
    assert np.linalg.norm(x_cg - x_lu) <= 1e-13 * np.linalg.norm(x_lu)
    n = prob.n
    b = prob.stage_rhs(x_cg, [], [], 0.1)
    assert np.linalg.norm(b[:n]) < 1e-12 * np.linalg.norm(b[n:2 * n])


def test_mass_conservation_and_energy(small_pfc):
    prob, x = small_pfc
    m0 = prob.mass(x)
    energies = [prob.energy(x)]
    tau = 0.1
    for _ in range(4):
        res = pfc_step(prob, x, tau)
        if res.accepted:
            x = res.x_new
            energies.append(prob.energy(x))
        tau = res.tau_next
        assert abs(prob.mass(x) - m0) < 1e-11 * abs(m0)
    if any(b > a for a, b in zip(energies, energies[1:])):
        warnings.warn(f"energy rose on some accepted step: {energies}")
    assert energies[-1] < energies[0]


def test_temporal_order_on_pfc_system():
    prob = PFCProblem(structured_mesh(2, 2, 12.0), -0.4)
    n = prob.n
    x0 = prob.consistent_state(synth.initial_psi(2, 2, -0.3, 0.1, 3))
    T = 0.4

    def run(nsteps):
        x = x0.copy()
        for _ in range(nsteps):
            x = pfc_step(prob, x, T / nsteps, StepControl(atol=1e9, rtol=0.0), tol=1e-14, inner="exact").x_new
        return x[n:2 * n]

    ref = run(512)
    errs = [np.linalg.norm(run(k) - ref) for k in (16, 32, 64)]
    ords = [math.log2(a / b) for a, b in zip(errs, errs[1:])]
    assert all(o > 2.6 for o in ords), (errs, ords)


def test_step_control_rejects_and_shrinks(small_pfc):
    prob, x = small_pfc
    res = pfc_step(prob, x, 0.5, StepControl(atol=1e-9, rtol=1e-9))
    assert not res.accepted and res.err > 1.0 and res.tau_next < 0.5
    assert np.array_equal(res.x_new, x)
    # an accepted step right after a rejection does not grow the width
    ok = pfc_step(prob, x, res.tau_next, prev_rejected=True)
    assert ok.accepted and ok.tau_next <= res.tau_next
    free = pfc_step(prob, x, res.tau_next)
    assert free.tau_next > res.tau_next
    ctl = StepControl()
    assert next_tau(1.0, 0.0, ctl) == 5.0
    assert next_tau(1.0, 1e6, ctl) == 0.2
    assert next_tau(1.0, 1.0, ctl) == pytest.approx(0.9)
    e = np.array([1e-3, -1e-3])
    assert step_error(np.zeros(2), np.zeros(2), e, ctl) == pytest.approx(1.0)
