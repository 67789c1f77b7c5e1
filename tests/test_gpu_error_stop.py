"""The stage solve's solution-error stop on the GPU (options.err_tol), through the C ABI.

The stage solution is the exact solution of A^R y = b (Eq. 3.10).  Near the
critical width of Lemma 3 the relative residual understates the relative error
by up to four orders of magnitude, so every solve here is compared with a sparse
direct solve (library LU) of the oracle's A^R on the same seeded inputs, at the
widths the adaptive 2D 512^2 trajectory attempts (tau = 4.57, 6.88, 8.5; up to
0.9 tau*) on meshes of its spacing (h = 0.5) and of spacing 1, and at the widths
the 3D trajectory reaches (up to tau = 20).  Tolerance: 1e-8 relative (the
accuracy target of the stage solves), with err_tol at its default 1e-9.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle.mesh import structured_mesh
from oracle.rosenbrock import ROS3PW, PFCProblem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1501_06852_gb300 as pfc  # noqa: E402

# (dim, side, length, r, psi_bar, amp, widths)
CASES = {
    "2d-s32-h0.5": (2, 32, 16.0, -0.4, -0.3, 0.1, (4.57, 6.88, 8.5)),
    "2d-s32-h1": (2, 32, 32.0, -0.4, -0.3, 0.1, (4.57, 6.88, 8.5)),
    "3d-s6": (3, 6, 6.0, -0.3, -0.35, 0.05, (5.0, 10.0, 20.0)),
}

_cache = {}


def exact(name, tau):
    key = (name, tau)
    if key not in _cache:
        dim, side, L, r, pm, amp, _ = CASES[name]
        pk = ("prob", name)
        if pk not in _cache:
            prob = PFCProblem(structured_mesh(dim, side, L), r)
            _cache[pk] = (prob, prob.consistent_state(synth.initial_psi(dim, side, pm, amp, 2)))
        prob, x = _cache[pk]
        n = prob.n
        A = prob.stage_matrix(x[n:2 * n], tau)
        b = prob.stage_rhs(x, [], [], tau)
        _cache[key] = (x, b, spla.splu(A.tocsc()).solve(b))
    return _cache[key]


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


PARAMS = [(name, tau) for name, c in CASES.items() for tau in c[6]]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name,tau", PARAMS, ids=[f"{n}-tau{t}" for n, t in PARAMS])
def test_stage_solve_meets_1e8_against_direct_solve(name, tau, precision):
    dim, side, L, r = CASES[name][:4]
    x, b, y_ex = exact(name, tau)
    with pfc.PFCSolver(dim, side, L, r=r, precision=precision, max_outer=2000) as s:
        s.assemble(cuda(x), tau)
        y, st = s.stage_solve(cuda(b))
        err = rel(host(y), y_ex)
        assert st.status == 0 and st.rel_residual <= 1e-10
        assert st.err_est <= 1e-9 and 0.0 < st.sigma_min < 1.0
        assert err <= 1e-8, (err, st)
        # the estimate is not below the true error by more than a small factor
        assert err <= 2.0 * st.err_est, (err, st.err_est)
        # a second solve on the context starts from the learned residual target and
        # still meets the tolerance
        y2, st2 = s.stage_solve(cuda(b))
        assert st2.status == 0 and rel(host(y2), y_ex) <= 1e-8


def test_plain_residual_stop_misses_near_critical_width():
    """err_tol = 0 keeps the residual test alone: at 0.9 tau* on the h = 0.5 mesh a
    1e-11 residual leaves an error above 1e-8, which the default rule removes."""
    name, tau = "2d-s32-h0.5", 8.5
    dim, side, L, r = CASES[name][:4]
    x, b, y_ex = exact(name, tau)
    with pfc.PFCSolver(dim, side, L, r=r, outer_tol=1e-11, err_tol=0.0, max_outer=2000) as s:
        s.assemble(cuda(x), tau)
        y, st = s.stage_solve(cuda(b))
        assert st.status == 0 and math.isnan(st.err_est)
        assert rel(host(y), y_ex) > 1e-8
    with pfc.PFCSolver(dim, side, L, r=r, outer_tol=1e-11, max_outer=2000) as s:
        s.assemble(cuda(x), tau)
        y, st = s.stage_solve(cuda(b))
        assert st.status == 0 and rel(host(y), y_ex) <= 1e-8


def test_fresh_contexts_give_the_same_bits():
    """The learned residual target is per context: the same solve on two fresh
    contexts gives the same bits and statistics."""
    name, tau = "2d-s32-h0.5", 4.57
    dim, side, L, r = CASES[name][:4]
    x, b, _ = exact(name, tau)
    out = []
    for _ in range(2):
        with pfc.PFCSolver(dim, side, L, r=r, precision="fp32") as s:
            s.assemble(cuda(x), tau)
            out.append(s.stage_solve(cuda(b)))
    (y1, s1), (y2, s2) = out
    assert torch.equal(y1, y2) and s1 == s2


def test_unreachable_error_tolerance_ends_at_the_cap_not_converged():
    """An error tolerance the solve cannot reach ends at max_outer with
    PFC_ERR_NOT_CONVERGED, even though the residual test passed on the way."""
    name, tau = "2d-s32-h1", 4.57
    dim, side, L, r = CASES[name][:4]
    x, b, _ = exact(name, tau)
    with pfc.PFCSolver(dim, side, L, r=r, outer_tol=1e-3, err_tol=1e-300, max_outer=40) as s:
        s.assemble(cuda(x), tau)
        _, st = s.stage_solve(cuda(b), check=False)
        assert st.status == 4 and st.outer_its == 40


def test_width_guard_caps_the_next_width_at_lemma3():
    """tau_guard: the width after an accepted step is capped at tau_guard tau*(r, <psi>) / gamma
    with <psi> the mean density of the state (Lemma 3)."""
    dim, side, L, r, pm, amp = 2, 16, 16.0, -0.4, -0.3, 0.1
    prob = PFCProblem(structured_mesh(dim, side, L), r)
    x0 = prob.consistent_state(synth.initial_psi(dim, side, pm, amp, 4))
    mean_psi = prob.mass(x0) / L ** dim
    cap = 0.9 * pfc.critical_tau(r, mean_psi) / ROS3PW.gamma
    with pfc.PFCSolver(dim, side, L, r=r, step_atol=1e3, step_rtol=1e3, tau_guard=0.9) as s:
        acc, err, tau_next, _ = s.step(cuda(x0), 2.0)
        assert acc and cap < 10.0 and tau_next == pytest.approx(cap, rel=1e-12)
    with pfc.PFCSolver(dim, side, L, r=r, step_atol=1e3, step_rtol=1e3) as s:
        acc, err, tau_next, _ = s.step(cuda(x0), 2.0)
        assert acc and tau_next == pytest.approx(10.0, rel=1e-12)
