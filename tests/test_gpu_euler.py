"""Parity of the linearised semi-implicit Euler step (Section 3, Eq. 3.4) on the GPU
with the FP64 oracle, through the C ABI.

The reference solution of each step is a sparse direct solve of the oracle's Euler
system (the exact x_{k+1} up to rounding); the GPU step, solved to an outer
relative residual of 1e-11 or 1e-12, must match it to relative L2 1e-8, the
accuracy target of the stage solves.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle.mesh import structured_mesh
from oracle.rosenbrock import PFCProblem, euler_matrix, euler_rhs, euler_step

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1501_06852_gb300 as pfc  # noqa: E402

# (dim, side, L, r, psi_mean, amp): the 2D/3D parameter sets of the paper's
# experiments (2D r = psi_mean = -0.35; 3D r = -0.3, psi_mean = -0.34), with a
# P2 dof spacing of about pi/4, plus ragged and minimal meshes
CASES = [
    (2, 24, 24 * np.pi / 2, -0.35, -0.35, 0.1),   # 2401 dofs per field, several slices
    (2, 5, 5 * np.pi / 2, -0.35, -0.35, 0.1),     # 121 dofs: a partial last slice
    (3, 4, 4 * np.pi / 2, -0.3, -0.34, 0.05),     # Kuhn tetrahedra, 729 dofs
    (2, 1, 1.0, -0.35, -0.35, 0.1),               # 9 dofs
    (3, 1, 1.0, -0.3, -0.34, 0.05),               # 27 dofs
]
IDS = [f"{c[0]}d-s{c[1]}" for c in CASES]

_probs = {}


def problem(dim, side, L, r):
    key = (dim, side, L, r)
    if key not in _probs:
        _probs[key] = PFCProblem(structured_mesh(dim, side, L), r)
    return _probs[key]


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def start(case, seed=1):
    dim, side, L, r, pm, amp = case
    prob = problem(dim, side, L, r)
    return prob, prob.consistent_state(synth.initial_psi(dim, side, pm, amp, seed))


def exact_step(prob, x, tau):
    psi = x[prob.n:2 * prob.n]
    return spla.spsolve(euler_matrix(prob, psi, tau).tocsc(), euler_rhs(prob, psi))


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("inner_op", [0, 1], ids=["sell", "stencil"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_euler_step_parity(case, precision, inner_op):
    dim, side, L, r, pm, amp = case
    prob, x0 = start(case)
    want = exact_step(prob, x0, 0.1)
    with pfc.PFCSolver(dim, side, L, r=r, precision=precision, outer_tol=1e-11, inner_operator=inner_op) as s:
        st = cuda(x0)
        stats = s.euler_step(st, 0.1)
        got = host(st)
    assert stats.status == 0 and stats.rel_residual <= 1e-11
    assert stats.inner_calls == 5 * (stats.outer_its + 1)  # + the solution-error test
    assert rel(got, want) <= 1e-8, (rel(got, want), stats)


@pytest.mark.parametrize("tau", [0.01, 1.0, 10.0])
def test_euler_step_parity_tau_sweep(tau):
    """The step widths of the paper's time-step study, float32 inner solves."""
    case = CASES[0]
    dim, side, L, r, pm, amp = case
    prob, x0 = start(case)
    want = exact_step(prob, x0, tau)
    with pfc.PFCSolver(dim, side, L, r=r, precision="fp32", outer_tol=1e-12) as s:
        st = cuda(x0)
        stats = s.euler_step(st, tau)
        got = host(st)
    assert stats.status == 0
    assert rel(got, want) <= 1e-8, (rel(got, want), stats)


def test_euler_outer_iterations_match_oracle():
    """Same method, same tolerance: the GPU's FP64 FGMRES and the oracle's take the
    same number of outer iterations (up to one, from rounding near the threshold);
    residual test alone on both sides."""
    case = CASES[0]
    dim, side, L, r, pm, amp = case
    prob, x0 = start(case)
    for tau in (0.1, 1.0):
        _, ost = euler_step(prob, x0, tau, tol=1e-8)
        with pfc.PFCSolver(dim, side, L, r=r, precision="fp64", outer_tol=1e-8, pcg_variant=0, err_tol=0.0) as s:
            stats = s.euler_step(cuda(x0), tau)
        assert abs(stats.outer_its - ost.outer_iterations) <= 1, (tau, stats.outer_its, ost.outer_iterations)


def test_euler_trajectory_matches_oracle():
    """Five consecutive steps: every state matches the oracle's exact step from the
    oracle's previous state, mass is conserved and the GPU trajectory stays on the
    oracle's."""
    case = CASES[2]
    dim, side, L, r, pm, amp = case
    prob, x = start(case, seed=7)
    m0 = prob.mass(x)
    with pfc.PFCSolver(dim, side, L, r=r, precision="fp32", outer_tol=1e-12) as s:
        st = cuda(x)
        for k in range(5):
            s.euler_step(st, 0.5)
            x = exact_step(prob, x, 0.5)
            got = host(st)
            assert rel(got, x) <= 1e-8, k
            assert abs(prob.mass(got) - m0) <= 1e-10 * abs(m0)


def test_euler_operator_uses_gamma_one():
    """After an Euler step the context's block operator is A of Eq. (3.4) (the
    (1,1) block is M, not M / gamma); a following Rosenbrock assembly restores
    M / gamma."""
    case = CASES[1]
    dim, side, L, r, pm, amp = case
    prob, x0 = start(case)
    v = synth.random_vector(3 * prob.n, 9)
    A = euler_matrix(prob, x0[prob.n:2 * prob.n], 0.3)
    AR = prob.stage_matrix(x0[prob.n:2 * prob.n], 0.3)
    with pfc.PFCSolver(dim, side, L, r=r) as s:
        s.euler_step(cuda(x0), 0.3)
        got = host(s.apply(pfc.OP_AR, cuda(v)))
        assert np.abs(got - A @ v).max() <= 1e-12 * (abs(A) @ np.abs(v)).max()
        s.assemble(cuda(x0), 0.3)
        got = host(s.apply(pfc.OP_AR, cuda(v)))
        assert np.abs(got - AR @ v).max() <= 1e-12 * (abs(AR) @ np.abs(v)).max()


def test_euler_invalid_arguments_leave_state():
    case = CASES[1]
    dim, side, L, r, pm, amp = case
    prob, x0 = start(case)
    with pfc.PFCSolver(dim, side, L, r=r) as s:
        st = cuda(x0)
        for tau in (0.0, -1.0, float("nan"), float("inf")):
            with pytest.raises(pfc.PFCError) as ei:
                s.euler_step(st, tau)
            assert ei.value.status == 1
        bad = x0.copy()
        bad[prob.n + 2] = np.nan
        sb = cuda(bad)
        with pytest.raises(pfc.PFCError) as ei:
            s.euler_step(sb, 0.1)
        assert ei.value.status == 5
        assert np.array_equal(host(sb), bad, equal_nan=True)
        s.euler_step(st, 0.1)          # the context stays usable
        assert rel(host(st), exact_step(prob, x0, 0.1)) <= 1e-8
