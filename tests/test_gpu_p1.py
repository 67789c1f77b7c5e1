"""Parity of the P1 discretisation (options.degree = 1; Section 3, p = 1) on the GPU with
the FP64 oracle, through the C ABI: operators, stage right-hand sides, stage solves,
Ros3Pw steps and Euler steps, in 2D and 3D, with both inner operators."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import assembly
from oracle.mesh import structured_mesh
from oracle.rosenbrock import ROS3PW, PFCProblem, StepControl, euler_matrix, euler_rhs, pfc_step

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1501_06852_gb300 as pfc  # noqa: E402

CASES = [
    (2, 40, 40 * np.pi / 4, -0.35, -0.35, 0.1),   # 1681 vertices
    (2, 7, 7 * np.pi / 4, -0.35, -0.35, 0.1),     # 64 vertices: two slices
    (3, 8, 8 * np.pi / 4, -0.3, -0.34, 0.05),     # 729 vertices
    (2, 1, 1.0, -0.35, -0.35, 0.1),               # 4 vertices
]
IDS = [f"{c[0]}d-s{c[1]}" for c in CASES]
_probs = {}


def problem(dim, side, L, r):
    key = (dim, side, L, r)
    if key not in _probs:
        _probs[key] = PFCProblem(structured_mesh(dim, side, L, degree=1), r)
    return _probs[key]


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def start(case, seed=41):
    dim, side, L, r, pm, amp = case
    prob = problem(dim, side, L, r)
    return prob, prob.consistent_state(synth.initial_psi(dim, side, pm, amp, seed, degree=1))


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_p1_operators(case):
    dim, side, L, r, pm, amp = case
    prob, x = start(case)
    n = prob.n
    tau = 0.2
    v = synth.random_vector(n, 42)
    v3 = synth.random_vector(3 * n, 43)
    with pfc.PFCSolver(dim, side, L, r=r, degree=1) as s:
        assert s.n == n
        s.assemble(cuda(x), tau)
        for op, A in ((pfc.OP_M, prob.M), (pfc.OP_K, prob.K), (pfc.OP_A01, prob.a01(x[n:2 * n]))):
            got = host(s.apply(op, cuda(v)))
            scale = abs(A) @ np.abs(v)
            assert np.all(np.abs(got - A @ v) <= 1e-12 * (scale + scale.max() * 1e-3))
        AR = prob.stage_matrix(x[n:2 * n], tau)
        got = host(s.apply(pfc.OP_AR, cuda(v3)))
        scale = abs(AR) @ np.abs(v3)
        assert np.all(np.abs(got - AR @ v3) <= 1e-12 * (scale + scale.max() * 1e-3))


@pytest.mark.parametrize("case", CASES[:3], ids=IDS[:3])
def test_p1_stage_rhs(case):
    dim, side, L, r, pm, amp = case
    prob, x = start(case)
    n = prob.n
    tau = 0.2
    ys = [synth.random_vector(3 * n, 50 + j) * 1e-2 for j in range(2)]
    with pfc.PFCSolver(dim, side, L, r=r, degree=1) as s:
        s.assemble(cuda(x), tau)
        for i in range(3):
            xi = x + sum(ROS3PW.a(i, j) * ys[j] for j in range(i))
            want = prob.stage_rhs(xi, [y[n:2 * n] for y in ys[:i]], [ROS3PW.c(i, j) for j in range(i)], tau)
            got = host(s.stage_rhs(i, cuda(xi), cuda(np.concatenate(ys[:i])) if i else None))
            assert rel(got, want) <= 1e-12, i


@pytest.mark.parametrize("inner_op", [0, 1], ids=["sell", "stencil"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_p1_stage_solve(case, precision, inner_op):
    dim, side, L, r, pm, amp = case
    prob, x = start(case)
    n = prob.n
    tau = 0.2
    A = prob.stage_matrix(x[n:2 * n], tau)
    b = prob.stage_rhs(x, [], [], tau)
    want = spla.spsolve(A.tocsc(), b)
    with pfc.PFCSolver(dim, side, L, r=r, degree=1, precision=precision, outer_tol=1e-12,
                       inner_operator=inner_op) as s:
        s.assemble(cuda(x), tau)
        y, st = s.stage_solve(cuda(b))
        got = host(y)
    assert st.status == 0
    assert rel(got, want) <= 1e-8, (rel(got, want), st)


@pytest.mark.parametrize("case", CASES[:3], ids=IDS[:3])
def test_p1_step_and_euler(case):
    dim, side, L, r, pm, amp = case
    prob, x0 = start(case)
    n = prob.n
    ref = pfc_step(prob, x0, 0.1, StepControl(), tol=1e-13)
    want_e = spla.spsolve(euler_matrix(prob, x0[n:2 * n], 0.3).tocsc(), euler_rhs(prob, x0[n:2 * n]))
    with pfc.PFCSolver(dim, side, L, r=r, degree=1, precision="fp32", outer_tol=1e-12) as s:
        st = cuda(x0)
        acc, err, tau_next, stats = s.step(st, 0.1)
        got = host(st)
        se = cuda(x0)
        s.euler_step(se, 0.3)
        got_e = host(se)
    assert acc == ref.accepted
    assert err == pytest.approx(ref.err, rel=1e-6)
    if acc:
        assert rel(got - x0, ref.x_new - x0) <= 1e-8
    assert rel(got_e, want_e) <= 1e-8


def test_p1_invalid_degree():
    with pytest.raises(pfc.PFCError):
        pfc.PFCSolver(2, 4, 4.0, degree=3)
