"""Parity of the PFC1 (mobility psi^+ = psi - psi_min) path on the GPU with the FP64
oracle, through the C ABI: the block operator, the stage right-hand sides, stage
solves, Ros3Pw steps and linearised Euler steps (Eq. 2.3, 3.4, 3.10).

References: the oracle's matrices and right-hand sides; for solutions, a sparse
direct solve of the oracle's system.  The noisy start here has a small amplitude
(0.01) so that |grad mu| stays moderate and the F(mu) block does not dominate M.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle.mesh import structured_mesh
from oracle.rosenbrock import ROS3PW, PFCProblem, StepControl, euler_matrix, euler_rhs, pfc_step

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1501_06852_gb300 as pfc  # noqa: E402

CASES = [
    (2, 16, 16 * np.pi / 2, -0.35, -0.35),   # 1089 dofs per field
    (2, 5, 5 * np.pi / 2, -0.35, -0.35),     # ragged last slice
    (3, 3, 3 * np.pi / 2, -0.3, -0.34),      # Kuhn tetrahedra, 343 dofs
]
IDS = [f"{c[0]}d-s{c[1]}" for c in CASES]
AMP = 0.01
_probs = {}


def problem(dim, side, L, r):
    key = (dim, side, L, r)
    if key not in _probs:
        _probs[key] = PFCProblem(structured_mesh(dim, side, L), r, model=1)
    return _probs[key]


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def start(case, seed=21):
    dim, side, L, r, pm = case
    prob = problem(dim, side, L, r)
    return prob, prob.consistent_state(synth.initial_psi(dim, side, pm, AMP, seed))


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_pfc1_block_operator(case):
    dim, side, L, r, pm = case
    prob, x = start(case)
    n = prob.n
    tau = 0.07
    A = prob.stage_matrix(x[n:2 * n], tau, mu_k=x[:n])
    v = synth.random_vector(3 * n, 22)
    with pfc.PFCSolver(dim, side, L, r=r, model=1) as s:
        s.assemble(cuda(x), tau)
        got = host(s.apply(pfc.OP_AR, cuda(v)))
    scale = abs(A) @ np.abs(v)
    assert np.all(np.abs(got - A @ v) <= 1e-12 * (scale + scale.max() * 1e-3))


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_pfc1_stage_rhs(case):
    dim, side, L, r, pm = case
    prob, x = start(case)
    n = prob.n
    tau = 0.07
    ys = [synth.random_vector(3 * n, 30 + j) * 1e-3 for j in range(2)]
    with pfc.PFCSolver(dim, side, L, r=r, model=1) as s:
        s.assemble(cuda(x), tau)
        for i in range(3):
            xi = x + sum(ROS3PW.a(i, j) * ys[j] for j in range(i))
            want = prob.stage_rhs(xi, [y[n:2 * n] for y in ys[:i]], [ROS3PW.c(i, j) for j in range(i)], tau)
            got = host(s.stage_rhs(i, cuda(xi), cuda(np.concatenate(ys[:i])) if i else None))
            assert rel(got, want) <= 1e-12, i


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_pfc1_stage_solve(case, precision):
    dim, side, L, r, pm = case
    prob, x = start(case)
    n = prob.n
    tau = 0.07
    A = prob.stage_matrix(x[n:2 * n], tau, mu_k=x[:n])
    b = prob.stage_rhs(x, [], [], tau)
    want = spla.spsolve(A.tocsc(), b)
    with pfc.PFCSolver(dim, side, L, r=r, model=1, precision=precision, outer_tol=1e-12) as s:
        s.assemble(cuda(x), tau)
        y, st = s.stage_solve(cuda(b))
        got = host(y)
    assert st.status == 0 and st.rel_residual <= 1e-12
    assert rel(got, want) <= 1e-8, (rel(got, want), st)


@pytest.mark.parametrize("case", [CASES[0], CASES[2]], ids=[IDS[0], IDS[2]])
def test_pfc1_step(case):
    dim, side, L, r, pm = case
    prob, x0 = start(case)
    n = prob.n
    ref = pfc_step(prob, x0, 0.05, StepControl(), tol=1e-13)
    with pfc.PFCSolver(dim, side, L, r=r, model=1, precision="fp32", outer_tol=1e-12) as s:
        st = cuda(x0)
        acc, err, tau_next, stats = s.step(st, 0.05)
        got = host(st)
    assert acc == ref.accepted
    assert err == pytest.approx(ref.err, rel=1e-6)
    assert tau_next == pytest.approx(ref.tau_next, rel=1e-6)
    if acc:
        assert rel(got - x0, ref.x_new - x0) <= 1e-8
        assert abs(prob.mass(got) - prob.mass(x0)) <= 1e-9 * abs(prob.mass(x0))


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_pfc1_euler_step(case):
    dim, side, L, r, pm = case
    prob, x0 = start(case)
    n = prob.n
    psi_k = x0[n:2 * n]
    want = spla.spsolve(euler_matrix(prob, psi_k, 0.2).tocsc(), euler_rhs(prob, psi_k))
    with pfc.PFCSolver(dim, side, L, r=r, model=1, precision="fp32", outer_tol=1e-12) as s:
        st = cuda(x0)
        stats = s.euler_step(st, 0.2)
        got = host(st)
    assert stats.status == 0
    assert rel(got, want) <= 1e-8


def test_pfc1_invalid_model_and_mobility():
    with pytest.raises(pfc.PFCError):
        pfc.PFCSolver(2, 4, 4.0, model=3)
    case = CASES[1]
    dim, side, L, r, pm = case
    prob, x = start(case)
    # psi_min above the density: the mean mobility is negative
    with pfc.PFCSolver(dim, side, L, r=r, model=1, psi_min=1.0) as s:
        with pytest.raises(pfc.PFCError) as ei:
            s.assemble(cuda(x), 0.1)
        assert ei.value.status == 1
