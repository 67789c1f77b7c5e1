"""Parity of the P(S_D) preconditioner (Section 4.1: S_D = M - 2 delta K + delta K
M_D^{-1} K, step (3) by a fixed number of Jacobi-PCG iterations, Table 2) on the GPU
with the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle.mesh import structured_mesh
from oracle.rosenbrock import ROS3PW, PFCProblem, euler_matrix, euler_rhs
from oracle.solvers import PCH

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1501_06852_gb300 as pfc  # noqa: E402

CASES = [
    (2, 32, 32.0, -0.4, -0.3, 0.1),
    (2, 5, 5.0, -0.4, -0.3, 0.1),
    (3, 4, 4.0, -0.3, -0.35, 0.05),
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


def start(case):
    dim, side, L, r, pm, amp = case
    prob = problem(dim, side, L, r)
    return prob, prob.consistent_state(synth.initial_psi(dim, side, pm, amp, 31))


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_psd_application_matches_oracle(case):
    """One application of P(S_D)^{-1} in float64: steps (1), (2), (5) solved tightly on
    both sides, step (3) the same 20 PCG iterations."""
    dim, side, L, r, pm, amp = case
    prob, x = start(case)
    n = prob.n
    tau = 0.1
    v = synth.random_vector(3 * n, 32)
    pc = PCH(prob.M, prob.K, tau, ROS3PW.gamma, inner="pcg", inner_rtol=1e-13, schur="sd", sd_its=20)
    want = pc.apply(v)
    with pfc.PFCSolver(dim, side, L, r=r, schur=1, schur_its=20, inner_rtol=1e-13) as s:
        s.assemble(cuda(x), tau)
        got = host(s.apply(pfc.OP_PCH, cuda(v)))
    assert rel(got, want) <= 1e-9, rel(got, want)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_psd_stage_solve(case, precision):
    dim, side, L, r, pm, amp = case
    prob, x = start(case)
    n = prob.n
    tau = 0.1
    A = prob.stage_matrix(x[n:2 * n], tau)
    b = prob.stage_rhs(x, [], [], tau)
    want = spla.spsolve(A.tocsc(), b)
    with pfc.PFCSolver(dim, side, L, r=r, schur=1, precision=precision, outer_tol=1e-12) as s:
        s.assemble(cuda(x), tau)
        y, st = s.stage_solve(cuda(b))
        got = host(y)
    assert st.status == 0 and st.rel_residual <= 1e-12
    assert st.inner_calls == 4 * (st.outer_its + 1)  # + the solution-error test
    assert rel(got, want) <= 1e-8, (rel(got, want), st)


def test_psd_euler_step():
    case = CASES[0]
    dim, side, L, r, pm, amp = case
    prob, x0 = start(case)
    n = prob.n
    psi_k = x0[n:2 * n]
    want = spla.spsolve(euler_matrix(prob, psi_k, 0.1).tocsc(), euler_rhs(prob, psi_k))
    with pfc.PFCSolver(dim, side, L, r=r, schur=1, precision="fp32", outer_tol=1e-12) as s:
        st = cuda(x0)
        stats = s.euler_step(st, 0.1)
        got = host(st)
    assert stats.status == 0 and stats.inner_calls == 4 * (stats.outer_its + 1)
    assert rel(got, want) <= 1e-8


def test_psd_invalid_options():
    for kw in ({"schur": 2}, {"schur": 1, "schur_its": 0}):
        with pytest.raises(pfc.PFCError):
            pfc.PFCSolver(2, 4, 4.0, **kw)
