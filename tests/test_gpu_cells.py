"""Cell kernels of the float inner solves (P2, cell-major rows) against the oracle.

The cell kernels run the Chronopoulos-Gear Jacobi-PCG of the P_CH inner solves
(Table 2) with one grid barrier per iteration: each block recomputes the halo of
u = D r in shared memory instead of waiting for its neighbours.  In exact arithmetic
they give the iterates of the textbook Jacobi-PCG, so every solve is compared with the
oracle's ``pcg_jacobi`` (float64): the float32 solve meets its residual target in the
float64 norm (up to the float32 rounding of the iteration), takes the same number of
iterations within 2, and lands on the same iterate to 1e-4 relative.  Stage solves
(Eq. 3.10) meet the method's 1e-8 against the oracle.  Sizes: 2D sides 2 to 32 (tiny
tiles), 256 at h = 0.5 and the 512^2 benchmark mesh (1.05M rows per field); 3D sides 2
to 16 (cells of eight rows, 3D tiles and rings).
"""
import math

import numpy as np
import pytest

import synth
from oracle.mesh import structured_mesh
from oracle.rosenbrock import ROS3PW, PFCProblem
from oracle.solvers import pcg_jacobi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1501_06852_gb300 as pfc  # noqa: E402

_probs = {}


def problem(side, L, r=-0.4):
    key = (side, L, r)
    if key not in _probs:
        _probs[key] = PFCProblem(structured_mesh(2, side, L), r)
    return _probs[key]


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def state(prob, side, seed=1):
    n = prob.n
    return np.concatenate([synth.random_vector(n, seed + 100), synth.initial_psi(2, side, -0.3, 0.1, seed),
                           synth.random_vector(n, seed + 200)])


def inner_matrices(prob, tau):
    delta = math.sqrt(ROS3PW.gamma * tau)
    return [prob.M, (prob.M + delta * prob.K).tocsr(), (prob.M + math.sqrt(delta) * prob.K).tocsr()]


def test_cell_kernels_run_where_they_apply():
    on = dict(precision="fp32")
    with pfc.PFCSolver(2, 8, 8.0, **on) as s:
        assert s.cell_kernels
    with pfc.PFCSolver(2, 8, 8.0, precision="fp16") as s:
        assert s.cell_kernels
    for kw in (dict(precision="fp64"), dict(precision="fp32", cells=0), dict(precision="fp32", inner_operator=0),
               dict(precision="fp32", smem_window=1), dict(precision="fp32", pcg_variant=1),
               dict(precision="fp32", degree=1)):
        with pfc.PFCSolver(2, 8, 8.0, **kw) as s:
            assert not s.cell_kernels, kw
    with pfc.PFCSolver(3, 4, 4.0, precision="fp32") as s:
        assert s.cell_kernels
    with pfc.PFCSolver(3, 4, 4.0, precision="fp32", cells=0) as s:
        assert not s.cell_kernels
    # a single-cell mesh has no interior row: the host keeps the cell kernels off
    with pfc.PFCSolver(2, 1, 1.0, precision="fp32") as s:
        assert not s.cell_kernels


SIDES = [(32, 32.0), (5, 5.0), (2, 2.0), (256, 128.0)]


@pytest.mark.parametrize("side,L", SIDES, ids=[f"s{s}" for s, _ in SIDES])
def test_cell_pcg_matches_oracle(side, L):
    prob = problem(side, L)
    x = state(prob, side)
    tau = 2.3
    b = synth.random_vector(prob.n, 8)
    with pfc.PFCSolver(2, side, L, r=-0.4, precision="fp32") as s:
        assert s.cell_kernels
        s.assemble(cuda(x), tau)
        for which, A in enumerate(inner_matrices(prob, tau)):
            for rtol in (1e-3, 1e-5):
                got, its = s.pcg(which, cuda(b), rtol)
                got = host(got)
                ref = pcg_jacobi(A, b, rtol, 10000)
                res = np.linalg.norm(b - A @ got) / np.linalg.norm(b)
                assert res <= rtol * 1.05 + 2e-6, (which, rtol, res)
                assert abs(its - ref.iterations) <= 2, (which, rtol, its, ref.iterations)
                if its == ref.iterations:
                    assert np.linalg.norm(got - ref.x) <= 1e-4 * np.linalg.norm(ref.x)


@pytest.mark.parametrize("side,L", SIDES[:3], ids=[f"s{s}" for s, _ in SIDES[:3]])
def test_cell_and_lexicographic_orders_agree(side, L):
    """The same fp32 Chronopoulos-Gear iterates on the cell kernels and on the
    per-warp lexicographic path (two barriers per iteration)."""
    prob = problem(side, L)
    x = state(prob, side)
    tau = 0.7
    b = synth.random_vector(prob.n, 9)
    out = {}
    for cells in (1, 0):
        with pfc.PFCSolver(2, side, L, r=-0.4, precision="fp32", pcg_variant=3, cells=cells) as s:
            assert s.cell_kernels == (cells == 1)
            s.assemble(cuda(x), tau)
            out[cells] = [s.pcg(which, cuda(b), 1e-4) for which in range(3)]
    for (g1, i1), (g0, i0) in zip(out[1], out[0]):
        assert abs(i1 - i0) <= 1
        if i1 == i0:
            a, c = host(g1), host(g0)
            assert np.linalg.norm(a - c) <= 1e-4 * np.linalg.norm(c)


def _oracle_stage(side, L, tau):
    prob = problem(side, L)
    x = prob.consistent_state(synth.initial_psi(2, side, -0.3, 0.1, 1), tol=1e-15, solver="pcg")
    A = prob.stage_matrix(x[prob.n:2 * prob.n], tau)
    b = prob.stage_rhs(x, [], [], tau)
    y, st = prob.stage_solve(A, b, tau, tol=1e-13, err_tol=1e-11)
    assert st.converged
    return x, b, y


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("side,L,tau", [(32, 32.0, 0.1), (32, 16.0, 4.57), (5, 5.0, 1.0), (2, 2.0, 0.1)],
                         ids=["s32-tau0.1", "s32-h0.5-tau4.57", "s5-tau1", "s2-tau0.1"])
def test_cell_stage_solves_match_oracle(side, L, tau, precision):
    x, b, yref = _oracle_stage(side, L, tau)
    with pfc.PFCSolver(2, side, L, r=-0.4, precision=precision) as s:
        assert s.cell_kernels
        s.assemble(cuda(x), tau)
        y, st = s.stage_solve(cuda(b))
        y = host(y)
    err = np.linalg.norm(y - yref) / np.linalg.norm(yref)
    assert st.status == 0 and err <= 1e-8, (err, st)
    assert st.inner_calls == 5 * (st.outer_its + 1)


def test_cell_pcg_on_the_benchmark_mesh():
    """One inner solve per operator on the 2D 512^2 mesh (1,050,625 rows per field,
    152 blocks of about seven lattice lines): residual and iteration count against the
    oracle's float64 Jacobi-PCG."""
    w = synth.C2_2D_LARGE
    prob = PFCProblem(structured_mesh(w.dim, w.side, w.length), w.r)
    n = prob.n
    x = np.concatenate([synth.random_vector(n, 301), synth.initial_psi(w.dim, w.side, w.psi_mean, w.amp, w.seed),
                        synth.random_vector(n, 302)])
    tau = 4.57
    b = synth.random_vector(n, 304)
    with pfc.PFCSolver(w.dim, w.side, w.length, r=w.r, precision="fp32") as s:
        assert s.cell_kernels
        s.assemble(cuda(x), tau)
        for which, A in enumerate(inner_matrices(prob, tau)):
            got, its = s.pcg(which, cuda(b), 1e-3)
            got = host(got)
            ref = pcg_jacobi(A, b, 1e-3, 10000)
            res = np.linalg.norm(b - A @ got) / np.linalg.norm(b)
            assert res <= 1.05e-3, (which, res)
            assert abs(its - ref.iterations) <= 2, (which, its, ref.iterations)
            if its == ref.iterations:
                assert np.linalg.norm(got - ref.x) <= 1e-4 * np.linalg.norm(ref.x)


# ---------------------------------------------------------------------------- 3D
_probs3 = {}


def problem3(side, L, r=-0.3):
    key = (side, L, r)
    if key not in _probs3:
        _probs3[key] = PFCProblem(structured_mesh(3, side, L), r)
    return _probs3[key]


SIDES3 = [(4, 4.0), (2, 2.0), (7, 7.0), (16, 16.0)]


@pytest.mark.parametrize("side,L", SIDES3, ids=[f"3d-s{s}" for s, _ in SIDES3])
def test_cell3d_pcg_matches_oracle(side, L):
    prob = problem3(side, L)
    n = prob.n
    x = np.concatenate([synth.random_vector(n, 101), synth.initial_psi(3, side, -0.35, 0.05, 1),
                        synth.random_vector(n, 201)])
    tau = 2.3
    b = synth.random_vector(n, 8)
    with pfc.PFCSolver(3, side, L, r=-0.3, precision="fp32") as s:
        assert s.cell_kernels
        s.assemble(cuda(x), tau)
        for which, A in enumerate(inner_matrices(prob, tau)):
            for rtol in (1e-3, 1e-5):
                got, its = s.pcg(which, cuda(b), rtol)
                got = host(got)
                ref = pcg_jacobi(A, b, rtol, 10000)
                res = np.linalg.norm(b - A @ got) / np.linalg.norm(b)
                assert res <= rtol * 1.05 + 2e-6, (which, rtol, res)
                assert abs(its - ref.iterations) <= 2, (which, rtol, its, ref.iterations)
                if its == ref.iterations:
                    assert np.linalg.norm(got - ref.x) <= 1e-4 * np.linalg.norm(ref.x)


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("side,L,tau", [(4, 4.0, 0.1), (6, 6.0, 5.0), (2, 2.0, 1.0)],
                         ids=["3d-s4-tau0.1", "3d-s6-tau5", "3d-s2-tau1"])
def test_cell3d_stage_solves_match_oracle(side, L, tau, precision):
    prob = problem3(side, L)
    x = prob.consistent_state(synth.initial_psi(3, side, -0.35, 0.05, 1), tol=1e-15, solver="pcg")
    A = prob.stage_matrix(x[prob.n:2 * prob.n], tau)
    b = prob.stage_rhs(x, [], [], tau)
    yref, ost = prob.stage_solve(A, b, tau, tol=1e-13, err_tol=1e-11)
    assert ost.converged
    with pfc.PFCSolver(3, side, L, r=-0.3, precision=precision) as s:
        assert s.cell_kernels
        s.assemble(cuda(x), tau)
        y, st = s.stage_solve(cuda(b))
        y = host(y)
    err = np.linalg.norm(y - yref) / np.linalg.norm(yref)
    assert st.status == 0 and err <= 1e-8, (err, st)
