"""Serving: each simulation's result is the same alone and in the mix, bit for bit.

Four simulations of different sizes and dimensions are advanced three steps each,
once one at a time with pfc_step, once launch by launch through the stage-wise
entry points with start times one launch apart (so that launches solve the first
stage of some steps beside the second and third stages of others), and once
through the continuous-batching server.  Every
simulation's context keeps a fixed block count (options.grid_blocks), so its row
partition and reduction order are the same in both runs: final states and next
step widths are equal bit for bit."""
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1501_06852_gb300 as pfc  # noqa: E402
from paper_1501_06852_gb300 import serving  # noqa: E402

WL = [synth.Workload("a", 2, 6, 6.0, -0.4, -0.3, 0.1, 31, 0.1, 1),
      synth.Workload("b", 2, 40, 40.0, -0.3, -0.25, 0.1, 32, 0.1, 1),
      synth.Workload("c", 3, 5, 5.0, -0.3, -0.35, 0.05, 33, 0.1, 1),
      synth.Workload("d", 2, 64, 64.0, -0.45, -0.35, 0.1, 34, 0.1, 1)]
STEPS = 3


def _psi(w):
    return synth.initial_psi(w.dim, w.side, w.psi_mean, w.amp, w.seed)


def _alone(w):
    with _solver(w) as s:
        x = s.init_state(torch.from_numpy(_psi(w)).cuda())
        tau = 0.1
        for _ in range(STEPS):
            _, _, tau, st = s.step(x, tau)
            assert all(t.status == 0 for t in st)
        return x.cpu(), tau


def _solver(w):
    return pfc.PFCSolver(w.dim, w.side, w.length, r=w.r, precision="fp32", outer_tol=1e-10, err_tol=1e-9,
                         tau_max=serving.TAU_MAX_UNGUARDED, tau_guard=serving.TAU_GUARD,
                         grid_blocks=serving.default_blocks(w))


def test_stage_launches_in_a_mix_give_the_same_bits_as_alone():
    """Launch by launch: simulations start one launch apart, so every launch after the
    first solves different stages of different steps side by side."""
    alone = [_alone(w) for w in WL]
    solvers = [_solver(w) for w in WL]
    try:
        states = [s.init_state(torch.from_numpy(_psi(w)).cuda()) for s, w in zip(solvers, WL)]
        taus = [0.1] * len(WL)
        left = [STEPS] * len(WL)
        start = [0, 0, 1, 2]
        mixed = 0
        launch = 0
        while any(left):
            for k, s in enumerate(solvers):
                if left[k] and s.stage == -1 and launch >= start[k]:
                    s.step_begin(states[k], taus[k])
            busy = [s for s in solvers if s.stage in (0, 1, 2)]
            mixed += len({s.stage for s in busy}) > 1
            pfc.batch_stage_advance(busy)
            for k, s in enumerate(solvers):
                if s.stage == 3:
                    acc, _, taus[k], st = s.step_finish(states[k], taus[k])
                    assert all(t.status == 0 for t in st)
                    left[k] -= 1
            launch += 1
        assert mixed >= 3
        for k, (x_ref, tau_ref) in enumerate(alone):
            x = states[k].cpu()
            assert torch.equal(x, x_ref), (k, float((x - x_ref).norm() / x_ref.norm()))
            assert taus[k] == tau_ref
    finally:
        for s in solvers:
            s.close()


def test_server_results_are_the_same_bits_as_alone():
    alone = [_alone(w) for w in WL]
    reqs = [synth.Request(0.0, 0, WL[0]), synth.Request(0.0, 1, WL[1]),
            synth.Request(0.02, 2, WL[2]), synth.Request(0.04, 3, WL[3])]
    reqs += [synth.Request(0.0, k, w) for _ in range(STEPS - 1) for k, w in enumerate(WL)]
    srv = serving.Server(budget_bytes=8 << 30, precision="fp32", outer_tol=1e-10, err_tol=1e-9, initial_psi=_psi)
    try:
        rep = srv.run(reqs)
        assert len(rep.served) == len(reqs)
        for k, (x_ref, tau_ref) in enumerate(alone):
            x = srv.sims[k].state.cpu()
            assert torch.equal(x, x_ref), (k, float((x - x_ref).norm() / x_ref.norm()))
            assert srv.sims[k].tau == tau_ref
    finally:
        srv.close()


def test_stage_api_matches_pfc_step():
    """pfc_step_begin + three pfc_batch_stage_advance + pfc_step_finish on one context
    is pfc_step, bit for bit (fixed block count)."""
    w = WL[1]
    kw = dict(r=w.r, precision="fp32", grid_blocks=serving.default_blocks(w))
    outs = []
    for staged in (False, True):
        with pfc.PFCSolver(w.dim, w.side, w.length, **kw) as s:
            x = s.init_state(torch.from_numpy(_psi(w)).cuda())
            if staged:
                s.step_begin(x, 0.2)
                assert s.stage == 0
                for k in range(3):
                    pfc.batch_stage_advance([s])
                    assert s.stage == k + 1
                with pytest.raises(pfc.PFCError):
                    pfc.batch_stage_advance([s])
                res = s.step_finish(x, 0.2)
                assert s.stage == -1
            else:
                res = s.step(x, 0.2)
            outs.append((x.cpu(), res[0], res[1], res[2]))
    (x0, a0, e0, t0), (x1, a1, e1, t1) = outs
    assert torch.equal(x0, x1) and a0 == a1 and e0 == e1 and t0 == t1
