"""Serving: each simulation's result is the same alone and in the mix.

Four simulations of different sizes and dimensions are advanced three steps each,
once one at a time with pfc_step and once through the continuous-batching server
(where they share batched launches).  The final states agree to relative 1e-7
(three steps of stage solves that each match to the 1e-8 solver tolerance) and the
next step widths to 1e-3."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1501_06852_gb300 as pfc  # noqa: E402
from paper_1501_06852_gb300 import serving  # noqa: E402

WL = [synth.Workload("a", 2, 6, 6.0, -0.4, -0.3, 0.1, 31, 0.1, 1),
      synth.Workload("b", 2, 10, 10.0, -0.3, -0.25, 0.1, 32, 0.1, 1),
      synth.Workload("c", 3, 3, 3.0, -0.3, -0.35, 0.05, 33, 0.1, 1),
      synth.Workload("d", 2, 14, 14.0, -0.45, -0.35, 0.1, 34, 0.1, 1)]
STEPS = 3


def _psi(w):
    return synth.initial_psi(w.dim, w.side, w.psi_mean, w.amp, w.seed)


def _alone(w):
    cap = pfc.critical_tau(w.r, w.psi_mean)
    tau_max = 1e9 if cap == float("inf") else 0.9 * cap / pfc.ROS3PW_GAMMA
    with pfc.PFCSolver(w.dim, w.side, w.length, r=w.r, precision="fp32", outer_tol=1e-10, tau_max=tau_max) as s:
        x = s.init_state(torch.from_numpy(_psi(w)).cuda())
        tau = min(0.1, tau_max)
        for _ in range(STEPS):
            _, _, tau, _ = s.step(x, tau)
        return x.cpu(), tau


def test_results_alone_and_in_the_mix_agree():
    alone = [_alone(w) for w in WL]
    reqs = [synth.Request(0.0, k, w) for _ in range(STEPS) for k, w in enumerate(WL)]
    srv = serving.Server(budget_bytes=8 << 30, precision="fp32", outer_tol=1e-10, initial_psi=_psi)
    try:
        rep = srv.run(reqs)
        assert len(rep.served) == len(reqs)
        assert max(b[2] for b in rep.batches) == len(WL)       # they did share batches
        for k, (x_ref, tau_ref) in enumerate(alone):
            x = srv.sims[k].state.cpu()
            assert float((x - x_ref).norm() / x_ref.norm()) <= 1e-7
            # tau_next = tau * 0.9 err^(-1/3), and err is the norm of sum (mhat_j - m_j) y_j,
            # a combination about 1e-3 the size of the increments: stage solutions that agree
            # to the solver tolerance (their block partition, hence reduction order, differs
            # with the batch's composition) move err, and tau, by up to ~1e-4
            assert srv.sims[k].tau == pytest.approx(tau_ref, rel=1e-3)
    finally:
        srv.close()
