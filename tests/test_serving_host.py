"""Host logic of the continuous-batching server, on CPU with a fake solver:
stage-wise scheduling (a step takes three launches; a request that arrives while
others are in flight joins the next launch, beside their later stages), one step
in flight per simulation, admission by footprint, LRU eviction of idle
simulations to host memory and their restoration, and refusal of a simulation
larger than the budget.  No GPU is involved."""
import time

import numpy as np
import pytest
import torch

import synth
from paper_1501_06852_gb300 import serving

STAGE_S = 0.02   # one fake stage launch
STEP_S = 3 * STAGE_S


class FakeSolver:
    live = 0

    def __init__(self, dim, side, length, **kw):
        self.n = (2 * side + 1) ** dim
        FakeSolver.live += 1
        self.closed = False

    def init_state(self, psi0):
        return torch.cat([torch.zeros_like(psi0), psi0, torch.zeros_like(psi0)])

    stage = -1

    def step_begin(self, state, tau):
        assert self.stage == -1
        self.stage = 0

    def step_finish(self, state, tau, check=True):
        assert self.stage == 3
        self.stage = -1
        state += 1.0
        return True, 0.1, tau * 1.5, [None] * 3

    def close(self):
        if not self.closed:
            FakeSolver.live -= 1
            self.closed = True


def fake_batch_stage_advance(solvers):
    """One launch: every solver's stage advances by one (a step takes three)."""
    time.sleep(STAGE_S)
    for s in solvers:
        assert 0 <= s.stage <= 2
        s.stage += 1


@pytest.fixture
def fakes(monkeypatch):
    FakeSolver.live = 0
    monkeypatch.setattr(serving, "PFCSolver", FakeSolver)
    monkeypatch.setattr(serving, "batch_stage_advance", fake_batch_stage_advance)
    monkeypatch.setattr(serving, "footprint_bytes", lambda dim, side, precision="fp32", restart=30: side * 100)


def _wl(sid, side):
    return synth.Workload(f"s{sid}", 2, side, float(side), -0.4, -0.3, 0.1, 10 + sid, 0.1, 1)


def _psi(w):
    return synth.initial_psi(w.dim, w.side, w.psi_mean, w.amp, w.seed)


def test_stage_wise_batches_one_step_per_sim(fakes):
    wl = [_wl(k, 4) for k in range(3)]
    reqs = [synth.Request(0.0, 0, wl[0]), synth.Request(0.0, 0, wl[0]), synth.Request(0.0, 1, wl[1]),
            synth.Request(STAGE_S * 1.5, 2, wl[2]), synth.Request(STAGE_S * 0.5, 1, wl[1])]
    srv = serving.Server(10 ** 9, initial_psi=_psi, device="cpu")
    rep = srv.run(reqs)
    # every step took three launches of its simulation
    assert sum(b[2] for b in rep.batches) == 3 * len(reqs)
    # sim 2 arrived during the first steps and joined a launch beside their later stages
    mixed = [b for b in rep.batches if len(set(b[4])) > 1]
    assert mixed and any(0 in b[4] and (1 in b[4] or 2 in b[4]) for b in mixed)
    per_sim = {}
    for s in rep.served:
        per_sim.setdefault(s.sim_id, []).append(s)
    # one step in flight per simulation: sim 0's second step starts after its first is done
    assert len(per_sim[0]) == 2 and per_sim[0][0].done <= per_sim[0][1].start + 1e-9
    # a late request does not wait for whole steps: sim 2 finishes 3 launches after it starts
    s2 = per_sim[2][0]
    assert s2.done - s2.start < 4.5 * STAGE_S + 0.05
    # each served step advanced its simulation exactly once
    assert float(srv.sims[0].state[0]) == 2.0 and float(srv.sims[1].state[0]) == 2.0
    s = rep.summary()
    assert s["requests"] == 5 and s["p99_ms"] >= s["p50_ms"] > 0 and s["launches_with_mixed_stages"] >= 1
    srv.close()
    assert FakeSolver.live == 0


def test_lru_eviction_and_restore(fakes):
    wl = [_wl(k, 10) for k in range(3)]      # 1000 bytes each, budget fits two
    reqs = [synth.Request(0.0, 0, wl[0]), synth.Request(0.0, 1, wl[1]),
            synth.Request(STEP_S * 1.5, 2, wl[2]), synth.Request(STEP_S * 3.5, 0, wl[0])]
    srv = serving.Server(2000, initial_psi=_psi, device="cpu")
    rep = srv.run(reqs)
    assert rep.evictions >= 2 and rep.admissions == 4
    assert srv.resident_bytes <= 2000
    # sim 0 was evicted and restored with its state: two steps applied in total
    assert float(srv.sims[0].state[0]) == 2.0
    assert srv.sims[0].tau == pytest.approx(0.1 * 1.5 * 1.5)
    srv.close()


def test_simulation_larger_than_budget_is_refused(fakes):
    srv = serving.Server(500, initial_psi=_psi, device="cpu")
    with pytest.raises(RuntimeError):
        srv.run([synth.Request(0.0, 0, _wl(0, 10))])
    srv.close()


def test_footprint_grows_with_size():
    a = serving.footprint_bytes(2, 64)
    b = serving.footprint_bytes(2, 256)
    c = serving.footprint_bytes(3, 32)
    assert 0 < a < b and c > 0
