"""Host logic of the continuous-batching server, on CPU with a fake solver:
FIFO batches with one request per simulation, requests that arrive during a batch
joining the next one, admission by footprint, LRU eviction of idle simulations to
host memory and their restoration, and refusal of a simulation larger than the
budget.  No GPU is involved."""
import time

import numpy as np
import pytest
import torch

import synth
from paper_1501_06852_gb300 import serving

STEP_S = 0.05


class FakeSolver:
    live = 0

    def __init__(self, dim, side, length, **kw):
        self.n = (2 * side + 1) ** dim
        FakeSolver.live += 1
        self.closed = False

    def init_state(self, psi0):
        return torch.cat([torch.zeros_like(psi0), psi0, torch.zeros_like(psi0)])

    def close(self):
        if not self.closed:
            FakeSolver.live -= 1
            self.closed = True


def fake_batch_step(solvers, states, taus, check=True):
    time.sleep(STEP_S)
    for x in states:
        x += 1.0
    return [True] * len(states), [0.1] * len(states), [t * 1.5 for t in taus], [[None] * 3 for _ in states]


@pytest.fixture
def fakes(monkeypatch):
    FakeSolver.live = 0
    monkeypatch.setattr(serving, "PFCSolver", FakeSolver)
    monkeypatch.setattr(serving, "batch_step", fake_batch_step)
    monkeypatch.setattr(serving, "footprint_bytes", lambda dim, side, precision="fp32", restart=30: side * 100)


def _wl(sid, side):
    return synth.Workload(f"s{sid}", 2, side, float(side), -0.4, -0.3, 0.1, 10 + sid, 0.1, 1)


def _psi(w):
    return synth.initial_psi(w.dim, w.side, w.psi_mean, w.amp, w.seed)


def test_continuous_batches_one_request_per_sim(fakes):
    wl = [_wl(k, 4) for k in range(3)]
    reqs = [synth.Request(0.0, 0, wl[0]), synth.Request(0.0, 0, wl[0]), synth.Request(0.0, 1, wl[1]),
            synth.Request(0.01, 2, wl[2]), synth.Request(STEP_S * 0.5, 1, wl[1])]
    srv = serving.Server(10 ** 9, initial_psi=_psi, device="cpu")
    rep = srv.run(reqs)
    sizes = [b[2] for b in rep.batches]
    assert sum(sizes) == 5
    # the first batch holds sims 0 and 1 (and 2 if it arrived in time); sim 0's second request waits
    assert sizes[0] >= 2 and max(sizes) <= 3
    per_sim = {}
    for s in rep.served:
        per_sim.setdefault(s.sim_id, []).append(s)
    assert len(per_sim[0]) == 2 and per_sim[0][0].done < per_sim[0][1].start + 1e-9
    # each served step advanced its simulation exactly once
    assert float(srv.sims[0].state[0]) == 2.0 and float(srv.sims[1].state[0]) == 2.0
    s = rep.summary()
    assert s["requests"] == 5 and s["p99_ms"] >= s["p50_ms"] > 0
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
