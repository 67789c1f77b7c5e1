"""Continuous-batching server for PFC time-step requests (host logic only).

Requests ask to advance one simulation (identified by ``sim_id``) by one Ros3Pw
step.  The server keeps each admitted simulation resident on the device (its
context with mesh, matrices and Krylov workspace, its state and its step width)
and admits new simulations by device-memory footprint.  It schedules by stage:
every iteration of its loop is one batched persistent launch
(``batch_stage_advance``) that solves the next stage of every step in flight, so
a request that arrives while others are on the GPU starts its step (assembly,
then its first stage) in the very next launch, next to the second and third
stages of the steps already running, and a finished step returns as soon as its
third stage is done.  Each simulation's context keeps a fixed block count
(``grid_blocks``), so its results are the same bits alone and in any mix.  Idle
simulations are evicted least-recently-used first when the footprint budget
needs room; their state and step width move to host memory and come back when
the simulation is requested again.

Not part of the paper: its runs advance one simulation at a time.
"""
from __future__ import annotations

import statistics
import time
from collections import OrderedDict, deque
from dataclasses import dataclass, field

import ctypes

from . import PFCSolver, batch_stage_advance, lib, _Options

# Step-width limit where Lemma 3 gives no critical step width (the paper's adaptive
# runs reach tau of about 18, Section 7), and the library's Lemma-3 guard
# (options.tau_guard: gamma tau <= 0.9 tau*(r, <psi>)).
TAU_MAX_UNGUARDED = 20.0
TAU_GUARD = 0.9


def default_blocks(workload) -> int:
    """Fixed persistent-solver blocks of a simulation: about one block per 64 slices
    of 32 rows, between 2 and 76 (half of a GB300's SMs), so that several
    simulations share each launch and a large one still spreads over many SMs."""
    n = (2 * workload.side + 1) ** workload.dim
    return max(2, min(76, n // (32 * 64)))


def footprint_bytes(dim: int, side: int, precision: str = "fp32", restart: int = 30) -> int:
    o = _Options()
    lib.pfc_default_options(ctypes.byref(o))
    o.precision = {"fp64": 0, "fp32": 1, "fp16": 2}[precision]
    o.restart = restart
    return int(lib.pfc_footprint_bytes(dim, side, ctypes.byref(o)))


@dataclass
class Sim:
    sim_id: int
    workload: object
    solver: PFCSolver | None = None
    state: object = None            # device tensor while resident, host tensor when evicted
    tau: float = 0.1
    bytes: int = 0
    steps: int = 0
    accepted: int = 0
    last_used: float = 0.0


@dataclass
class Served:
    sim_id: int
    arrival: float
    start: float          # the launch that solved the step's first stage began
    done: float
    accepted: bool
    batch_size: int       # steps in flight in that first launch

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class ServeReport:
    served: list = field(default_factory=list)
    batches: list = field(default_factory=list)     # launches: (t_start, t_end, size, resident_bytes, stages)
    admissions: int = 0
    evictions: int = 0
    wall_s: float = 0.0

    def summary(self) -> dict:
        lat = sorted(s.latency for s in self.served)

        def pct(q):
            if not lat:
                return None
            k = (len(lat) - 1) * q / 100.0
            lo, hi = int(k), min(int(k) + 1, len(lat) - 1)
            return lat[lo] + (lat[hi] - lat[lo]) * (k - lo)

        sizes = [b[2] for b in self.batches]
        mixed = sum(1 for b in self.batches if len(set(b[4])) > 1)
        return {
            "requests": len(self.served),
            "p50_ms": None if not lat else 1e3 * pct(50),
            "p99_ms": None if not lat else 1e3 * pct(99),
            "mean_ms": None if not lat else 1e3 * statistics.mean(lat),
            "stage_solves_per_s": 3 * len(self.served) / self.wall_s if self.wall_s else None,
            "steps_per_s": len(self.served) / self.wall_s if self.wall_s else None,
            "launches": len(self.batches),
            "mean_batch": statistics.mean(sizes) if sizes else 0,
            "launches_with_mixed_stages": mixed,
            "max_batch": max(sizes) if sizes else 0,
            "admissions": self.admissions,
            "evictions": self.evictions,
            "max_resident_bytes": max((b[3] for b in self.batches), default=0),
            "wall_s": self.wall_s,
        }


class Server:
    """Admits simulations by footprint and advances them stage by stage in batched launches."""

    def __init__(self, budget_bytes: int, precision: str = "fp32", outer_tol: float = 1e-10,
                 err_tol: float = 1e-9, max_batch: int = 64, initial_psi=None, tau0: float = 0.1,
                 device: str = "cuda", blocks=default_blocks, autotune: bool = False):
        import torch

        self.torch = torch
        self.device = device
        self.budget = int(budget_bytes)
        self.precision = precision
        self.outer_tol = outer_tol
        self.err_tol = err_tol
        self.max_batch = max_batch
        self.tau0 = tau0
        self.blocks = blocks               # callable(workload) -> fixed solver blocks
        self.autotune = autotune           # per size class solver configuration (autotune.tuned)
        self.initial_psi = initial_psi     # callable(workload) -> numpy psi0
        self.sims: dict[int, Sim] = {}
        self.resident: "OrderedDict[int, Sim]" = OrderedDict()
        self.resident_bytes = 0
        self.report = ServeReport()

    # -- residency --------------------------------------------------------------
    def _evict_for(self, need: int, busy: set) -> bool:
        while self.resident_bytes + need > self.budget:
            victim = next((sid for sid in self.resident if sid not in busy), None)
            if victim is None:
                return False
            sim = self.resident.pop(victim)
            sim.state = sim.state.cpu()
            sim.solver.close()
            sim.solver = None
            self.resident_bytes -= sim.bytes
            self.report.evictions += 1
        return True

    def _admit(self, sim: Sim, busy: set) -> bool:
        if sim.solver is not None:
            self.resident.move_to_end(sim.sim_id)
            return True
        w = sim.workload
        need = footprint_bytes(w.dim, w.side, self.precision)
        if need > self.budget or not self._evict_for(need, busy):
            return False
        cfg = self._config(w)
        sim.solver = PFCSolver(w.dim, w.side, w.length, r=w.r, precision=self.precision,
                               outer_tol=self.outer_tol, err_tol=self.err_tol, tau_max=TAU_MAX_UNGUARDED,
                               tau_guard=TAU_GUARD, grid_blocks=self.blocks(w), **cfg)
        sim.bytes = need
        torch = self.torch
        if sim.state is None:
            psi0 = torch.from_numpy(self.initial_psi(w)).to(self.device)
            sim.state = sim.solver.init_state(psi0)
            sim.tau = self.tau0
        else:
            sim.state = sim.state.to(self.device)
        self.resident[sim.sim_id] = sim
        self.resident_bytes += need
        self.report.admissions += 1
        return True

    def _config(self, w) -> dict:
        if not self.autotune:
            return {}
        from . import autotune

        return autotune.tuned(w.dim, w.side, w.length, self.precision)

    def prepare(self, requests: list) -> None:
        """Tunes every size class the requests use before serving (autotune on)."""
        for q in requests:
            self._config(q.workload)

    # -- loop -------------------------------------------------------------------
    def run(self, requests: list) -> ServeReport:
        """Serves ``requests`` (objects with arrival_s, sim_id, workload) in real time."""
        pending: deque = deque(sorted(requests, key=lambda q: q.arrival_s))
        waiting: list = []                      # arrived, step not begun (FIFO)
        inflight: "OrderedDict[int, tuple]" = OrderedDict()   # sim_id -> (request, sim, first launch, size)
        t0 = time.perf_counter()
        while pending or waiting or inflight:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival_s <= now:
                waiting.append(pending.popleft())
            # begin the steps of arrived requests: one step in flight per simulation,
            # oldest request first, admitted by footprint
            rest = []
            for q in waiting:
                if len(inflight) < self.max_batch and q.sim_id not in inflight:
                    sim = self.sims.get(q.sim_id)
                    if sim is None:
                        sim = self.sims[q.sim_id] = Sim(q.sim_id, q.workload)
                    if self._admit(sim, set(inflight)):
                        sim.solver.step_begin(sim.state, sim.tau)
                        inflight[q.sim_id] = (q, sim, None, 0)
                        continue
                rest.append(q)
            waiting = rest
            if not inflight:
                if waiting:
                    raise RuntimeError("a simulation does not fit the footprint budget")
                time.sleep(max(0.0, min(0.01, pending[0].arrival_s - now)))
                continue
            # one batched launch: the next stage of every step in flight
            sims = [v[1] for v in inflight.values()]
            stages = [s.solver.stage for s in sims]
            start = time.perf_counter() - t0
            batch_stage_advance([s.solver for s in sims])
            done = time.perf_counter() - t0
            self.report.batches.append((start, done, len(sims), self.resident_bytes, stages))
            for sid in list(inflight):
                q, sim, first, size = inflight[sid]
                if first is None:
                    inflight[sid] = (q, sim, start, len(sims))
                    first, size = start, len(sims)
                if sim.solver.stage != 3:
                    continue
                # a stage solve that hit its iteration cap rejects the step (state kept,
                # tau shrunk) like an error estimate above 1
                acc, _, tn, _ = sim.solver.step_finish(sim.state, sim.tau, check=False)
                fin = time.perf_counter() - t0
                sim.tau = tn
                sim.steps += 1
                sim.accepted += int(acc)
                sim.last_used = fin
                self.report.served.append(Served(sid, q.arrival_s, first, fin, acc, size))
                del inflight[sid]
        self.report.wall_s = time.perf_counter() - t0
        return self.report

    def close(self):
        for sim in list(self.resident.values()):
            if sim.solver is not None:
                sim.solver.close()
                sim.solver = None
        self.resident.clear()
        self.resident_bytes = 0
