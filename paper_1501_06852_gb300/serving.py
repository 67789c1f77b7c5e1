"""Continuous-batching server for PFC time-step requests (host logic only).

Requests ask to advance one simulation (identified by ``sim_id``) by one Ros3Pw
step.  The server keeps each admitted simulation resident on the device (its
context with mesh, matrices and Krylov workspace, its state and its step width),
admits new simulations by device-memory footprint, and advances every simulation
that has an arrived request in one batched step (``batch_step``: one persistent
launch per stage for all of them).  Requests that arrive while a batch runs join
the next batch.  Idle simulations are evicted least-recently-used first when the
footprint budget needs room; their state and step width move to host memory and
come back when the simulation is requested again.

Not part of the paper: its runs advance one simulation at a time.
"""
from __future__ import annotations

import statistics
import time
from collections import OrderedDict, deque
from dataclasses import dataclass, field

from . import PFCSolver, batch_step, critical_tau, lib, ROS3PW_GAMMA, _Options

import ctypes


# Step-width limit where Lemma 3 gives no critical step width (the paper's adaptive
# runs reach tau of about 18, Section 7).
TAU_MAX_UNGUARDED = 20.0


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
    start: float
    done: float
    accepted: bool
    batch_size: int

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class ServeReport:
    served: list = field(default_factory=list)
    batches: list = field(default_factory=list)     # (t_start, t_end, size, resident_bytes)
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
        return {
            "requests": len(self.served),
            "p50_ms": None if not lat else 1e3 * pct(50),
            "p99_ms": None if not lat else 1e3 * pct(99),
            "mean_ms": None if not lat else 1e3 * statistics.mean(lat),
            "stage_solves_per_s": 3 * len(self.served) / self.wall_s if self.wall_s else None,
            "steps_per_s": len(self.served) / self.wall_s if self.wall_s else None,
            "batches": len(self.batches),
            "mean_batch": statistics.mean(sizes) if sizes else 0,
            "max_batch": max(sizes) if sizes else 0,
            "admissions": self.admissions,
            "evictions": self.evictions,
            "max_resident_bytes": max((b[3] for b in self.batches), default=0),
            "wall_s": self.wall_s,
        }


class Server:
    """Admits simulations by footprint and advances them in continuous batches."""

    def __init__(self, budget_bytes: int, precision: str = "fp32", outer_tol: float = 1e-10,
                 max_batch: int = 64, initial_psi=None, tau0: float = 0.1, device: str = "cuda"):
        import torch

        self.torch = torch
        self.device = device
        self.budget = int(budget_bytes)
        self.precision = precision
        self.outer_tol = outer_tol
        self.max_batch = max_batch
        self.tau0 = tau0
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
        cap = critical_tau(w.r, w.psi_mean)
        tau_max = TAU_MAX_UNGUARDED if cap == float("inf") else min(TAU_MAX_UNGUARDED, 0.9 * cap / ROS3PW_GAMMA)
        sim.solver = PFCSolver(w.dim, w.side, w.length, r=w.r, precision=self.precision,
                               outer_tol=self.outer_tol, tau_max=tau_max)
        sim.bytes = need
        torch = self.torch
        if sim.state is None:
            psi0 = torch.from_numpy(self.initial_psi(w)).to(self.device)
            sim.state = sim.solver.init_state(psi0)
            sim.tau = min(self.tau0, tau_max)
        else:
            sim.state = sim.state.to(self.device)
        self.resident[sim.sim_id] = sim
        self.resident_bytes += need
        self.report.admissions += 1
        return True

    # -- loop -------------------------------------------------------------------
    def run(self, requests: list) -> ServeReport:
        """Serves ``requests`` (objects with arrival_s, sim_id, workload) in real time."""
        torch = self.torch
        pending: deque = deque(sorted(requests, key=lambda q: q.arrival_s))
        waiting: list = []                      # arrived, not yet served (FIFO)
        t0 = time.perf_counter()
        while pending or waiting:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival_s <= now:
                waiting.append(pending.popleft())
            if not waiting:
                time.sleep(max(0.0, min(0.01, pending[0].arrival_s - now)))
                continue
            # one request per simulation per batch, oldest first, admitted by footprint
            batch, taken, rest = [], set(), []
            for q in waiting:
                if len(batch) < self.max_batch and q.sim_id not in taken:
                    sim = self.sims.get(q.sim_id)
                    if sim is None:
                        sim = self.sims[q.sim_id] = Sim(q.sim_id, q.workload)
                    if self._admit(sim, taken):
                        batch.append((q, sim))
                        taken.add(q.sim_id)
                        continue
                rest.append(q)
            waiting = rest
            if not batch:
                raise RuntimeError("a simulation does not fit the footprint budget")
            start = time.perf_counter() - t0
            sims = [sim for _, sim in batch]
            # a stage solve that hits its iteration cap rejects that simulation's step
            # (state kept, tau shrunk) like an error estimate above 1
            acc, errs, taus, _ = batch_step([s.solver for s in sims], [s.state for s in sims],
                                            [s.tau for s in sims], check=False)
            if self.device != "cpu":
                torch.cuda.synchronize()
            done = time.perf_counter() - t0
            for (q, sim), a, tn in zip(batch, acc, taus):
                sim.tau = tn
                sim.steps += 1
                sim.accepted += int(a)
                sim.last_used = done
                self.report.served.append(Served(q.sim_id, q.arrival_s, start, done, a, len(batch)))
            self.report.batches.append((start, done, len(batch), self.resident_bytes))
        self.report.wall_s = time.perf_counter() - t0
        return self.report

    def close(self):
        for sim in list(self.resident.values()):
            if sim.solver is not None:
                sim.solver.close()
                sim.solver = None
        self.resident.clear()
        self.resident_bytes = 0
