"""Seeded synthetic inputs for the PFC stage solver.

This module is the only code shared by the FP64 CPU oracle (``oracle/``) and the
CUDA path (``paper_1501_06852_gb300``).  It holds random-number generation and the
workload recipes (sizes, parameters, seeds) and none of the method's arithmetic:
no mesh, no finite elements, no solver.

Random numbers come from SplitMix64 (G. L. Steele, D. Lea, C. H. Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014): the j-th output of a
generator seeded with ``seed`` is ``mix64(seed + (j + 1) * 0x9E3779B97F4A7C15)``
(all arithmetic mod 2**64), which is the sequence of successive ``next()`` calls
of the published generator.  Uniforms in [0, 1) take the top 53 bits.

Initial states follow the crystallisation set-up of the paper (Section 7: a
start well away from equilibrium, noise around a mean density psi_bar):
``psi0_j = psi_bar + amp * (2 u_j - 1)`` with ``j`` the lexicographic P2 dof index.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of a SplitMix64 stream seeded with ``seed``."""
    j = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + j * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _C1
        z = (z ^ (z >> np.uint64(27))) * _C2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1): top 53 bits of each SplitMix64 output times 2**-53."""
    return (splitmix64(seed, count, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def p2_dofs_per_field(dim: int, side: int) -> int:
    """Number of P2 lattice points of a structured grid with ``side`` cells per axis."""
    return (2 * side + 1) ** dim


def dofs_per_field(dim: int, side: int, degree: int = 2) -> int:
    """Lattice points of a structured grid with ``side`` cells per axis: P2 (degree 2)
    uses the half-spacing lattice, P1 (degree 1) the vertices."""
    return (degree * side + 1) ** dim


def initial_psi(dim: int, side: int, psi_mean: float, amp: float, seed: int, degree: int = 2) -> np.ndarray:
    """Seeded noise psi0 (lexicographic dof order, x fastest), float64."""
    n = dofs_per_field(dim, side, degree)
    return psi_mean + amp * (2.0 * uniform01(seed, n) - 1.0)


def random_vector(n: int, seed: int) -> np.ndarray:
    """A seeded test vector with entries uniform in [-1, 1)."""
    return 2.0 * uniform01(seed, n) - 1.0


@dataclass(frozen=True)
class Workload:
    """One PFC simulation: mesh, model parameter, initial noise and time-step data."""

    name: str
    dim: int
    side: int
    length: float
    r: float
    psi_mean: float
    amp: float
    seed: int
    tau0: float
    steps: int
    outer_tol: float = 1e-10

    @property
    def n(self) -> int:
        return p2_dofs_per_field(self.dim, self.side)

    @property
    def unknowns(self) -> int:
        return 3 * self.n


# Workload recipes.  Sizes and parameters follow the paper's 2D/3D crystallisation
# settings (Section 7) scaled to structured square/cube grids.
C1_2D_SMALL = Workload("2d-s32-L32", 2, 32, 32.0, -0.4, -0.3, 0.1, 1, 0.1, 1, 1e-10)
C2_2D_LARGE = Workload("2d-s512-L256", 2, 512, 256.0, -0.4, -0.3, 0.1, 2, 0.1, 20, 1e-10)
C3_3D = Workload("3d-s64-L64", 3, 64, 64.0, -0.3, -0.35, 0.05, 3, 0.1, 5, 1e-10)

# Lattice spacing d = 4 pi / sqrt(3) of the one-mode crystal approximation the
# paper sizes its domains by (Section 7: Omega = [N d]^dim, P2 dof spacing about pi/4).
LATTICE_D = 4.0 * math.pi / math.sqrt(3.0)
# The ~66,000-unknown comparison problems of the paper's solver tables (Section 7,
# Tables 3-5), linearised Euler steps at tau = 0.1: 2D [16 d]^2 with 74^2 squares
# (3 x 149^2 = 66,603 unknowns; r = psi_bar = -0.35) and 3D [3 d]^3 with 14^3 cubes
# (3 x 29^3 = 73,167 unknowns; r = -0.3, psi_bar = -0.34), both with dof spacing
# within 1.5 % of pi/4.
C0_2D_EULER = Workload("2d-s74-L16d", 2, 74, 16 * LATTICE_D, -0.35, -0.35, 0.1, 6, 0.1, 20, 1e-8)
C0_3D_EULER = Workload("3d-s14-L3d", 3, 14, 3 * LATTICE_D, -0.3, -0.34, 0.05, 7, 0.1, 20, 1e-8)


def batched_instances(count: int = 256, seed: int = 4, lo: int = 16, hi: int = 256) -> list[Workload]:
    """Independent 2D instances of uneven size (log-uniform side in [lo, hi], h = 1).

    Parameter draws: side = round(exp(U(ln lo, ln hi))), r ~ U(-0.5, -0.2),
    psi_mean ~ U(-0.4, -0.2), noise amplitude 0.1, per-instance seed 1000 + b.
    """
    u = uniform01(seed, 3 * count).reshape(count, 3)
    out = []
    for b in range(count):
        side = int(round(math.exp(math.log(lo) + u[b, 0] * (math.log(hi) - math.log(lo)))))
        r = -0.5 + 0.3 * u[b, 1]
        psi_mean = -0.4 + 0.2 * u[b, 2]
        out.append(Workload(f"batch{b}", 2, side, float(side), r, psi_mean, 0.1, 1000 + b, 0.1, 1))
    return out


@dataclass
class Request:
    """One serving request: advance simulation ``sim_id`` by one time step."""

    arrival_s: float
    sim_id: int
    workload: Workload


def serving_stream(count: int = 2000, rate_hz: float = 50.0, sims: int = 64, seed: int = 5) -> list[Request]:
    """Poisson arrivals of time-step requests over ``sims`` long-lived simulations.

    80 % of the simulations are 2D (side log-uniform in [32, 512]) and 20 % 3D
    (side log-uniform in [16, 48]); h = 1; parameters drawn as for the batched
    instances.  Requests pick a simulation uniformly at random.
    """
    u = uniform01(seed, 5 * sims).reshape(sims, 5)
    wl = []
    for s in range(sims):
        if u[s, 0] < 0.8:
            lo, hi, dim = 32, 512, 2
        else:
            lo, hi, dim = 16, 48, 3
        side = int(round(math.exp(math.log(lo) + u[s, 1] * (math.log(hi) - math.log(lo)))))
        r = -0.5 + 0.3 * u[s, 2]
        psi_mean = -0.4 + 0.2 * u[s, 3]
        wl.append(Workload(f"sim{s}", dim, side, float(side), r, psi_mean, 0.1, 2000 + s, 0.1, 1))
    ua = uniform01(seed + 1, 2 * count).reshape(count, 2)
    t = 0.0
    reqs = []
    for i in range(count):
        t += -math.log(1.0 - ua[i, 0]) / rate_hz
        sid = min(int(ua[i, 1] * sims), sims - 1)
        reqs.append(Request(t, sid, wl[sid]))
    return reqs
