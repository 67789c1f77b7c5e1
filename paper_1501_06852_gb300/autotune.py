"""Autotuner for the runtime shape of the persistent solver.

For a problem class (dimension, side, inner precision) it times the inner solve
of each candidate configuration on the device and keeps the fastest:

* ``inner_operator``: assembled SELL-32 values and indices, or structured stencils;
* ``pcg_variant``: textbook, pipelined or Chronopoulos-Gear Jacobi-PCG;
* ``cells`` (structured stencils, Chronopoulos-Gear, float inner solves): the cell
  kernels (one grid barrier per iteration, rings recomputed in shared memory) or the
  per-warp form in lexicographic rows.

(The persistent kernel runs 1024-thread blocks, one per SM, so the grid's
residency is not a candidate.)

The timing unit is a fixed-iteration PCG solve with M + sqrt(delta) K, the matrix of
the preconditioner's most frequent inner solves (steps 3.1 and 3.2), through
pfc_pcg with a tolerance no solve reaches, so every candidate runs the same
number of iterations.  A candidate whose pipelined recurrences drift (float32) is
not excluded here: FGMRES absorbs it at the price of outer iterations, which this
per-iteration timing does not see; ``pcg_variant`` candidates are therefore
limited to the forms that keep the outer iteration count (textbook and
Chronopoulos-Gear in float32/float16; all three in float64).
Results are cached per process.  ``tuned`` gives the configuration of a size
class (the mesh side rounded down to a power of two, at the same spacing), so that a
batch or a server with many sizes tunes a handful of classes, not every size.
"""
from __future__ import annotations

import itertools
import math
import time

_CACHE: dict = {}


def candidates(precision: str):
    variants = (0, 1, 3) if precision == "fp64" else (0, 3)
    out = []
    for io, v in itertools.product((0, 1), variants):
        if precision != "fp64" and io == 1 and v == 3:
            out += [dict(inner_operator=io, pcg_variant=v, cells=1), dict(inner_operator=io, pcg_variant=v, cells=0)]
        else:
            out.append(dict(inner_operator=io, pcg_variant=v, cells=0))
    return out


def size_class(side: int) -> int:
    """The largest power of two not above side, between 8 and 512 (the class is timed on
    a mesh no larger than any of its members)."""
    return int(min(512, max(8, 2 ** math.floor(math.log2(max(side, 1))))))


def tuned(dim: int, side: int, length: float, precision: str = "fp32", **kw) -> dict:
    """Tuned options of the size class of (dim, side): the fastest configuration
    timed on the class's representative mesh at the same spacing."""
    rep = size_class(side)
    return tune(dim, rep, length * rep / side, precision, **kw)["config"]


def tune(dim: int, side: int, length: float, precision: str = "fp32", iters: int = 60, reps: int = 2,
         r: float = -0.4, psi_mean: float = -0.3, tau: float = 1.0) -> dict:
    """Fastest configuration for this problem class; returns {"config", "us_per_iteration", "all"}."""
    key = (dim, side, float(length), precision)
    if key in _CACHE:
        return _CACHE[key]
    import torch

    import synth
    from . import PFCSolver

    psi0 = torch.from_numpy(synth.initial_psi(dim, side, psi_mean, 0.1, 7)).cuda()
    rhs = torch.from_numpy(synth.random_vector((2 * side + 1) ** dim, 8)).cuda()
    results = []
    for cfg in candidates(precision):
        with PFCSolver(dim, side, length, r=r, precision=precision, max_inner=iters, **cfg) as s:
            x = s.init_state(psi0)
            s.assemble(x, tau)
            s.pcg(2, rhs, 1e-30)                       # warm-up
            best = float("inf")
            for _ in range(reps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, its = s.pcg(2, rhs, 1e-30)
                torch.cuda.synchronize()
                best = min(best, (time.perf_counter() - t0) / max(its, 1))
            results.append((best * 1e6, cfg))
    results.sort(key=lambda t: t[0])
    out = {"config": results[0][1], "us_per_iteration": results[0][0],
           "all": [{"us_per_iteration": t, **c} for t, c in results]}
    _CACHE[key] = out
    return out
