"""GB300 (sm_103a) solver for the Rosenbrock stages of the P2 phase-field-crystal equation.

Thin Python binding over the C ABI of ``libpfc.so`` (declared in ``include/pfc.h``):
argument marshalling only.  Every step of the method (assembly, stage
right-hand side, FGMRES with the P_CH block preconditioner, Jacobi-PCG, the
Ros3Pw step and its error estimate) runs in the library's CUDA kernels.
PyTorch provides device memory and the CUDA stream.

Importing the package (re)builds ``libpfc.so`` when it is missing or older than
its sources and then loads it; if it cannot be built or loaded the import fails
(there is no fallback path).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

from . import build as _build
from .build import LIB as _LIB_PATH

__all__ = ["PFCSolver", "PFCError", "SolveStats", "lib", "critical_tau", "ROS3PW_GAMMA",
           "batch_stage_solve", "batch_step", "batch_stage_advance",
           "OP_M", "OP_K", "OP_A01", "OP_AR", "OP_PCH", "PRECISIONS"]

OP_M, OP_K, OP_A01, OP_AR, OP_PCH = 0, 1, 2, 3, 4
PRECISIONS = {"fp64": 0, "fp32": 1, "fp16": 2}
ROS3PW_GAMMA = 0.78867513459481287
STATUS = {0: "PFC_OK", 1: "PFC_ERR_INVALID", 2: "PFC_ERR_OOM", 3: "PFC_ERR_CUDA",
          4: "PFC_ERR_NOT_CONVERGED", 5: "PFC_ERR_NONFINITE", 6: "PFC_ERR_TIMEOUT"}


class _Options(ctypes.Structure):
    _fields_ = [("r", ctypes.c_double), ("outer_tol", ctypes.c_double), ("inner_rtol", ctypes.c_double),
                ("restart", ctypes.c_int), ("max_outer", ctypes.c_int), ("max_inner", ctypes.c_int),
                ("precision", ctypes.c_int), ("step_atol", ctypes.c_double), ("step_rtol", ctypes.c_double),
                ("tau_max", ctypes.c_double), ("blocks_per_sm", ctypes.c_int), ("pcg_variant", ctypes.c_int),
                ("inner_operator", ctypes.c_int),
                ("smem_window", ctypes.c_int),
                ("model", ctypes.c_int),
                ("psi_min", ctypes.c_double),
                ("schur", ctypes.c_int),
                ("schur_its", ctypes.c_int),
                ("degree", ctypes.c_int),
                ("err_tol", ctypes.c_double),
                ("tau_guard", ctypes.c_double),
                ("grid_blocks", ctypes.c_int),
                ("cells", ctypes.c_int)]


class _Stats(ctypes.Structure):
    _fields_ = [("outer_its", ctypes.c_int), ("restarts", ctypes.c_int), ("inner_its", ctypes.c_longlong),
                ("inner_calls", ctypes.c_int), ("inner_capped", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("status", ctypes.c_int), ("phase_ms", ctypes.c_double * 8),
                ("err_est", ctypes.c_double), ("sigma_min", ctypes.c_double)]


def _load():
    if _build._stale():
        _build.build()
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is missing and could not be built")
    L = ctypes.CDLL(_LIB_PATH)
    P, D, I, V = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, None
    sig = {
        "pfc_default_options": (V, [ctypes.POINTER(_Options)]),
        "pfc_setup_mesh": (I, [ctypes.POINTER(P), I, I, D, ctypes.POINTER(_Options), P]),
        "pfc_num_dofs": (ctypes.c_int64, [P]),
        "pfc_footprint_bytes": (ctypes.c_size_t, [I, I, ctypes.POINTER(_Options)]),
        "pfc_assemble": (I, [P, P, D]),
        "pfc_stage_rhs": (I, [P, I, P, P, P]),
        "pfc_stage_solve": (I, [P, P, P, ctypes.POINTER(_Stats)]),
        "pfc_step": (I, [P, P, ctypes.POINTER(D), ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(_Stats)]),
        "pfc_euler_step": (I, [P, P, D, ctypes.POINTER(_Stats)]),
        "pfc_init_state": (I, [P, P, P]),
        "pfc_apply": (I, [P, I, P, P]),
        "pfc_pcg": (I, [P, I, P, P, D, ctypes.POINTER(I)]),
        "pfc_selftest_barrier_timeout": (I, [P, D]),
        "pfc_host_pattern": (I, [I, I, D, ctypes.POINTER(ctypes.c_int64)]),
        "pfc_host_stencil": (I, [I, I, D, ctypes.POINTER(ctypes.c_int64)]),
        "pfc_host_cells": (I, [I, I, D, ctypes.POINTER(ctypes.c_int64)]),
        "pfc_cell_kernels": (I, [P]),
        "pfc_host_partition": (I, [I, I, D, I, I, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(ctypes.c_int64)]),
        "pfc_batch_stage_solve": (I, [ctypes.POINTER(P), I, ctypes.POINTER(P), ctypes.POINTER(P),
                                      ctypes.POINTER(_Stats)]),
        "pfc_batch_step": (I, [ctypes.POINTER(P), I, ctypes.POINTER(P), ctypes.POINTER(D), ctypes.POINTER(I),
                               ctypes.POINTER(D), ctypes.POINTER(_Stats)]),
        "pfc_set_timing": (I, [P, I]),
        "pfc_step_begin": (I, [P, P, D]),
        "pfc_batch_stage_advance": (I, [ctypes.POINTER(P), I]),
        "pfc_step_finish": (I, [P, P, ctypes.POINTER(D), ctypes.POINTER(I), ctypes.POINTER(D),
                                ctypes.POINTER(_Stats)]),
        "pfc_step_stage": (I, [P]),
        "pfc_step_combine_static": (I, [ctypes.c_int64, P, P, D, D, P, P, P]),
        "pfc_counters": (I, [P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                             ctypes.POINTER(D)]),
        "pfc_last_error": (ctypes.c_char_p, [P]),
        "pfc_status_string": (ctypes.c_char_p, [I]),
        "pfc_critical_tau": (D, [D, D]),
        "pfc_destroy": (V, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


lib = _load()


class PFCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


@dataclass
class SolveStats:
    outer_its: int
    restarts: int
    inner_its: int
    inner_calls: int
    inner_capped: int
    rel_residual: float
    status: int
    phase_ms: tuple = ()
    err_est: float = float("nan")
    sigma_min: float = float("inf")

    @classmethod
    def _from(cls, s: _Stats) -> "SolveStats":
        return cls(s.outer_its, s.restarts, s.inner_its, s.inner_calls, s.inner_capped, s.rel_residual, s.status,
                   tuple(s.phase_ms), s.err_est, s.sigma_min)


def critical_tau(r: float, psi_bar: float) -> float:
    """Critical time-step width of Lemma 3, from the library (pfc_critical_tau); inf when none."""
    return float(lib.pfc_critical_tau(float(r), float(psi_bar)))


def default_options() -> dict:
    o = _Options()
    lib.pfc_default_options(ctypes.byref(o))
    return {k: getattr(o, k) for k, _ in _Options._fields_}


def host_pattern(dim: int, side: int, length: float = 1.0) -> dict:
    """Sizes from the host mesh/pattern builder (no GPU needed)."""
    out = (ctypes.c_int64 * 4)()
    st = lib.pfc_host_pattern(dim, side, float(length), out)
    if st != 0:
        raise PFCError(st, "host_pattern")
    return {"n": out[0], "nnz": out[1], "nnz_sell": out[2], "elements": out[3]}


def _handles(solvers):
    arr = (ctypes.c_void_p * len(solvers))()
    for k, s in enumerate(solvers):
        arr[k] = s._h.value
    return arr


def batch_stage_solve(solvers, bs):
    """One batched launch solving A^R_k y_k = b_k for every solver (see pfc_batch_stage_solve)."""
    if len(solvers) != len(bs) or not solvers:
        raise ValueError("one right-hand side per solver")
    ys = [s._new(3 * s.n) for s in solvers]
    bp = (ctypes.c_void_p * len(bs))(*[s._vec(b, 3 * s.n, "b").value for s, b in zip(solvers, bs)])
    yp = (ctypes.c_void_p * len(ys))(*[y.data_ptr() for y in ys])
    stats = (_Stats * len(solvers))()
    st = lib.pfc_batch_stage_solve(_handles(solvers), len(solvers), bp, yp, stats)
    if st != 0:
        raise PFCError(st, lib.pfc_last_error(solvers[0]._h).decode())
    return ys, [SolveStats._from(x) for x in stats]


def batch_step(solvers, states, taus, check: bool = True):
    """One Ros3Pw step attempt for every solver in one batch (see pfc_batch_step).
    states are updated in place where accepted.  Returns (accepted, errs, taus_next, stats[k][3])."""
    k = len(solvers)
    if len(states) != k or len(taus) != k or k == 0:
        raise ValueError("one state and one tau per solver")
    sp = (ctypes.c_void_p * k)(*[s._vec(x, 3 * s.n, "state").value for s, x in zip(solvers, states)])
    tt = (ctypes.c_double * k)(*[float(t) for t in taus])
    acc = (ctypes.c_int * k)()
    errs = (ctypes.c_double * k)()
    stats = (_Stats * (3 * k))()
    st = lib.pfc_batch_step(_handles(solvers), k, sp, tt, acc, errs, stats)
    if check and st != 0:
        raise PFCError(st, lib.pfc_last_error(solvers[0]._h).decode())
    out = [[SolveStats._from(stats[3 * i + j]) for j in range(3)] for i in range(k)]
    return [bool(a) for a in acc], list(errs), list(tt), out


def batch_stage_advance(solvers):
    """One batched launch solving every solver's next stage of its begun step
    (pfc_batch_stage_advance); each solver's stage advances by one."""
    if not solvers:
        raise ValueError("no solvers")
    st = lib.pfc_batch_stage_advance(_handles(solvers), len(solvers))
    if st != 0:
        raise PFCError(st, lib.pfc_last_error(solvers[0]._h).decode())


def host_partition(dim: int, side: int, length: float, nparts: int, degree: int = 2) -> dict:
    """Row-block (strip) partition of one instance over nparts devices (pfc_host_partition):
    {"begin": row offsets (nparts + 1), "halo": [(below, above)] * nparts, "nnz": per part}."""
    b = (ctypes.c_int64 * (nparts + 1))()
    h = (ctypes.c_int64 * (2 * nparts))()
    z = (ctypes.c_int64 * nparts)()
    st = lib.pfc_host_partition(dim, side, float(length), degree, nparts, b, h, z)
    if st != 0:
        raise PFCError(st, "host_partition")
    return {"begin": list(b), "halo": [(h[2 * k], h[2 * k + 1]) for k in range(nparts)], "nnz": list(z)}


def host_stencil(dim: int, side: int, length: float = 1.0) -> dict:
    """Stencil sizes from the host builder (no GPU needed)."""
    out = (ctypes.c_int64 * 3)()
    st = lib.pfc_host_stencil(dim, side, float(length), out)
    if st != 0:
        raise PFCError(st, "host_stencil")
    return {"interior_rows": out[0], "boundary_nnz": out[1], "stencil_entries": out[2]}


def host_cells(side: int, length: float = 1.0, dim: int = 2) -> dict:
    """Row and cell classes of the P2 cell-major order from the host builder (no GPU needed)."""
    out = (ctypes.c_int64 * 4)()
    st = lib.pfc_host_cells(dim, side, float(length), out)
    if st != 0:
        raise PFCError(st, "host_cells")
    return {"classes": out[0], "entries": out[1], "pattern_ok": out[2] > 0, "cell_classes": out[2],
            "rows": out[3]}


class PFCSolver:
    """One PFC simulation instance on the current CUDA device.

    Vectors are float64 CUDA tensors in lexicographic P2 dof order; a state has
    3n entries [mu | psi | omega].  All work runs on the CUDA stream current at
    construction (or ``stream``)."""

    def __init__(self, dim: int, side: int, length: float, r: float = -0.4, precision: str = "fp64",
                 outer_tol: float = 1e-10, inner_rtol: float = 1e-3, restart: int = 30, max_outer: int = 600,
                 max_inner: int = 1000, step_atol: float = 1e-3, step_rtol: float = 1e-3,
                 tau_max: float = 1e9, blocks_per_sm: int = 0, pcg_variant: int = 2,
                 inner_operator: int = 1, smem_window: int | None = None, model: int = 2, psi_min: float = -1.5,
                 schur: int = 0, schur_its: int = 20, degree: int = 2, err_tol: float = 1e-9,
                 tau_guard: float = 0.0, grid_blocks: int = 0, cells: int | None = None, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise PFCError(3, "no CUDA device: the PFC solver runs only on the GPU")
        self._torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        o = _Options()
        lib.pfc_default_options(ctypes.byref(o))
        o.r, o.outer_tol, o.inner_rtol = r, outer_tol, inner_rtol
        o.restart, o.max_outer, o.max_inner = restart, max_outer, max_inner
        o.precision = PRECISIONS[precision]
        o.step_atol, o.step_rtol, o.tau_max, o.blocks_per_sm = step_atol, step_rtol, tau_max, blocks_per_sm
        o.pcg_variant = pcg_variant
        o.inner_operator = inner_operator
        if smem_window is not None:        # else the library's default (pfc_default_options)
            o.smem_window = smem_window
        o.model = model
        o.psi_min = psi_min
        o.schur = schur
        o.schur_its = schur_its
        o.degree = degree
        o.err_tol = err_tol
        o.tau_guard = tau_guard
        o.grid_blocks = grid_blocks
        if cells is not None:              # else the library's default (pfc_default_options)
            o.cells = cells
        self.options = o
        self.dim, self.side, self.length, self.r, self.precision = dim, side, float(length), r, precision
        h = ctypes.c_void_p()
        st = lib.pfc_setup_mesh(ctypes.byref(h), dim, side, float(length), ctypes.byref(o),
                                ctypes.c_void_p(self.stream.cuda_stream))
        if st != 0:
            msg = lib.pfc_last_error(h).decode() if h.value else ""
            if h.value:
                lib.pfc_destroy(h)
            raise PFCError(st, msg)
        self._h = h
        self.n = int(lib.pfc_num_dofs(h))

    # --- marshalling helpers ------------------------------------------------
    def _vec(self, t, count: int, name: str):
        torch = self._torch
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or t.device != self.device:
            raise TypeError(f"{name} must be a float64 tensor on {self.device}")
        if not t.is_contiguous() or t.numel() != count:
            raise ValueError(f"{name} must be contiguous with {count} entries")
        return ctypes.c_void_p(t.data_ptr())

    def _new(self, count: int):
        return self._torch.empty(count, dtype=self._torch.float64, device=self.device)

    def _check(self, st: int):
        if st != 0:
            raise PFCError(st, lib.pfc_last_error(self._h).decode())

    # --- API ------------------------------------------------------------------
    def init_state(self, psi0):
        state = self._new(3 * self.n)
        self._check(lib.pfc_init_state(self._h, self._vec(psi0, self.n, "psi0"), self._vec(state, 3 * self.n, "state")))
        return state

    def assemble(self, state, tau: float):
        self._check(lib.pfc_assemble(self._h, self._vec(state, 3 * self.n, "state"), float(tau)))

    def stage_rhs(self, nprev: int, x_stage, y_prev=None):
        b = self._new(3 * self.n)
        yp = self._vec(y_prev, nprev * 3 * self.n, "y_prev") if nprev > 0 else None
        self._check(lib.pfc_stage_rhs(self._h, nprev, self._vec(x_stage, 3 * self.n, "x_stage"), yp,
                                      self._vec(b, 3 * self.n, "b")))
        return b

    def stage_solve(self, b, y=None, check: bool = True):
        y = self._new(3 * self.n) if y is None else y
        s = _Stats()
        st = lib.pfc_stage_solve(self._h, self._vec(b, 3 * self.n, "b"), self._vec(y, 3 * self.n, "y"),
                                 ctypes.byref(s))
        if check:
            self._check(st)
        return y, SolveStats._from(s)

    def step(self, state, tau: float, check: bool = True):
        """One Ros3Pw step attempt; state (device, 3n) is updated in place if accepted.
        Returns (accepted, err, tau_next, [SolveStats] * 3)."""
        t = ctypes.c_double(tau)
        acc = ctypes.c_int(0)
        err = ctypes.c_double(0.0)
        stats = (_Stats * 3)()
        st = lib.pfc_step(self._h, self._vec(state, 3 * self.n, "state"), ctypes.byref(t), ctypes.byref(acc),
                          ctypes.byref(err), stats)
        if check:
            self._check(st)
        return bool(acc.value), err.value, t.value, [SolveStats._from(s) for s in stats]

    def step_begin(self, state, tau: float):
        """Assembly for a stage-wise step (pfc_step_begin); the stages are solved by
        batch_stage_advance and the step completed by step_finish."""
        self._check(lib.pfc_step_begin(self._h, self._vec(state, 3 * self.n, "state"), float(tau)))

    @property
    def stage(self) -> int:
        """-1 no begun step, 0..2 next stage, 3 ready for step_finish (pfc_step_stage)."""
        return int(lib.pfc_step_stage(self._h))

    def step_finish(self, state, tau: float, check: bool = True):
        """Completes a stage-wise step like step(): returns (accepted, err, tau_next, stats)."""
        t = ctypes.c_double(tau)
        acc = ctypes.c_int(0)
        err = ctypes.c_double(0.0)
        stats = (_Stats * 3)()
        st = lib.pfc_step_finish(self._h, self._vec(state, 3 * self.n, "state"), ctypes.byref(t), ctypes.byref(acc),
                                 ctypes.byref(err), stats)
        if check:
            self._check(st)
        return bool(acc.value), err.value, t.value, [SolveStats._from(s) for s in stats]

    def euler_step(self, state, tau: float, check: bool = True) -> "SolveStats":
        """One linearised semi-implicit Euler step (Eq. 3.4) with step width tau; state
        (device, 3n) is overwritten with x_{k+1} when the solve succeeds."""
        stats = _Stats()
        st = lib.pfc_euler_step(self._h, self._vec(state, 3 * self.n, "state"), float(tau), ctypes.byref(stats))
        if check:
            self._check(st)
        return SolveStats._from(stats)

    def apply(self, op: int, x):
        m = 3 * self.n if op in (OP_AR, OP_PCH) else self.n
        y = self._new(m)
        self._check(lib.pfc_apply(self._h, op, self._vec(x, m, "x"), self._vec(y, m, "y")))
        return y

    def pcg(self, which: int, b, rtol: float):
        x = self._new(self.n)
        its = ctypes.c_int(0)
        self._check(lib.pfc_pcg(self._h, which, self._vec(b, self.n, "b"), self._vec(x, self.n, "x"), float(rtol),
                                ctypes.byref(its)))
        return x, its.value

    def set_timing(self, enable: bool = True):
        self._check(lib.pfc_set_timing(self._h, 1 if enable else 0))

    @property
    def cell_kernels(self) -> bool:
        """Whether this context's float32/float16 inner solves run the cell kernels."""
        return bool(lib.pfc_cell_kernels(self._h))

    def counters(self) -> dict:
        """Kernels launched by this context, persistent-solver launches and their summed event time."""
        a, b, ms = ctypes.c_longlong(0), ctypes.c_longlong(0), ctypes.c_double(0.0)
        self._check(lib.pfc_counters(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(ms)))
        return {"kernel_launches": a.value, "solver_launches": b.value, "solver_ms": ms.value}

    def selftest_barrier_timeout(self, limit_seconds: float = 0.2) -> int:
        return int(lib.pfc_selftest_barrier_timeout(self._h, float(limit_seconds)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.pfc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
