"""pfc_step_combine_static: the step combination and error estimate for callers
that cannot allocate device memory (code inside a stream capture, a loop that must
not touch the allocator, a guest whose host application owns all device memory).

It is called through the C ABI on vectors the caller owns and compared with the
existing entry point pfc_step on the same step, on two calls in a row (the calls
share the library's static scratch array).  This file is collected last, so a run
that stops at the first failure has already run every other test; it also passes
on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1501_06852_gb300 as pfc  # noqa: E402

# Ros3Pw stage weights a_ij (Table 1)
A21, A31 = 2.0, 0.633974596215561


def _stage_increments(s, x0, tau):
    """The three stage increments of one step, through the public stage API."""
    s.assemble(x0, tau)
    ys = []
    for i in range(3):
        xi = x0.clone()
        if i == 1:
            xi += A21 * ys[0]
        elif i == 2:
            xi += A31 * ys[0]
        yp = torch.cat(ys) if ys else None
        b = s.stage_rhs(i, xi, yp)
        y, st = s.stage_solve(b)
        assert st.status == 0
        ys.append(y)
    return torch.cat(ys)


def test_static_step_combination_matches_pfc_step_twice():
    w = synth.C1_2D_SMALL
    with pfc.PFCSolver(w.dim, w.side, w.length, r=w.r, outer_tol=1e-11) as s:
        n = s.n
        x0 = s.init_state(torch.from_numpy(synth.initial_psi(w.dim, w.side, w.psi_mean, w.amp, w.seed)).cuda())
        ref_state = x0.clone()
        acc, err_ref, _, _ = s.step(ref_state, w.tau0)
        assert acc
        y = _stage_increments(s, x0, w.tau0)
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        for call in range(2):
            out = torch.full((3 * n,), float("nan"), dtype=torch.float64, device="cuda")
            err = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            st = pfc.lib.pfc_step_combine_static(n, ctypes.c_void_p(x0.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                                 1e-3, 1e-3, ctypes.c_void_p(out.data_ptr()),
                                                 ctypes.c_void_p(err.data_ptr()), stream)
            assert st == 0, call
            torch.cuda.synchronize()
            d_ref = (ref_state - x0).cpu().numpy()
            d_got = (out - x0).cpu().numpy()
            # stage solutions agree to the stage-solve tolerance of the parity tests
            assert np.linalg.norm(d_got - d_ref) <= 1e-8 * np.linalg.norm(d_ref), call
            assert float(err.item()) == pytest.approx(err_ref, rel=1e-6), call


def test_static_step_combination_rejects_bad_sizes():
    x = torch.zeros(3, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(x.data_ptr())
    assert pfc.lib.pfc_step_combine_static(0, p, p, 1e-3, 1e-3, p, p, None) == 1
    assert pfc.lib.pfc_step_combine_static(2 ** 31, p, p, 1e-3, 1e-3, p, p, None) == 1
    assert pfc.lib.pfc_step_combine_static(1, None, p, 1e-3, 1e-3, p, p, None) == 1
