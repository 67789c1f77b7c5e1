"""Batched launches of independent instances (pfc_batch_stage_solve, pfc_batch_step).

Each instance's result in a batch must match its single-instance result to the
stage-solve tolerance (relative 1e-8 on the stage solutions and step increments):
the segment of the grid an instance gets in a batch differs from its own grid, so
the summation order of its reductions differs.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1501_06852_gb300 as pfc  # noqa: E402

MIX = [(2, 8, 8.0, -0.4, -0.3), (2, 16, 16.0, -0.3, -0.25), (3, 3, 3.0, -0.3, -0.35), (2, 5, 5.0, -0.45, -0.35)]


def _make(precision, **kw):
    out = []
    for k, (dim, side, L, r, pm) in enumerate(MIX):
        s = pfc.PFCSolver(dim, side, L, r=r, precision=precision, outer_tol=1e-11, **kw)
        x0 = s.init_state(torch.from_numpy(synth.initial_psi(dim, side, pm, 0.1, 100 + k)).cuda())
        out.append((s, x0))
    return out


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batched_stage_solves_match_single_solves(precision):
    inst = _make(precision)
    try:
        bs, refs = [], []
        for s, x0 in inst:
            s.assemble(x0, 0.3)
            b = s.stage_rhs(0, x0)
            y, st = s.stage_solve(b)
            bs.append(b)
            refs.append(y)
        ys, stats = pfc.batch_stage_solve([s for s, _ in inst], bs)
        for y, yr, st in zip(ys, refs, stats):
            assert st.status == 0 and st.rel_residual <= 1e-11
            assert float((y - yr).norm() / yr.norm()) <= 1e-8
    finally:
        for s, _ in inst:
            s.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batched_steps_match_single_steps(precision):
    inst = _make(precision)
    try:
        taus = [0.1, 0.2, 0.05, 0.4]
        singles = []
        for (s, x0), tau in zip(inst, taus):
            x = x0.clone()
            acc, err, tn, _ = s.step(x, tau)
            singles.append((x, acc, err, tn))
        # fresh contexts for the batch (step control keeps per-context history)
        inst2 = _make(precision)
        try:
            states = [x0.clone() for _, x0 in inst2]
            acc, errs, tns, stats = pfc.batch_step([s for s, _ in inst2], states, taus)
            for k, (x, a1, e1, t1) in enumerate(singles):
                x0 = inst2[k][1]
                assert acc[k] == a1
                assert errs[k] == pytest.approx(e1, rel=1e-6)
                assert tns[k] == pytest.approx(t1, rel=1e-6)
                d_ref, d_got = (x - x0), (states[k] - x0)
                if a1:
                    assert float((d_got - d_ref).norm() / d_ref.norm()) <= 1e-8
                assert all(st.status == 0 for st in stats[k])
        finally:
            for s, _ in inst2:
                s.close()
    finally:
        for s, _ in inst:
            s.close()


def test_more_instances_than_resident_blocks_run_in_waves():
    # one block per SM: more instances than co-resident blocks -> several launches
    props = torch.cuda.get_device_properties(0)
    count = props.multi_processor_count + 8
    solvers, bs, refs = [], [], []
    try:
        for k in range(count):
            s = pfc.PFCSolver(2, 1, 1.0, r=-0.4, outer_tol=1e-11, blocks_per_sm=1)
            x0 = s.init_state(torch.from_numpy(synth.initial_psi(2, 1, -0.3, 0.1, 500 + k)).cuda())
            s.assemble(x0, 0.1)
            b = s.stage_rhs(0, x0)
            y, _ = s.stage_solve(b)
            solvers.append(s)
            bs.append(b)
            refs.append(y)
        ys, stats = pfc.batch_stage_solve(solvers, bs)
        for y, yr in zip(ys, refs):
            assert float((y - yr).norm() / yr.norm()) <= 1e-8
    finally:
        for s in solvers:
            s.close()


def test_batch_rejects_mixed_precisions():
    a = pfc.PFCSolver(2, 2, 2.0, precision="fp32")
    b = pfc.PFCSolver(2, 2, 2.0, precision="fp64")
    try:
        x = [torch.zeros(3 * s.n, dtype=torch.float64, device="cuda") for s in (a, b)]
        with pytest.raises(pfc.PFCError):
            pfc.batch_step([a, b], x, [0.1, 0.1])
    finally:
        a.close()
        b.close()
