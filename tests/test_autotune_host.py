"""Candidate lists of the autotuner (host logic)."""
from paper_1501_06852_gb300 import autotune


def test_candidates_keep_outer_iteration_safe_forms():
    c32 = autotune.candidates("fp32")
    assert all(c["pcg_variant"] in (0, 3) for c in c32)          # no pipelined form in float32
    assert {c["inner_operator"] for c in c32} == {0, 1}
    assert {c["blocks_per_sm"] for c in c32} == {1, 2}
    assert {c["pcg_variant"] for c in autotune.candidates("fp64")} == {0, 1, 3}
