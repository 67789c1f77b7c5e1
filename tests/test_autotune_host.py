"""Candidate lists of the autotuner (host logic)."""
from paper_1501_06852_gb300 import autotune


def test_candidates_keep_outer_iteration_safe_forms():
    c32 = autotune.candidates("fp32")
    assert all(c["pcg_variant"] in (0, 3) for c in c32)          # no pipelined form in float32
    assert {c["inner_operator"] for c in c32} == {0, 1}
    assert {c["pcg_variant"] for c in autotune.candidates("fp64")} == {0, 1, 3}


def test_cell_kernels_are_a_candidate_of_the_float_forms():
    c32 = autotune.candidates("fp32")
    cells = [c for c in c32 if c["cells"] == 1]
    assert cells == [dict(inner_operator=1, pcg_variant=3, cells=1)]
    assert dict(inner_operator=1, pcg_variant=3, cells=0) in c32
    assert all(c["cells"] == 0 for c in autotune.candidates("fp64"))


def test_size_classes_are_powers_of_two():
    assert [autotune.size_class(s) for s in (1, 16, 22, 31, 32, 48, 63, 255, 256, 700)] == \
        [8, 16, 16, 16, 32, 32, 32, 128, 256, 512]
