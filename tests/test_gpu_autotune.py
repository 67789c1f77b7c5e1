"""The autotuner times every candidate and returns the fastest one."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1501_06852_gb300 import autotune  # noqa: E402


def test_autotune_picks_the_fastest_candidate():
    res = autotune.tune(2, 16, 16.0, "fp32", iters=20, reps=1)
    times = [c["us_per_iteration"] for c in res["all"]]
    assert len(times) == len(autotune.candidates("fp32"))
    assert res["us_per_iteration"] == min(times)
    assert res["config"] in autotune.candidates("fp32")
    assert autotune.tune(2, 16, 16.0, "fp32") is res      # cached
