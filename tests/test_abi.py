"""The C ABI library loads on a CPU-only machine, exports every symbol that
include/pfc.h declares, and its host logic (options, status codes, mesh and
SELL pattern builder, argument checks) behaves as documented.  No GPU calls."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    from paper_1501_06852_gb300 import build as b
    b.build()
    import paper_1501_06852_gb300 as p
    return p


def _declared():
    text = open(os.path.join(ROOT, "include", "pfc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pfc_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(pkg):
    names = _declared()
    assert len(names) >= 16
    lib = ctypes.CDLL(pkg.build.LIB)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_default_options(pkg):
    o = pkg.default_options()
    assert o["restart"] == 30 and o["inner_rtol"] == 1e-3 and o["outer_tol"] == 1e-10
    assert o["precision"] == 0 and o["step_atol"] == 1e-3 and o["step_rtol"] == 1e-3
    assert o["pcg_variant"] == 2 and o["inner_operator"] == 1 and o["smem_window"] == 0
    assert o["model"] == 2 and o["psi_min"] == -1.5 and o["schur"] == 0 and o["schur_its"] == 20
    assert o["degree"] == 2 and o["err_tol"] == 1e-9 and o["tau_guard"] == 0.0 and o["grid_blocks"] == 0
    assert o["cells"] == 1


def test_status_strings(pkg):
    for k, v in pkg.STATUS.items():
        assert pkg.lib.pfc_status_string(k).decode() == v
    assert pkg.lib.pfc_status_string(99).decode() == "PFC_UNKNOWN"


@pytest.mark.parametrize("side", [1, 2, 3, 5, 8, 32])
def test_host_pattern_2d(pkg, side):
    hp = pkg.host_pattern(2, side, float(side))
    assert hp["n"] == (2 * side + 1) ** 2
    assert hp["nnz"] == 46 * side * side + 16 * side + 1
    assert hp["elements"] == 2 * side * side
    n_pad = (hp["n"] + 31) // 32 * 32
    assert hp["nnz"] <= hp["nnz_sell"] <= 19 * n_pad


@pytest.mark.parametrize("side", [1, 2, 3, 6])
def test_host_pattern_3d(pkg, side):
    hp = pkg.host_pattern(3, side, float(side))
    assert hp["n"] == (2 * side + 1) ** 3
    assert hp["nnz"] == 230 * side ** 3 + 138 * side ** 2 + 24 * side + 1
    assert hp["elements"] == 6 * side ** 3
    assert hp["nnz_sell"] >= hp["nnz"]


def test_sell_padding_is_small_at_benchmark_size(pkg):
    hp = pkg.host_pattern(2, 512, 256.0)
    assert hp["nnz"] == 12066817
    assert hp["nnz_sell"] / hp["nnz"] < 1.02


def test_invalid_arguments_rejected_before_any_gpu_call(pkg):
    lib = pkg.lib
    out = (ctypes.c_int64 * 4)()
    assert lib.pfc_host_pattern(4, 2, 1.0, out) == 1
    assert lib.pfc_host_pattern(2, 0, 1.0, out) == 1
    assert lib.pfc_host_pattern(2, 2, -1.0, out) == 1
    h = ctypes.c_void_p()
    st = lib.pfc_setup_mesh(ctypes.byref(h), 5, 4, 1.0, None, None)
    assert st == 1
    assert b"dim" in lib.pfc_last_error(h)
    lib.pfc_destroy(h)
    assert lib.pfc_assemble(None, None, 0.1) == 1
    assert lib.pfc_stage_solve(None, None, None, None) == 1
    assert lib.pfc_num_dofs(None) == 0
    lib.pfc_destroy(None)


def test_footprint_grows_with_size_and_precision(pkg):
    f = pkg.lib.pfc_footprint_bytes
    assert f(2, 64, None) < f(2, 128, None) < f(2, 512, None)
    assert f(3, 16, None) > 0 and f(4, 16, None) == 0
    o = pkg._Options()
    pkg.lib.pfc_default_options(ctypes.byref(o))
    o.precision = 1
    assert f(2, 512, ctypes.byref(o)) > f(2, 512, None)


def test_critical_tau_export(pkg):
    """pfc_critical_tau (Lemma 3) against the widths the paper prints and the oracle's closed form."""
    from oracle import analysis
    for line in open(os.path.join(ROOT, "tests", "golden", "lemma3_critical_tau.txt")):
        if line.strip() and not line.startswith("#"):
            r, pb, printed, digits = (float(v) for v in line.split())
            got = pkg.lib.pfc_critical_tau(r, pb)
            assert float(f"{got:.{int(digits)}g}") == pytest.approx(printed, rel=1e-12)
    for r in (-0.5, -0.4, -0.35, -0.2, -0.05):
        for pb in (0.0, -0.1, -0.2, -0.3, -0.35, -0.5):
            want = analysis.critical_tau(r, pb)
            got = pkg.critical_tau(r, pb)
            assert got == want if math.isinf(want) else got == pytest.approx(want, rel=1e-14)
    assert pkg.critical_tau(-0.3, -0.35) == float("inf")


def test_width_guard_option_checked(pkg):
    o = pkg._Options()
    pkg.lib.pfc_default_options(ctypes.byref(o))
    for bad in (-0.1, 1.0, float("nan")):
        o.tau_guard = bad
        h = ctypes.c_void_p()
        assert pkg.lib.pfc_setup_mesh(ctypes.byref(h), 2, 2, 2.0, ctypes.byref(o), None) == 1
        assert b"tau_guard" in pkg.lib.pfc_last_error(h)
        pkg.lib.pfc_destroy(h)
    o.tau_guard = 0.0
    for bad in (-1e-9, float("inf"), float("nan")):
        o.err_tol = bad
        h = ctypes.c_void_p()
        assert pkg.lib.pfc_setup_mesh(ctypes.byref(h), 2, 2, 2.0, ctypes.byref(o), None) == 1
        assert b"err_tol" in pkg.lib.pfc_last_error(h)
        pkg.lib.pfc_destroy(h)


def test_static_step_combination_size_limit(pkg):
    """pfc_step_combine_static rejects n beyond (2^31 - 1 - 2^18) / 3 before touching the GPU
    (its kernel's 32-bit index steps by 2^18 past 3n)."""
    limit = (2 ** 31 - 1 - 2 ** 18) // 3
    assert limit == 715740501
    dummy = ctypes.c_void_p(256)   # never dereferenced: the size check comes first
    f = pkg.lib.pfc_step_combine_static
    assert f(limit + 1, dummy, dummy, 1e-3, 1e-3, dummy, dummy, None) == 1
    assert f((2 ** 31 - 1) // 3, dummy, dummy, 1e-3, 1e-3, dummy, dummy, None) == 1
    assert f(0, dummy, dummy, 1e-3, 1e-3, dummy, dummy, None) == 1


def test_no_cuda_means_loud_failure(pkg):
    import torch
    if torch.cuda.is_available():
        pytest.skip("CUDA present")
    with pytest.raises(pkg.PFCError):
        pkg.PFCSolver(2, 4, 4.0)
