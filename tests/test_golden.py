"""Values printed in the paper (tests/golden/*) against the oracle's closed forms."""
import math
import os

import pytest

from oracle import analysis

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    for line in open(os.path.join(GOLDEN, name)):
        if line.strip() and not line.startswith("#"):
            yield [float(v) for v in line.split()]


def test_lemma3_worked_values():
    rows = list(_rows("lemma3_critical_tau.txt"))
    assert len(rows) == 2
    for r, psi_bar, printed, digits in rows:
        got = analysis.critical_tau(r, psi_bar)
        # the paper prints 5 significant digits
        assert float(f"{got:.{int(digits)}g}") == pytest.approx(printed, rel=1e-12)


def test_lemma3_no_critical_width_in_liquid_phase():
    # psi_bar^2 >= -r/3 leaves no critical width (Lemma 3)
    assert analysis.critical_tau(-0.3, -0.35) == math.inf
    # and the symbol is zero exactly at tau* at the critical wave number k^2 = 2/3 + sqrt(alpha)/3
    r, pb = -0.4, -0.3
    ts = analysis.critical_tau(r, pb)
    k2 = 2.0 / 3.0 + math.sqrt(1 - 3 * r - 9 * pb * pb) / 3.0
    assert abs(analysis.symbol_A0(k2, ts, r, pb)) < 1e-12
    assert min(analysis.symbol_A0(0.01 * i, 0.99 * ts, r, pb) for i in range(1, 400)) > 0


def test_critical_tau_for_p_is_one():
    # tau_natural = 1 for P (Section 6.1): its q-denominator vanishes at k^2 = 1, tau = 1
    den = lambda k2, tau: tau * k2 ** 3 + (math.sqrt(tau) - 2 * tau) * k2 ** 2 - math.sqrt(tau) * k2 + 1
    assert abs(den(1.0, 1.0)) < 1e-15
    assert min(den(0.01 * i, 0.99) for i in range(1, 400)) > 0
    # P_CH's denominator stays positive for every tau (Section 6.1), so the third
    # eigenvalue of Q_CH changes sign only with the symbol of A_0: it is positive for
    # every wave number below Lemma 3's critical width and reaches zero at it
    r, pb = -0.35, 0.0
    ts = analysis.critical_tau(r, pb)
    k2s = [0.01 * i for i in range(0, 1000)]
    for tau in (1e-3, 0.01, 0.1, 1.0, 10.0, 100.0, 1e4):
        assert min(analysis.qch_denominator(k2, tau) for k2 in k2s) > 0
    for tau in (0.01, 0.1, 0.5 * ts, 0.99 * ts):
        assert min(analysis.qch_eigenvalue(k2, tau, r, pb) for k2 in k2s) > 0
    kc = 2.0 / 3.0 + math.sqrt(1 - 3 * r - 9 * pb * pb) / 3.0
    assert abs(analysis.qch_eigenvalue(kc, ts, r, pb)) < 1e-12
    assert analysis.qch_eigenvalue(kc, 1.5 * ts, r, pb) < 0


def test_interval_convergence_factor():
    assert analysis.interval_convergence_factor(1.0, 1.0) == 0.0
    assert analysis.interval_convergence_factor(1.0, 9.0) == pytest.approx(0.5)
