"""Closed forms of the paper's spectral analysis (Section 6).

TEST INFRASTRUCTURE (see ``oracle/__init__``).
"""
from __future__ import annotations

import math


def critical_tau(r: float, psi_bar: float = 0.0) -> float:
    """Lemma 3: the symbol of the linearised operator reaches zero once
    tau >= tau* = 27 / (2 (sqrt(alpha) - 1)(sqrt(alpha) + 2)^2), alpha = 1 - 3r - 9 psi_bar^2.
    Returns +inf when no critical width exists (alpha <= 1, i.e. psi_bar^2 >= -r/3)."""
    alpha = 1.0 - 3.0 * r - 9.0 * psi_bar * psi_bar
    if alpha <= 1.0:
        return math.inf
    sa = math.sqrt(alpha)
    return 27.0 / (2.0 * (sa - 1.0) * (sa + 2.0) ** 2)


def symbol_A0(k2: float, tau: float, r: float, psi_bar: float = 0.0) -> float:
    """Stabilised symbol (Eq. 6.6): 1 + tau[(3 psi_bar^2 + 1 + r) k^2 - 2 k^4 + k^6]."""
    return 1.0 + tau * ((3.0 * psi_bar ** 2 + 1.0 + r) * k2 - 2.0 * k2 ** 2 + k2 ** 3)


def q_eigenvalue(k2: float, tau: float, r: float, psi_bar: float = 0.0) -> float:
    """Third eigenvalue of Q = A P^{-1} (Eq. 6.8)."""
    st = math.sqrt(tau)
    den = tau * k2 ** 3 + (st - 2.0 * tau) * k2 ** 2 - st * k2 + 1.0
    return symbol_A0(k2, tau, r, psi_bar) / den


def qch_denominator(k2: float, tau: float) -> float:
    """Denominator of the third eigenvalue of Q_CH (Eq. 6.9)."""
    return tau * k2 ** 3 + (math.sqrt(tau) + 2.0 * tau ** 0.75) * k2 ** 2 \
        + (math.sqrt(tau) + 2.0 * tau ** 0.25) * k2 + 1.0


def qch_eigenvalue(k2: float, tau: float, r: float, psi_bar: float = 0.0) -> float:
    """Third eigenvalue of Q_CH = A P_CH^{-1} (Eq. 6.9)."""
    return symbol_A0(k2, tau, r, psi_bar) / qch_denominator(k2, tau)


def lemma2_lambda(mu: float, delta: float) -> float:
    """Eigenvalue of S_CH^{-1} S for the eigenvalue mu of M^{-1}K (Lemma 2).
    Reading of the garbled formula: S = M - 2 delta K + delta K M^{-1} K and
    S_CH = (M + sqrt(delta) K) M^{-1} (M + sqrt(delta) K) give
    lambda(mu) = (1 - 2 delta mu + delta mu^2) / (1 + sqrt(delta) mu)^2."""
    return (1.0 - 2.0 * delta * mu + delta * mu * mu) / (1.0 + math.sqrt(delta) * mu) ** 2


def lemma2_bounds(delta: float) -> tuple[float, float]:
    return (1.0 - math.sqrt(delta)) / 2.0, 1.0


def interval_convergence_factor(alpha: float, beta: float) -> float:
    """Eq. (5.8): rho = (sqrt(kappa) - 1)/(sqrt(kappa) + 1), kappa = beta/alpha."""
    k = beta / alpha
    return (math.sqrt(k) - 1.0) / (math.sqrt(k) + 1.0)
