"""Ros3Pw Rosenbrock stages for the PFC2 and PFC1 models, step combination and step control.

TEST INFRASTRUCTURE (see ``oracle/__init__``).

Section 3.1 writes the Rosenbrock scheme in its modified form (Eq. 3.6, 3.7):

    (1/(tau gamma)) MM y_i - J_F(x^k)[y_i] = F(x_i) + sum_{j<i} (c_ij / tau) MM y_j,
    x_i = x^k + sum_{j<i} a_ij y_j,
    x^{k+1} = x^k + sum_j m_j y_j,   xhat^{k+1} = x^k + sum_j mhat_j y_j,

with MM = diag(0, 1, 0) for x = (mu, psi, omega).  For the PFC2 model (H^{-1}
gradient flow, Eq. 2.2) the mobility is 1, so K_+ = K and F(mu) = 0, and the
stage system is Eq. (3.10):

    A^R = [[M, -(1+r) M + 2 K + N(psi_k), K],
           [tau K, M / gamma, 0],
           [0, K, M]]

with the right-hand side of the weak form (3.9) and its second component
multiplied by tau:

    b0 = -M mu_i + (1+r) M psi_i - 2 K psi_i - K omega_i + l(psi_i^3)
    b1 = -tau K mu_i + sum_{j<i} c_ij M dpsi_j
    b2 = -M omega_i - K psi_i

For the PFC1 model (Wasserstein flow, Eq. 2.3, mobility psi^+ = psi - psi_min with
psi_min = -1.5) the second block row of Eq. (3.10) becomes

    [tau K_+(psi_k), M / gamma + tau F(mu_k), 0],   b1 = -tau K_+(psi_i) mu_i + sum_{j<i} c_ij M dpsi_j

(K_+ and F as in ``assembly``).  Readings: psi^+ is psi - psi_min without clipping
(the Jacobian of Section 3.1 is taken under that assumption), and the preconditioner
uses the constant-mobility approximation K_+ ~ M0 K of Section 4 with M0 the mean of
psi_k^+ over the domain and F dropped: P_CH is built as for PFC2 with tau replaced by
M0 tau.

Reading of Table 1 (garbled): the diagonal entries "a22", "a33", "c11", "c22",
"c33" of the printed table are stage-time sums of the standard form and are not
entries of the modified-form matrices; for this autonomous system they are
unused.  The entries used are gamma, a21, a31, a32 = 0, c21, c31, c32, m, mhat.

Reading of the step-size control (the paper defers to Hairer-Wanner and Lang,
Section 3.1): error vector e = xhat^{k+1} - x^{k+1} restricted to psi (the
differential component, MM = diag(0, 1, 0)); err = RMS of
e_j / (atol + rtol * max(|psi^k_j|, |psi^{k+1}_j|)) with atol = rtol = 1e-3;
accept iff err <= 1; tau_new = tau * min(5, max(0.2, 0.9 err^{-1/3})) (embedded
order 2), except that an accepted step right after a rejected one may not grow
the width (fac <= 1; Hairer & Wanner, Solving ODEs II, Section IV.8).  Parity
unpinned: this is a convention, not a result of the paper.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import assembly
from .mesh import Mesh
from .solvers import PCH, fgmres


@dataclass(frozen=True)
class Ros3Pw:
    """Coefficients of Table 1 (modified form)."""

    gamma: float = 0.78867513459481287
    a21: float = 2.0
    a31: float = 0.633974596215561
    a32: float = 0.0
    c21: float = -2.53589838486225
    c31: float = -1.62740473580836
    c32: float = -0.274519052838329
    m: tuple = (1.63397459621556, 0.294228634059948, 1.07179676972449)
    mhat: tuple = (1.99444650053487, 0.654700538379252, 1.07179676972449)

    def a(self, i: int, j: int) -> float:
        return {(1, 0): self.a21, (2, 0): self.a31, (2, 1): self.a32}.get((i, j), 0.0)

    def c(self, i: int, j: int) -> float:
        return {(1, 0): self.c21, (2, 0): self.c31, (2, 1): self.c32}.get((i, j), 0.0)


ROS3PW = Ros3Pw()


def rosenbrock_ode_step(f, jac, x: np.ndarray, tau: float, coef: Ros3Pw = ROS3PW):
    """One step of Eq. (3.6)/(3.7) for an ODE x' = f(x) (MM = I), dense Jacobian.

    Returns (x^{k+1}, xhat^{k+1}).  Used to check the coefficient reading.
    """
    n = x.size
    A = np.eye(n) / (tau * coef.gamma) - jac(x)
    ys = []
    for i in range(3):
        xi = x + sum(coef.a(i, j) * ys[j] for j in range(i))
        b = f(xi) + sum(coef.c(i, j) / tau * ys[j] for j in range(i))
        ys.append(np.linalg.solve(A, b))
    xn = x + sum(coef.m[j] * ys[j] for j in range(3))
    xh = x + sum(coef.mhat[j] * ys[j] for j in range(3))
    return xn, xh


@dataclass
class PFCProblem:
    """Mesh, constant matrices and parameters of one PFC simulation (model 2: PFC2,
    mobility 1; model 1: PFC1, mobility psi - psi_min)."""

    mesh: Mesh
    r: float
    M: sp.csr_matrix = None
    K: sp.csr_matrix = None
    ref: assembly.Reference = None
    model: int = 2
    psi_min: float = -1.5

    def __post_init__(self):
        self.ref = self.ref or assembly.Reference(self.mesh.dim, degree=self.mesh.degree)
        if self.M is None:
            self.M = assembly.mass_matrix(self.mesh, self.ref)
        if self.K is None:
            self.K = assembly.stiffness_matrix(self.mesh, self.ref)

    @property
    def n(self) -> int:
        return self.mesh.n

    def split(self, x):
        n = self.n
        return x[:n], x[n:2 * n], x[2 * n:]

    # --- Eq. (3.10) -------------------------------------------------------
    def a01(self, psi_k: np.ndarray) -> sp.csr_matrix:
        N = assembly.nonlinear_mass(self.mesh, psi_k, self.ref)
        return (-(1.0 + self.r) * self.M + 2.0 * self.K + N).tocsr()

    def kplus(self, psi: np.ndarray) -> sp.csr_matrix:
        """K_+(psi): K for PFC2, the mobility stiffness of psi - psi_min for PFC1."""
        if self.model == 2:
            return self.K
        return assembly.mobility_stiffness(self.mesh, psi - self.psi_min, self.ref)

    def m0(self, psi: np.ndarray) -> float:
        """Mean mobility <psi^+> = (1^T M psi) / (1^T M 1) - psi_min (PFC1); 1 for PFC2."""
        if self.model == 2:
            return 1.0
        one = np.ones(self.n)
        return float(one @ (self.M @ psi)) / float(one @ (self.M @ one)) - self.psi_min

    def stage_matrix(self, psi_k: np.ndarray, tau: float, coef: Ros3Pw = ROS3PW,
                     mu_k: np.ndarray | None = None) -> sp.csr_matrix:
        M, K = self.M, self.K
        a11 = M / coef.gamma
        if self.model == 1:
            a11 = a11 + tau * assembly.mobility_derivative(self.mesh, mu_k, self.ref)
        return sp.bmat([[M, self.a01(psi_k), K],
                        [tau * self.kplus(psi_k), a11, None],
                        [None, K, M]], format="csr")

    def stage_rhs(self, x_i: np.ndarray, dpsi_prev: list, c_row: list, tau: float) -> np.ndarray:
        """b_i^R of Eq. (3.10) for stage value x_i and previous increments dpsi_j with weights c_ij."""
        M, K, r = self.M, self.K, self.r
        mu, psi, om = self.split(x_i)
        b0 = -(M @ mu) + (1.0 + r) * (M @ psi) - 2.0 * (K @ psi) - K @ om \
            + assembly.load_cubed(self.mesh, psi, self.ref)
        b1 = -tau * (self.kplus(psi) @ mu)
        for cij, dpsi in zip(c_row, dpsi_prev):
            b1 = b1 + cij * (M @ dpsi)
        b2 = -(M @ om) - K @ psi
        return np.concatenate([b0, b1, b2])

    # --- stage solve (Section 4, Section 7) --------------------------------
    def stage_solve(self, A: sp.csr_matrix, b: np.ndarray, tau: float, tol: float = 1e-13,
                    inner: str = "pcg", restart: int = 30, max_outer: int = 2000, coef: Ros3Pw = ROS3PW,
                    m0: float = 1.0, schur: str = "ch", err_tol: float = 0.0):
        """FGMRES with P(S_CH) (or P(S_D), schur="sd"); m0 is the mean mobility of the
        constant-mobility approximation; err_tol > 0 adds the solution-error stop
        (``solvers.fgmres``)."""
        pc = PCH(self.M, self.K, m0 * tau, coef.gamma, inner=inner, schur=schur)
        y, st = fgmres(lambda v: A @ v, b, pc.apply, tol, restart, max_outer, err_tol)
        st.inner = pc.log
        return y, st

    # --- initial state ----------------------------------------------------
    def consistent_state(self, psi0: np.ndarray, tol: float = 1e-14, solver: str = "lu") -> np.ndarray:
        """(mu0, psi0, omega0) with M omega0 = -K psi0 and
        M mu0 = l(psi0^3) + (1+r) M psi0 - 2 K psi0 - K omega0 (Eq. 2.4 in weak form).
        Reading: the paper does not say how mu and omega start; this makes the
        algebraic rows of the DAE hold at t = 0.  solver: "lu" (sparse LU of M) or
        "pcg" (Jacobi-PCG to a relative residual tol; M is well conditioned, so this
        is the cheap route on large meshes)."""
        import scipy.sparse.linalg as spla
        if solver == "lu":
            lu = spla.splu(self.M.tocsc())
            solve = lu.solve
        elif solver == "pcg":
            from .solvers import pcg_jacobi

            def solve(rhs):
                res = pcg_jacobi(self.M, rhs, tol, 10000)
                if not res.converged:
                    raise RuntimeError("consistent_state: PCG with M did not converge")
                return res.x
        else:
            raise ValueError("solver must be 'lu' or 'pcg'")
        om = solve(-(self.K @ psi0))
        rhs = assembly.load_cubed(self.mesh, psi0, self.ref) + (1.0 + self.r) * (self.M @ psi0) \
            - 2.0 * (self.K @ psi0) - self.K @ om
        mu = solve(rhs)
        return np.concatenate([mu, psi0, om])

    # --- diagnostics ------------------------------------------------------
    def mass(self, x: np.ndarray) -> float:
        """Integral of psi: 1^T M psi (conserved by the H^{-1} flow with Neumann BC)."""
        return float(np.ones(self.n) @ (self.M @ self.split(x)[1]))

    def energy(self, x: np.ndarray) -> float:
        """Swift-Hohenberg energy, Eq. (2.1): int 1/4 psi^4 + 1/2 (1+r) psi^2 - |grad psi|^2 + 1/2 (Lap psi)^2,
        with Lap psi represented by omega solving M omega = -K psi."""
        import scipy.sparse.linalg as spla
        psi = self.split(x)[1]
        om = spla.splu(self.M.tocsc()).solve(-(self.K @ psi))
        quart = float(psi @ assembly.load_cubed(self.mesh, psi, self.ref))
        return 0.25 * quart + 0.5 * (1.0 + self.r) * float(psi @ (self.M @ psi)) \
            - float(psi @ (self.K @ psi)) + 0.5 * float(om @ (self.M @ om))


@dataclass
class StepControl:
    atol: float = 1e-3
    rtol: float = 1e-3
    fac_min: float = 0.2
    fac_max: float = 5.0
    safety: float = 0.9
    tau_max: float = 1e9


def step_error(psi_k: np.ndarray, psi_new: np.ndarray, e_psi: np.ndarray, ctl: StepControl) -> float:
    sc = ctl.atol + ctl.rtol * np.maximum(np.abs(psi_k), np.abs(psi_new))
    return math.sqrt(float(np.mean((e_psi / sc) ** 2)))


def next_tau(tau: float, err: float, ctl: StepControl) -> float:
    fac = ctl.fac_max if err == 0.0 else min(ctl.fac_max, max(ctl.fac_min, ctl.safety * err ** (-1.0 / 3.0)))
    return min(tau * fac, ctl.tau_max)


@dataclass
class StepResult:
    x_new: np.ndarray
    accepted: bool
    err: float
    tau_next: float
    ys: list
    rhs: list
    stats: list = field(default_factory=list)


def pfc_step(prob: PFCProblem, x_k: np.ndarray, tau: float, ctl: StepControl = StepControl(),
             tol: float = 1e-13, inner: str = "pcg", coef: Ros3Pw = ROS3PW,
             prev_rejected: bool = False, err_tol: float = 0.0) -> StepResult:
    """One attempted Ros3Pw step (Eq. 3.6, 3.7, 3.10) with the error estimate.

    The matrix N(psi) is frozen at psi^k for all three stages (W-method).
    ``prev_rejected``: the previous attempt was rejected (no growth after it)."""
    n = prob.n
    mu_k, psi_k, _ = prob.split(x_k)
    A = prob.stage_matrix(psi_k, tau, coef, mu_k=mu_k)
    m0 = prob.m0(psi_k)
    ys, rhs, stats = [], [], []
    for i in range(3):
        x_i = x_k + sum(coef.a(i, j) * ys[j] for j in range(i))
        b = prob.stage_rhs(x_i, [y[n:2 * n] for y in ys], [coef.c(i, j) for j in range(i)], tau)
        y, st = prob.stage_solve(A, b, tau, tol=tol, inner=inner, coef=coef, m0=m0, err_tol=err_tol)
        ys.append(y)
        rhs.append(b)
        stats.append(st)
    x_new = x_k + sum(coef.m[j] * ys[j] for j in range(3))
    e = sum((coef.mhat[j] - coef.m[j]) * ys[j] for j in range(3))
    err = step_error(psi_k, x_new[n:2 * n], e[n:2 * n], ctl)
    accepted = err <= 1.0
    tau_next = next_tau(tau, err, ctl)
    if accepted and prev_rejected:
        tau_next = min(tau_next, tau)
    return StepResult(x_new if accepted else x_k.copy(), accepted, err, tau_next, ys, rhs, stats)


# --- linearised semi-implicit Euler (Section 3, Eq. 3.3-3.4) -----------------------
def euler_matrix(prob: PFCProblem, psi_k: np.ndarray, tau: float) -> sp.csr_matrix:
    """A of the linearised semi-implicit Euler step (Eq. 3.4):
    [[M, -(1+r) M + N(psi_k) + 2 K, K], [tau K_+(psi_k), M, 0], [0, K, M]]
    (K_+ = K for PFC2; the mobility is taken at psi_k, as in Eq. 3.3)."""
    M, K = prob.M, prob.K
    return sp.bmat([[M, prob.a01(psi_k), K], [tau * prob.kplus(psi_k), M, None], [None, K, M]], format="csr")


def euler_rhs(prob: PFCProblem, psi_k: np.ndarray) -> np.ndarray:
    """b0 = (-2 psi_k^3, phi), b1 = M psi_k, b2 = 0."""
    n = prob.n
    return np.concatenate([-2.0 * assembly.load_cubed(prob.mesh, psi_k, prob.ref), prob.M @ psi_k, np.zeros(n)])


def euler_step(prob: PFCProblem, x_k: np.ndarray, tau: float, tol: float = 1e-13, inner: str = "pcg",
               restart: int = 30, max_outer: int = 2000, schur: str = "ch", err_tol: float = 0.0):
    """x_{k+1} = A^{-1} b by FGMRES(restart) with P_CH built for gamma = 1 (Section 4)."""
    psi_k = prob.split(x_k)[1]
    A = euler_matrix(prob, psi_k, tau)
    b = euler_rhs(prob, psi_k)
    pc = PCH(prob.M, prob.K, prob.m0(psi_k) * tau, 1.0, inner=inner, schur=schur)
    x, st = fgmres(lambda v: A @ v, b, pc.apply, tol, restart, max_outer, err_tol)
    st.inner = pc.log
    return x, st
