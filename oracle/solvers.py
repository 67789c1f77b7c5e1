"""Krylov solvers and the block preconditioner P_CH.

TEST INFRASTRUCTURE (see ``oracle/__init__``).

* ``pcg_jacobi``  - conjugate gradients with the diagonal (Jacobi) preconditioner,
  the inner solver of every preconditioner step (Section 7, Table 2: "PCG",
  preconditioner "diag", relative tolerance 1e-3).  Reading: zero start,
  stop when the unpreconditioned residual satisfies ||r||_2 <= rtol ||b||_2.
* ``fgmres``      - flexible GMRES with right preconditioning (Section 4: the
  system A P^{-1} (P x) = b; Saad 1993), restart 30 and modified Gram-Schmidt
  (Section 7).  Reading: zero initial guess; Givens rotations on the Hessenberg
  matrix; after each cycle the true residual b - A x is recomputed and the
  solve stops once ||b - A x||_2 <= tol ||b||_2 (and, with err_tol > 0, once
  the solution-error estimate below is at most err_tol).
* ``PCH``         - the block preconditioner of Eq. (4.1) with the Cahn-Hilliard
  approximation S_CH of the Schur complement (Section 4.2), applied in the
  steps (1), (2), (3.1), (3.2), (4), (5); or, with ``schur="sd"``, with the
  diagonal approximation S_D = M - 2 delta K + delta K M_D^{-1} K, M_D = diag(M)
  (Section 4.1), whose step (3) S_D x1 = M y1 runs a fixed number of Jacobi-PCG
  iterations (Table 2: 20).

Reading of the outer stopping rule (the paper gives no outer tolerance): the
stage solution is needed to a relative error, not a relative residual, and the
ratio of the two grows with tau (the stage matrix nears singularity as
gamma tau approaches the critical width of Lemma 3).  With right
preconditioning the error of an iterate x is e = A^{-1} r = P^{-1} (A P^{-1})^{-1} r,
so ``fgmres(err_tol=...)`` estimates

    E = ||P^{-1} r||_2 / (||x||_2 sigma),   sigma = min over the cycles so far of
                                            the smallest singular value of the
                                            cycle's Hessenberg matrix H_k,

(H_k represents A P^{-1} on the cycle's Krylov space, so 1 / sigma estimates
||(A P^{-1})^{-1}||) and, once the residual test passes, stops only if
E <= err_tol; otherwise it tightens the residual target to
(||r|| / ||b||) (err_tol / E) / 2 and runs another cycle, whose first
preconditioned vector is the P^{-1} r just computed.

Readings of garbled or silent passages (each applies to ``PCH.apply``):

* Step (2) prints ``b_1 - tau K y_1`` on its right-hand side; the forward
  substitution with the lower factor of Eq. (4.1) needs ``b_1 - tau K y_0``,
  which is what is used.
* The preconditioner is derived for gamma = 1 (Section 4).  In a Rosenbrock
  stage the (psi, psi) block is M/gamma, so the second block row is scaled by
  gamma: P is built with tau_e = gamma * tau, delta = sqrt(tau_e), and applied to
  (v0, gamma * v1, v2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


@dataclass
class PCGResult:
    x: np.ndarray
    iterations: int
    converged: bool


def pcg_jacobi(A: sp.csr_matrix, b: np.ndarray, rtol: float, maxit: int) -> PCGResult:
    """Jacobi-preconditioned CG for SPD A from x0 = 0.  rtol = 0 runs maxit iterations.
    Reading: if p^T A p <= 0 (A not positive definite along p) the iteration stops
    and returns the current iterate."""
    dinv = 1.0 / A.diagonal()
    x = np.zeros_like(b)
    bnorm = math.sqrt(float(b @ b))
    if bnorm == 0.0:
        return PCGResult(x, 0, True)
    r = b.copy()
    z = dinv * r
    p = z.copy()
    rz = float(r @ z)
    for it in range(1, maxit + 1):
        q = A @ p
        pq = float(p @ q)
        if not pq > 0.0:
            return PCGResult(x, it - 1, False)
        alpha = rz / pq
        x += alpha * p
        r -= alpha * q
        if math.sqrt(float(r @ r)) <= rtol * bnorm:
            return PCGResult(x, it, True)
        z = dinv * r
        rz_new = float(r @ z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return PCGResult(x, maxit, False)


@dataclass
class FGMRESStats:
    outer_iterations: int = 0
    restarts: int = 0
    rel_residual: float = float("nan")
    converged: bool = False
    err_estimate: float = float("nan")   # E of the last solution-error test (err_tol > 0)
    sigma: float = float("inf")          # smallest singular value of the cycles' H_k
    history: list = field(default_factory=list)   # Givens residual estimates / ||b||


def fgmres(apply_A, b: np.ndarray, apply_Pinv, tol: float, restart: int = 30,
           max_outer: int = 1000, err_tol: float = 0.0) -> tuple[np.ndarray, FGMRESStats]:
    """Right-preconditioned flexible GMRES(restart) with modified Gram-Schmidt.
    err_tol > 0 adds the solution-error test of the module docstring."""
    st = FGMRESStats()
    x = np.zeros_like(b)
    bnorm = math.sqrt(float(b @ b))
    if bnorm == 0.0:
        st.rel_residual, st.converged = 0.0, True
        return x, st
    tol_r = tol
    z_first = None                            # P^{-1} v_0 of the next cycle, when already computed
    while True:
        r = b - apply_A(x)
        beta = math.sqrt(float(r @ r))
        st.rel_residual = beta / bnorm
        if beta <= tol_r * bnorm:
            if err_tol <= 0.0 or beta == 0.0:
                st.converged = True
                return x, st
            if st.outer_iterations < max_outer:
                z_first = apply_Pinv(r / beta)
                xnorm = math.sqrt(float(x @ x))
                st.err_estimate = beta * math.sqrt(float(z_first @ z_first)) / (xnorm * st.sigma)
                if st.err_estimate <= err_tol:
                    st.converged = True
                    return x, st
                tol_r = st.rel_residual * (err_tol / st.err_estimate) * 0.5
        if st.outer_iterations >= max_outer:
            return x, st
        m = restart
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        k = 0
        for j in range(m):
            z = z_first if (j == 0 and z_first is not None) else apply_Pinv(V[j])
            z_first = None
            Z.append(z)
            w = apply_A(z)
            for i in range(j + 1):            # modified Gram-Schmidt
                H[i, j] = float(w @ V[i])
                w = w - H[i, j] * V[i]
            hnext = math.sqrt(float(w @ w))
            H[j + 1, j] = hnext
            for i in range(j):                # previous Givens rotations on column j
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            st.outer_iterations += 1
            k = j + 1
            st.history.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= tol_r * bnorm or hnext == 0.0 or st.outer_iterations >= max_outer:
                break
            V.append(w / hnext)
        # the rotated k x k triangle has the singular values of the cycle's H_k
        st.sigma = min(st.sigma, float(np.linalg.svd(H[:k, :k], compute_uv=False)[-1]))
        y = np.zeros(k)                       # back substitution with the rotated H
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        for i in range(k):
            x = x + y[i] * Z[i]
        st.restarts += 1


@dataclass
class InnerLog:
    calls: int = 0
    iterations: int = 0
    per_call: list = field(default_factory=list)


class PCH:
    """Block preconditioner P(S_CH) (Eq. 4.1, Section 4.2) for one Rosenbrock stage matrix.

    ``inner`` chooses the SPD solves: "pcg" (Jacobi-PCG, rtol 1e-3 by default, as
    in Table 2) or "exact" (sparse direct solves; used by the spectral tests).
    """

    def __init__(self, M, K, tau: float, gamma: float, inner: str = "pcg",
                 inner_rtol: float = 1e-3, max_inner: int = 10000, schur: str = "ch", sd_its: int = 20):
        self.M, self.K = M.tocsr(), K.tocsr()
        self.gamma = gamma
        self.tau_e = gamma * tau
        self.delta = math.sqrt(self.tau_e)
        self.MdK = (self.M + self.delta * self.K).tocsr()            # step (2)
        self.MsK = (self.M + math.sqrt(self.delta) * self.K).tocsr() # steps (3.1), (3.2)
        self.schur, self.sd_its = schur, sd_its
        mats = [self.M, self.MdK, self.MsK]
        if schur == "sd":
            # S_D = M - 2 delta K + delta K M_D^{-1} K, M_D = diag(M)   (Section 4.1)
            md_inv = sp.diags(1.0 / self.M.diagonal())
            self.SD = (self.M - 2.0 * self.delta * self.K + self.delta * (self.K @ md_inv @ self.K)).tocsr()
            mats.append(self.SD)
        elif schur != "ch":
            raise ValueError("schur must be 'ch' or 'sd'")
        self.inner, self.inner_rtol, self.max_inner = inner, inner_rtol, max_inner
        self.log = InnerLog()
        self.n = M.shape[0]
        if inner == "exact":
            import scipy.sparse.linalg as spla
            self._lu = {id(A): spla.splu(A.tocsc()) for A in mats}

    def _solve(self, A, b, fixed_its: int = 0):
        if self.inner == "exact":
            return self._lu[id(A)].solve(b)
        res = pcg_jacobi(A, b, 0.0, fixed_its) if fixed_its else pcg_jacobi(A, b, self.inner_rtol, self.max_inner)
        self.log.calls += 1
        self.log.iterations += res.iterations
        self.log.per_call.append(res.iterations)
        return res.x

    def apply(self, v: np.ndarray) -> np.ndarray:
        n = self.n
        v0, v1, v2 = v[:n], v[n:2 * n], v[2 * n:]
        y0 = self._solve(self.M, v0)                                       # (1)  M y0 = v0
        y1 = self._solve(self.MdK, self.gamma * v1 - self.tau_e * (self.K @ y0))  # (2)
        if self.schur == "sd":
            x1 = self._solve(self.SD, self.M @ y1, self.sd_its)            # (3)  S_D x1 = M y1
        else:
            w = self._solve(self.MsK, self.M @ y1)                         # (3.1)
            x1 = self._solve(self.MsK, self.M @ w)                         # (3.2)
        x0 = y0 + (y1 - x1) / self.delta                                   # (4)
        x2 = self._solve(self.M, v2 - self.K @ x1)                         # (5)
        return np.concatenate([x0, x1, x2])
