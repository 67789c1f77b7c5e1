"""Gauss-Jacobi quadrature and collapsed (conical-product) rules on simplices.

TEST INFRASTRUCTURE (see ``oracle/__init__``).

The paper integrates the P2 forms of Section 3 exactly; the nonlinear mass
N(psi) = ((-3 psi^2 phi_j, phi_i)) and the load (psi^3, phi_i) have polynomial
integrands of degree 8 on each affine element.  Any rule exact to that degree
gives the same matrices up to rounding.  This module builds one such family from
first principles:

* 1-D Gauss-Jacobi nodes/weights by the Golub-Welsch eigenvalue method
  (G. H. Golub, J. H. Welsch, Math. Comp. 23 (1969)) from the three-term
  recurrence of the monic Jacobi polynomials.
* Simplex rules by the Duffy collapse: the unit square (cube) maps onto the
  reference triangle (tetrahedron) and the Jacobian factor is absorbed into the
  Jacobi weights of the collapsed directions.
"""
from __future__ import annotations

import math

import numpy as np


def gauss_jacobi(npts: int, alpha: float, beta: float) -> tuple[np.ndarray, np.ndarray]:
    """Nodes/weights on [-1, 1] for the weight (1-x)^alpha (1+x)^beta; exact to degree 2n-1."""
    a, b = float(alpha), float(beta)
    # diagonal of the Jacobi matrix
    diag = np.empty(npts)
    for i in range(npts):
        s = 2 * i + a + b
        if i == 0:
            diag[i] = (b - a) / (a + b + 2.0)
        else:
            diag[i] = (b * b - a * a) / (s * (s + 2.0))
    # off-diagonal (square root of the recurrence coefficients b_n, n >= 1)
    off = np.empty(max(npts - 1, 0))
    for i in range(1, npts):
        s = 2 * i + a + b
        num = 4.0 * i * (i + a) * (i + b) * (i + a + b)
        den = s * s * (s + 1.0) * (s - 1.0)
        off[i - 1] = math.sqrt(num / den)
    jac = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    nodes, vecs = np.linalg.eigh(jac)
    mu0 = 2.0 ** (a + b + 1.0) * math.gamma(a + 1.0) * math.gamma(b + 1.0) / math.gamma(a + b + 2.0)
    weights = mu0 * vecs[0, :] ** 2
    return nodes, weights


def simplex_rule(dim: int, npts: int) -> tuple[np.ndarray, np.ndarray]:
    """Collapsed Gauss rule on the reference simplex {xi_k >= 0, sum xi_k <= 1}.

    Returns (points [Q, dim], weights [Q]); exact for polynomials of total degree
    <= 2*npts - 1.  Weights sum to the simplex volume 1/dim!.
    """
    if dim == 2:
        xu, wu = gauss_jacobi(npts, 1.0, 0.0)   # collapsed direction: factor (1-u)
        xv, wv = gauss_jacobi(npts, 0.0, 0.0)
        u = (xu + 1.0) / 2.0
        v = (xv + 1.0) / 2.0
        wu = wu / 4.0                          # (1-u) = (1-x)/2, du = dx/2
        wv = wv / 2.0
        U, V = np.meshgrid(u, v, indexing="ij")
        W = np.outer(wu, wv)
        pts = np.stack([U.ravel(), ((1.0 - U) * V).ravel()], axis=1)
        return pts, W.ravel()
    if dim == 3:
        xu, wu = gauss_jacobi(npts, 2.0, 0.0)   # factor (1-u)^2
        xv, wv = gauss_jacobi(npts, 1.0, 0.0)   # factor (1-v)
        xw, ww = gauss_jacobi(npts, 0.0, 0.0)
        u = (xu + 1.0) / 2.0
        v = (xv + 1.0) / 2.0
        w = (xw + 1.0) / 2.0
        wu = wu / 8.0
        wv = wv / 4.0
        ww = ww / 2.0
        U, V, Wc = np.meshgrid(u, v, w, indexing="ij")
        pts = np.stack(
            [U.ravel(), ((1.0 - U) * V).ravel(), ((1.0 - U) * (1.0 - V) * Wc).ravel()], axis=1
        )
        weights = (wu[:, None, None] * wv[None, :, None] * ww[None, None, :]).ravel()
        return pts, weights
    raise ValueError("dim must be 2 or 3")
