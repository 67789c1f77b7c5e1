"""P2 (and P1) Lagrange bases on the reference simplex.

TEST INFRASTRUCTURE (see ``oracle/__init__``).

The paper's finite element space V_h uses piecewise polynomials of degree p = 2
on simplices (Section 3).  In barycentric coordinates lambda_0..lambda_d the
Lagrange basis of degree 2 is lambda_k (2 lambda_k - 1) at the vertices and
4 lambda_a lambda_b at the edge midpoints.  Reference coordinates xi give
lambda_k = xi_k (k >= 1) and lambda_0 = 1 - sum(xi).

Local numbering: vertices 0..d first, then the edges in ``EDGES[dim]`` order.
The P1 basis (p = 1, also used in the paper's experiments) is lambda_k at the vertices.
"""
from __future__ import annotations

import numpy as np

EDGES = {
    2: [(0, 1), (1, 2), (0, 2)],
    3: [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)],
}


def nloc(dim: int) -> int:
    return (dim + 1) * (dim + 2) // 2


def barycentric(xi: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """lambda [Q, d+1] at reference points xi [Q, d] and their constant xi-gradients [d+1, d]."""
    q, d = xi.shape
    lam = np.empty((q, d + 1))
    lam[:, 0] = 1.0 - xi.sum(axis=1)
    lam[:, 1:] = xi
    glam = np.zeros((d + 1, d))
    glam[0, :] = -1.0
    glam[1:, :] = np.eye(d)
    return lam, glam


def basis(xi: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Values [Q, nloc] and reference gradients [Q, nloc, d] of the P2 basis at points xi."""
    q, d = xi.shape
    lam, glam = barycentric(xi)
    nb = nloc(d)
    val = np.empty((q, nb))
    grad = np.empty((q, nb, d))
    for k in range(d + 1):
        val[:, k] = lam[:, k] * (2.0 * lam[:, k] - 1.0)
        grad[:, k, :] = (4.0 * lam[:, k] - 1.0)[:, None] * glam[k][None, :]
    for e, (a, b) in enumerate(EDGES[d]):
        val[:, d + 1 + e] = 4.0 * lam[:, a] * lam[:, b]
        grad[:, d + 1 + e, :] = 4.0 * (lam[:, b][:, None] * glam[a][None, :] + lam[:, a][:, None] * glam[b][None, :])
    return val, grad


def basis_p1(xi: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Values [Q, d+1] and reference gradients [Q, d+1, d] of the P1 basis at points xi."""
    q, d = xi.shape
    lam, glam = barycentric(xi)
    return lam, np.broadcast_to(glam[None, :, :], (q, d + 1, d)).copy()


def nodes(dim: int) -> np.ndarray:
    """Reference coordinates [nloc, d] of the P2 nodes in local order."""
    verts = np.zeros((dim + 1, dim))
    verts[1:, :] = np.eye(dim)
    mids = [0.5 * (verts[a] + verts[b]) for a, b in EDGES[dim]]
    return np.vstack([verts, np.array(mids)])
