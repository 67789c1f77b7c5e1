"""Finite element assembly of the PFC matrices and load vectors.

TEST INFRASTRUCTURE (see ``oracle/__init__``).

Definitions (Section 3, the block matrices below Eq. 3.4):

* mass          M_ij = (phi_j, phi_i)
* stiffness     K_ij = (grad phi_j, grad phi_i)
* nonlinear mass N(psi)_ij = (-3 psi^2 phi_j, phi_i)
* load vector   l(u)_i = (u, phi_i), used with u = psi^3 in the stage right-hand side.

PFC1 (mobility psi^+ = psi - psi_min, Eq. 2.3 and the matrices of Eq. 3.10):

* mobility stiffness  K_+(psi)_ij = (psi^+ grad phi_j, grad phi_i)
* mobility derivative F(mu)_ij   = (phi_j grad mu, grad phi_i)
* mobility load       k(psi, mu)_i = (psi^+ grad mu, grad phi_i) = (K_+(psi) mu)_i, assembled
  directly (one integrand, no matrix) so that tests can pin K_+ and F against it.

Each element integral is evaluated with the collapsed Gauss rule of
``quadrature.simplex_rule`` after the affine map x = X0 + J xi; gradients follow
the chain rule grad_x = J^{-T} grad_xi.  The default rule has 5 points per
direction, exact to degree 9 (the N and l(psi^3) integrands have degree 8 for P2).
Global matrices are summed from element contributions (COO -> CSR).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import p2
from .mesh import Mesh
from .quadrature import simplex_rule

DEFAULT_POINTS = 5
_CHUNK = 1 << 16


class Reference:
    """Basis values/gradients of the P2 (or P1) element at the quadrature points of one rule."""

    def __init__(self, dim: int, npts: int = DEFAULT_POINTS, degree: int = 2):
        self.xi, self.w = simplex_rule(dim, npts)
        self.degree = degree
        basis = p2.basis if degree == 2 else p2.basis_p1
        self.phi, self.dphi = basis(self.xi)   # [Q, nl], [Q, nl, d]


def _geometry(verts: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """|det J| [E] and J^{-1} [E, d, d] for element vertex coordinates [E, d+1, d]."""
    jac = np.transpose(verts[:, 1:, :] - verts[:, :1, :], (0, 2, 1))   # columns = edge vectors
    det = np.linalg.det(jac)
    inv = np.linalg.inv(jac)
    return np.abs(det), inv


def _to_csr(mesh: Mesh, emats_iter) -> sp.csr_matrix:
    n = mesh.n
    total = None
    for dofs, emat in emats_iter:
        nl = dofs.shape[1]
        rows = np.repeat(dofs, nl, axis=1).ravel()
        cols = np.tile(dofs, (1, nl)).ravel()
        part = sp.coo_matrix((emat.ravel(), (rows, cols)), shape=(n, n)).tocsr()
        total = part if total is None else total + part
    total.sum_duplicates()
    total.sort_indices()
    return total


def element_mass(mesh: Mesh, ref: Reference, sl=slice(None)) -> np.ndarray:
    det, _ = _geometry(mesh.elem_verts[sl])
    return np.einsum("e,q,qa,qb->eab", det, ref.w, ref.phi, ref.phi, optimize=True)


def element_stiffness(mesh: Mesh, ref: Reference, sl=slice(None)) -> np.ndarray:
    det, inv = _geometry(mesh.elem_verts[sl])
    # physical gradients: grad_x phi_a = J^{-T} grad_xi phi_a  ->  [E, Q, nl, d]
    gx = np.einsum("eji,qaj->eqai", inv, ref.dphi, optimize=True)
    return np.einsum("e,q,eqai,eqbi->eab", det, ref.w, gx, gx, optimize=True)


def element_nonlinear_mass(mesh: Mesh, ref: Reference, psi: np.ndarray, sl=slice(None)) -> np.ndarray:
    det, _ = _geometry(mesh.elem_verts[sl])
    psi_q = psi[mesh.elem_dofs[sl]] @ ref.phi.T                 # [E, Q]
    coef = -3.0 * psi_q ** 2
    return np.einsum("e,q,eq,qa,qb->eab", det, ref.w, coef, ref.phi, ref.phi, optimize=True)


def element_mobility_stiffness(mesh: Mesh, ref: Reference, coef: np.ndarray, sl=slice(None)) -> np.ndarray:
    """(c grad phi_b, grad phi_a) for c the P2 function with coefficients coef."""
    det, inv = _geometry(mesh.elem_verts[sl])
    gx = np.einsum("eji,qaj->eqai", inv, ref.dphi, optimize=True)
    c_q = coef[mesh.elem_dofs[sl]] @ ref.phi.T                   # [E, Q]
    return np.einsum("e,q,eq,eqai,eqbi->eab", det, ref.w, c_q, gx, gx, optimize=True)


def element_mobility_derivative(mesh: Mesh, ref: Reference, mu: np.ndarray, sl=slice(None)) -> np.ndarray:
    """Row a, column b: (phi_b grad mu, grad phi_a)."""
    det, inv = _geometry(mesh.elem_verts[sl])
    gx = np.einsum("eji,qaj->eqai", inv, ref.dphi, optimize=True)   # [E, Q, nl, d]
    gmu = np.einsum("ea,eqai->eqi", mu[mesh.elem_dofs[sl]], gx, optimize=True)
    return np.einsum("e,q,eqi,eqai,qb->eab", det, ref.w, gmu, gx, ref.phi, optimize=True)


def _chunks(mesh: Mesh):
    e = mesh.elem_dofs.shape[0]
    for s in range(0, e, _CHUNK):
        yield slice(s, min(s + _CHUNK, e))


def mass_matrix(mesh: Mesh, ref: Reference | None = None) -> sp.csr_matrix:
    ref = ref or Reference(mesh.dim, degree=mesh.degree)
    return _to_csr(mesh, ((mesh.elem_dofs[s], element_mass(mesh, ref, s)) for s in _chunks(mesh)))


def stiffness_matrix(mesh: Mesh, ref: Reference | None = None) -> sp.csr_matrix:
    ref = ref or Reference(mesh.dim, degree=mesh.degree)
    return _to_csr(mesh, ((mesh.elem_dofs[s], element_stiffness(mesh, ref, s)) for s in _chunks(mesh)))


def nonlinear_mass(mesh: Mesh, psi: np.ndarray, ref: Reference | None = None) -> sp.csr_matrix:
    """N(psi) = ((-3 psi^2 phi_j, phi_i)) for psi given by its P2 coefficients."""
    ref = ref or Reference(mesh.dim, degree=mesh.degree)
    return _to_csr(
        mesh, ((mesh.elem_dofs[s], element_nonlinear_mass(mesh, ref, psi, s)) for s in _chunks(mesh))
    )


def load_cubed(mesh: Mesh, psi: np.ndarray, ref: Reference | None = None) -> np.ndarray:
    """l(psi^3)_i = (psi_h^3, phi_i), psi_h the P2 function with coefficients psi."""
    ref = ref or Reference(mesh.dim, degree=mesh.degree)
    out = np.zeros(mesh.n)
    for s in _chunks(mesh):
        det, _ = _geometry(mesh.elem_verts[s])
        psi_q = psi[mesh.elem_dofs[s]] @ ref.phi.T
        le = np.einsum("e,q,eq,qa->ea", det, ref.w, psi_q ** 3, ref.phi, optimize=True)
        np.add.at(out, mesh.elem_dofs[s].ravel(), le.ravel())
    return out


def mobility_stiffness(mesh: Mesh, psi_plus: np.ndarray, ref: Reference | None = None) -> sp.csr_matrix:
    """K_+(psi) = ((psi^+ grad phi_j, grad phi_i)) for psi^+ given by its P2 coefficients."""
    ref = ref or Reference(mesh.dim, degree=mesh.degree)
    return _to_csr(mesh, ((mesh.elem_dofs[s], element_mobility_stiffness(mesh, ref, psi_plus, s))
                          for s in _chunks(mesh)))


def mobility_derivative(mesh: Mesh, mu: np.ndarray, ref: Reference | None = None) -> sp.csr_matrix:
    """F(mu) = ((phi_j grad mu, grad phi_i)): the derivative of K_+(psi) mu in psi."""
    ref = ref or Reference(mesh.dim, degree=mesh.degree)
    return _to_csr(mesh, ((mesh.elem_dofs[s], element_mobility_derivative(mesh, ref, mu, s))
                          for s in _chunks(mesh)))


def mobility_load(mesh: Mesh, psi_plus: np.ndarray, mu: np.ndarray, ref: Reference | None = None) -> np.ndarray:
    """k_i = (psi^+ grad mu, grad phi_i), integrated directly."""
    ref = ref or Reference(mesh.dim, degree=mesh.degree)
    out = np.zeros(mesh.n)
    for s in _chunks(mesh):
        det, inv = _geometry(mesh.elem_verts[s])
        gx = np.einsum("eji,qaj->eqai", inv, ref.dphi, optimize=True)
        gmu = np.einsum("ea,eqai->eqi", mu[mesh.elem_dofs[s]], gx, optimize=True)
        c_q = psi_plus[mesh.elem_dofs[s]] @ ref.phi.T
        le = np.einsum("e,q,eq,eqi,eqai->ea", det, ref.w, c_q, gmu, gx, optimize=True)
        np.add.at(out, mesh.elem_dofs[s].ravel(), le.ravel())
    return out


def pattern_nnz(mesh: Mesh) -> int:
    """Nonzeros of one P2-P2 block (all blocks share this pattern)."""
    ones = (np.ones((d.shape[0], d.shape[1], d.shape[1])) for d in [mesh.elem_dofs])
    return _to_csr(mesh, zip([mesh.elem_dofs], ones)).nnz
