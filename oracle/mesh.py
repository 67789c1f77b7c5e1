"""Structured simplicial meshes and the P2 (or P1) degree-of-freedom lattice.

TEST INFRASTRUCTURE (see ``oracle/__init__``).

The paper works on conforming simplicial meshes and uses regular simplicial
meshes of a square/cube in its experiments (Section 3, Section 7).  The meshes
here are:

* 2D: ``side x side`` squares of width h = L/side; square (i, j) is cut along the
  diagonal from vertex (i, j) to (i+1, j+1) into the triangles
  (v_ij, v_i+1,j, v_i+1,j+1) and (v_ij, v_i,j+1, v_i+1,j+1).
* 3D: ``side^3`` cubes; each cube is cut into the 6 Kuhn tetrahedra, one per
  permutation pi of the axes, with vertices v0 = corner, v_{k+1} = v_k + e_{pi_k}.

The P2 dofs are the points of the half-spacing lattice, (2 side + 1)^dim of them,
numbered lexicographically with x fastest.  Vertex (i, j[, k]) is lattice point
(2i, 2j[, 2k]) and the node of edge (a, b) is the lattice midpoint of its ends.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np

from .p2 import EDGES


@dataclass
class Mesh:
    dim: int
    side: int
    length: float
    n: int                 # P2 dofs per field
    coords: np.ndarray     # [n, dim] dof coordinates
    elem_dofs: np.ndarray  # [E, nloc] global P2 dof index per local node
    elem_verts: np.ndarray # [E, dim+1, dim] vertex coordinates
    degree: int = 2        # 2: P2 dofs (half-spacing lattice); 1: P1 dofs (the vertices)

    @property
    def h(self) -> float:
        return self.length / self.side


def _vertex_paths(dim: int) -> list[np.ndarray]:
    """Vertex offsets (in cell units) of the simplices of one cell, path ordered."""
    if dim == 2:
        return [np.array([[0, 0], [1, 0], [1, 1]]), np.array([[0, 0], [0, 1], [1, 1]])]
    paths = []
    for perm in itertools.permutations(range(3)):
        v = np.zeros((4, 3), dtype=np.int64)
        for k, ax in enumerate(perm):
            v[k + 1] = v[k]
            v[k + 1, ax] += 1
        paths.append(v)
    return paths


def structured_mesh(dim: int, side: int, length: float, degree: int = 2) -> Mesh:
    """P2 dofs on the half-spacing lattice (degree 2) or P1 dofs on the vertices (degree 1)."""
    m = degree * side + 1
    n = m ** dim
    h = length / side
    cells = np.stack(np.meshgrid(*[np.arange(side)] * dim, indexing="ij"), axis=-1).reshape(-1, dim)
    # order cells with x fastest to match the dof numbering convention
    cells = cells[np.lexsort(tuple(cells[:, k] for k in range(dim)))]
    elem_lat = []
    for path in _vertex_paths(dim):
        vl = degree * (cells[:, None, :] + path[None, :, :])     # [C, d+1, d] lattice coords
        if degree == 2:
            mids = [(vl[:, a, :] + vl[:, b, :]) // 2 for a, b in EDGES[dim]]
            elem_lat.append(np.concatenate([vl, np.stack(mids, axis=1)], axis=1))
        else:
            elem_lat.append(vl)
    lat = np.concatenate(elem_lat, axis=0)                        # [E, nloc, d]
    stride = m ** np.arange(dim)
    elem_dofs = (lat * stride).sum(axis=-1)
    elem_verts = lat[:, : dim + 1, :].astype(np.float64) * (h / degree)
    grid = np.stack(np.meshgrid(*[np.arange(m)] * dim, indexing="ij"), axis=-1).reshape(-1, dim)
    idx = (grid * stride).sum(axis=-1)
    coords = np.empty((n, dim))
    coords[idx] = grid * (h / degree)
    return Mesh(dim, side, float(length), n, coords, elem_dofs.astype(np.int64), elem_verts, degree)
