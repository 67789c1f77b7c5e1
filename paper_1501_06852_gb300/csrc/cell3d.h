// Interior stencil of the 3D P2 inner operators in the cell-major row order.
//
// Cell-major order (3D, P2, structured stencils): the half-spacing lattice points
// (x, y, z), 0 <= x, y, z <= 2 side, are grouped into the 2 x 2 x 2 cells
// (cx, cy, cz) = (x / 2, y / 2, z / 2), cx, cy, cz = 0 .. side, numbered
// (cz (side + 1) + cy)(side + 1) + cx; the eight rows of cell c are 8c + sub,
// sub = (x & 1) + 2 (y & 1) + 4 (z & 1) (the dof type of the row).  Points with a
// coordinate 2 side + 1 hold no dof (padding rows).  Two float4 loads of a vector at
// cell c read the eight dofs of one lattice cell (sub 0..3, then 4..7).
//
// On the Kuhn triangulation of the structured mesh (each cube cut into the six
// tetrahedra along its main diagonal, one per ordering of the axes), a P2 dof couples
// to the dofs of the tetrahedra that contain it: the vertex row to 65 lattice points,
// the edge rows to 27 or 19.  Two points of a tetrahedron differ by a vector whose
// components never have opposite signs, so every coupling of a cell's rows falls in
// one of the fifteen cells offset by (dx, dy, dz) in {0, 1}^3 or {-1, 0}^3:
// PFC_CELL3D_DX/DY/DZ below, own cell at index 7.  PFC_CELL3D_ENTRIES lists the 230
// couplings of an interior cell grouped by source cell: L(q) starts the couplings read
// from source cell q, X(t, q, sub) is output row type t reading row sub of cell q.  The
// host checks at set-up that the interior stencils it extracted from the assembled
// pattern are exactly these couplings (and disables the cell kernels otherwise).
#pragma once

namespace pfc {

constexpr int kCell3dEntries = 230;
constexpr int kCell3dSrc = 15;

#define PFC_CELL3D_DX {-1, 0, -1, 0, -1, 0, -1, 0, 1, 0, 1, 0, 1, 0, 1}
#define PFC_CELL3D_DY {-1, -1, 0, 0, -1, -1, 0, 0, 0, 1, 1, 0, 0, 1, 1}
#define PFC_CELL3D_DZ {-1, -1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1}

// clang-format off
#define PFC_CELL3D_ENTRIES(X, L) \
  L(0) \
  X(0, 0, 0) X(0, 0, 1) X(0, 0, 2) X(0, 0, 3) X(0, 0, 4) X(0, 0, 5) \
  X(0, 0, 6) X(0, 0, 7) \
  L(1) \
  X(0, 1, 0) X(0, 1, 2) X(0, 1, 4) X(0, 1, 6) X(0, 1, 7) X(1, 1, 0) \
  X(1, 1, 2) X(1, 1, 4) X(1, 1, 6) X(1, 1, 7) \
  L(2) \
  X(0, 2, 0) X(0, 2, 1) X(0, 2, 4) X(0, 2, 5) X(0, 2, 7) X(2, 2, 0) \
  X(2, 2, 1) X(2, 2, 4) X(2, 2, 5) X(2, 2, 7) \
  L(3) \
  X(0, 3, 0) X(0, 3, 4) X(0, 3, 5) X(0, 3, 6) X(0, 3, 7) X(1, 3, 0) \
  X(1, 3, 4) X(1, 3, 5) X(1, 3, 7) X(2, 3, 0) X(2, 3, 4) X(2, 3, 6) \
  X(2, 3, 7) X(3, 3, 0) X(3, 3, 4) X(3, 3, 5) X(3, 3, 6) X(3, 3, 7) \
  L(4) \
  X(0, 4, 0) X(0, 4, 1) X(0, 4, 2) X(0, 4, 3) X(0, 4, 7) X(4, 4, 0) \
  X(4, 4, 1) X(4, 4, 2) X(4, 4, 3) X(4, 4, 7) \
  L(5) \
  X(0, 5, 0) X(0, 5, 2) X(0, 5, 3) X(0, 5, 6) X(0, 5, 7) X(1, 5, 0) \
  X(1, 5, 2) X(1, 5, 3) X(1, 5, 7) X(4, 5, 0) X(4, 5, 2) X(4, 5, 6) \
  X(4, 5, 7) X(5, 5, 0) X(5, 5, 2) X(5, 5, 3) X(5, 5, 6) X(5, 5, 7) \
  L(6) \
  X(0, 6, 0) X(0, 6, 1) X(0, 6, 3) X(0, 6, 5) X(0, 6, 7) X(2, 6, 0) \
  X(2, 6, 1) X(2, 6, 3) X(2, 6, 7) X(4, 6, 0) X(4, 6, 1) X(4, 6, 5) \
  X(4, 6, 7) X(6, 6, 0) X(6, 6, 1) X(6, 6, 3) X(6, 6, 5) X(6, 6, 7) \
  L(7) \
  X(0, 7, 0) X(0, 7, 1) X(0, 7, 2) X(0, 7, 3) X(0, 7, 4) X(0, 7, 5) \
  X(0, 7, 6) X(0, 7, 7) X(1, 7, 0) X(1, 7, 1) X(1, 7, 3) X(1, 7, 5) \
  X(1, 7, 7) X(2, 7, 0) X(2, 7, 2) X(2, 7, 3) X(2, 7, 6) X(2, 7, 7) \
  X(3, 7, 0) X(3, 7, 1) X(3, 7, 2) X(3, 7, 3) X(3, 7, 7) X(4, 7, 0) \
  X(4, 7, 4) X(4, 7, 5) X(4, 7, 6) X(4, 7, 7) X(5, 7, 0) X(5, 7, 1) \
  X(5, 7, 4) X(5, 7, 5) X(5, 7, 7) X(6, 7, 0) X(6, 7, 2) X(6, 7, 4) \
  X(6, 7, 6) X(6, 7, 7) X(7, 7, 0) X(7, 7, 1) X(7, 7, 2) X(7, 7, 3) \
  X(7, 7, 4) X(7, 7, 5) X(7, 7, 6) X(7, 7, 7) \
  L(8) \
  X(0, 8, 0) X(0, 8, 2) X(0, 8, 4) X(0, 8, 6) X(1, 8, 0) X(1, 8, 2) \
  X(1, 8, 4) X(1, 8, 6) X(3, 8, 0) X(3, 8, 2) X(3, 8, 6) X(5, 8, 0) \
  X(5, 8, 4) X(5, 8, 6) X(7, 8, 0) X(7, 8, 2) X(7, 8, 4) X(7, 8, 6) \
  L(9) \
  X(0, 9, 0) X(0, 9, 1) X(0, 9, 4) X(0, 9, 5) X(2, 9, 0) X(2, 9, 1) \
  X(2, 9, 4) X(2, 9, 5) X(3, 9, 0) X(3, 9, 1) X(3, 9, 5) X(6, 9, 0) \
  X(6, 9, 4) X(6, 9, 5) X(7, 9, 0) X(7, 9, 1) X(7, 9, 4) X(7, 9, 5) \
  L(10) \
  X(0, 10, 0) X(0, 10, 4) X(1, 10, 0) X(1, 10, 4) X(2, 10, 0) X(2, 10, 4) \
  X(3, 10, 0) X(3, 10, 4) X(7, 10, 0) X(7, 10, 4) \
  L(11) \
  X(0, 11, 0) X(0, 11, 1) X(0, 11, 2) X(0, 11, 3) X(4, 11, 0) X(4, 11, 1) \
  X(4, 11, 2) X(4, 11, 3) X(5, 11, 0) X(5, 11, 1) X(5, 11, 3) X(6, 11, 0) \
  X(6, 11, 2) X(6, 11, 3) X(7, 11, 0) X(7, 11, 1) X(7, 11, 2) X(7, 11, 3) \
  L(12) \
  X(0, 12, 0) X(0, 12, 2) X(1, 12, 0) X(1, 12, 2) X(4, 12, 0) X(4, 12, 2) \
  X(5, 12, 0) X(5, 12, 2) X(7, 12, 0) X(7, 12, 2) \
  L(13) \
  X(0, 13, 0) X(0, 13, 1) X(2, 13, 0) X(2, 13, 1) X(4, 13, 0) X(4, 13, 1) \
  X(6, 13, 0) X(6, 13, 1) X(7, 13, 0) X(7, 13, 1) \
  L(14) \
  X(0, 14, 0) X(1, 14, 0) X(2, 14, 0) X(3, 14, 0) X(4, 14, 0) X(5, 14, 0) \
  X(6, 14, 0) X(7, 14, 0)
// clang-format on

}  // namespace pfc
