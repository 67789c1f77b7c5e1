// Interior stencil of the 2D P2 inner operators in the cell-major row order.
//
// Cell-major order (2D, P2, structured stencils): the half-spacing lattice points
// (x, y), 0 <= x, y <= 2 side, are grouped into the 2 x 2 cells (cx, cy) =
// (x / 2, y / 2), cx, cy = 0 .. side, numbered cy (side + 1) + cx; the four rows of
// cell c are 4c + sub, sub = (x & 1) + 2 (y & 1) (0 vertex, 1 x-edge, 2 y-edge,
// 3 diagonal-edge midpoint, which is also the dof type of the row).  Points with
// x or y = 2 side + 1 hold no dof (padding rows).  A float4 load of a vector at
// cell c reads the four dofs of one lattice cell.
//
// On the structured triangulation (each square cut by the diagonal from (i, j) to
// (i+1, j+1)), a P2 dof couples to the dofs of the triangles that contain it: the
// vertex row to 19 lattice points within +-2 in x and y, each edge row to 9.  In cell
// terms every coupling of a cell's rows falls in the seven cells
//     q:  0 (-1,-1)  1 (0,-1)  2 (-1,0)  3 (0,0)  4 (1,0)  5 (0,1)  6 (1,1)
// (cells (1,-1) and (-1,1) lie across the diagonals and are never reached).
// PFC_CELL2D_ENTRIES lists, for every nonzero of an interior row, X(t, q, sub):
// output row type t, source cell q, source row sub inside that cell, in the order
// the kernel accumulates them.  The host checks at set-up that the interior
// stencils it extracted from the assembled pattern are exactly these couplings
// (and disables the cell kernels otherwise), and maps each entry to its weight.
#pragma once

namespace pfc {

constexpr int kCell2dEntries = 46;
constexpr int kCell2dSrc = 7;

// cell offsets (dx, dy) of the seven source cells
#define PFC_CELL2D_DX {-1, 0, -1, 0, 1, 0, 1}
#define PFC_CELL2D_DY {-1, -1, 0, 0, 0, 1, 1}

// clang-format off
#define PFC_CELL2D_ENTRIES(X)                                                                   \
  X(0, 0, 0) X(0, 0, 1) X(0, 1, 0) X(0, 0, 2) X(0, 0, 3) X(0, 1, 2) X(0, 1, 3)                   \
  X(0, 2, 0) X(0, 2, 1) X(0, 3, 0) X(0, 3, 1) X(0, 4, 0) X(0, 2, 3) X(0, 3, 2)                   \
  X(0, 3, 3) X(0, 4, 2) X(0, 5, 0) X(0, 5, 1) X(0, 6, 0)                                         \
  X(1, 1, 0) X(1, 1, 2) X(1, 1, 3) X(1, 3, 0) X(1, 3, 1) X(1, 4, 0) X(1, 3, 3)                   \
  X(1, 4, 2) X(1, 6, 0)                                                                          \
  X(2, 2, 0) X(2, 2, 1) X(2, 3, 0) X(2, 2, 3) X(2, 3, 2) X(2, 3, 3) X(2, 5, 0)                   \
  X(2, 5, 1) X(2, 6, 0)                                                                          \
  X(3, 3, 0) X(3, 3, 1) X(3, 4, 0) X(3, 3, 2) X(3, 3, 3) X(3, 4, 2) X(3, 5, 0)                   \
  X(3, 5, 1) X(3, 6, 0)
// clang-format on

}  // namespace pfc
