// Internal declarations of the PFC stage-solver library (host and device).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace pfc {

constexpr int kSellC = 32;          // SELL slice height = warp width
constexpr int kSellSigma = 1024;    // rows sorted by length inside windows of this size
constexpr int kMaxRestart = 40;     // FGMRES restart cap (shared-memory Hessenberg)
constexpr int kMaxLocal = 10;       // P2 nodes per tetrahedron
constexpr int kMaxPairs = 55;       // unordered local pairs for tetrahedra

// Exact integrals of P2 basis products on one simplex type, built from
// barycentric monomials: int_T lambda^e = |T| d! prod(e_k!) / (|e| + d)!.
struct RefTensors {
  int dim = 0, nl = 0, npairs = 0, ntypes = 0;
  double vol = 0.0;                          // |T| of every element of the structured mesh
  std::vector<int> pair_i, pair_j;           // unordered pair p -> (i <= j)
  std::vector<int> pair_index;               // nl*nl -> p
  std::vector<double> mass;                  // ntypes x npairs: int phi_i phi_j
  std::vector<double> stiff;                 // ntypes x npairs: int grad phi_i . grad phi_j
  std::vector<double> quartic;               // npairs(ab) x npairs(ij): w_ab int phi_a phi_b phi_i phi_j, w_ab = 2 (a != b), 1
  std::vector<double> mob;                   // ntypes x nl x nl x nl: int phi_a grad phi_b . grad phi_c (physical)
};

// Structured mesh, P2 dofs, SELL-C-sigma pattern and the maps the assembly
// kernels gather through.  All indices are int32.
struct HostSetup {
  int dim = 0, side = 0;
  int degree = 2;                 // Lagrange degree: 2 (P2) or 1 (P1)
  double length = 0.0, h = 0.0;
  int lat = 0;                    // degree * side + 1 lattice points per axis
  int n = 0;                      // dofs per field
  int n_pad = 0;                  // internal rows (a multiple of kSellC, >= n)
  int nslices = 0;
  int64_t nnz = 0;                // true nonzeros of one block
  int64_t nnz_sell = 0;           // stored slots (with padding)
  int E = 0;                      // elements
  int nl = 0;                     // local nodes per element
  int ntypes = 0;                 // element types per cell (2 or 6)
  std::vector<int> perm;          // internal row -> lexicographic dof (size n_pad; -1: no dof)
  std::vector<int> iperm;         // lexicographic dof -> internal row (size n)
  std::vector<int> slice_ptr;     // nslices + 1 (slot offsets)
  std::vector<int> cols;          // nnz_sell internal column indices (padding: the row itself)
  std::vector<int> diag_pos;      // n_pad (-1 for padding rows)
  std::vector<int> elem_int;      // nl x E (SoA) internal dof of local node l of element e
  std::vector<int> contrib_ptr;   // nnz_sell + 1
  std::vector<int> contrib_idx;   // p * E + e for each element pair landing on a slot
  std::vector<int> dof_ptr;       // n_pad + 1
  std::vector<int> dof_idx;       // l * E + e for each element incident to a row
  RefTensors ref;
  // Structured stencils of the constant matrices (only with sigma == 1, where the
  // internal order is lexicographic):
  // dof type t = lattice-coordinate parities;
  // every row whose incident elements all exist ("interior") has the stencil of
  // its type: M_i,i+off[k] = st_wM[k], K_i,i+off[k] = st_wK[k], k in
  // [st_start[t], st_start[t+1]).
  int sigma = kSellSigma;
  int ntypes_dof = 0;
  std::vector<int> st_start;      // ntypes_dof + 1
  std::vector<int> st_off;
  std::vector<double> st_wM, st_wK;
  std::vector<unsigned char> rowinfo;  // n_pad: bits 0-2 dof type, bit 3 interior
  // Cell-major row order (P2 with structured stencils, cells = 1; cell2d.h, cell3d.h):
  // row 2^dim c + sub holds lattice point (2 cx + (sub & 1), 2 cy + ((sub >> 1) & 1),
  // 2 cz + (sub >> 2)) of cell c = (cz cell_S + cy) cell_S + cx.  Row classes (built in that order only): every row's stencil
  // (column offsets with its M and K weights); class t < ntypes_dof is the interior
  // stencil of dof type t, class ntypes_dof has no entries (rows that hold no dof),
  // the others are the distinct stencils of the rows with a missing element.
  int cells = 0;
  int cell_S = 0;                 // cells per lattice line (side + 1)
  std::vector<int> cls_start;     // classes + 1
  std::vector<int> cls_off;
  std::vector<double> cls_wM, cls_wK;
  std::vector<unsigned char> rowclass;  // n_pad class of each row (empty unless cells)
};

bool build_reference(int dim, double h, RefTensors& out, std::string& err, int degree = 2);
bool build_setup(int dim, int side, double length, HostSetup& out, std::string& err, int sigma = kSellSigma,
                 int degree = 2, int cells = 0);

// Strip partition of the lexicographic rows over nparts devices (row-block solve):
// begin (nparts + 1 row offsets), halo (ghost rows below / above each part), the
// nonzeros of one block held by each part.
bool build_partition(int dim, int side, double length, int degree, int nparts, std::vector<int64_t>& begin,
                     std::vector<int64_t>& halo, std::vector<int64_t>& part_nnz, std::string& err);

// Bytes of device memory a context of this size holds (estimate used for admission).
size_t footprint_estimate(int dim, int side, int restart, int precision, int degree = 2, int model = 2);

}  // namespace pfc
