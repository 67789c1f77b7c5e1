// Structured simplicial mesh, P2 (or P1) dof lattice, SELL-C-sigma pattern and the
// gather maps of the assembly kernels (host side, once per instance).
//
// Mesh (Section 3 and Section 7 use regular simplicial meshes): side^dim cells of
// width h = length / side; cell c splits into the simplices whose vertices follow
// a monotone lattice path from the cell's low corner to its high corner (2 in 2D,
// the 6 Kuhn tetrahedra in 3D).  P2 dofs are the half-spacing lattice points,
// numbered lexicographically (x fastest); the node of edge (a, b) is the lattice
// midpoint of its end points.  P1 dofs (degree 1) are the vertices themselves.
//
// Device layout.  All blocks of the stage matrix (M, K, A01 and the inner
// matrices) share one sparsity pattern, stored once as SELL-32-sigma: slices of
// 32 rows, each stored column-major with the width of its longest row.  The row
// order IS the internal dof order of every device vector, so a SpMV writes y[row]
// coalesced and a vector update touches 32 consecutive rows per warp.  Without
// structured stencils rows are sorted by length (descending) inside windows of
// kSellSigma lexicographic rows; with them (sigma = 1) the order is lexicographic,
// or, for P2 with cells = 1, cell-major (2 x 2 or 2 x 2 x 2 lattice cells of four or
// eight consecutive rows, cell2d.h / cell3d.h).  Padding rows hold no dof; padding slots point at their own row
// with value 0.
#include <algorithm>
#include <cstring>
#include <map>
#include <numeric>

#include "internal.h"

#ifdef _OPENMP
#include <omp.h>
#endif

namespace pfc {

void element_path(int dim, int t, int verts[4][3]);
void local_edge(int dim, int e, int& a, int& b);

bool build_setup(int dim, int side, double length, HostSetup& S, std::string& err, int sigma, int degree,
                 int cells) {
  if (dim != 2 && dim != 3) {
    err = "dim must be 2 or 3";
    return false;
  }
  if (side < 1 || !(length > 0.0)) {
    err = "side must be >= 1 and length > 0";
    return false;
  }
  if (degree != 1 && degree != 2) {
    err = "degree must be 1 or 2";
    return false;
  }
  const int64_t lat = degree * (int64_t)side + 1;
  const int64_t n64 = dim == 2 ? lat * lat : lat * lat * lat;
  const int64_t cells64 = dim == 2 ? (int64_t)side * side : (int64_t)side * side * side;
  const int ntypes = dim == 2 ? 2 : 6;
  const int nl = degree == 1 ? dim + 1 : (dim == 2 ? 6 : 10);
  const int np = nl * (nl + 1) / 2;
  if (n64 > (1LL << 28) || cells64 * ntypes * np > (1LL << 31) - 1) {
    err = "mesh too large for 32-bit indices";
    return false;
  }
  S = HostSetup{};
  S.dim = dim;
  S.degree = degree;
  S.side = side;
  S.length = length;
  S.h = length / side;
  S.lat = (int)lat;
  S.n = (int)n64;
  S.ntypes = ntypes;
  S.nl = nl;
  S.sigma = sigma < 1 ? 1 : sigma;
  if (!build_reference(dim, S.h, S.ref, err, degree)) return false;
  const int n = S.n;
  const int E = (int)(cells64 * ntypes);
  S.E = E;

  // --- elements: cell-major (x fastest), types inner ---------------------------
  std::vector<int> elem_lex((size_t)E * nl);
  int path[6][4][3];
  for (int t = 0; t < ntypes; ++t) element_path(dim, t, path[t]);
  for (int64_t c = 0; c < cells64; ++c) {
    int ci = (int)(c % side), cj = (int)((c / side) % side), ck = dim == 3 ? (int)(c / ((int64_t)side * side)) : 0;
    for (int t = 0; t < ntypes; ++t) {
      int e = (int)(c * ntypes + t);
      int L[10][3];
      for (int k = 0; k <= dim; ++k) {
        L[k][0] = degree * (ci + path[t][k][0]);
        L[k][1] = degree * (cj + path[t][k][1]);
        L[k][2] = degree * (ck + path[t][k][2]);
      }
      int ne = degree == 1 ? 0 : (dim == 2 ? 3 : 6);
      for (int q = 0; q < ne; ++q) {
        int a, b;
        local_edge(dim, q, a, b);
        for (int x = 0; x < 3; ++x) L[dim + 1 + q][x] = (L[a][x] + L[b][x]) / 2;
      }
      for (int l = 0; l < nl; ++l)
        elem_lex[(size_t)e * nl + l] = (int)(L[l][0] + lat * (L[l][1] + lat * (int64_t)L[l][2]));
    }
  }

  // --- dof -> (element, local) incidence ---------------------------------------
  std::vector<int> inc_ptr(n + 1, 0), inc(E * (size_t)nl);
  for (size_t q = 0; q < elem_lex.size(); ++q) inc_ptr[elem_lex[q] + 1]++;
  for (int i = 0; i < n; ++i) inc_ptr[i + 1] += inc_ptr[i];
  {
    std::vector<int> fill(inc_ptr.begin(), inc_ptr.end() - 1);
    for (int e = 0; e < E; ++e)
      for (int l = 0; l < nl; ++l) inc[fill[elem_lex[(size_t)e * nl + l]]++] = l * E + e;
  }

  // --- row lengths (lexicographic) ---------------------------------------------
  std::vector<int> len(n);
#pragma omp parallel
  {
    std::vector<int> buf;
#pragma omp for schedule(static)
    for (int i = 0; i < n; ++i) {
      buf.clear();
      for (int q = inc_ptr[i]; q < inc_ptr[i + 1]; ++q) {
        int e = inc[q] % E;
        for (int l = 0; l < nl; ++l) buf.push_back(elem_lex[(size_t)e * nl + l]);
      }
      std::sort(buf.begin(), buf.end());
      len[i] = (int)(std::unique(buf.begin(), buf.end()) - buf.begin());
    }
  }
  S.nnz = 0;
  for (int i = 0; i < n; ++i) S.nnz += len[i];

  // --- internal row order ------------------------------------------------------
  // perm: internal row -> lexicographic dof, -1 for the padding rows.
  // SELL-32-sigma: rows sorted by length inside windows of sigma lexicographic rows
  // (sigma = 1 with structured stencils: lexicographic, padding rows at the end), or
  // cell-major (P2 with structured stencils and cells = 1): in 2D row 4 c + sub holds
  // lattice point (2 cx + (sub & 1), 2 cy + (sub >> 1)) of cell c = cy (side + 1) + cx,
  // in 3D row 8 c + sub likewise with z; the points with a coordinate 2 side + 1 and the
  // rows past the last cell are padding.
  S.iperm.assign(n, -1);
  S.cells = (cells && degree == 2 && S.sigma == 1) ? 1 : 0;
  if (S.cells) {
    // 2^dim rows per cell: row cr c + sub holds (2 cx + (sub & 1), 2 cy + ((sub >> 1) & 1),
    // 2 cz + (sub >> 2)) of cell c = (cz cs + cy) cs + cx
    const int64_t cs = side + 1, cr = dim == 2 ? 4 : 8, ncell = dim == 2 ? cs * cs : cs * cs * cs;
    S.cell_S = (int)cs;
    S.n_pad = (int)((cr * ncell + kSellC - 1) / kSellC * kSellC);
    S.perm.assign(S.n_pad, -1);
    for (int64_t p = 0; p < cr * ncell; ++p) {
      const int64_t c = p / cr, sub = p % cr;
      const int64_t x = 2 * (c % cs) + (sub & 1), y = 2 * ((c / cs) % cs) + ((sub >> 1) & 1);
      const int64_t z = dim == 3 ? 2 * (c / (cs * cs)) + (sub >> 2) : 0;
      if (x < lat && y < lat && z < (dim == 3 ? lat : 1)) {
        const int64_t i = (z * lat + y) * lat + x;
        S.perm[p] = (int)i;
        S.iperm[i] = (int)p;
      }
    }
  } else {
    S.n_pad = (n + kSellC - 1) / kSellC * kSellC;
    S.perm.assign(S.n_pad, -1);
    std::iota(S.perm.begin(), S.perm.begin() + n, 0);
    for (int w0 = 0; w0 < n; w0 += S.sigma) {
      int w1 = std::min(n, w0 + S.sigma);
      std::stable_sort(S.perm.begin() + w0, S.perm.begin() + w1, [&](int a, int b) { return len[a] > len[b]; });
    }
    for (int p = 0; p < n; ++p) S.iperm[S.perm[p]] = p;
  }
  S.nslices = S.n_pad / kSellC;
  S.slice_ptr.assign(S.nslices + 1, 0);
  for (int s = 0; s < S.nslices; ++s) {
    int w = 0;
    for (int l = 0; l < kSellC; ++l) {
      const int i = S.perm[s * kSellC + l];
      if (i >= 0) w = std::max(w, len[i]);
    }
    S.slice_ptr[s + 1] = S.slice_ptr[s] + w * kSellC;
  }
  S.nnz_sell = S.slice_ptr[S.nslices];
  if (S.nnz_sell > (1LL << 31) - 1) {
    err = "too many nonzeros for 32-bit slot indices";
    return false;
  }

  // --- columns, diagonal positions, slot contributions ---------------------------
  S.cols.assign(S.nnz_sell, 0);
  S.diag_pos.assign(S.n_pad, -1);
  std::vector<int> ccount(S.nnz_sell + 1, 0);
  S.elem_int.resize((size_t)nl * E);
  for (int e = 0; e < E; ++e)
    for (int l = 0; l < nl; ++l) S.elem_int[(size_t)l * E + e] = S.iperm[elem_lex[(size_t)e * nl + l]];

  auto row_cols = [&](int i, std::vector<int>& buf) {
    buf.clear();
    for (int q = inc_ptr[i]; q < inc_ptr[i + 1]; ++q) {
      int e = inc[q] % E;
      for (int l = 0; l < nl; ++l) buf.push_back(S.iperm[elem_lex[(size_t)e * nl + l]]);
    }
    std::sort(buf.begin(), buf.end());
    buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
  };
  const RefTensors& R = S.ref;
  // pass 1: columns, diagonal, contribution counts
#pragma omp parallel
  {
    std::vector<int> buf;
#pragma omp for schedule(static)
    for (int p = 0; p < S.n_pad; ++p) {
      int s = p / kSellC, lane = p % kSellC;
      int base = S.slice_ptr[s] + lane;
      int w = (S.slice_ptr[s + 1] - S.slice_ptr[s]) / kSellC;
      const int i = S.perm[p];
      if (i < 0) {
        for (int j = 0; j < w; ++j) S.cols[base + j * kSellC] = p;
        continue;
      }
      row_cols(i, buf);
      for (int j = 0; j < w; ++j) S.cols[base + j * kSellC] = j < (int)buf.size() ? buf[j] : p;
      for (int j = 0; j < (int)buf.size(); ++j)
        if (buf[j] == p) S.diag_pos[p] = base + j * kSellC;
      for (int q = inc_ptr[i]; q < inc_ptr[i + 1]; ++q) {
        int e = inc[q] % E;
        for (int lc = 0; lc < nl; ++lc) {
          int col = S.elem_int[(size_t)lc * E + e];
          int j = (int)(std::lower_bound(buf.begin(), buf.end(), col) - buf.begin());
          ccount[base + j * kSellC + 1]++;
        }
      }
    }
  }
  for (int64_t q = 0; q < S.nnz_sell; ++q) ccount[q + 1] += ccount[q];
  S.contrib_ptr = ccount;
  S.contrib_idx.assign(S.contrib_ptr[S.nnz_sell], 0);
  // pass 2: contribution lists (each row owns its slots, so rows run in parallel)
#pragma omp parallel
  {
    std::vector<int> buf;
#pragma omp for schedule(static)
    for (int p = 0; p < S.n_pad; ++p) {
      const int i = S.perm[p];
      if (i < 0) continue;
      int s = p / kSellC, lane = p % kSellC;
      int base = S.slice_ptr[s] + lane;
      row_cols(i, buf);
      std::vector<int> next(buf.size(), 0);
      for (int q = inc_ptr[i]; q < inc_ptr[i + 1]; ++q) {
        int e = inc[q] % E, li = inc[q] / E;
        for (int lc = 0; lc < nl; ++lc) {
          int col = S.elem_int[(size_t)lc * E + e];
          int j = (int)(std::lower_bound(buf.begin(), buf.end(), col) - buf.begin());
          int slot = base + j * kSellC;
          int pr = R.pair_index[li * nl + lc];
          S.contrib_idx[S.contrib_ptr[slot] + next[j]++] = pr * E + e;
        }
      }
    }
  }

  // --- dof gather map for element load vectors ---------------------------------
  S.dof_ptr.assign(S.n_pad + 1, 0);
  for (int p = 0; p < S.n_pad; ++p) {
    const int i = S.perm[p];
    int c = i >= 0 ? inc_ptr[i + 1] - inc_ptr[i] : 0;
    S.dof_ptr[p + 1] = S.dof_ptr[p] + c;
  }
  S.dof_idx.resize(S.dof_ptr[S.n_pad]);
  for (int p = 0; p < S.n_pad; ++p) {
    const int i = S.perm[p];
    if (i >= 0) std::copy(inc.begin() + inc_ptr[i], inc.begin() + inc_ptr[i + 1], S.dof_idx.begin() + S.dof_ptr[p]);
  }

  // --- structured stencils of M and K (sigma == 1: lexicographic order) -----------
  // Row p's columns are p + offset; the offsets of an interior row (all incident
  // elements present) depend only on its dof type t (the lattice coordinate
  // parities), so every type has one stencil.
  S.ntypes_dof = 1 << dim;
  S.rowinfo.assign(S.n_pad, 0);
  if (S.sigma == 1) {
    auto dof_type = [&](int i) {
      const int a = i % (int)lat, b = (int)((i / lat) % lat), c = dim == 3 ? (int)(i / (lat * lat)) : 0;
      return (a & 1) | ((b & 1) << 1) | ((c & 1) << 2);
    };
    // rows whose incident-element count is the maximum of their type have all
    // their elements, hence the interior stencil of the type
    std::vector<int> maxinc(S.ntypes_dof, 0), rep(S.ntypes_dof, -1);
    for (int i = 0; i < n; ++i) {
      const int t = dof_type(i), k = inc_ptr[i + 1] - inc_ptr[i];
      if (k > maxinc[t]) {
        maxinc[t] = k;
        rep[t] = i;
      }
    }
    S.st_start.assign(S.ntypes_dof + 1, 0);
    S.st_off.clear();
    S.st_wM.clear();
    S.st_wK.clear();
    std::vector<int> buf;
    for (int t = 0; t < S.ntypes_dof; ++t) {
      const int i = rep[t];
      if (i >= 0) {
        row_cols(i, buf);
        const int p = S.iperm[i];
        const int s_ = p / kSellC, lane = p % kSellC, base = S.slice_ptr[s_] + lane;
        for (int j = 0; j < (int)buf.size(); ++j) {
          const int slot = base + j * kSellC;
          double m = 0.0, k = 0.0;
          for (int q = S.contrib_ptr[slot]; q < S.contrib_ptr[slot + 1]; ++q) {
            const int idx = S.contrib_idx[q], pr = idx / E, e = idx - pr * E, et = e % ntypes;
            m += R.mass[(size_t)et * R.npairs + pr];
            k += R.stiff[(size_t)et * R.npairs + pr];
          }
          S.st_off.push_back(buf[j] - p);
          S.st_wM.push_back(m);
          S.st_wK.push_back(k);
        }
      }
      S.st_start[t + 1] = (int)S.st_off.size();
    }
    // interior: same element count AND the same column offsets as the type's
    // representative (translation invariance then gives the same values)
#pragma omp parallel
    {
      std::vector<int> rb;
#pragma omp for schedule(static)
      for (int p = 0; p < S.n_pad; ++p) {
        const int i = S.perm[p];
        if (i < 0) continue;
        const int t = dof_type(i);
        bool interior = (inc_ptr[i + 1] - inc_ptr[i]) == maxinc[t];
        if (interior) {
          row_cols(i, rb);
          const int k0 = S.st_start[t], len = S.st_start[t + 1] - k0;
          interior = (int)rb.size() == len;
          for (int j = 0; interior && j < len; ++j) interior = rb[j] - p == S.st_off[k0 + j];
        }
        S.rowinfo[p] = (unsigned char)(t | (interior ? 8 : 0));
      }
    }
  }

  // --- row classes (cell-major order) ---------------------------------------------
  // A row's stencil: its columns as offsets from the row with the M and K values of
  // the slot (the same sums of element contributions the assembly kernel forms).  On
  // the uniform mesh the rows with a missing element fall into a few classes (by
  // dof type and the side or corner they lie on); rows with equal stencils share one.
  if (S.cells) {
    const int nt = S.ntypes_dof;
    S.cls_start.assign(1, 0);
    for (int t = 0; t < nt; ++t) {
      for (int k = S.st_start[t]; k < S.st_start[t + 1]; ++k) {
        S.cls_off.push_back(S.st_off[k]);
        S.cls_wM.push_back(S.st_wM[k]);
        S.cls_wK.push_back(S.st_wK[k]);
      }
      S.cls_start.push_back((int)S.cls_off.size());
    }
    S.cls_start.push_back((int)S.cls_off.size());   // class nt: no entries
    S.rowclass.assign(S.n_pad, (unsigned char)nt);
    struct Key {
      std::vector<int> off;
      std::vector<double> m, k;
      bool operator<(const Key& o) const {
        if (off != o.off) return off < o.off;
        if (m != o.m) return m < o.m;
        return k < o.k;
      }
    };
    std::map<Key, int> seen;
    std::vector<int> buf;
    for (int p = 0; p < S.n_pad; ++p) {
      const int i = S.perm[p];
      if (i < 0) continue;
      if (S.rowinfo[p] & 8) {
        S.rowclass[p] = (unsigned char)(S.rowinfo[p] & 7);
        continue;
      }
      row_cols(i, buf);
      const int s_ = p / kSellC, lane = p % kSellC, base = S.slice_ptr[s_] + lane;
      Key key;
      for (int j = 0; j < (int)buf.size(); ++j) {
        const int slot = base + j * kSellC;
        double m = 0.0, k = 0.0;
        for (int q = S.contrib_ptr[slot]; q < S.contrib_ptr[slot + 1]; ++q) {
          const int idx = S.contrib_idx[q], pr = idx / E, e = idx - pr * E, et = e % ntypes;
          m += R.mass[(size_t)et * R.npairs + pr];
          k += R.stiff[(size_t)et * R.npairs + pr];
        }
        key.off.push_back(buf[j] - p);
        key.m.push_back(m);
        key.k.push_back(k);
      }
      auto it = seen.find(key);
      int id;
      if (it != seen.end()) {
        id = it->second;
      } else {
        id = (int)S.cls_start.size() - 1;
        for (size_t j = 0; j < key.off.size(); ++j) {
          S.cls_off.push_back(key.off[j]);
          S.cls_wM.push_back(key.m[j]);
          S.cls_wK.push_back(key.k[j]);
        }
        S.cls_start.push_back((int)S.cls_off.size());
        seen.emplace(std::move(key), id);
      }
      S.rowclass[p] = (unsigned char)std::min(id, 255);
    }
  }
  return true;
}

size_t footprint_estimate(int dim, int side, int restart, int precision, int degree, int model) {
  const double lat = degree * side + 1.0;
  const double n = dim == 2 ? lat * lat : lat * lat * lat;
  const double nnz_row = degree == 1 ? (dim == 2 ? 7.2 : 15.2) : (dim == 2 ? 11.6 : 28.6);  // slots per row
  const double nnz = n * nnz_row;
  const double E = dim == 2 ? 2.0 * side * side : 6.0 * side * side * side;
  const double nl = degree == 1 ? dim + 1 : (dim == 2 ? 6 : 10), np = nl * (nl + 1) / 2;
  double b = 0;
  b += nnz * 4;                             // columns
  b += nnz * 8 * 5;                         // M, K, A01, M+dK, M+sK (float64)
  b += precision == 0 ? 0 : nnz * (precision == 1 ? 4 : 2) * 4;
  b += nnz * 4 + E * nl * nl * 4;           // contribution map
  b += E * np * 8 + E * nl * 4 * 2;         // element buffer, element dofs, dof map
  b += n * 8 * 3 * (2.0 * restart + 1 + 8); // Krylov bases and step vectors
  b += n * 8 * 12;                          // inner vectors, diagonals
  if (model == 1) b += nnz * 8 * 2 + E * np * 8 * 2;  // PFC1: A10, A11 and the wider element buffer
  return (size_t)(b * 1.05) + (64u << 20);
}

}  // namespace pfc

namespace pfc {

// Strip partition of one instance for a row-block solve over several devices (the
// paper's PETSc/MPI runs partition the rows in contiguous blocks, Section 7).  With
// lexicographic numbering a contiguous block of rows made of whole lattice lines
// (2D) or planes (3D) is a strip (slab) of the domain, and a row's columns reach at
// most `degree` lines (planes) up or down, so a part exchanges ghost values with its
// two neighbours only, provided every part holds at least `degree` lines.  Parts are
// cut at line boundaries so that their nonzeros are as equal as the lines allow.
bool build_partition(int dim, int side, double length, int degree, int nparts, std::vector<int64_t>& begin,
                     std::vector<int64_t>& halo, std::vector<int64_t>& part_nnz, std::string& err) {
  HostSetup S;
  if (!build_setup(dim, side, length, S, err, kSellSigma, degree)) return false;
  const int64_t lat = S.lat, n = S.n;
  const int64_t line = dim == 2 ? lat : lat * lat;   // rows per line (2D) / plane (3D)
  const int64_t nlines = n / line;
  if (nparts < 1 || (int64_t)nparts * degree > nlines) {
    err = "every part needs at least `degree` lattice lines: nparts must be in 1.." + std::to_string(nlines / degree);
    return false;
  }
  // per lexicographic row: true nonzeros and the lowest / highest column
  std::vector<int64_t> rnnz(n, 0), cmin(n, n), cmax(n, -1);
  for (int p = 0; p < S.n_pad; ++p) {
    const int i = S.perm[p];
    if (i < 0) continue;
    const int s = p / kSellC, lane = p % kSellC, base = S.slice_ptr[s] + lane;
    const int w = (S.slice_ptr[s + 1] - S.slice_ptr[s]) / kSellC;
    for (int j = 0; j < w; ++j) {
      const int slot = base + j * kSellC;
      if (S.contrib_ptr[slot + 1] == S.contrib_ptr[slot]) continue;   // padding slot
      const int64_t col = S.perm[S.cols[slot]];
      rnnz[i] += 1;
      cmin[i] = std::min(cmin[i], col);
      cmax[i] = std::max(cmax[i], col);
    }
  }
  std::vector<int64_t> lnnz(nlines + 1, 0);   // prefix sums of nonzeros by line
  for (int64_t l = 0; l < nlines; ++l) {
    int64_t t = 0;
    for (int64_t i = l * line; i < (l + 1) * line; ++i) t += rnnz[i];
    lnnz[l + 1] = lnnz[l] + t;
  }
  // cut points: the line where the nonzero prefix reaches k / nparts of the total,
  // kept at least `degree` lines apart
  std::vector<int64_t> cut(nparts + 1, 0);
  cut[nparts] = nlines;
  for (int k = 1; k < nparts; ++k) {
    const int64_t target = lnnz[nlines] * k / nparts;
    int64_t l = (int64_t)(std::lower_bound(lnnz.begin(), lnnz.end(), target) - lnnz.begin());
    l = std::max(l, cut[k - 1] + degree);
    l = std::min(l, nlines - (int64_t)(nparts - k) * degree);
    cut[k] = l;
  }
  begin.assign(nparts + 1, 0);
  halo.assign(2 * (size_t)nparts, 0);
  part_nnz.assign(nparts, 0);
  for (int k = 0; k <= nparts; ++k) begin[k] = cut[k] * line;
  for (int k = 0; k < nparts; ++k) {
    int64_t lo = n, hi = -1;
    for (int64_t i = begin[k]; i < begin[k + 1]; ++i) {
      lo = std::min(lo, cmin[i]);
      hi = std::max(hi, cmax[i]);
    }
    halo[2 * k] = begin[k] - lo;             // ghost rows below the part
    halo[2 * k + 1] = hi + 1 - begin[k + 1]; // ghost rows above it
    part_nnz[k] = lnnz[cut[k + 1]] - lnnz[cut[k]];
    // ghosts come from the neighbouring parts only
    if ((k > 0 && lo < begin[k - 1]) || (k + 1 < nparts && hi >= begin[k + 2])) {
      err = "a part's columns reach past its neighbours";
      return false;
    }
  }
  return true;
}

}  // namespace pfc
