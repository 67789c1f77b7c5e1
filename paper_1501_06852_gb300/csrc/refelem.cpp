// Reference-element tensors of the P2 Lagrange element, computed exactly.
//
// Every P2 basis function is a polynomial in the barycentric coordinates
// lambda_0..lambda_d of its simplex: lambda_k (2 lambda_k - 1) at vertex k and
// 4 lambda_a lambda_b at the midpoint of edge (a, b) (Section 3: V_h with p = 2).
// Products of such polynomials are expanded into barycentric monomials and
// integrated with the closed form
//     int_T lambda^e dx = |T| d! prod_k e_k! / (|e| + d)!,
// so the mass matrix, the stiffness matrix (through grad phi = sum_k
// d phi / d lambda_k grad lambda_k) and the quartic tensor that gives the
// nonlinear mass N(psi)_ij = (-3 psi^2 phi_j, phi_i) are exact to rounding, as is
// the mobility tensor int phi_a grad phi_b . grad phi_c of the PFC1 model, from
// which K_+(psi) = ((psi^+ grad phi_j, grad phi_i)), F(mu) = ((phi_j grad mu,
// grad phi_i)) and the load (psi^+ grad mu, grad phi_i) follow (Eq. 3.10).
#include <array>
#include <cmath>
#include <map>

#include "internal.h"

namespace pfc {
namespace {

using Mono = std::array<int, 4>;
using Poly = std::map<Mono, double>;

Poly mul(const Poly& a, const Poly& b) {
  Poly out;
  for (const auto& [ea, ca] : a)
    for (const auto& [eb, cb] : b) {
      Mono e{ea[0] + eb[0], ea[1] + eb[1], ea[2] + eb[2], ea[3] + eb[3]};
      out[e] += ca * cb;
    }
  return out;
}

Poly dlambda(const Poly& a, int k) {
  Poly out;
  for (const auto& [e, c] : a) {
    if (e[k] == 0) continue;
    Mono f = e;
    f[k] -= 1;
    out[f] += c * e[k];
  }
  return out;
}

double fact(int k) {
  double f = 1.0;
  for (int i = 2; i <= k; ++i) f *= i;
  return f;
}

// integral over a simplex of unit volume
double integrate(const Poly& a, int dim) {
  double s = 0.0;
  for (const auto& [e, c] : a) {
    int tot = e[0] + e[1] + e[2] + e[3];
    s += c * fact(dim) * fact(e[0]) * fact(e[1]) * fact(e[2]) * fact(e[3]) / fact(tot + dim);
  }
  return s;
}

Mono unit(int k, int p) {
  Mono m{0, 0, 0, 0};
  m[k] = p;
  return m;
}

// Local node order: vertices 0..d, then edges.
const int kEdges2[3][2] = {{1, 2}, {0, 2}, {0, 1}};
const int kEdges3[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

// P1: lambda_k at vertex k
std::vector<Poly> p1_basis(int dim) {
  std::vector<Poly> b;
  for (int k = 0; k <= dim; ++k) {
    Poly p;
    p[unit(k, 1)] = 1.0;
    b.push_back(p);
  }
  return b;
}

std::vector<Poly> p2_basis(int dim) {
  std::vector<Poly> b;
  for (int k = 0; k <= dim; ++k) {
    Poly p;
    p[unit(k, 2)] = 2.0;
    p[unit(k, 1)] = -1.0;
    b.push_back(p);
  }
  int ne = dim == 2 ? 3 : 6;
  for (int e = 0; e < ne; ++e) {
    int a = dim == 2 ? kEdges2[e][0] : kEdges3[e][0];
    int c = dim == 2 ? kEdges2[e][1] : kEdges3[e][1];
    Mono m{0, 0, 0, 0};
    m[a] += 1;
    m[c] += 1;
    Poly p;
    p[m] = 4.0;
    b.push_back(p);
  }
  return b;
}

}  // namespace

// Vertex offsets (cell units) of element type t: a monotone lattice path from
// the cell corner to the opposite corner (2D: x then y / y then x; 3D: the 6
// axis permutations, the Kuhn tetrahedra).
void element_path(int dim, int t, int verts[4][3]) {
  static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  static const int perms2[2][2] = {{0, 1}, {1, 0}};
  for (int k = 0; k < 4; ++k)
    for (int c = 0; c < 3; ++c) verts[k][c] = 0;
  for (int k = 0; k < dim; ++k) {
    int ax = dim == 2 ? perms2[t][k] : perms[t][k];
    for (int c = 0; c < 3; ++c) verts[k + 1][c] = verts[k][c];
    verts[k + 1][ax] += 1;
  }
}

void local_edge(int dim, int e, int& a, int& b) {
  a = dim == 2 ? kEdges2[e][0] : kEdges3[e][0];
  b = dim == 2 ? kEdges2[e][1] : kEdges3[e][1];
}

bool build_reference(int dim, double h, RefTensors& out, std::string& err, int degree) {
  if (dim != 2 && dim != 3) {
    err = "dim must be 2 or 3";
    return false;
  }
  if (degree != 1 && degree != 2) {
    err = "degree must be 1 or 2";
    return false;
  }
  const int nl = degree == 1 ? dim + 1 : (dim == 2 ? 6 : 10);
  const int ntypes = dim == 2 ? 2 : 6;
  out = RefTensors{};
  out.dim = dim;
  out.nl = nl;
  out.ntypes = ntypes;
  out.pair_index.assign(nl * nl, -1);
  for (int i = 0; i < nl; ++i)
    for (int j = i; j < nl; ++j) {
      out.pair_index[i * nl + j] = out.pair_index[j * nl + i] = (int)out.pair_i.size();
      out.pair_i.push_back(i);
      out.pair_j.push_back(j);
    }
  const int np = (int)out.pair_i.size();
  out.npairs = np;

  std::vector<Poly> phi = degree == 2 ? p2_basis(dim) : p1_basis(dim);
  // unit-volume integrals
  std::vector<double> mref(np), quart((size_t)np * np);
  for (int p = 0; p < np; ++p) mref[p] = integrate(mul(phi[out.pair_i[p]], phi[out.pair_j[p]]), dim);
  std::vector<Poly> prod(np);
  for (int p = 0; p < np; ++p) prod[p] = mul(phi[out.pair_i[p]], phi[out.pair_j[p]]);
  for (int pa = 0; pa < np; ++pa) {
    double w = out.pair_i[pa] == out.pair_j[pa] ? 1.0 : 2.0;
    for (int pb = 0; pb < np; ++pb) quart[(size_t)pa * np + pb] = w * integrate(mul(prod[pa], prod[pb]), dim);
  }
  // D[i][k][j][l] = int d_k phi_i d_l phi_j (unit volume)
  const int nb = dim + 1;
  std::vector<double> D((size_t)nl * nb * nl * nb);
  for (int i = 0; i < nl; ++i)
    for (int k = 0; k < nb; ++k) {
      Poly di = dlambda(phi[i], k);
      for (int j = 0; j < nl; ++j)
        for (int l = 0; l < nb; ++l)
          D[((i * nb + k) * nl + j) * nb + l] = integrate(mul(di, dlambda(phi[j], l)), dim);
    }

  // Dm[a][b][k][c][l] = int phi_a d_k phi_b d_l phi_c (unit volume)
  std::vector<double> Dm((size_t)nl * nl * nb * nl * nb);
  for (int a = 0; a < nl; ++a)
    for (int b = 0; b < nl; ++b)
      for (int k = 0; k < nb; ++k) {
        const Poly ab = mul(phi[a], dlambda(phi[b], k));
        for (int c = 0; c < nl; ++c)
          for (int l = 0; l < nb; ++l)
            Dm[((((size_t)a * nl + b) * nb + k) * nl + c) * nb + l] = integrate(mul(ab, dlambda(phi[c], l)), dim);
      }
  out.mob.assign((size_t)ntypes * nl * nl * nl, 0.0);
  out.mass.assign((size_t)ntypes * np, 0.0);
  out.stiff.assign((size_t)ntypes * np, 0.0);
  double vol0 = -1.0;
  for (int t = 0; t < ntypes; ++t) {
    int v[4][3];
    element_path(dim, t, v);
    // B = [X1 - X0, ..., Xd - X0] (columns), X in physical units
    double B[3][3] = {{0}};
    for (int c = 0; c < dim; ++c)
      for (int r = 0; r < dim; ++r) B[r][c] = h * (v[c + 1][r] - v[0][r]);
    double det, inv[3][3];
    if (dim == 2) {
      det = B[0][0] * B[1][1] - B[0][1] * B[1][0];
      inv[0][0] = B[1][1] / det;
      inv[0][1] = -B[0][1] / det;
      inv[1][0] = -B[1][0] / det;
      inv[1][1] = B[0][0] / det;
    } else {
      det = B[0][0] * (B[1][1] * B[2][2] - B[1][2] * B[2][1]) - B[0][1] * (B[1][0] * B[2][2] - B[1][2] * B[2][0]) +
            B[0][2] * (B[1][0] * B[2][1] - B[1][1] * B[2][0]);
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
          int r1 = (c + 1) % 3, r2 = (c + 2) % 3, c1 = (r + 1) % 3, c2 = (r + 2) % 3;
          inv[r][c] = (B[r1][c1] * B[r2][c2] - B[r1][c2] * B[r2][c1]) / det;
        }
    }
    if (det == 0.0) {
      err = "degenerate element";
      return false;
    }
    double vol = std::fabs(det) / (dim == 2 ? 2.0 : 6.0);
    if (vol0 < 0) vol0 = vol;
    // grad lambda_k, k >= 1: row k-1 of B^{-1}; grad lambda_0 = -sum
    double g[4][3] = {{0}};
    for (int k = 1; k <= dim; ++k)
      for (int c = 0; c < dim; ++c) {
        g[k][c] = inv[k - 1][c];
        g[0][c] -= inv[k - 1][c];
      }
    double G[4][4];
    for (int a = 0; a < nb; ++a)
      for (int b = 0; b < nb; ++b) {
        double s = 0;
        for (int c = 0; c < dim; ++c) s += g[a][c] * g[b][c];
        G[a][b] = s;
      }
    for (int p = 0; p < np; ++p) {
      int i = out.pair_i[p], j = out.pair_j[p];
      double s = 0.0;
      for (int k = 0; k < nb; ++k)
        for (int l = 0; l < nb; ++l) s += G[k][l] * D[((i * nb + k) * nl + j) * nb + l];
      out.stiff[(size_t)t * np + p] = vol * s;
      out.mass[(size_t)t * np + p] = vol * mref[p];
    }
    for (int a = 0; a < nl; ++a)
      for (int b = 0; b < nl; ++b)
        for (int c = 0; c < nl; ++c) {
          double s = 0.0;
          for (int k = 0; k < nb; ++k)
            for (int l = 0; l < nb; ++l) s += G[k][l] * Dm[((((size_t)a * nl + b) * nb + k) * nl + c) * nb + l];
          out.mob[(((size_t)t * nl + a) * nl + b) * nl + c] = vol * s;
        }
  }
  out.vol = vol0;
  out.quartic.resize((size_t)np * np);
  for (size_t q = 0; q < quart.size(); ++q) out.quartic[q] = vol0 * quart[q];
  return true;
}

}  // namespace pfc
