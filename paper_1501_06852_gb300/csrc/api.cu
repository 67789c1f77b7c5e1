// C ABI of the PFC stage solver: context set-up, per-step assembly, stage
// right-hand side, stage solve and the Ros3Pw step (see include/pfc.h).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <functional>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <string>

#include "device.cuh"
#include "internal.h"
#include "launch.h"
#include "pfc.h"

#ifndef PFC_BOUNDARY_COST
#define PFC_BOUNDARY_COST 1
#endif
#ifndef PFC_VEC_COST
#define PFC_VEC_COST 320
#endif

namespace {

// Ros3Pw in the modified Rosenbrock form (Table 1 of Praetorius & Voigt).  The
// printed diagonal entries "a22", "a33", "c11", "c22", "c33" are stage-time sums
// of the standard form; the PFC system is autonomous, so they are unused.
constexpr double kGamma = 0.78867513459481287;
constexpr double kA[3][2] = {{0.0, 0.0}, {2.0, 0.0}, {0.633974596215561, 0.0}};
constexpr double kC[3][2] = {{0.0, 0.0}, {-2.53589838486225, 0.0}, {-1.62740473580836, -0.274519052838329}};
constexpr double kM[3] = {1.63397459621556, 0.294228634059948, 1.07179676972449};
constexpr double kMhat[3] = {1.99444650053487, 0.654700538379252, 1.07179676972449};

struct Layout {
  size_t off = 0;
  size_t take(size_t bytes) {
    off = (off + 255) & ~size_t(255);
    const size_t o = off;
    off += bytes;
    return o;
  }
};

std::mutex g_const_mutex;
bool g_const_done[4][64] = {};   // element kind (P2 tri, P2 tet, P1 tri, P1 tet) x device

}  // namespace

struct pfc_ctx {
  pfc_options opt{};
  int device = 0;
  cudaStream_t stream = nullptr;
  int dim = 0, side = 0;
  double length = 0.0;
  int n = 0, n_pad = 0, nslices = 0, E = 0, nl = 0, np = 0, ntypes = 0;
  long long nnz_sell = 0, nnz = 0, ncontrib = 0;
  int prec = 0;
  double vol = 0.0;
  int G = 0;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  // pattern and maps
  int *slice_ptr = nullptr, *cols = nullptr, *diag = nullptr, *perm = nullptr, *elem = nullptr;
  int *cptr = nullptr, *cidx = nullptr, *dptr = nullptr, *didx = nullptr, *blk = nullptr;
  // structured stencils (inner_operator == 1)
  unsigned char* rowinfo = nullptr;
  int *st_start = nullptr, *st_off = nullptr;
  double *st_wM = nullptr, *st_wK = nullptr;
  int st_types = 0;
  int st_halo = 0;              // largest |stencil offset|
  int win_cap = 0;              // floats of the shared-memory SpMV window (0: off)
  int tma = 0, tma_lat = 0, tma_plane = 0, tma_S = 0, tma_cap = 0;   // chunked windows (smem_window 2)
  // cell kernels (2D P2 cell-major rows, float inner vectors): row classes and windows
  int cells = 0;                // rows in cell-major order
  int cell_ok = 0;              // the cell kernels run the Chronopoulos-Gear inner solves
  int cell_S = 0;
  int ccls_n = 0;               // cell classes
  double *ccls_wM = nullptr, *ccls_wK = nullptr;
  unsigned char* cellclass = nullptr;
  int cell_rep[8] = {};         // an interior row of each dof type
  int cell_gx = 0, cell_gy = 0, cell_gz = 0, cell_wcap = 0, cell_ccap = 0, cell_rcap = 0;   // tiling of its own grid
  double *mass_tab = nullptr, *stiff_tab = nullptr;
  // float64 matrices
  double *Mv = nullptr, *Kv = nullptr, *Av = nullptr, *MdKv = nullptr, *MsKv = nullptr;
  double *dM = nullptr, *dMdK = nullptr, *dMsK = nullptr;
  // inner (float32 / float16) matrices and float32 Jacobi inverses
  void *iM = nullptr, *iK = nullptr, *iMdK = nullptr, *iMsK = nullptr;
  float *fdM = nullptr, *fdMdK = nullptr, *fdMsK = nullptr;
  // vectors in internal order
  double *xk = nullptr, *xi = nullptr, *ys = nullptr, *bv = nullptr, *xnew = nullptr, *tmp3 = nullptr;
  double *dvec = nullptr, *lvec = nullptr, *tmpn = nullptr, *ebuf = nullptr;
  double *V = nullptr, *Z = nullptr;
  void* ivec = nullptr;
  // control
  unsigned* arrive = nullptr;
  int* errw = nullptr;
  double4_32a* part = nullptr;
  pfc::DevStats* stats = nullptr;   // 4 slots
  double* step_part = nullptr;
  double* err_scalar = nullptr;
  double* kappa = nullptr;      // {error / residual ratio, tau} of the last error-tested solve

  // pinned host mirrors
  pfc::DevStats* h_stats = nullptr;
  double* h_err = nullptr;
  int* h_errw = nullptr;
  bool assembled = false;
  bool last_rejected = false;   // the previous pfc_step attempt was rejected
  int step_stage = -1;          // stage-wise step (pfc_step_begin): next stage 0..2, 3 = ready to finish
  bool fixed_grid = false;      // options.grid_blocks > 0: the solver always uses G blocks
  double tau = 0.0, delta = 0.0;
  double gamma = kGamma;        // scaling of the (1,1) block: Ros3Pw gamma, or 1 for the Euler system
  // PFC1 (model 1): second block row A10 = tau K_+(psi_k), A11 = M / gamma + tau F(mu_k),
  // the element mobility tensor, int phi_j per row, and the mean mobility M0
  int model = 2;
  double psi_min = -1.5;
  double m0 = 1.0;
  double *A10v = nullptr, *A11v = nullptr, *mob = nullptr, *wint = nullptr;
  // P(S_D): Jacobi inverse of diag(S_D) in float64 and float32
  double* dSD = nullptr;
  float* fdSD = nullptr;
  // batched launches: this instance's warp slice ranges for a segment of blk_b_G blocks
  std::vector<long long> slice_cost_prefix;   // host, nslices + 1
  int* blk_b = nullptr;                       // device, G * W + 1
  int* h_blk_b = nullptr;                     // pinned staging
  int blk_b_G = 0;
  // accounting: kernels launched, persistent-solver launches and their event time
  long long launches = 0, solver_launches = 0;
  double solver_ms = 0.0;
  bool timing = false;
  cudaEvent_t ev[4][2] = {};
  bool ev_pending[4] = {};
  std::string last_error;
};

namespace {

pfc_status fail(pfc_ctx* c, pfc_status st, const std::string& msg) {
  if (c) c->last_error = msg;
  return st;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(c, PFC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));      \
  } while (0)

// A kernel launch through one of the launch wrappers, counted per context.
#define LAUNCH(call)  \
  do {                \
    CK(call);         \
    c->launches += 1; \
  } while (0)

size_t inner_elem_bytes(int prec) { return prec == 1 ? 4 : prec == 2 ? 2 : 8; }

pfc::SolveArgs base_args(pfc_ctx* c, int prec) {
  pfc::SolveArgs a{};
  a.n_pad = c->n_pad;
  a.slice_ptr = c->slice_ptr;
  a.cols = c->cols;
  a.blk = c->blk;
  a.Mv = c->Mv;
  a.Kv = c->Kv;
  a.Av = c->Av;
  a.A10 = c->model == 1 ? c->A10v : nullptr;
  a.schur = c->opt.schur;
  a.schur_its = c->opt.schur_its;
  a.dSD = prec == 0 ? (const void*)c->dSD : (const void*)c->fdSD;
  a.A11 = c->model == 1 ? c->A11v : nullptr;
  if (prec == 0) {
    a.iM = c->Mv;
    a.iK = c->Kv;
    a.iMdK = c->MdKv;
    a.iMsK = c->MsKv;
    a.dM = c->dM;
    a.dMdK = c->dMdK;
    a.dMsK = c->dMsK;
  } else {
    a.iM = c->iM;
    a.iK = c->iK;
    a.iMdK = c->iMdK;
    a.iMsK = c->iMsK;
    a.dM = c->fdM;
    a.dMdK = c->fdMdK;
    a.dMsK = c->fdMsK;
  }
  a.tau = c->tau;
  a.gamma = c->gamma;
  a.inv_gamma = 1.0 / c->gamma;
  a.tau_e = c->gamma * c->tau * c->m0;  // PFC1: constant-mobility approximation K_+ ~ M0 K
  a.inv_delta = c->delta > 0 ? 1.0 / c->delta : 0.0;
  a.tol = c->opt.outer_tol;
  a.err_tol = c->opt.err_tol;
  a.kappa = c->kappa;
  a.inner_rtol = c->opt.inner_rtol;
  a.restart = c->opt.restart;
  a.max_outer = c->opt.max_outer;
  a.max_inner = c->opt.max_inner;
  a.V = c->V;
  a.Z = c->Z;
  a.ivec = c->ivec;
  a.arrive = c->arrive;
  a.err = c->errw;
  a.part = c->part;
  a.stats = c->stats;
  a.spin_limit_ns = 2000000000ULL;
  a.barrier_extra = 0;
  // 2 = automatic: the pipelined form in float64; the Chronopoulos-Gear form in
  // float32/float16, where the pipelined recurrences drift and cost outer iterations
  a.pcg_variant = c->opt.pcg_variant == 2 ? (prec == 0 ? 1 : 3) : c->opt.pcg_variant;
  a.stencil = c->opt.inner_operator == 1 ? 1 : 0;
  a.rowinfo = c->rowinfo;
  a.st_start = c->st_start;
  a.st_off = c->st_off;
  a.st_wM = c->st_wM;
  a.st_wK = c->st_wK;
  a.st_types = c->st_types;
  a.st_halo = c->st_halo;
  a.win_cap = c->win_cap;
  a.tma = c->tma;
  a.lat = c->tma_lat;
  a.plane = c->tma_plane;
  a.tma_S = c->tma_S;
  a.tma_cap = c->tma_cap;
  const double cK[4] = {0.0, 1.0, c->delta, std::sqrt(c->delta)};
  const double cM[4] = {1.0, 0.0, 1.0, 1.0};
  for (int k = 0; k < 4; ++k) {
    a.op_cK[k] = cK[k];
    a.op_cM[k] = cM[k];
  }
  a.cells = (prec != 0 && c->cell_ok) ? 1 : 0;
  a.cell_S = c->cell_S;
  a.cell_dim = c->dim;
  a.cell_gx = c->cell_gx;
  a.cell_gz = c->cell_gz;
  a.cell_gy = c->cell_gy;
  a.cell_wcap = c->cell_wcap;
  a.cell_ccap = c->cell_ccap;
  a.cell_rcap = c->cell_rcap;
  a.ccls_n = c->ccls_n;
  a.ccls_wM = c->ccls_wM;
  a.ccls_wK = c->ccls_wK;
  a.cellclass = c->cellclass;
  for (int t = 0; t < 8; ++t) a.cell_rep[t] = c->cell_rep[t];
  a.prof = c->timing ? 1 : 0;
  return a;
}

// Tables of the cell kernels built on the host from the row classes.
struct CellTables {
  int ncc = 0;                          // cell classes (class 0: every row interior)
  std::vector<unsigned char> cellclass; // n_pad / 2^dim
  std::vector<double> wM, wK;           // ncc x couplings (46 in 2D, 230 in 3D)
  int rep[8] = {-1, -1, -1, -1, -1, -1, -1, -1};   // an interior row of each dof type
};

// The hard-coded couplings of an interior cell (cell2d.h, cell3d.h): output row type t,
// source cell q at cell offset (dx, dy, dz), source row sub.
struct CellEnt {
  int t, q, sub;
};
const std::vector<CellEnt>& cell_entries(int dim) {
  static const std::vector<CellEnt> e2 = {
#define PFC_CELL_ENT(t, q, sub) {t, q, sub},
      PFC_CELL2D_ENTRIES(PFC_CELL_ENT)};
  static const std::vector<CellEnt> e3 = {
#define PFC_CELL_NOP(q)
      PFC_CELL3D_ENTRIES(PFC_CELL_ENT, PFC_CELL_NOP)};
#undef PFC_CELL_NOP
#undef PFC_CELL_ENT
  return dim == 2 ? e2 : e3;
}

// Whether the cell kernels may run on this cell-major setup, and their tables: the
// interior stencil of each dof type must be exactly its couplings in cell2d.h /
// cell3d.h, and every other row's stencil a subset of the couplings of its type (true
// for the rows on the sides of a structured mesh, whose elements are a subset of an
// interior row's).  A cell's class is the tuple of its rows' classes; its weights are
// those of the couplings, 0 where a row lacks one.  At most 255 classes.
bool cell_pattern_ok(const pfc::HostSetup& S, CellTables* out) {
  const int nt = S.ntypes_dof, dim = S.dim;
  const int ncls = (int)S.cls_start.size() - 1;
  if (!S.cells || nt != (1 << dim) || ncls > 255) return false;
  const std::vector<CellEnt>& tab = cell_entries(dim);
  static const int dx2[] = PFC_CELL2D_DX, dy2[] = PFC_CELL2D_DY;
  static const int dx3[] = PFC_CELL3D_DX, dy3[] = PFC_CELL3D_DY, dz3[] = PFC_CELL3D_DZ;
  const long long cs = S.cell_S;
  const int E = (int)tab.size();
  std::vector<long long> off(E);
  for (int e = 0; e < E; ++e) {
    const int q = tab[e].q;
    const long long dc = dim == 2 ? dy2[q] * cs + dx2[q] : (dz3[q] * cs + dy3[q]) * cs + dx3[q];
    off[e] = nt * dc + tab[e].sub - tab[e].t;
  }
  // the interior stencils have exactly the couplings of their type
  for (int t = 0; t < nt; ++t) {
    int count = 0;
    for (int e = 0; e < E; ++e) {
      if (tab[e].t != t) continue;
      ++count;
      bool found = false;
      for (int j = S.cls_start[t]; j < S.cls_start[t + 1]; ++j) found = found || S.cls_off[j] == off[e];
      if (!found) return false;
    }
    if (count != S.cls_start[t + 1] - S.cls_start[t]) return false;
  }
  CellTables T;
  std::map<uint64_t, int> ids;
  auto row_class = [&](uint64_t key, int t) { return (int)((key >> (8 * t)) & 255u); };
  auto add_class = [&](uint64_t key) -> bool {
    for (int t = 0; t < nt; ++t) {
      const int k = row_class(key, t);
      int used = 0;
      for (int e = 0; e < E; ++e) {
        if (tab[e].t != t) continue;
        for (int j = S.cls_start[k]; j < S.cls_start[k + 1]; ++j)
          if (S.cls_off[j] == off[e]) ++used;
      }
      if (used != S.cls_start[k + 1] - S.cls_start[k]) return false;   // a coupling outside the pattern
    }
    for (int e = 0; e < E; ++e) {
      const int k = row_class(key, tab[e].t);
      double m = 0.0, kk = 0.0;
      for (int j = S.cls_start[k]; j < S.cls_start[k + 1]; ++j)
        if (S.cls_off[j] == off[e]) {
          m = S.cls_wM[j];
          kk = S.cls_wK[j];
        }
      T.wM.push_back(m);
      T.wK.push_back(kk);
    }
    const int id = (int)ids.size();
    ids.emplace(key, id);
    return true;
  };
  uint64_t interior = 0;
  for (int t = 0; t < nt; ++t) interior |= (uint64_t)t << (8 * t);
  if (!add_class(interior)) return false;
  const int ncell = S.n_pad / nt;
  T.cellclass.resize(ncell);
  for (int c = 0; c < ncell; ++c) {
    uint64_t key = 0;
    for (int t = 0; t < nt; ++t) key |= (uint64_t)S.rowclass[(size_t)nt * c + t] << (8 * t);
    auto it = ids.find(key);
    if (it == ids.end()) {
      if (ids.size() >= 255 || !add_class(key)) return false;
      it = ids.find(key);
    }
    T.cellclass[c] = (unsigned char)it->second;
    if (it->second == 0 && T.rep[0] < 0)
      for (int t = 0; t < nt; ++t) T.rep[t] = nt * c + t;
  }
  if (T.rep[0] < 0) return false;   // no interior cell
  T.ncc = (int)ids.size();
  if (out) *out = std::move(T);
  return true;
}

// Tiles of the cell kernels for a grid of G blocks: gx x gy (x gz) <= G boxes of the
// cell grid (S cells per axis; block b owns tile (b % gx, (b / gx) % gy, b / (gx gy))),
// chosen to minimise the work of the largest tile: its cells plus its ring, which
// costs about 0.4 of an own cell (four reads against about ten accesses).  wcap: cells
// of the largest tile with its ring; ccap: of the largest tile; rcap: of the largest ring.
void cell_tiling(int dim, int S, int G, int& gx, int& gy, int& gz, int& wcap, int& ccap, int& rcap) {
  double best = 1e300;
  gx = gy = gz = 1;
  for (int z = 1; z <= (dim == 3 ? std::min(G, S) : 1); ++z) {
    for (int x = 1; x <= std::min(G / z, S); ++x) {
      const int y = std::min(G / (x * z), S);
      if (y < 1) break;
      const double tw = (S + x - 1) / x, th = (S + y - 1) / y, td = dim == 3 ? (S + z - 1) / z : 1;
      const double own = tw * th * td;
      const double ring = dim == 3 ? (tw + 2) * (th + 2) * (td + 2) - own : (tw + 2) * (th + 2) - own;
      const double cost = own + 0.4 * ring;
      if (cost < best) {
        best = cost;
        gx = x;
        gy = y;
        gz = z;
      }
    }
  }
  const int tw = (S + gx - 1) / gx, th = (S + gy - 1) / gy, td = dim == 3 ? (S + gz - 1) / gz : 1;
  wcap = (tw + 2) * (th + 2) * (dim == 3 ? td + 2 : 1);
  ccap = tw * th * td;
  rcap = wcap - ccap;
}

pfc_status status_from_err(int err) {
  if (err & pfc::kErrTimeout) return PFC_ERR_TIMEOUT;
  if (err & pfc::kErrNonfinite) return PFC_ERR_NONFINITE;
  if (err & pfc::kErrOuterCap) return PFC_ERR_NOT_CONVERGED;
  return PFC_OK;
}

// Lemma 3 (Section 6): the symbol of the linearised PFC2 operator about a constant
// density psi_bar reaches zero once the effective width gamma tau is at least
// tau* = 27 / (2 (sqrt(alpha) - 1)(sqrt(alpha) + 2)^2), alpha = 1 - 3 r - 9 psi_bar^2;
// for alpha <= 1 (psi_bar^2 >= -r / 3) there is no critical width (infinity).
double critical_tau(double r, double psi_bar) {
  const double alpha = 1.0 - 3.0 * r - 9.0 * psi_bar * psi_bar;
  if (!(alpha > 1.0)) return INFINITY;
  const double sa = std::sqrt(alpha);
  return 27.0 / (2.0 * (sa - 1.0) * (sa + 2.0) * (sa + 2.0));
}

// Mean density <psi^k> = (int psi^k) / |Omega| onto c->err_scalar[1] (after the step
// reduction has consumed c->step_part), for the width guard of pfc_step.
pfc_status enqueue_mean_psi(pfc_ctx* c) {
  const int parts = pfc::step_partials();
  LAUNCH(pfc::launch_dot_partials(c->n_pad, c->wint, c->xk + c->n_pad, c->step_part, parts, c->stream));
  LAUNCH(pfc::launch_sum_partials(parts, c->step_part, 1.0 / std::pow(c->length, c->dim), c->err_scalar + 1,
                                  c->stream));
  return PFC_OK;
}

bool width_guard_on(const pfc_ctx* c) { return c->opt.tau_guard > 0.0 && c->model == 2; }

// Upper bound of the next step width: tau_max, and with the guard on (PFC2)
// gamma tau <= tau_guard tau*(r, <psi^k>).
double width_cap(const pfc_ctx* c, double mean_psi) {
  double cap = c->opt.tau_max;
  if (width_guard_on(c)) cap = std::min(cap, c->opt.tau_guard * critical_tau(c->opt.r, mean_psi) / kGamma);
  return cap;
}

// Enqueue one persistent-kernel launch; stats go to c->stats[slot].
pfc_status run_solver(pfc_ctx* c, pfc::SolveArgs a, int prec, int slot) {
  a.stats = c->stats + slot;
  CK(cudaMemsetAsync(c->arrive, 0, sizeof(unsigned) * (4 + (size_t)c->G), c->stream));
  CK(cudaMemsetAsync(c->errw + slot, 0, sizeof(int), c->stream));
  CK(cudaMemsetAsync(a.stats, 0, sizeof(pfc::DevStats), c->stream));
  a.err = c->errw + slot;
  if (c->timing) CK(cudaEventRecord(c->ev[slot][0], c->stream));
  LAUNCH(pfc::launch_solve(prec, c->G, a, c->stream));
  c->solver_launches += 1;
  if (c->timing) {
    CK(cudaEventRecord(c->ev[slot][1], c->stream));
    c->ev_pending[slot] = true;
  }
  return PFC_OK;
}

// After a stream synchronisation: add the event time of the finished solver launches.
void harvest(pfc_ctx* c) {
  for (int k = 0; k < 4; ++k) {
    if (!c->ev_pending[k]) continue;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, c->ev[k][0], c->ev[k][1]) == cudaSuccess) c->solver_ms += ms;
    c->ev_pending[k] = false;
  }
}

void fill_stats(const pfc::DevStats& d, int err, pfc_solve_stats* s) {
  if (!s) return;
  s->outer_its = d.outer_its;
  s->restarts = d.restarts;
  s->inner_its = d.inner_its;
  s->inner_calls = d.inner_calls;
  s->inner_capped = d.inner_capped;
  s->rel_residual = d.rel_residual;
  s->status = status_from_err(err);
  for (int k = 0; k < 8; ++k) s->phase_ms[k] = d.prof_ns[k] * 1e-6;
  s->err_est = d.err_est;
  s->sigma_min = d.sigma;
}

// b^R from the stage value c->xi and (when with_d) d = sum c_ij dpsi_j in c->dvec:
// element loads (psi_i^3, phi) and, for PFC1, (psi_i^+ grad mu_i, grad phi), then
// the row kernel.
pfc_status rhs_at_stage(pfc_ctx* c, bool with_d) {
  const int np = c->n_pad;
  LAUNCH(pfc::launch_elem_load(c->nl, c->E, c->elem, c->xi + np, c->vol, c->ebuf, c->stream));
  double* lbuf2 = nullptr;
  if (c->model == 1) {
    lbuf2 = c->ebuf + (size_t)c->nl * c->E;
    LAUNCH(pfc::launch_elem_mobload(c->nl, c->E, c->ntypes, c->elem, c->xi + np, c->xi, c->psi_min, c->mob, lbuf2,
                                    c->stream));
  }
  LAUNCH(pfc::launch_rhs(c->nslices, c->slice_ptr, c->cols, c->Mv, c->Kv, c->dptr, c->didx, c->ebuf, c->xi,
                         with_d ? c->dvec : nullptr, c->opt.r, c->tau, lbuf2, c->bv, c->stream));
  return PFC_OK;
}

// b_i^R for stage nprev from c->xi (stage value) and the increments c->ys.
pfc_status stage_rhs_internal(pfc_ctx* c, int nprev) {
  const int np = c->n_pad;
  const double c0 = nprev > 0 ? kC[nprev][0] : 0.0, c1 = nprev > 1 ? kC[nprev][1] : 0.0;
  if (nprev > 0) LAUNCH(pfc::launch_combine_field(np, c->ys + np, c0, nprev > 1 ? c->ys + 3 * np + np : nullptr, c1, c->dvec, c->stream));
  return rhs_at_stage(c, nprev > 0);
}

// with_f: the Rosenbrock matrix (A11 = M / gamma + tau F(mu_k)); false for the Euler
// system, whose mobility is explicit (A11 = M).
pfc_status assemble_internal(pfc_ctx* c, double tau, double gamma = kGamma, bool with_f = true) {
  const int np = c->n_pad;
  LAUNCH(pfc::launch_elem_quartic(c->nl, c->E, c->elem, c->xk + np, c->vol, c->ebuf, c->stream));
  LAUNCH(pfc::launch_assemble_a01(c->nnz_sell, c->cptr, c->cidx, c->ebuf, c->Mv, c->Kv, c->opt.r, c->Av, c->stream));
  c->tau = tau;
  c->gamma = gamma;
  c->m0 = 1.0;
  if (c->model == 1) {
    // M0 = <psi_k^+> = (sum_j int phi_j psi_j) / |Omega| - psi_min
    const int parts = pfc::step_partials();
    LAUNCH(pfc::launch_dot_partials(np, c->wint, c->xk + np, c->step_part, parts, c->stream));
    LAUNCH(pfc::launch_sum_partials(parts, c->step_part, 1.0, c->err_scalar + 1, c->stream));
    CK(cudaMemcpyAsync(c->h_err + 1, c->err_scalar + 1, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const double omega = std::pow(c->length, c->dim);
    c->m0 = c->h_err[1] / omega - c->psi_min;
    if (!(c->m0 > 0.0) || !std::isfinite(c->m0))
      return fail(c, PFC_ERR_INVALID, "PFC1: the mean mobility <psi - psi_min> must be positive");
    LAUNCH(pfc::launch_elem_mobility(c->nl, c->E, c->ntypes, c->elem, c->xk + np, c->xk, c->psi_min, c->mob, c->ebuf,
                                     c->stream));
    LAUNCH(pfc::launch_assemble_mob(c->nl, c->nnz_sell, c->cptr, c->cidx, c->cols, c->elem, c->E, c->ebuf, c->Mv, tau,
                                    1.0 / gamma, with_f ? 1 : 0, c->A10v, c->A11v, c->stream));
  }
  c->delta = std::sqrt(gamma * tau * c->m0);
  if (c->opt.schur == 1)
    LAUNCH(pfc::launch_sd_diag_inv(c->nslices, c->slice_ptr, c->cols, c->Mv, c->Kv, c->diag, c->dM, c->delta, c->dSD,
                                   c->prec ? c->fdSD : nullptr, c->stream));
  const double sdelta = std::sqrt(c->delta);
  LAUNCH(pfc::launch_inner_mats(c->prec, c->nnz_sell, c->Mv, c->Kv, c->delta, sdelta, c->MdKv, c->MsKv, c->iMdK, c->iMsK,
                            c->stream));
  LAUNCH(pfc::launch_diag_inv(np, c->diag, c->MdKv, c->dMdK, c->prec ? c->fdMdK : nullptr, c->stream));
  LAUNCH(pfc::launch_diag_inv(np, c->diag, c->MsKv, c->dMsK, c->prec ? c->fdMsK : nullptr, c->stream));
  c->assembled = true;
  return PFC_OK;
}

pfc_status check_ctx(pfc_ctx* c) {
  if (!c) return PFC_ERR_INVALID;
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return fail(c, PFC_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  return PFC_OK;
}

// The end of a step attempt after its three stage solves (Eq. 3.6, 3.7):
// x^{k+1} and the embedded error estimate, one synchronisation, accept/reject,
// the next width.  Shared by pfc_step and pfc_step_finish.
pfc_status finish_step(pfc_ctx* c, double* state, double* tau, int* accepted, double* err, pfc_solve_stats* stats) {
  const int np = c->n_pad;
  const size_t np3 = 3 * (size_t)np;
  pfc_status st = PFC_OK;
  double e[3];
  for (int j = 0; j < 3; ++j) e[j] = kMhat[j] - kM[j];
  LAUNCH(pfc::launch_step_combine(np, c->xk, c->ys, c->ys + np3, c->ys + 2 * np3, kM, e, c->opt.step_atol, c->opt.step_rtol,
                              c->xnew, c->step_part, pfc::step_partials(), c->stream));
  LAUNCH(pfc::launch_reduce_partials(pfc::step_partials(), c->step_part, 1.0 / c->n, c->err_scalar, c->stream));
  if (width_guard_on(c)) {
    st = enqueue_mean_psi(c);
    if (st != PFC_OK) return st;
  }
  CK(cudaMemcpyAsync(c->h_stats, c->stats, sizeof(pfc::DevStats) * 3, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(c->h_errw, c->errw, sizeof(int) * 3, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(c->h_err, c->err_scalar, sizeof(double) * 2, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  harvest(c);
  int werr = 0;
  for (int i = 0; i < 3; ++i) {
    fill_stats(c->h_stats[i], c->h_errw[i], stats ? stats + i : nullptr);
    werr |= c->h_errw[i];
  }
  const double ev = c->h_err[0];
  if (err) *err = ev;
  st = status_from_err(werr);
  if (st == PFC_ERR_TIMEOUT || st == PFC_ERR_NONFINITE || !std::isfinite(ev)) {
    if (accepted) *accepted = 0;
    return fail(c, st == PFC_OK ? PFC_ERR_NONFINITE : st, "step failed in a stage solve");
  }
  const bool acc = ev <= 1.0 && st == PFC_OK;
  if (accepted) *accepted = acc ? 1 : 0;
  if (acc) LAUNCH(pfc::launch_scatter_out(c->n, np, 3, c->perm, c->xnew, state, c->stream));
  double fac = ev == 0.0 ? 5.0 : std::min(5.0, std::max(0.2, 0.9 * std::pow(ev, -1.0 / 3.0)));
  if (acc && c->last_rejected) fac = std::min(fac, 1.0);  // no growth right after a rejection
  c->last_rejected = !acc;
  *tau = std::min(*tau * fac, width_cap(c, c->h_err[1]));
  if (st != PFC_OK) return fail(c, st, "a stage solve did not converge");
  return PFC_OK;
}

// ---------------------------------------------------------------- batches
// Device and pinned staging buffers of batched launches (per device, grown on demand).
struct BatchSpace {
  char* dev = nullptr;
  char* host = nullptr;
  size_t bytes = 0;
};
std::mutex g_batch_mutex;
BatchSpace g_batch[64];

pfc_status batch_space(pfc_ctx* c, size_t need, BatchSpace*& out) {
  BatchSpace& b = g_batch[c->device];
  if (b.bytes < need) {
    if (b.dev) {
      cudaStreamSynchronize(c->stream);
      cudaFree(b.dev);
      cudaFreeHost(b.host);
      b = BatchSpace{};
    }
    size_t bytes = std::max<size_t>(need, 1 << 16);
    if (cudaMalloc((void**)&b.dev, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, PFC_ERR_OOM, "batch workspace allocation failed");
    }
    if (cudaMallocHost((void**)&b.host, bytes) != cudaSuccess) {
      cudaFree(b.dev);
      b = BatchSpace{};
      return fail(c, PFC_ERR_OOM, "batch staging allocation failed");
    }
    b.bytes = bytes;
  }
  out = &b;
  return PFC_OK;
}

// Warp slice ranges of instance c for a segment of G blocks (cost balanced as at set-up).
pfc_status prepare_segment(pfc_ctx* c, int G) {
  if (c->blk_b_G == G) return PFC_OK;
  const int W = pfc::solve_threads() / 32;
  const std::vector<long long>& pre = c->slice_cost_prefix;
  auto split = [&](int lo, int hi, int parts, int* out) {
    out[0] = lo;
    int s = lo;
    for (int k = 1; k < parts; ++k) {
      const long long target = pre[lo] + (pre[hi] - pre[lo]) * k / parts;
      while (s < hi && pre[s] < target) ++s;
      out[k] = std::max(s, out[k - 1]);
    }
    out[parts] = hi;
  };
  // the staging buffer may still feed an earlier copy: wait for the stream first
  CK(cudaStreamSynchronize(c->stream));
  std::vector<int> bb(G + 1), wb(W + 1);
  split(0, c->nslices, G, bb.data());
  for (int b = 0; b < G; ++b) {
    split(bb[b], bb[b + 1], W, wb.data());
    for (int w = 0; w < W; ++w) c->h_blk_b[(size_t)b * W + w] = wb[w];
  }
  c->h_blk_b[(size_t)G * W] = c->nslices;
  CK(cudaMemcpyAsync(c->blk_b, c->h_blk_b, sizeof(int) * ((size_t)G * W + 1), cudaMemcpyHostToDevice, c->stream));
  c->blk_b_G = G;
  return PFC_OK;
}

// Splits `count` instances into waves that fit one co-resident grid and gives each
// instance a segment proportional to its rows (at least one block, at most its
// own grid).  Returns the waves as [first, last) instance ranges with block counts.
void plan_segments(pfc_ctx* const* ctxs, int count, int max_blocks, std::vector<int>& Gs,
                   std::vector<std::pair<int, int>>& waves) {
  Gs.assign(count, 1);
  waves.clear();
  bool fixed = true;
  for (int k = 0; k < count; ++k) fixed = fixed && ctxs[k]->fixed_grid;
  if (fixed) {
    // every instance keeps its own block count (its partition, hence its results, do not
    // depend on the rest of the batch); waves fill the co-resident grid in order
    int lo = 0, used = 0;
    for (int k = 0; k < count; ++k) {
      Gs[k] = std::min(ctxs[k]->G, max_blocks);
      if (k > lo && used + Gs[k] > max_blocks) {
        waves.emplace_back(lo, k);
        lo = k;
        used = 0;
      }
      used += Gs[k];
    }
    waves.emplace_back(lo, count);
    return;
  }
  for (int lo = 0; lo < count; lo += max_blocks) {
    const int hi = std::min(count, lo + max_blocks);
    long long rows = 0;
    for (int k = lo; k < hi; ++k) rows += ctxs[k]->n_pad;
    int spare = max_blocks - (hi - lo);
    // proportional shares, capped by each instance's own grid, in a few rounds
    for (int round = 0; round < 4 && spare > 0; ++round) {
      long long w = 0;
      for (int k = lo; k < hi; ++k)
        if (Gs[k] < ctxs[k]->G) w += ctxs[k]->n_pad;
      if (w == 0) break;
      int given = 0;
      for (int k = lo; k < hi; ++k) {
        if (Gs[k] >= ctxs[k]->G) continue;
        int add = (int)((long long)spare * ctxs[k]->n_pad / w);
        add = std::min(add, ctxs[k]->G - Gs[k]);
        Gs[k] += add;
        given += add;
      }
      spare -= given;
      if (given == 0) break;
    }
    (void)rows;
    waves.emplace_back(lo, hi);
  }
}

// Enqueues the batched FGMRES solves for every instance: b = ctx->bv, y = ys + slot * 3 n_pad
// (or tmp3 when to_tmp), stats and error word in `slot`, with slot = slots[k] of the
// instance (its own stage) or the common `slot` when slots is null.
pfc_status run_batch(pfc_ctx* const* ctxs_in, int count, int slot, bool to_tmp, BatchSpace* space, size_t region,
                     const int* slots = nullptr) {
  // Instances are taken largest first, so that when they need several waves each wave
  // holds instances of similar size (a wave lasts as long as its largest solve).  All
  // outputs are per context, so the order changes nothing else.
  std::vector<int> idx(count);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return ctxs_in[x]->n_pad > ctxs_in[y]->n_pad; });
  std::vector<pfc_ctx*> order(count);
  std::vector<int> slot_of(count);
  for (int k = 0; k < count; ++k) {
    order[k] = ctxs_in[idx[k]];
    slot_of[k] = slots ? slots[idx[k]] : slot;
  }
  pfc_ctx* const* ctxs = order.data();
  pfc_ctx* c0 = ctxs[0];      // stream, device and precision are shared by all
  pfc_ctx* c = ctxs_in[0];    // errors are reported on the caller's first context
  int occ = 0;
  CK(pfc::batch_occupancy(c0->prec, &occ, 0));
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c0->device));
  int bps = occ;
  if (c0->opt.blocks_per_sm > 0) bps = std::min(bps, c0->opt.blocks_per_sm);
  const int max_blocks = std::min(sms * bps, pfc::solve_threads());
  if (max_blocks < 1) return fail(c0, PFC_ERR_CUDA, "batched solver does not fit on an SM");
  std::vector<int> Gs;
  std::vector<std::pair<int, int>> waves;
  plan_segments(ctxs, count, max_blocks, Gs, waves);
  for (int k = 0; k < count; ++k) {
    pfc_status st = prepare_segment(ctxs[k], Gs[k]);
    if (st != PFC_OK) return st;
  }
  char* hbase = space->host + region;
  char* dbase = space->dev + region;
  size_t off = 0;
  for (const auto& wv : waves) {
    const int n = wv.second - wv.first;
    pfc::SolveArgs* hargs = (pfc::SolveArgs*)(hbase + off);
    int* hseg = (int*)(hbase + off + sizeof(pfc::SolveArgs) * n);
    hseg[0] = 0;
    // cell kernels: the wave's dynamic shared memory holds the widest tile window among
    // the instances that can have one at the residency the wave needs (in their segment
    // partition); an instance whose window does not fit takes the per-warp form
    std::vector<size_t> needs(n, 0);
    size_t dyn = 0;
    {
      for (int i = 0; i < n; ++i) {
        pfc_ctx* ck = ctxs[wv.first + i];
        if (!(ck->prec != 0 && ck->cell_ok)) continue;
        int gx = 0, gy = 0, gz = 0, wcap = 0, ccap = 0, rcap = 0;
        cell_tiling(ck->dim, ck->cell_S, Gs[wv.first + i], gx, gy, gz, wcap, ccap, rcap);
        needs[i] = pfc::cell_smem_bytes(wcap, ck->dim == 3 ? 2 : 1, rcap, ck->ccls_n, ck->dim == 3 ? 232 : 48, ccap);
      }
      std::vector<size_t> cand(needs.begin(), needs.end());
      std::sort(cand.begin(), cand.end(), std::greater<size_t>());
      int blocks = 0;
      for (int i = 0; i < n; ++i) blocks += Gs[wv.first + i];
      const int need_bps = (blocks + sms - 1) / sms;
      for (size_t k = 0; k < cand.size() && cand[k] > 0; ++k) {
        if (k > 0 && cand[k] == cand[k - 1]) continue;
        int occ_c = 0;
        const bool ok = pfc::batch_occupancy(c0->prec, &occ_c, cand[k]) == cudaSuccess && occ_c >= need_bps;
        cudaGetLastError();
        if (ok) {
          dyn = cand[k];
          break;
        }
      }
    }
    for (int i = 0; i < n; ++i) {
      pfc_ctx* ck = ctxs[wv.first + i];
      c = ck;
      pfc::SolveArgs a = base_args(ck, ck->prec);
      a.win_cap = 0;  // segments of different instances: no shared-memory window
      a.tma = 0;
      a.mode = 0;
      const int sk = slot_of[wv.first + i];
      a.b = ck->bv;
      a.y = to_tmp ? ck->tmp3 : ck->ys + (size_t)sk * 3 * ck->n_pad;
      a.blk = ck->blk_b;
      if (a.cells) {
        if (needs[i] > 0 && needs[i] <= dyn)
          cell_tiling(ck->dim, ck->cell_S, Gs[wv.first + i], a.cell_gx, a.cell_gy, a.cell_gz, a.cell_wcap,
                      a.cell_ccap, a.cell_rcap);
        else a.cells = 0;
      }
      a.stats = ck->stats + sk;
      a.err = ck->errw + sk;
      hargs[i] = a;
      hseg[i + 1] = hseg[i] + Gs[wv.first + i];
      CK(cudaMemsetAsync(ck->arrive, 0, sizeof(unsigned) * (4 + (size_t)ck->G), ck->stream));
      CK(cudaMemsetAsync(ck->errw + sk, 0, sizeof(int), ck->stream));
      CK(cudaMemsetAsync(ck->stats + sk, 0, sizeof(pfc::DevStats), ck->stream));
    }
    c = ctxs_in[0];
    const size_t bytes = sizeof(pfc::SolveArgs) * n + sizeof(int) * (n + 1);
    CK(cudaMemcpyAsync(dbase + off, hbase + off, bytes, cudaMemcpyHostToDevice, c0->stream));
    pfc::BatchArgs ba;
    ba.inst = (const pfc::SolveArgs*)(dbase + off);
    ba.seg = (const int*)(dbase + off + sizeof(pfc::SolveArgs) * n);
    ba.count = n;
    CK(pfc::launch_solve_batch(c0->prec, hseg[n], ba, c0->stream, dyn));
    c0->launches += 1;
    c0->solver_launches += 1;
    off += (bytes + 255) & ~size_t(255);
  }
  return PFC_OK;
}

size_t batch_region_bytes(int count) {
  return ((sizeof(pfc::SolveArgs) + sizeof(int)) * (size_t)count + 256 * ((size_t)count + 2) + 255) & ~size_t(255);
}

pfc_status check_batch(pfc_ctx* const* ctxs, int count) {
  if (!ctxs || count < 1) return PFC_ERR_INVALID;
  for (int k = 0; k < count; ++k)
    if (!ctxs[k]) return PFC_ERR_INVALID;
  pfc_ctx* c = ctxs[0];
  pfc_status st = check_ctx(c);
  if (st != PFC_OK) return st;
  for (int k = 1; k < count; ++k) {
    if (ctxs[k]->device != c->device || ctxs[k]->stream != c->stream || ctxs[k]->prec != c->prec)
      return fail(c, PFC_ERR_INVALID, "batched contexts must share device, stream and precision");
    for (int j = 0; j < k; ++j)
      if (ctxs[j] == ctxs[k]) return fail(c, PFC_ERR_INVALID, "a context appears twice in a batch");
  }
  return PFC_OK;
}

}  // namespace

extern "C" {

void pfc_default_options(pfc_options* o) {
  if (!o) return;
  o->r = -0.4;
  o->outer_tol = 1e-10;
  o->inner_rtol = 1e-3;
  o->restart = 30;
  o->max_outer = 600;
  o->max_inner = 1000;
  o->precision = PFC_PREC_FP64;
  o->step_atol = 1e-3;
  o->step_rtol = 1e-3;
  o->tau_max = 1e9;
  o->blocks_per_sm = 0;
  o->pcg_variant = 2;
  o->inner_operator = 1;
  o->smem_window = 0;
  o->model = 2;
  o->psi_min = -1.5;
  o->schur = 0;
  o->schur_its = 20;
  o->degree = 2;
  o->err_tol = 1e-9;
  o->tau_guard = 0.0;
  o->grid_blocks = 0;
  o->cells = 1;
}

double pfc_critical_tau(double r, double psi_bar) { return critical_tau(r, psi_bar); }

const char* pfc_status_string(int s) {
  switch (s) {
    case PFC_OK: return "PFC_OK";
    case PFC_ERR_INVALID: return "PFC_ERR_INVALID";
    case PFC_ERR_OOM: return "PFC_ERR_OOM";
    case PFC_ERR_CUDA: return "PFC_ERR_CUDA";
    case PFC_ERR_NOT_CONVERGED: return "PFC_ERR_NOT_CONVERGED";
    case PFC_ERR_NONFINITE: return "PFC_ERR_NONFINITE";
    case PFC_ERR_TIMEOUT: return "PFC_ERR_TIMEOUT";
    default: return "PFC_UNKNOWN";
  }
}

const char* pfc_last_error(const pfc_ctx* c) {
  if (!c) return "null context";
  return c->last_error.c_str();
}

int64_t pfc_num_dofs(const pfc_ctx* c) { return c ? (int64_t)c->n : 0; }

size_t pfc_footprint_bytes(int dim, int side, const pfc_options* opt) {
  pfc_options o;
  pfc_default_options(&o);
  if (opt) o = *opt;
  if ((dim != 2 && dim != 3) || side < 1) return 0;
  return pfc::footprint_estimate(dim, side, o.restart, o.precision, o.degree == 1 ? 1 : 2, o.model == 1 ? 1 : 2);
}

void pfc_destroy(pfc_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  for (int k = 0; k < 4; ++k)
    for (int j = 0; j < 2; ++j)
      if (c->ev[k][j]) cudaEventDestroy(c->ev[k][j]);
  if (c->arena) cudaFree(c->arena);
  if (c->h_stats) cudaFreeHost(c->h_stats);
  delete c;
}

pfc_status pfc_setup_mesh(pfc_ctx** out, int dim, int side, double length, const pfc_options* opt,
                          void* cuda_stream) {
  if (!out) return PFC_ERR_INVALID;
  *out = nullptr;
  pfc_ctx* c = new (std::nothrow) pfc_ctx();
  if (!c) return PFC_ERR_OOM;
  pfc_default_options(&c->opt);
  if (opt) c->opt = *opt;
  auto bail = [&](pfc_status st) {
    if (st != PFC_OK) {
      *out = c;  // keep the context so that pfc_last_error can be read; caller destroys it
    }
    return st;
  };
  if ((dim != 2 && dim != 3) || side < 1 || !(length > 0.0))
    return bail(fail(c, PFC_ERR_INVALID, "dim must be 2 or 3, side >= 1, length > 0"));
  if (c->opt.restart < 1 || c->opt.restart > pfc::kMaxRestart)
    return bail(fail(c, PFC_ERR_INVALID, "restart must be in 1..40"));
  if (c->opt.precision < 0 || c->opt.precision > 2) return bail(fail(c, PFC_ERR_INVALID, "precision must be 0, 1 or 2"));
  if (c->opt.pcg_variant < 0 || c->opt.pcg_variant > 3)
    return bail(fail(c, PFC_ERR_INVALID, "pcg_variant must be 0, 1, 2 or 3"));
  if (c->opt.inner_operator < 0 || c->opt.inner_operator > 1)
    return bail(fail(c, PFC_ERR_INVALID, "inner_operator must be 0 or 1"));
  if (c->opt.smem_window < 0 || c->opt.smem_window > 2)
    return bail(fail(c, PFC_ERR_INVALID, "smem_window must be 0, 1 or 2"));
  if ((c->opt.model != 1 && c->opt.model != 2) || !std::isfinite(c->opt.psi_min))
    return bail(fail(c, PFC_ERR_INVALID, "model must be 1 (PFC1) or 2 (PFC2) and psi_min finite"));
  if ((c->opt.schur != 0 && c->opt.schur != 1) || c->opt.schur_its < 1)
    return bail(fail(c, PFC_ERR_INVALID, "schur must be 0 (S_CH) or 1 (S_D) and schur_its >= 1"));
  if (c->opt.degree != 1 && c->opt.degree != 2) return bail(fail(c, PFC_ERR_INVALID, "degree must be 1 or 2"));
  if (!(c->opt.err_tol >= 0.0) || !std::isfinite(c->opt.err_tol))
    return bail(fail(c, PFC_ERR_INVALID, "err_tol must be finite and >= 0"));
  if (!(c->opt.tau_guard >= 0.0) || !(c->opt.tau_guard < 1.0))
    return bail(fail(c, PFC_ERR_INVALID, "tau_guard must be in [0, 1)"));
  if (c->opt.grid_blocks < 0) return bail(fail(c, PFC_ERR_INVALID, "grid_blocks must be >= 0"));
  if (c->opt.cells != 0 && c->opt.cells != 1) return bail(fail(c, PFC_ERR_INVALID, "cells must be 0 or 1"));
  c->model = c->opt.model;
  c->psi_min = c->opt.psi_min;
  if (!(c->opt.outer_tol > 0.0) || !(c->opt.inner_rtol > 0.0) || c->opt.max_outer < 1 || c->opt.max_inner < 1)
    return bail(fail(c, PFC_ERR_INVALID, "tolerances must be > 0 and iteration caps >= 1"));
  c->stream = (cudaStream_t)cuda_stream;
  c->dim = dim;
  c->side = side;
  c->length = length;
  c->prec = c->opt.precision;
  {
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) return bail(fail(c, PFC_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e)));
  }

  pfc::HostSetup S;
  std::string err;
  const bool stencil = c->opt.inner_operator == 1;
  // Cell-major rows only where the cell kernels can run them (2D P2 structured
  // stencils, float32/float16 Chronopoulos-Gear inner solves, no staged window);
  // elsewhere, or when the checks below turn the kernels down, lexicographic rows
  // (the per-warp gathers of the other paths are faster in that order).
  bool try_cells = stencil && c->opt.cells && c->opt.degree == 2 && c->prec != 0 &&
                   c->opt.smem_window == 0 && (c->opt.pcg_variant == 2 || c->opt.pcg_variant == 3);
retry_layout:
  if (!pfc::build_setup(dim, side, length, S, err, stencil ? 1 : pfc::kSellSigma, c->opt.degree,
                        try_cells ? 1 : 0))
    return bail(fail(c, PFC_ERR_INVALID, err));
  if (stencil) {
    // the kernel pads every type to the longest stencil (rounded up to 4) and adds
    // one all-padding type
    int longest = 0;
    for (int t = 0; t < S.ntypes_dof; ++t) longest = std::max(longest, S.st_start[t + 1] - S.st_start[t]);
    const int stride = (longest + 3) & ~3;
    if (S.ntypes_dof > 8 || (S.ntypes_dof + 1) * stride > pfc::kMaxStencil)
      return bail(fail(c, PFC_ERR_INVALID, "structured stencil larger than the kernel's table"));
  }
  c->n = S.n;
  c->n_pad = S.n_pad;
  c->nslices = S.nslices;
  c->E = S.E;
  c->nl = S.nl;
  c->np = S.ref.npairs;
  c->ntypes = S.ntypes;
  c->nnz_sell = S.nnz_sell;
  c->nnz = S.nnz;
  c->ncontrib = (long long)S.contrib_idx.size();
  c->vol = S.ref.vol;

  // persistent grid: co-resident blocks, no more blocks than slices
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || sms < 1)
    return bail(fail(c, PFC_ERR_CUDA, "cannot query the SM count"));
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device);
  if (!coop) return bail(fail(c, PFC_ERR_CUDA, "device does not support cooperative launch"));
  int occ0 = 0, occ1 = 0;
  if (pfc::solve_occupancy(0, &occ0) != cudaSuccess) return bail(fail(c, PFC_ERR_CUDA, "occupancy query failed"));
  occ1 = occ0;
  if (c->prec != 0 && pfc::solve_occupancy(c->prec, &occ1) != cudaSuccess)
    return bail(fail(c, PFC_ERR_CUDA, "occupancy query failed"));
  int bps = std::min(occ0, occ1);
  if (c->opt.blocks_per_sm > 0) bps = std::min(bps, c->opt.blocks_per_sm);
  if (bps < 1) return bail(fail(c, PFC_ERR_CUDA, "solver kernel does not fit on an SM"));
  c->G = std::max(1, std::min(std::min(sms * bps, c->nslices), pfc::solve_threads()));
  if (c->opt.grid_blocks > 0) {
    c->G = std::min(c->G, c->opt.grid_blocks);
    c->fixed_grid = true;
  }
  // Slice ranges: blocks and, inside each block, warps get contiguous runs of
  // slices of equal cost, cost(slice) = 32 * (width + 10) ~ bytes of one SpMV
  // row plus the vector traffic of the inner iteration.  With structured stencils
  // a slice holding rows with a missing element (boundary rows, which read their
  // assembled SELL values and indices) costs kBoundaryExtra more per such row and
  // slot: in 3D whole lattice planes are boundary rows, and without the extra
  // weight the blocks holding them set the pace of every phase.
  constexpr long long kBoundaryExtra = PFC_BOUNDARY_COST;
  const int W = pfc::solve_threads() / 32;
  std::vector<int> blk((size_t)c->G * W + 1, 0);
  {
    std::vector<long long> pre(S.nslices + 1, 0);
    for (int s = 0; s < S.nslices; ++s) {
      const long long width = (S.slice_ptr[s + 1] - S.slice_ptr[s]) / 32;
      long long cost = 32 * width + PFC_VEC_COST;
      if (stencil) {
        int nb = 0;
        for (int l = 0; l < 32; ++l)
          if (!(S.rowinfo[(size_t)s * 32 + l] & 8)) ++nb;
        cost += kBoundaryExtra * nb * width;
        // cell kernels: every cell costs the same (its vector traffic and the couplings
        // of cell2d.h, with its class's weights)
        if (S.cells && c->prec != 0) cost = 64;
      }
      pre[s + 1] = pre[s] + cost;
    }
    auto split = [&](int lo, int hi, int parts, int* out) {  // out[0..parts]
      out[0] = lo;
      int s = lo;
      for (int k = 1; k < parts; ++k) {
        const long long target = pre[lo] + (pre[hi] - pre[lo]) * k / parts;
        while (s < hi && pre[s] < target) ++s;
        out[k] = std::max(s, out[k - 1]);
      }
      out[parts] = hi;
    };
    c->slice_cost_prefix = pre;
    std::vector<int> bb(c->G + 1);
    split(0, S.nslices, c->G, bb.data());
    for (int b = 0; b < c->G; ++b) {
      std::vector<int> wb(W + 1);
      split(bb[b], bb[b + 1], W, wb.data());
      for (int w = 0; w < W; ++w) blk[(size_t)b * W + w] = wb[w];
    }
    blk[(size_t)c->G * W] = S.nslices;
  }

  // Cell kernels (2D P2 rows in cell-major order): they run the Chronopoulos-Gear inner
  // solves of float32/float16 contexts without a staged window, once the host has
  // checked that the interior stencils it extracted are the couplings of cell2d.h,
  // that every other row's stencil stays inside the block window (one lattice line of
  // cells and one cell on each side), and that the window and tables of the widest
  // block fit in shared memory at the grid's residency.
  CellTables ct;
  if (S.cells) {
    c->cells = 1;
    c->cell_S = S.cell_S;
    bool ok = c->prec != 0 && c->opt.smem_window == 0 && (c->opt.pcg_variant == 2 || c->opt.pcg_variant == 3) &&
              cell_pattern_ok(S, &ct);
    if (ok) {
      c->ccls_n = ct.ncc;
      for (int t = 0; t < 8; ++t) c->cell_rep[t] = ct.rep[t];
      cell_tiling(dim, c->cell_S, c->G, c->cell_gx, c->cell_gy, c->cell_gz, c->cell_wcap, c->cell_ccap,
                  c->cell_rcap);
      const size_t dyn = pfc::cell_smem_bytes(c->cell_wcap, dim == 3 ? 2 : 1, c->cell_rcap, c->ccls_n,
                                              dim == 3 ? 232 : 48, c->cell_ccap);
      const int need = (c->G + sms - 1) / sms;
      int occ_c = 0;
      ok = pfc::solve_occupancy(c->prec, &occ_c, dyn) == cudaSuccess && occ_c >= need;
      cudaGetLastError();
    }
    c->cell_ok = ok ? 1 : 0;
  }
  if (S.cells && !c->cell_ok) {
    try_cells = false;
    c->cells = c->cell_S = c->ccls_n = 0;
    goto retry_layout;
  }

  // Shared-memory window of the stencil SpMV (float inner vectors): block b reads
  // the source vector on its rows [rs, re) widened by the stencil reach on both
  // sides, rounded out to multiples of 4 floats.  It is used only if the largest
  // window keeps the residency the grid was sized with.
  if (stencil) {
    for (int v : S.st_off) c->st_halo = std::max(c->st_halo, v < 0 ? -v : v);
  }
  if (stencil && c->prec != 0 && c->opt.smem_window == 1) {
    int winmax = 0;
    for (int b = 0; b < c->G; ++b) {
      const int rs = blk[(size_t)b * W] * 32, re = blk[(size_t)(b + 1) * W] * 32;
      const int lo = std::max(0, rs - c->st_halo) & ~3;
      const int hi = std::min(c->n_pad, (re + c->st_halo + 3) & ~3);
      winmax = std::max(winmax, hi - lo);
    }
    const int need = (c->G + sms - 1) / sms;  // blocks per SM the grid needs co-resident
    int occ_w = 0;
    if (winmax > 0 && pfc::solve_occupancy(c->prec, &occ_w, (size_t)winmax * sizeof(float)) == cudaSuccess &&
        occ_w >= need)
      c->win_cap = winmax;
    cudaGetLastError();
  }

  // Chunked windows (smem_window 2, float inner vectors): every block walks its rows
  // in chunks of one row per thread, and the source window of a chunk (its lattice
  // lines +- 2, in 3D in the five planes around it) is bulk-copied into one of two
  // shared-memory buffers.  Sizes: a chunk spans at most maxlines lines; 3D plane
  // segments sit S apart with S = plane (mod 4), so that each copy starts 16-byte
  // aligned.  Used only if two buffers keep the grid's residency.
  if (stencil && c->prec != 0 && c->opt.smem_window == 2 && !S.cells) {   // lexicographic lines only
    const int chunk = pfc::solve_threads();
    const long long lat = (long long)c->opt.degree * side + 1;
    const long long plane = dim == 3 ? lat * lat : 0;
    if (dim == 2 || plane >= chunk) {
      const long long maxlines = (chunk - 1) / lat + 2;
      const long long span = (maxlines + 4) * lat + 8;
      long long S = 0, cap = 0;
      if (dim == 2) {
        cap = (span + 8 + 3) & ~3LL;
      } else {
        S = span + 4;
        while (((S - plane) % 4 + 4) % 4 != 0) ++S;
        cap = (5 * S + 8 + 3) & ~3LL;
      }
      const size_t dyn = 2 * (size_t)cap * sizeof(float);
      const int need = (c->G + sms - 1) / sms;
      int occ_t = 0;
      if (pfc::solve_occupancy(c->prec, &occ_t, dyn) == cudaSuccess && occ_t >= need) {
        c->tma = 1;
        c->tma_lat = (int)lat;
        c->tma_plane = (int)plane;
        c->tma_S = (int)S;
        c->tma_cap = (int)cap;
      }
      cudaGetLastError();
    }
  }

  // ---- device layout (one allocation) ----
  const size_t np3 = 3 * (size_t)c->n_pad;
  const size_t ib = inner_elem_bytes(c->prec);
  Layout L;
  const size_t o_slice = L.take(sizeof(int) * (S.nslices + 1));
  const size_t o_cols = L.take(sizeof(int) * S.nnz_sell);
  const size_t o_diag = L.take(sizeof(int) * S.n_pad);
  const size_t o_perm = L.take(sizeof(int) * S.n_pad);
  const size_t o_elem = L.take(sizeof(int) * S.elem_int.size());
  const size_t o_cptr = L.take(sizeof(int) * S.contrib_ptr.size());
  const size_t o_cidx = L.take(sizeof(int) * std::max<size_t>(1, S.contrib_idx.size()));
  const size_t o_dptr = L.take(sizeof(int) * S.dof_ptr.size());
  const size_t o_didx = L.take(sizeof(int) * std::max<size_t>(1, S.dof_idx.size()));
  const size_t o_blk = L.take(sizeof(int) * blk.size());
  const size_t o_blkb = L.take(sizeof(int) * blk.size());
  const size_t o_ri = L.take(S.rowinfo.size());
  const size_t o_sts = L.take(sizeof(int) * std::max<size_t>(1, S.st_start.size()));
  const size_t o_sto = L.take(sizeof(int) * std::max<size_t>(1, S.st_off.size()));
  const size_t o_stm = L.take(sizeof(double) * std::max<size_t>(1, S.st_wM.size()));
  const size_t o_stk = L.take(sizeof(double) * std::max<size_t>(1, S.st_wK.size()));
  const size_t o_cm = L.take(sizeof(double) * std::max<size_t>(1, ct.wM.size()));
  const size_t o_ck = L.take(sizeof(double) * std::max<size_t>(1, ct.wK.size()));
  const size_t o_cc = L.take(std::max<size_t>(1, ct.cellclass.size()));
  const size_t o_mt = L.take(sizeof(double) * S.ref.mass.size());
  const size_t o_st = L.take(sizeof(double) * S.ref.stiff.size());
  const size_t vals = sizeof(double) * S.nnz_sell;
  const size_t o_M = L.take(vals), o_K = L.take(vals), o_A = L.take(vals), o_MdK = L.take(vals), o_MsK = L.take(vals);
  const size_t o_dM = L.take(sizeof(double) * c->n_pad), o_dMdK = L.take(sizeof(double) * c->n_pad),
               o_dMsK = L.take(sizeof(double) * c->n_pad);
  size_t o_iM = 0, o_iK = 0, o_iMdK = 0, o_iMsK = 0, o_f1 = 0, o_f2 = 0, o_f3 = 0;
  if (c->prec) {
    o_iM = L.take(ib * S.nnz_sell);
    o_iK = L.take(ib * S.nnz_sell);
    o_iMdK = L.take(ib * S.nnz_sell);
    o_iMsK = L.take(ib * S.nnz_sell);
    o_f1 = L.take(sizeof(float) * c->n_pad);
    o_f2 = L.take(sizeof(float) * c->n_pad);
    o_f3 = L.take(sizeof(float) * c->n_pad);
  }
  const size_t vec_begin = L.take(0);
  const size_t o_xk = L.take(sizeof(double) * np3), o_xi = L.take(sizeof(double) * np3),
               o_ys = L.take(sizeof(double) * np3 * 3), o_bv = L.take(sizeof(double) * np3),
               o_xnew = L.take(sizeof(double) * np3), o_tmp3 = L.take(sizeof(double) * np3);
  const size_t o_dvec = L.take(sizeof(double) * c->n_pad), o_lvec = L.take(sizeof(double) * c->n_pad),
               o_tmpn = L.take(sizeof(double) * c->n_pad);
  // element buffer: N(psi) pair values (PFC2); PFC1 needs 3 values per pair
  const size_t o_ebuf = L.take(sizeof(double) * (size_t)c->np * c->E * (c->model == 1 ? 3 : 1));
  const size_t o_V = L.take(sizeof(double) * np3 * (c->opt.restart + 1));
  const size_t o_Z = L.take(sizeof(double) * np3 * c->opt.restart);
  const size_t o_ivec = L.take((size_t)pfc::kInnerVecs * c->n_pad * 8);
  const size_t vec_end = L.take(0);
  // barrier counter (+3 spare words), then one phase flag per block (neighbour sync)
  const size_t o_arr = L.take(sizeof(unsigned) * (4 + (size_t)c->G));
  const size_t o_errw = L.take(sizeof(int) * 8);
  const size_t o_part = L.take(sizeof(double4_32a) * pfc::solve_ring() * c->G);
  const size_t o_stats = L.take(sizeof(pfc::DevStats) * 4);
  const size_t o_sp = L.take(sizeof(double) * pfc::step_partials());
  const size_t o_es = L.take(sizeof(double) * 2);
  const size_t o_kappa = L.take(sizeof(double) * 2);
  size_t o_a10 = 0, o_a11 = 0, o_mob = 0;
  if (c->model == 1) {
    o_a10 = L.take(sizeof(double) * S.nnz_sell);
    o_a11 = L.take(sizeof(double) * S.nnz_sell);
    o_mob = L.take(sizeof(double) * S.ref.mob.size());
  }
  const size_t o_wint = L.take(sizeof(double) * c->n_pad);
  const size_t o_dsd = L.take(sizeof(double) * c->n_pad);
  const size_t o_fdsd = L.take(sizeof(float) * c->n_pad);
  c->arena_bytes = L.take(0);
  {
    cudaError_t e = cudaMalloc((void**)&c->arena, c->arena_bytes);
    if (e != cudaSuccess) {
      c->arena = nullptr;
      cudaGetLastError();
      return bail(fail(c, PFC_ERR_OOM, "cudaMalloc of " + std::to_string(c->arena_bytes) + " bytes failed"));
    }
  }
  char* A = c->arena;
  c->slice_ptr = (int*)(A + o_slice);
  c->cols = (int*)(A + o_cols);
  c->diag = (int*)(A + o_diag);
  c->perm = (int*)(A + o_perm);
  c->elem = (int*)(A + o_elem);
  c->cptr = (int*)(A + o_cptr);
  c->cidx = (int*)(A + o_cidx);
  c->dptr = (int*)(A + o_dptr);
  c->didx = (int*)(A + o_didx);
  c->blk = (int*)(A + o_blk);
  c->blk_b = (int*)(A + o_blkb);
  c->rowinfo = (unsigned char*)(A + o_ri);
  c->st_start = (int*)(A + o_sts);
  c->st_off = (int*)(A + o_sto);
  c->st_wM = (double*)(A + o_stm);
  c->st_wK = (double*)(A + o_stk);
  c->st_types = stencil ? S.ntypes_dof : 0;
  c->ccls_wM = (double*)(A + o_cm);
  c->ccls_wK = (double*)(A + o_ck);
  c->cellclass = (unsigned char*)(A + o_cc);
  c->mass_tab = (double*)(A + o_mt);
  c->stiff_tab = (double*)(A + o_st);
  c->Mv = (double*)(A + o_M);
  c->Kv = (double*)(A + o_K);
  c->Av = (double*)(A + o_A);
  c->MdKv = (double*)(A + o_MdK);
  c->MsKv = (double*)(A + o_MsK);
  c->dM = (double*)(A + o_dM);
  c->dMdK = (double*)(A + o_dMdK);
  c->dMsK = (double*)(A + o_dMsK);
  if (c->prec) {
    c->iM = A + o_iM;
    c->iK = A + o_iK;
    c->iMdK = A + o_iMdK;
    c->iMsK = A + o_iMsK;
    c->fdM = (float*)(A + o_f1);
    c->fdMdK = (float*)(A + o_f2);
    c->fdMsK = (float*)(A + o_f3);
  }
  c->xk = (double*)(A + o_xk);
  c->xi = (double*)(A + o_xi);
  c->ys = (double*)(A + o_ys);
  c->bv = (double*)(A + o_bv);
  c->xnew = (double*)(A + o_xnew);
  c->tmp3 = (double*)(A + o_tmp3);
  c->dvec = (double*)(A + o_dvec);
  c->lvec = (double*)(A + o_lvec);
  c->tmpn = (double*)(A + o_tmpn);
  c->ebuf = (double*)(A + o_ebuf);
  c->V = (double*)(A + o_V);
  c->Z = (double*)(A + o_Z);
  c->ivec = (void*)(A + o_ivec);
  c->arrive = (unsigned*)(A + o_arr);
  c->errw = (int*)(A + o_errw);
  c->part = (double4_32a*)(A + o_part);
  c->stats = (pfc::DevStats*)(A + o_stats);
  c->step_part = (double*)(A + o_sp);
  c->err_scalar = (double*)(A + o_es);
  c->kappa = (double*)(A + o_kappa);
  c->wint = (double*)(A + o_wint);
  c->dSD = (double*)(A + o_dsd);
  c->fdSD = (float*)(A + o_fdsd);
  if (c->model == 1) {
    c->A10v = (double*)(A + o_a10);
    c->A11v = (double*)(A + o_a11);
    c->mob = (double*)(A + o_mob);
  }
  {
    cudaError_t e = cudaMallocHost((void**)&c->h_stats, sizeof(pfc::DevStats) * 4 + sizeof(double) * 2 + sizeof(int) * 8 +
                                                         sizeof(int) * blk.size());
    if (e != cudaSuccess) return bail(fail(c, PFC_ERR_OOM, "cudaMallocHost failed"));
    c->h_err = (double*)(c->h_stats + 4);
    c->h_errw = (int*)(c->h_err + 2);
    c->h_blk_b = c->h_errw + 8;
  }

  for (int k = 0; k < 4; ++k)
    for (int j = 0; j < 2; ++j)
      if (cudaEventCreate(&c->ev[k][j]) != cudaSuccess) return bail(fail(c, PFC_ERR_CUDA, "cudaEventCreate failed"));

  // ---- uploads ----
#define UP(dst, vec) CK_SETUP(cudaMemcpy(dst, vec.data(), sizeof(vec[0]) * vec.size(), cudaMemcpyHostToDevice))
#define CK_SETUP(call)                                                                         \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return bail(fail(c, PFC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_))); \
  } while (0)
  UP(c->slice_ptr, S.slice_ptr);
  UP(c->cols, S.cols);
  UP(c->diag, S.diag_pos);
  UP(c->perm, S.perm);
  UP(c->elem, S.elem_int);
  UP(c->cptr, S.contrib_ptr);
  if (!S.contrib_idx.empty()) UP(c->cidx, S.contrib_idx);
  UP(c->dptr, S.dof_ptr);
  if (!S.dof_idx.empty()) UP(c->didx, S.dof_idx);
  UP(c->blk, blk);
  UP(c->rowinfo, S.rowinfo);
  if (stencil) {
    UP(c->st_start, S.st_start);
    UP(c->st_off, S.st_off);
    UP(c->st_wM, S.st_wM);
    UP(c->st_wK, S.st_wK);
  }
  if (c->cell_ok) {
    UP(c->ccls_wM, ct.wM);
    UP(c->ccls_wK, ct.wK);
    UP(c->cellclass, ct.cellclass);
  }
  UP(c->mass_tab, S.ref.mass);
  UP(c->stiff_tab, S.ref.stiff);
  {
    std::lock_guard<std::mutex> lk(g_const_mutex);
    const int di = (dim - 2) + (S.degree == 1 ? 2 : 0);
    if (c->device < 0 || c->device >= 64) return bail(fail(c, PFC_ERR_INVALID, "device index out of range"));
    if (!g_const_done[di][c->device]) {
      std::vector<double> unit(S.ref.quartic.size());
      for (size_t q = 0; q < unit.size(); ++q) unit[q] = S.ref.quartic[q] / S.ref.vol;
      CK_SETUP(pfc::upload_quartic(S.nl, unit.data(), S.ref.npairs));
      CK_SETUP(pfc::upload_pairs(S.nl, S.ref.pair_j.data(), S.ref.npairs));
      g_const_done[di][c->device] = true;
    }
  }
  CK_SETUP(cudaMemsetAsync(A + vec_begin, 0, vec_end - vec_begin, c->stream));
  CK_SETUP(cudaMemsetAsync(A + o_arr, 0, c->arena_bytes - o_arr, c->stream));
  // the mobility tensor lies in the zeroed tail: upload it after, on the same stream
  if (c->model == 1)
    CK_SETUP(cudaMemcpyAsync(c->mob, S.ref.mob.data(), sizeof(double) * S.ref.mob.size(), cudaMemcpyHostToDevice,
                             c->stream));
  CK_SETUP(pfc::launch_assemble_mk(c->nnz_sell, c->cptr, c->cidx, c->E, c->ntypes, c->np, c->mass_tab, c->stiff_tab,
                                   c->Mv, c->Kv, c->stream));
  CK_SETUP(pfc::launch_diag_inv(c->n_pad, c->diag, c->Mv, c->dM, c->prec ? c->fdM : nullptr, c->stream));
  // int phi_j = row sums of M (padding rows: 0), for the mean mobility of PFC1
  CK_SETUP(pfc::launch_row_sums(c->nslices, c->slice_ptr, c->Mv, c->wint, c->stream));
  if (c->prec) {
    CK_SETUP(pfc::launch_convert(c->prec, c->nnz_sell, c->Mv, c->iM, c->stream));
    CK_SETUP(pfc::launch_convert(c->prec, c->nnz_sell, c->Kv, c->iK, c->stream));
  }
  CK_SETUP(cudaStreamSynchronize(c->stream));
#undef UP
#undef CK_SETUP
  *out = c;
  return PFC_OK;
}

pfc_status pfc_assemble(pfc_ctx* c, const double* state, double tau) {
  pfc_status st = check_ctx(c);
  if (st != PFC_OK) return st;
  if (!state || !(tau > 0.0) || !std::isfinite(tau)) return fail(c, PFC_ERR_INVALID, "state must be non-null and tau > 0");
  c->step_stage = -1;
  LAUNCH(pfc::launch_gather_in(c->n, c->n_pad, 3, c->perm, state, c->xk, c->stream));
  return assemble_internal(c, tau);
}

pfc_status pfc_stage_rhs(pfc_ctx* c, int nprev, const double* x_stage, const double* y_prev, double* b) {
  pfc_status st = check_ctx(c);
  if (st != PFC_OK) return st;
  if (!c->assembled) return fail(c, PFC_ERR_INVALID, "pfc_assemble must come first");
  if (nprev < 0 || nprev > 2 || !x_stage || !b || (nprev > 0 && !y_prev))
    return fail(c, PFC_ERR_INVALID, "bad stage_rhs arguments");
  const size_t n3 = 3 * (size_t)c->n;
  LAUNCH(pfc::launch_gather_in(c->n, c->n_pad, 3, c->perm, x_stage, c->xi, c->stream));
  for (int j = 0; j < nprev; ++j)
    LAUNCH(pfc::launch_gather_in(c->n, c->n_pad, 3, c->perm, y_prev + j * n3, c->ys + (size_t)j * 3 * c->n_pad, c->stream));
  st = stage_rhs_internal(c, nprev);
  if (st != PFC_OK) return st;
  LAUNCH(pfc::launch_scatter_out(c->n, c->n_pad, 3, c->perm, c->bv, b, c->stream));
  return PFC_OK;
}

pfc_status pfc_stage_solve(pfc_ctx* c, const double* b, double* y, pfc_solve_stats* stats) {
  pfc_status st = check_ctx(c);
  if (st != PFC_OK) return st;
  if (!c->assembled) return fail(c, PFC_ERR_INVALID, "pfc_assemble must come first");
  if (!b || !y) return fail(c, PFC_ERR_INVALID, "null vector");
  LAUNCH(pfc::launch_gather_in(c->n, c->n_pad, 3, c->perm, b, c->bv, c->stream));
  std::unique_lock<std::mutex> lk(g_batch_mutex, std::defer_lock);
  if (c->fixed_grid) {
    // fixed block count: the batched kernel, as in every batch (same bits alone and batched)
    lk.lock();
    BatchSpace* space = nullptr;
    st = batch_space(c, batch_region_bytes(1), space);
    if (st != PFC_OK) return st;
    pfc_ctx* one[1] = {c};
    st = run_batch(one, 1, 0, true, space, 0);
  } else {
    pfc::SolveArgs a = base_args(c, c->prec);
    a.mode = 0;
    a.b = c->bv;
    a.y = c->tmp3;
    st = run_solver(c, a, c->prec, 0);
  }
  if (st != PFC_OK) return st;
  LAUNCH(pfc::launch_scatter_out(c->n, c->n_pad, 3, c->perm, c->tmp3, y, c->stream));
  CK(cudaMemcpyAsync(c->h_stats, c->stats, sizeof(pfc::DevStats), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(c->h_errw, c->errw, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (lk.owns_lock()) lk.unlock();
  harvest(c);
  fill_stats(c->h_stats[0], c->h_errw[0], stats);
  st = status_from_err(c->h_errw[0]);
  if (st != PFC_OK) return fail(c, st, std::string("stage solve: ") + pfc_status_string(st));
  return PFC_OK;
}

pfc_status pfc_step(pfc_ctx* c, double* state, double* tau, int* accepted, double* err, pfc_solve_stats* stats) {
  pfc_status st = check_ctx(c);
  if (st != PFC_OK) return st;
  if (!state || !tau || !(*tau > 0.0) || !std::isfinite(*tau)) return fail(c, PFC_ERR_INVALID, "bad step arguments");
  const int np = c->n_pad;
  const size_t np3 = 3 * (size_t)np;
  c->step_stage = -1;
  LAUNCH(pfc::launch_gather_in(c->n, np, 3, c->perm, state, c->xk, c->stream));
  st = assemble_internal(c, *tau);
  if (st != PFC_OK) return st;
  if (c->fixed_grid) {
    // a context with a fixed block count solves through the batched kernel (as a batch
    // of one), the kernel every batched launch runs, so its results are the same bits
    // alone and in a batch
    std::lock_guard<std::mutex> lk(g_batch_mutex);
    BatchSpace* space = nullptr;
    const size_t region = batch_region_bytes(1);
    st = batch_space(c, 3 * region, space);
    if (st != PFC_OK) return st;
    pfc_ctx* one[1] = {c};
    for (int i = 0; i < 3; ++i) {
      LAUNCH(pfc::launch_stage_combine(np, c->xk, c->ys, c->ys + np3, i, kA[i][0], kA[i][1], kC[i][0], kC[i][1],
                                       c->xi, c->dvec, c->stream));
      st = rhs_at_stage(c, i > 0);
      if (st != PFC_OK) return st;
      st = run_batch(one, 1, i, false, space, (size_t)i * region);
      if (st != PFC_OK) return st;
    }
    // the staged launch arguments are read before this synchronisation returns
    return finish_step(c, state, tau, accepted, err, stats);
  }
  for (int i = 0; i < 3; ++i) {
    LAUNCH(pfc::launch_stage_combine(np, c->xk, c->ys, c->ys + np3, i, kA[i][0], kA[i][1], kC[i][0], kC[i][1], c->xi,
                                 c->dvec, c->stream));
    // d = sum_j c_ij dpsi_j comes from stage_combine; the RHS kernel reads it
    st = rhs_at_stage(c, i > 0);
    if (st != PFC_OK) return st;
    pfc::SolveArgs a = base_args(c, c->prec);
    a.mode = 0;
    a.b = c->bv;
    a.y = c->ys + i * np3;
    st = run_solver(c, a, c->prec, i);
    if (st != PFC_OK) return st;
  }
  return finish_step(c, state, tau, accepted, err, stats);
}

pfc_status pfc_step_begin(pfc_ctx* c, const double* state, double tau) {
  pfc_status st = check_ctx(c);
  if (st != PFC_OK) return st;
  if (!state || !(tau > 0.0) || !std::isfinite(tau)) return fail(c, PFC_ERR_INVALID, "bad step arguments");
  c->step_stage = -1;
  LAUNCH(pfc::launch_gather_in(c->n, c->n_pad, 3, c->perm, state, c->xk, c->stream));
  st = assemble_internal(c, tau);
  if (st != PFC_OK) return st;
  c->step_stage = 0;
  return PFC_OK;
}

int pfc_step_stage(const pfc_ctx* c) { return c ? c->step_stage : -1; }

pfc_status pfc_batch_stage_advance(pfc_ctx* const* ctxs, int count) {
  pfc_status st = check_batch(ctxs, count);
  if (st != PFC_OK) return st;
  pfc_ctx* c = ctxs[0];
  for (int k = 0; k < count; ++k)
    if (ctxs[k]->step_stage < 0 || ctxs[k]->step_stage > 2)
      return fail(c, PFC_ERR_INVALID, "every context needs a begun step with a stage left (pfc_step_begin)");
  std::lock_guard<std::mutex> lk(g_batch_mutex);
  BatchSpace* space = nullptr;
  st = batch_space(c, batch_region_bytes(count), space);
  if (st != PFC_OK) return st;
  std::vector<int> slots(count);
  for (int k = 0; k < count; ++k) {
    pfc_ctx* ck = ctxs[k];
    c = ck;
    const int i = ck->step_stage, np = ck->n_pad;
    const size_t np3 = 3 * (size_t)np;
    slots[k] = i;
    LAUNCH(pfc::launch_stage_combine(np, ck->xk, ck->ys, ck->ys + np3, i, kA[i][0], kA[i][1], kC[i][0], kC[i][1],
                                     ck->xi, ck->dvec, ck->stream));
    st = rhs_at_stage(ck, i > 0);
    if (st != PFC_OK) return st;
  }
  c = ctxs[0];
  st = run_batch(ctxs, count, 0, false, space, 0, slots.data());
  if (st != PFC_OK) return st;
  for (int k = 0; k < count; ++k) ctxs[k]->step_stage += 1;
  // the launch's arguments were staged in pinned memory that the next call reuses
  CK(cudaStreamSynchronize(c->stream));
  return PFC_OK;
}

pfc_status pfc_step_finish(pfc_ctx* c, double* state, double* tau, int* accepted, double* err,
                           pfc_solve_stats* stats) {
  pfc_status st = check_ctx(c);
  if (st != PFC_OK) return st;
  if (!state || !tau || !(*tau > 0.0) || !std::isfinite(*tau)) return fail(c, PFC_ERR_INVALID, "bad step arguments");
  if (c->step_stage != 3) return fail(c, PFC_ERR_INVALID, "the step's three stages have not been solved");
  c->step_stage = -1;
  return finish_step(c, state, tau, accepted, err, stats);
}

pfc_status pfc_euler_step(pfc_ctx* c, double* state, double tau, pfc_solve_stats* stats) {
  pfc_status st = check_ctx(c);
  if (st != PFC_OK) return st;
  if (!state || !(tau > 0.0) || !std::isfinite(tau)) return fail(c, PFC_ERR_INVALID, "bad euler step arguments");
  c->step_stage = -1;
  const int np = c->n_pad;
  LAUNCH(pfc::launch_gather_in(c->n, np, 3, c->perm, state, c->xk, c->stream));
  // A of Eq. (3.4): the stage matrix with gamma = 1, A01 = -(1+r) M + N(psi_k) + 2 K
  st = assemble_internal(c, tau, 1.0, false);
  if (st != PFC_OK) return st;
  LAUNCH(pfc::launch_elem_load(c->nl, c->E, c->elem, c->xk + np, c->vol, c->ebuf, c->stream));
  LAUNCH(pfc::launch_euler_rhs(c->nslices, np, c->slice_ptr, c->cols, c->Mv, c->dptr, c->didx, c->ebuf, c->xk + np,
                               c->bv, c->stream));
  pfc::SolveArgs a = base_args(c, c->prec);
  a.mode = 0;
  a.b = c->bv;
  a.y = c->xnew;
  st = run_solver(c, a, c->prec, 0);
  if (st != PFC_OK) return st;
  CK(cudaMemcpyAsync(c->h_stats, c->stats, sizeof(pfc::DevStats), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(c->h_errw, c->errw, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  harvest(c);
  fill_stats(c->h_stats[0], c->h_errw[0], stats);
  st = status_from_err(c->h_errw[0]);
  if (st != PFC_OK) return fail(c, st, std::string("euler step: ") + pfc_status_string(st));
  LAUNCH(pfc::launch_scatter_out(c->n, np, 3, c->perm, c->xnew, state, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return PFC_OK;
}

pfc_status pfc_init_state(pfc_ctx* c, const double* psi0, double* state) {
  pfc_status st = check_ctx(c);
  if (st != PFC_OK) return st;
  if (!psi0 || !state) return fail(c, PFC_ERR_INVALID, "null vector");
  const int np = c->n_pad;
  double* mu = c->xk;
  double* psi = c->xk + np;
  double* om = c->xk + 2 * np;
  LAUNCH(pfc::launch_gather_in(c->n, np, 1, c->perm, psi0, psi, c->stream));
  LAUNCH(pfc::launch_elem_load(c->nl, c->E, c->elem, psi, c->vol, c->ebuf, c->stream));
  LAUNCH(pfc::launch_dof_gather(np, c->dptr, c->didx, c->ebuf, c->lvec, c->stream));
  // M omega = -K psi
  LAUNCH(pfc::launch_spmv_combo(c->nslices, c->slice_ptr, c->cols, c->Mv, c->Kv, 0.0, nullptr, -1.0, psi, 0.0, nullptr, 0.0,
                            nullptr, c->tmpn, c->stream));
  pfc::SolveArgs a = base_args(c, 0);
  a.mode = 2;
  a.which = 0;
  a.inner_rtol = 1e-14;
  a.max_inner = 5000;
  a.b = c->tmpn;
  a.y = om;
  st = run_solver(c, a, 0, 3);
  if (st != PFC_OK) return st;
  // M mu = l(psi^3) + (1+r) M psi - 2 K psi - K omega
  LAUNCH(pfc::launch_spmv_combo(c->nslices, c->slice_ptr, c->cols, c->Mv, c->Kv, 1.0 + c->opt.r, psi, -2.0, psi, -1.0, om,
                            1.0, c->lvec, c->tmpn, c->stream));
  a.y = mu;
  st = run_solver(c, a, 0, 3);
  if (st != PFC_OK) return st;
  LAUNCH(pfc::launch_scatter_out(c->n, np, 3, c->perm, c->xk, state, c->stream));
  CK(cudaMemcpyAsync(c->h_errw, c->errw + 3, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  harvest(c);
  st = status_from_err(c->h_errw[0]);
  if (st != PFC_OK) return fail(c, st, "consistent initialisation failed");
  return PFC_OK;
}

pfc_status pfc_apply(pfc_ctx* c, int op, const double* x, double* y) {
  pfc_status st = check_ctx(c);
  if (st != PFC_OK) return st;
  if (!x || !y) return fail(c, PFC_ERR_INVALID, "null vector");
  if ((op == PFC_OP_A01 || op == PFC_OP_AR || op == PFC_OP_PCH) && !c->assembled)
    return fail(c, PFC_ERR_INVALID, "pfc_assemble must come first");
  const int np = c->n_pad;
  if (op == PFC_OP_M || op == PFC_OP_K || op == PFC_OP_A01) {
    LAUNCH(pfc::launch_gather_in(c->n, np, 1, c->perm, x, c->tmp3, c->stream));
    const double* vals = op == PFC_OP_M ? c->Mv : op == PFC_OP_K ? c->Kv : c->Av;
    LAUNCH(pfc::launch_spmv(c->nslices, c->slice_ptr, c->cols, vals, c->tmp3, c->xnew, c->stream));
    LAUNCH(pfc::launch_scatter_out(c->n, np, 1, c->perm, c->xnew, y, c->stream));
  } else if (op == PFC_OP_AR) {
    LAUNCH(pfc::launch_gather_in(c->n, np, 3, c->perm, x, c->tmp3, c->stream));
    LAUNCH(pfc::launch_spmv_ar(c->nslices, np, c->slice_ptr, c->cols, c->Mv, c->Kv, c->Av, c->tau, 1.0 / c->gamma,
                               c->model == 1 ? c->A10v : nullptr, c->model == 1 ? c->A11v : nullptr, c->tmp3,
                           c->xnew, c->stream));
    LAUNCH(pfc::launch_scatter_out(c->n, np, 3, c->perm, c->xnew, y, c->stream));
  } else if (op == PFC_OP_PCH) {
    LAUNCH(pfc::launch_gather_in(c->n, np, 3, c->perm, x, c->tmp3, c->stream));
    pfc::SolveArgs a = base_args(c, c->prec);
    a.mode = 1;
    a.b = c->tmp3;
    a.y = c->xnew;
    st = run_solver(c, a, c->prec, 0);
    if (st != PFC_OK) return st;
    LAUNCH(pfc::launch_scatter_out(c->n, np, 3, c->perm, c->xnew, y, c->stream));
  } else {
    return fail(c, PFC_ERR_INVALID, "unknown operator");
  }
  CK(cudaMemcpyAsync(c->h_errw, c->errw, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  harvest(c);
  st = op == PFC_OP_PCH ? status_from_err(c->h_errw[0]) : PFC_OK;
  if (st != PFC_OK) return fail(c, st, "preconditioner application failed");
  return PFC_OK;
}

pfc_status pfc_pcg(pfc_ctx* c, int which, const double* b, double* x, double rtol, int* iterations) {
  pfc_status st = check_ctx(c);
  if (st != PFC_OK) return st;
  if (!c->assembled) return fail(c, PFC_ERR_INVALID, "pfc_assemble must come first");
  if (!b || !x || which < 0 || which > 2 || !(rtol > 0.0)) return fail(c, PFC_ERR_INVALID, "bad pcg arguments");
  const int np = c->n_pad;
  LAUNCH(pfc::launch_gather_in(c->n, np, 1, c->perm, b, c->tmp3, c->stream));
  pfc::SolveArgs a = base_args(c, c->prec);
  a.mode = 2;
  a.which = which;
  a.inner_rtol = rtol;
  a.b = c->tmp3;
  a.y = c->xnew;
  st = run_solver(c, a, c->prec, 0);
  if (st != PFC_OK) return st;
  LAUNCH(pfc::launch_scatter_out(c->n, np, 1, c->perm, c->xnew, x, c->stream));
  CK(cudaMemcpyAsync(c->h_stats, c->stats, sizeof(pfc::DevStats), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(c->h_errw, c->errw, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  harvest(c);
  if (iterations) *iterations = c->h_stats[0].last_its;
  st = status_from_err(c->h_errw[0]);
  if (st != PFC_OK) return fail(c, st, "pcg failed");
  return PFC_OK;
}

pfc_status pfc_selftest_barrier_timeout(pfc_ctx* c, double limit_seconds) {
  pfc_status st = check_ctx(c);
  if (st != PFC_OK) return st;
  if (!(limit_seconds > 0.0) || limit_seconds > 10.0) return fail(c, PFC_ERR_INVALID, "limit must be in (0, 10] s");
  // A PCG launch whose barriers wait for one block more than the grid has: every
  // wait runs out after limit_seconds, the kernel sets the timeout bit and returns.
  pfc::SolveArgs a = base_args(c, 0);
  a.mode = 2;
  a.which = 0;
  a.b = c->tmpn;
  a.y = c->xnew;
  a.barrier_extra = 1;
  a.spin_limit_ns = (unsigned long long)(limit_seconds * 1e9);
  st = run_solver(c, a, 0, 0);
  if (st != PFC_OK) return st;
  CK(cudaMemcpyAsync(c->h_errw, c->errw, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  harvest(c);
  return status_from_err(c->h_errw[0]);
}

pfc_status pfc_batch_stage_solve(pfc_ctx* const* ctxs, int count, const double* const* b, double* const* y,
                                 pfc_solve_stats* stats) {
  pfc_status st = check_batch(ctxs, count);
  if (st != PFC_OK) return st;
  pfc_ctx* c = ctxs[0];
  if (!b || !y) return fail(c, PFC_ERR_INVALID, "null vector array");
  for (int k = 0; k < count; ++k) {
    if (!ctxs[k]->assembled) return fail(c, PFC_ERR_INVALID, "pfc_assemble must come first for every context");
    if (!b[k] || !y[k]) return fail(c, PFC_ERR_INVALID, "null vector");
  }
  std::lock_guard<std::mutex> lk(g_batch_mutex);
  BatchSpace* space = nullptr;
  st = batch_space(c, batch_region_bytes(count), space);
  if (st != PFC_OK) return st;
  for (int k = 0; k < count; ++k) {
    pfc_ctx* ck = ctxs[k];
    LAUNCH(pfc::launch_gather_in(ck->n, ck->n_pad, 3, ck->perm, b[k], ck->bv, ck->stream));
  }
  st = run_batch(ctxs, count, 0, true, space, 0);
  if (st != PFC_OK) return st;
  for (int k = 0; k < count; ++k) {
    pfc_ctx* ck = ctxs[k];
    LAUNCH(pfc::launch_scatter_out(ck->n, ck->n_pad, 3, ck->perm, ck->tmp3, y[k], ck->stream));
    CK(cudaMemcpyAsync(ck->h_stats, ck->stats, sizeof(pfc::DevStats), cudaMemcpyDeviceToHost, ck->stream));
    CK(cudaMemcpyAsync(ck->h_errw, ck->errw, sizeof(int), cudaMemcpyDeviceToHost, ck->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  pfc_status worst = PFC_OK;
  for (int k = 0; k < count; ++k) {
    fill_stats(ctxs[k]->h_stats[0], ctxs[k]->h_errw[0], stats ? stats + k : nullptr);
    pfc_status sk = status_from_err(ctxs[k]->h_errw[0]);
    if (sk != PFC_OK && worst == PFC_OK) worst = sk;
  }
  if (worst != PFC_OK) return fail(c, worst, "a batched stage solve failed");
  return PFC_OK;
}

pfc_status pfc_batch_step(pfc_ctx* const* ctxs, int count, double* const* states, double* taus, int* accepted,
                          double* errs, pfc_solve_stats* stats) {
  pfc_status st = check_batch(ctxs, count);
  if (st != PFC_OK) return st;
  pfc_ctx* c = ctxs[0];
  if (!states || !taus) return fail(c, PFC_ERR_INVALID, "null argument");
  for (int k = 0; k < count; ++k)
    if (!states[k] || !(taus[k] > 0.0) || !std::isfinite(taus[k])) return fail(c, PFC_ERR_INVALID, "bad step arguments");
  std::lock_guard<std::mutex> lk(g_batch_mutex);
  BatchSpace* space = nullptr;
  const size_t region = batch_region_bytes(count);
  st = batch_space(c, 3 * region, space);
  if (st != PFC_OK) return st;
  for (int k = 0; k < count; ++k) {
    pfc_ctx* ck = ctxs[k];
    c = ck;
    ck->step_stage = -1;
    LAUNCH(pfc::launch_gather_in(ck->n, ck->n_pad, 3, ck->perm, states[k], ck->xk, ck->stream));
    st = assemble_internal(ck, taus[k]);
    if (st != PFC_OK) return st;
  }
  c = ctxs[0];
  for (int i = 0; i < 3; ++i) {
    for (int k = 0; k < count; ++k) {
      pfc_ctx* ck = ctxs[k];
      c = ck;
      const int np = ck->n_pad;
      const size_t np3 = 3 * (size_t)np;
      LAUNCH(pfc::launch_stage_combine(np, ck->xk, ck->ys, ck->ys + np3, i, kA[i][0], kA[i][1], kC[i][0], kC[i][1],
                                       ck->xi, ck->dvec, ck->stream));
      st = rhs_at_stage(ck, i > 0);
      if (st != PFC_OK) return st;
    }
    c = ctxs[0];
    st = run_batch(ctxs, count, i, false, space, (size_t)i * region);
    if (st != PFC_OK) return st;
  }
  double e[3];
  for (int j = 0; j < 3; ++j) e[j] = kMhat[j] - kM[j];
  for (int k = 0; k < count; ++k) {
    pfc_ctx* ck = ctxs[k];
    c = ck;
    const int np = ck->n_pad;
    const size_t np3 = 3 * (size_t)np;
    LAUNCH(pfc::launch_step_combine(np, ck->xk, ck->ys, ck->ys + np3, ck->ys + 2 * np3, kM, e, ck->opt.step_atol,
                                    ck->opt.step_rtol, ck->xnew, ck->step_part, pfc::step_partials(), ck->stream));
    LAUNCH(pfc::launch_reduce_partials(pfc::step_partials(), ck->step_part, 1.0 / ck->n, ck->err_scalar, ck->stream));
    if (width_guard_on(ck)) {
      st = enqueue_mean_psi(ck);
      if (st != PFC_OK) return st;
    }
    CK(cudaMemcpyAsync(ck->h_stats, ck->stats, sizeof(pfc::DevStats) * 3, cudaMemcpyDeviceToHost, ck->stream));
    CK(cudaMemcpyAsync(ck->h_errw, ck->errw, sizeof(int) * 3, cudaMemcpyDeviceToHost, ck->stream));
    CK(cudaMemcpyAsync(ck->h_err, ck->err_scalar, sizeof(double) * 2, cudaMemcpyDeviceToHost, ck->stream));
  }
  c = ctxs[0];
  CK(cudaStreamSynchronize(c->stream));
  pfc_status worst = PFC_OK;
  for (int k = 0; k < count; ++k) {
    pfc_ctx* ck = ctxs[k];
    c = ck;
    int werr = 0;
    for (int i = 0; i < 3; ++i) {
      fill_stats(ck->h_stats[i], ck->h_errw[i], stats ? stats + 3 * k + i : nullptr);
      werr |= ck->h_errw[i];
    }
    const double ev = ck->h_err[0];
    if (errs) errs[k] = ev;
    pfc_status sk = status_from_err(werr);
    if (sk == PFC_ERR_TIMEOUT || sk == PFC_ERR_NONFINITE || !std::isfinite(ev)) {
      if (accepted) accepted[k] = 0;
      if (worst == PFC_OK) worst = sk == PFC_OK ? PFC_ERR_NONFINITE : sk;
      continue;
    }
    const bool acc = ev <= 1.0 && sk == PFC_OK;
    if (accepted) accepted[k] = acc ? 1 : 0;
    if (acc) LAUNCH(pfc::launch_scatter_out(ck->n, ck->n_pad, 3, ck->perm, ck->xnew, states[k], ck->stream));
    double fac = ev == 0.0 ? 5.0 : std::min(5.0, std::max(0.2, 0.9 * std::pow(ev, -1.0 / 3.0)));
    if (acc && ck->last_rejected) fac = std::min(fac, 1.0);
    ck->last_rejected = !acc;
    taus[k] = std::min(taus[k] * fac, width_cap(ck, ck->h_err[1]));
    if (sk != PFC_OK && worst == PFC_OK) worst = sk;
  }
  c = ctxs[0];
  if (worst != PFC_OK) return fail(c, worst, "a batched step failed");
  return PFC_OK;
}

pfc_status pfc_set_timing(pfc_ctx* c, int enable) {
  pfc_status st = check_ctx(c);
  if (st != PFC_OK) return st;
  c->timing = enable != 0;
  return PFC_OK;
}

pfc_status pfc_counters(const pfc_ctx* c, long long* launches, long long* solver_launches, double* solver_ms) {
  if (!c) return PFC_ERR_INVALID;
  if (launches) *launches = c->launches;
  if (solver_launches) *solver_launches = c->solver_launches;
  if (solver_ms) *solver_ms = c->solver_ms;
  return PFC_OK;
}

pfc_status pfc_host_stencil(int dim, int side, double length, int64_t* out3) {
  if (!out3) return PFC_ERR_INVALID;
  pfc::HostSetup S;
  std::string err;
  if (!pfc::build_setup(dim, side, length, S, err, 1)) return PFC_ERR_INVALID;
  int64_t interior = 0, bnnz = 0;
  for (int p = 0; p < S.n_pad; ++p)
    if (S.rowinfo[p] & 8) ++interior;
  // nonzeros of the rows that keep their assembled values (true row lengths; rows
  // that hold no dof have none)
  for (int p = 0; p < S.n_pad; ++p) {
    if ((S.rowinfo[p] & 8) || S.perm[p] < 0) continue;
    const int s = p / pfc::kSellC, lane = p % pfc::kSellC, base = S.slice_ptr[s] + lane;
    const int w = (S.slice_ptr[s + 1] - S.slice_ptr[s]) / pfc::kSellC;
    for (int j = 0; j < w; ++j)
      if (S.cols[base + j * pfc::kSellC] != p || S.diag_pos[p] == base + j * pfc::kSellC) ++bnnz;
  }
  out3[0] = interior;
  out3[1] = bnnz;
  out3[2] = (int64_t)S.st_off.size();
  return PFC_OK;
}

pfc_status pfc_host_partition(int dim, int side, double length, int degree, int nparts, int64_t* row_begin,
                              int64_t* halo, int64_t* part_nnz) {
  if (!row_begin || !halo || !part_nnz || nparts < 1) return PFC_ERR_INVALID;
  std::vector<int64_t> b, h, z;
  std::string err;
  if (!pfc::build_partition(dim, side, length, degree, nparts, b, h, z, err)) return PFC_ERR_INVALID;
  std::copy(b.begin(), b.end(), row_begin);
  std::copy(h.begin(), h.end(), halo);
  std::copy(z.begin(), z.end(), part_nnz);
  return PFC_OK;
}

pfc_status pfc_host_cells(int dim, int side, double length, int64_t* out4) {
  if (!out4) return PFC_ERR_INVALID;
  pfc::HostSetup S;
  std::string err;
  if (!pfc::build_setup(dim, side, length, S, err, 1, 2, 1)) return PFC_ERR_INVALID;
  CellTables T;
  out4[0] = (int64_t)S.cls_start.size() - 1;
  out4[1] = (int64_t)S.cls_off.size();
  out4[2] = cell_pattern_ok(S, &T) ? T.ncc : 0;
  int64_t rows = 0;
  for (int p = 0; p < S.n_pad; ++p)
    if (S.perm[p] >= 0) ++rows;
  out4[3] = rows;
  return PFC_OK;
}

int pfc_cell_kernels(const pfc_ctx* c) { return (c && c->prec != 0 && c->cell_ok) ? 1 : 0; }

pfc_status pfc_host_pattern(int dim, int side, double length, int64_t* out4) {
  if (!out4) return PFC_ERR_INVALID;
  pfc::HostSetup S;
  std::string err;
  if (!pfc::build_setup(dim, side, length, S, err)) return PFC_ERR_INVALID;
  out4[0] = S.n;
  out4[1] = S.nnz;
  out4[2] = S.nnz_sell;
  out4[3] = S.E;
  return PFC_OK;
}

}  // extern "C"
