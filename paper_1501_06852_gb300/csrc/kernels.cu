// Element assembly, stage right-hand side, stage/step combination and layout
// kernels of the PFC stage solver.
//
// Assembly is gather-based and free of atomics: an element kernel writes the
// element quantity of every element into a structure-of-arrays buffer
// (entry p of element e at p * E + e), and a slot (or row) kernel sums the
// contributions listed for it in a precomputed map, always in the same order.
// The nonlinear mass (Section 3) N(psi)_ij = -3 int psi^2 phi_j phi_i and the
// load (psi^3, phi_j) come from the exact quartic tensor of the P2 element,
// int phi_a phi_b phi_i phi_j, kept in constant memory per dimension.
#include <cuda_fp16.h>

#include "device.cuh"
#include "internal.h"
#include "launch.h"

namespace pfc {
namespace {

__constant__ double c_quart2[21 * 21];   // P2 triangles
__constant__ double c_quart3[55 * 55];   // P2 tetrahedra
__constant__ double c_quart1_2[6 * 6];   // P1 triangles
__constant__ double c_quart1_3[10 * 10]; // P1 tetrahedra
// second node of unordered local pair p = (i <= j), per element kind
__constant__ int c_pair_j2[21];
__constant__ int c_pair_j3[55];
__constant__ int c_pair_j1_2[6];
__constant__ int c_pair_j1_3[10];

constexpr int kBlock = 256;

inline int blocks_for(long long work, int per_block) {
  long long b = (work + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > 1048576) b = 1048576;
  return (int)b;
}

__global__ void k_assemble_mk(long long nnz, const int* __restrict__ cptr, const int* __restrict__ cidx, int E,
                              int ntypes, int np, const double* __restrict__ mass, const double* __restrict__ stiff,
                              double* Mv, double* Kv) {
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < nnz; s += (long long)gridDim.x * blockDim.x) {
    double m = 0.0, k = 0.0;
    for (int q = cptr[s]; q < cptr[s + 1]; ++q) {
      const int idx = cidx[q];
      const int pr = idx / E;
      const int e = idx - pr * E;
      const int t = e % ntypes;
      m += mass[t * np + pr];
      k += stiff[t * np + pr];
    }
    Mv[s] = m;
    Kv[s] = k;
  }
}

template <int NL>
__device__ __forceinline__ const double* quart_table();
template <>
__device__ __forceinline__ const double* quart_table<6>() {
  return c_quart2;
}
template <>
__device__ __forceinline__ const double* quart_table<10>() {
  return c_quart3;
}
template <>
__device__ __forceinline__ const double* quart_table<3>() {
  return c_quart1_2;
}
template <>
__device__ __forceinline__ const double* quart_table<4>() {
  return c_quart1_3;
}

template <int NL>
__device__ __forceinline__ const int* pair_j_table() {
  return NL == 6 ? c_pair_j2 : NL == 10 ? c_pair_j3 : NL == 3 ? c_pair_j1_2 : c_pair_j1_3;
}

// ebuf[p * E + e] = vol * int psi^2 phi_i phi_j (unit-volume tensor times vol), p = (i <= j)
template <int NL>
__global__ void __launch_bounds__(128) k_elem_quartic(int E, const int* __restrict__ elem,
                                                       const double* __restrict__ psi, double vol, double* ebuf) {
  constexpr int NP = NL * (NL + 1) / 2;
  const double* T = quart_table<NL>();
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
    double ps[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) ps[l] = psi[__ldg(elem + (size_t)l * E + e)];
    double cab[NP];
    {
      int t = 0;
#pragma unroll
      for (int a = 0; a < NL; ++a)
#pragma unroll
        for (int b = a; b < NL; ++b) cab[t++] = ps[a] * ps[b];
    }
#pragma unroll 1
    for (int p = 0; p < NP; ++p) {
      double s = 0.0;
#pragma unroll
      for (int q = 0; q < NP; ++q) s = fma(cab[q], T[q * NP + p], s);
      ebuf[(size_t)p * E + e] = vol * s;
    }
  }
}

// lbuf[l * E + e] = vol * int psi^3 phi_l over element e
template <int NL>
__global__ void __launch_bounds__(128) k_elem_load(int E, const int* __restrict__ elem, const double* __restrict__ psi,
                                                    double vol, double* lbuf) {
  constexpr int NP = NL * (NL + 1) / 2;
  const double* T = quart_table<NL>();
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
    double ps[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) ps[l] = psi[__ldg(elem + (size_t)l * E + e)];
    double cab[NP];
    {
      int t = 0;
#pragma unroll
      for (int a = 0; a < NL; ++a)
#pragma unroll
        for (int b = a; b < NL; ++b) cab[t++] = ps[a] * ps[b];
    }
    double lj[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) lj[l] = 0.0;
    int p = 0;
#pragma unroll
    for (int i = 0; i < NL; ++i) {
#pragma unroll
      for (int j = i; j < NL; ++j) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < NP; ++q) s = fma(cab[q], T[q * NP + p], s);
        lj[j] = fma(ps[i], s, lj[j]);
        if (i != j) lj[i] = fma(ps[j], s, lj[i]);
        ++p;
      }
    }
#pragma unroll
    for (int l = 0; l < NL; ++l) lbuf[(size_t)l * E + e] = vol * lj[l];
  }
}

__global__ void k_assemble_a01(long long nnz, const int* __restrict__ cptr, const int* __restrict__ cidx,
                               const double* __restrict__ ebuf, const double* __restrict__ Mv,
                               const double* __restrict__ Kv, double r, double* Av) {
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < nnz; s += (long long)gridDim.x * blockDim.x) {
    double q = 0.0;
    for (int c = cptr[s]; c < cptr[s + 1]; ++c) q += ebuf[cidx[c]];
    Av[s] = -(1.0 + r) * Mv[s] + 2.0 * Kv[s] - 3.0 * q;
  }
}

// ---------------------------------------------------------------- PFC1 mobility
// T = mob + t * NL^3 holds int phi_a grad phi_b . grad phi_c over an element of
// type t (t = e mod ntypes: elements are stored cell-major, types inner).
//
// Per element and unordered local pair p = (i <= j):
//   ebuf[(3p)   E + e] = (psi^+ grad phi_j, grad phi_i)      -> K_+(psi)
//   ebuf[(3p+1) E + e] = (phi_j grad mu, grad phi_i)         -> F(mu), row node i
//   ebuf[(3p+2) E + e] = (phi_i grad mu, grad phi_j)         -> F(mu), row node j
template <int NL>
__global__ void __launch_bounds__(128) k_elem_mobility(int E, int ntypes, const int* __restrict__ elem,
                                                        const double* __restrict__ psi, const double* __restrict__ mu,
                                                        double psi_min, const double* __restrict__ mob, double* ebuf) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
    const double* T = mob + (size_t)(e % ntypes) * NL * NL * NL;
    double pp[NL], mm[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      const int d = __ldg(elem + (size_t)l * E + e);
      pp[l] = psi[d] - psi_min;
      mm[l] = mu[d];
    }
    int p = 0;
#pragma unroll 1
    for (int i = 0; i < NL; ++i) {
#pragma unroll 1
      for (int j = i; j < NL; ++j) {
        double kp = 0.0, fij = 0.0, fji = 0.0;
#pragma unroll
        for (int a = 0; a < NL; ++a) {
          kp = fma(pp[a], __ldg(T + ((size_t)a * NL + i) * NL + j), kp);
          fij = fma(mm[a], __ldg(T + ((size_t)j * NL + a) * NL + i), fij);
          fji = fma(mm[a], __ldg(T + ((size_t)i * NL + a) * NL + j), fji);
        }
        ebuf[(size_t)(3 * p) * E + e] = kp;
        ebuf[(size_t)(3 * p + 1) * E + e] = fij;
        ebuf[(size_t)(3 * p + 2) * E + e] = fji;
        ++p;
      }
    }
  }
}

// lbuf[l E + e] = (psi^+ grad mu, grad phi_l) over element e
template <int NL>
__global__ void __launch_bounds__(128) k_elem_mobload(int E, int ntypes, const int* __restrict__ elem,
                                                       const double* __restrict__ psi, const double* __restrict__ mu,
                                                       double psi_min, const double* __restrict__ mob, double* lbuf) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
    const double* T = mob + (size_t)(e % ntypes) * NL * NL * NL;
    double pp[NL], mm[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      const int d = __ldg(elem + (size_t)l * E + e);
      pp[l] = psi[d] - psi_min;
      mm[l] = mu[d];
    }
#pragma unroll 1
    for (int c = 0; c < NL; ++c) {
      double s = 0.0;
#pragma unroll 1
      for (int a = 0; a < NL; ++a) {
        double t = 0.0;
#pragma unroll
        for (int b = 0; b < NL; ++b) t = fma(mm[b], __ldg(T + ((size_t)a * NL + b) * NL + c), t);
        s = fma(pp[a], t, s);
      }
      lbuf[(size_t)c * E + e] = s;
    }
  }
}

// A10 = tau K_+(psi_k), A11 = M / gamma + tau F(mu_k) (F only when with_f) on every
// slot: for a contribution of pair p = (i, j) of element e, the slot's column is
// node j (then the slot's row is node i) or node i.
template <int NL>
__global__ void k_assemble_mob(long long nnz, const int* __restrict__ cptr, const int* __restrict__ cidx,
                               const int* __restrict__ cols, const int* __restrict__ elem, int E,
                               const double* __restrict__ ebuf, const double* __restrict__ Mv, double tau,
                               double inv_gamma, int with_f, double* A10, double* A11) {
  const int* pj = pair_j_table<NL>();
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < nnz; s += (long long)gridDim.x * blockDim.x) {
    const int col = cols[s];
    double kp = 0.0, f = 0.0;
    for (int c = cptr[s]; c < cptr[s + 1]; ++c) {
      const int idx = cidx[c];
      const int p = idx / E;
      const int e = idx - p * E;
      kp += ebuf[(size_t)(3 * p) * E + e];
      if (with_f) {
        const int nj = __ldg(elem + (size_t)pj[p] * E + e);
        f += ebuf[(size_t)(3 * p + (nj == col ? 1 : 2)) * E + e];
      }
    }
    A10[s] = tau * kp;
    A11[s] = inv_gamma * Mv[s] + tau * f;
  }
}

// Jacobi inverse of S_D = M - 2 delta K + delta K M_D^{-1} K (Section 4.1):
//   d_i = M_ii - 2 delta K_ii + delta sum_j K_ij^2 / M_jj
// (mdinv = 1 / diag(M)), one thread per SELL row; padding rows get 0.
__global__ void k_sd_diag_inv(int nslices, const int* __restrict__ sp, const int* __restrict__ cols,
                              const double* __restrict__ Mv, const double* __restrict__ Kv,
                              const int* __restrict__ diag_pos, const double* __restrict__ mdinv, double delta,
                              double* out, float* fout) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= nslices) return;
  const int row = s * 32 + lane;
  const int dp = diag_pos[row];
  double v = 0.0;
  if (dp >= 0) {
    double kk = 0.0;
    for (int idx = sp[s] + lane; idx < sp[s + 1]; idx += 32) {
      const double k = Kv[idx];
      kk = fma(k * k, mdinv[cols[idx]], kk);
    }
    v = 1.0 / (Mv[dp] - 2.0 * delta * Kv[dp] + delta * kk);
  }
  out[row] = v;
  if (fout) fout[row] = (float)v;
}

// w[row] = sum of the row's stored values (SELL-32 slices, one warp per slice)
__global__ void k_row_sums(int nslices, const int* __restrict__ sp, const double* __restrict__ vals, double* w) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= nslices) return;
  double acc = 0.0;
  for (int idx = sp[s] + lane; idx < sp[s + 1]; idx += 32) acc += vals[idx];
  w[s * 32 + lane] = acc;
}

// partial[b] = sum over block b's strided share of a[i] * b[i] (fixed order)
__global__ void k_dot_partials(int n, const double* __restrict__ a, const double* __restrict__ b, double* partial) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) acc = fma(a[i], b[i], acc);
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

template <class TM>
__device__ __forceinline__ TM cvt_to(double v);
template <>
__device__ __forceinline__ float cvt_to<float>(double v) {
  return (float)v;
}
template <>
__device__ __forceinline__ __half cvt_to<__half>(double v) {
  return __double2half(v);
}
template <>
__device__ __forceinline__ double cvt_to<double>(double v) {
  return v;
}

template <class TM>
__global__ void k_inner_mats(long long nnz, const double* __restrict__ Mv, const double* __restrict__ Kv, double delta,
                             double sdelta, double* MdK, double* MsK, TM* iMdK, TM* iMsK) {
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < nnz; s += (long long)gridDim.x * blockDim.x) {
    const double m = Mv[s], k = Kv[s];
    const double md = fma(delta, k, m), ms = fma(sdelta, k, m);
    MdK[s] = md;
    MsK[s] = ms;
    if (iMdK) {
      iMdK[s] = cvt_to<TM>(md);
      iMsK[s] = cvt_to<TM>(ms);
    }
  }
}

template <class TM>
__global__ void k_convert(long long count, const double* __restrict__ src, TM* dst) {
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < count; s += (long long)gridDim.x * blockDim.x)
    dst[s] = cvt_to<TM>(src[s]);
}

__global__ void k_diag_inv(int n_pad, const int* __restrict__ diag, const double* __restrict__ A, double* dinv,
                           float* fdinv) {
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n_pad; row += gridDim.x * blockDim.x) {
    const int p = diag[row];
    const double v = p < 0 ? 0.0 : 1.0 / A[p];
    dinv[row] = v;
    if (fdinv) fdinv[row] = (float)v;
  }
}

// Stage right-hand side of Eq. (3.10) for one SELL-32 slice per warp:
//   b0 = -M mu + (1+r) M psi - 2 K psi - K omega + l,  b1 = -tau K mu + M d,  b2 = -M omega - K psi
__global__ void k_rhs(int nslices, int n_pad, const int* __restrict__ sp, const int* __restrict__ cols,
                      const double* __restrict__ Mv, const double* __restrict__ Kv, const int* __restrict__ dptr,
                      const int* __restrict__ didx, const double* __restrict__ lbuf, const double* __restrict__ x,
                      const double* __restrict__ d, double r, double tau, const double* __restrict__ lbuf2,
                      double* b) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= nslices) return;
  const int row = s * 32 + lane;
  const double* xm = x;
  const double* xp = x + n_pad;
  const double* xo = x + 2 * n_pad;
  double m_mu = 0, m_psi = 0, m_om = 0, m_d = 0, k_mu = 0, k_psi = 0, k_om = 0;
  const int end = sp[s + 1];
  for (int idx = sp[s] + lane; idx < end; idx += 32) {
    const int c = cols[idx];
    const double mv = Mv[idx], kv = Kv[idx];
    const double zm = xm[c], zp = xp[c], zo = xo[c];
    m_mu = fma(mv, zm, m_mu);
    m_psi = fma(mv, zp, m_psi);
    m_om = fma(mv, zo, m_om);
    k_mu = fma(kv, zm, k_mu);
    k_psi = fma(kv, zp, k_psi);
    k_om = fma(kv, zo, k_om);
    if (d) m_d = fma(mv, d[c], m_d);
  }
  double l = 0.0, l2 = 0.0;
  for (int q = dptr[row]; q < dptr[row + 1]; ++q) {
    l += lbuf[didx[q]];
    if (lbuf2) l2 += lbuf2[didx[q]];
  }
  b[row] = -m_mu + (1.0 + r) * m_psi - 2.0 * k_psi - k_om + l;
  // PFC2: -tau K mu; PFC1: -tau (psi^+ grad mu, grad phi) from the element loads
  b[n_pad + row] = -tau * (lbuf2 ? l2 : k_mu) + m_d;
  b[2 * n_pad + row] = -m_om - k_psi;
}

// Right-hand side of the linearised semi-implicit Euler system (Eq. 3.4):
// b0 = (-2 psi_k^3, phi) from the per-element loads, b1 = M psi_k, b2 = 0.
__global__ void k_euler_rhs(int nslices, int n_pad, const int* __restrict__ sp, const int* __restrict__ cols,
                            const double* __restrict__ Mv, const int* __restrict__ dptr,
                            const int* __restrict__ didx, const double* __restrict__ lbuf,
                            const double* __restrict__ psi, double* b) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= nslices) return;
  const int row = s * 32 + lane;
  double m_psi = 0.0;
  const int end = sp[s + 1];
  for (int idx = sp[s] + lane; idx < end; idx += 32) m_psi = fma(Mv[idx], psi[cols[idx]], m_psi);
  double l = 0.0;
  for (int q = dptr[row]; q < dptr[row + 1]; ++q) l += lbuf[didx[q]];
  b[row] = -2.0 * l;
  b[n_pad + row] = m_psi;
  b[2 * n_pad + row] = 0.0;
}

__global__ void k_dof_gather(int n_pad, const int* __restrict__ dptr, const int* __restrict__ didx,
                             const double* __restrict__ lbuf, double* out) {
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n_pad; row += gridDim.x * blockDim.x) {
    double l = 0.0;
    for (int q = dptr[row]; q < dptr[row + 1]; ++q) l += lbuf[didx[q]];
    out[row] = l;
  }
}

// out = alpha M u + beta K v + gam K w + delt l  (terms with a zero coefficient are skipped)
__global__ void k_spmv_combo(int nslices, const int* __restrict__ sp, const int* __restrict__ cols,
                             const double* __restrict__ Mv, const double* __restrict__ Kv, double alpha,
                             const double* __restrict__ u, double beta, const double* __restrict__ v, double gam,
                             const double* __restrict__ w, double delt, const double* __restrict__ l, double* out) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= nslices) return;
  const int row = s * 32 + lane;
  double mu = 0, kv_ = 0, kw = 0;
  const int end = sp[s + 1];
  for (int idx = sp[s] + lane; idx < end; idx += 32) {
    const int c = cols[idx];
    if (alpha != 0.0) mu = fma(Mv[idx], u[c], mu);
    if (beta != 0.0) kv_ = fma(Kv[idx], v[c], kv_);
    if (gam != 0.0) kw = fma(Kv[idx], w[c], kw);
  }
  double o = alpha * mu + beta * kv_ + gam * kw;
  if (delt != 0.0) o += delt * l[row];
  out[row] = o;
}

__global__ void k_spmv(int nslices, const int* __restrict__ sp, const int* __restrict__ cols,
                       const double* __restrict__ vals, const double* __restrict__ x, double* y) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= nslices) return;
  y[s * 32 + lane] = sell_row<double>(sp, cols, vals, x, s, lane);
}

__global__ void k_spmv_ar(int nslices, int n_pad, const int* __restrict__ sp, const int* __restrict__ cols,
                          const double* __restrict__ Mv, const double* __restrict__ Kv, const double* __restrict__ Av,
                          double tau, double inv_gamma, const double* __restrict__ A10,
                          const double* __restrict__ A11, const double* __restrict__ z, double* w) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= nslices) return;
  const int row = s * 32 + lane;
  double m_mu = 0, a_psi = 0, k_om = 0, k_mu = 0, m_psi = 0, k_psi = 0, m_om = 0;
  const int end = sp[s + 1];
  for (int idx = sp[s] + lane; idx < end; idx += 32) {
    const int c = cols[idx];
    const double mv = Mv[idx], kv = Kv[idx], av = Av[idx];
    const double zm = z[c], zp = z[n_pad + c], zo = z[2 * n_pad + c];
    m_mu = fma(mv, zm, m_mu);
    a_psi = fma(av, zp, a_psi);
    k_om = fma(kv, zo, k_om);
    // PFC1: the second block row is A10, A11 (see k_assemble_mob)
    k_mu = fma(A10 ? A10[idx] : kv, zm, k_mu);
    m_psi = fma(A11 ? A11[idx] : mv, zp, m_psi);
    k_psi = fma(kv, zp, k_psi);
    m_om = fma(mv, zo, m_om);
  }
  w[row] = m_mu + a_psi + k_om;
  w[n_pad + row] = A10 ? k_mu + m_psi : tau * k_mu + inv_gamma * m_psi;
  w[2 * n_pad + row] = k_psi + m_om;
}

// x_i = x^k + sum_{j<i} a_ij y_j (3 fields);  d = sum_{j<i} c_ij dpsi_j
__global__ void k_stage_combine(int n_pad, const double* __restrict__ xk, const double* __restrict__ y0,
                                const double* __restrict__ y1, int nprev, double a0, double a1, double c0, double c1,
                                double* xi, double* d) {
  const int n3 = 3 * n_pad;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += gridDim.x * blockDim.x) {
    double v = xk[i];
    double dv = 0.0;
    if (nprev > 0) {
      v = fma(a0, y0[i], v);
      dv = c0 * y0[i];
    }
    if (nprev > 1) {
      v = fma(a1, y1[i], v);
      dv = fma(c1, y1[i], dv);
    }
    xi[i] = v;
    if (i >= n_pad && i < 2 * n_pad) d[i - n_pad] = dv;
  }
}

constexpr int kStepParts = 1024;

// x^{k+1} = x^k + sum m_j y_j; per-block partial sums of (e_psi / sc)^2
__global__ void __launch_bounds__(kBlock) k_step_combine(int n_pad, const double* __restrict__ xk,
                                                          const double* __restrict__ y0, const double* __restrict__ y1,
                                                          const double* __restrict__ y2, double m0, double m1,
                                                          double m2, double e0, double e1, double e2, double atol,
                                                          double rtol, double* xnew, double* partial) {
  __shared__ double sw[kBlock / 32];
  const int n3 = 3 * n_pad;
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += gridDim.x * blockDim.x) {
    const double a = y0[i], b = y1[i], c = y2[i];
    const double xo = xk[i];
    const double xn = xo + m0 * a + m1 * b + m2 * c;
    xnew[i] = xn;
    if (i >= n_pad && i < 2 * n_pad) {
      const double e = e0 * a + e1 * b + e2 * c;
      const double sc = atol + rtol * fmax(fabs(xo), fabs(xn));
      const double t = e / sc;
      acc = fma(t, t, acc);
    }
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < kBlock / 32 ? sw[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
  }
}

__global__ void k_reduce_partials(int nparts, const double* __restrict__ partial, double scale, double* out) {
  __shared__ double sw[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += partial[i];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (int)(blockDim.x >> 5) ? sw[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) *out = sqrt(t * scale);
  }
}

// out = scale * sum of the partials (fixed order), no square root
__global__ void k_sum_partials(int nparts, const double* __restrict__ partial, double scale, double* out) {
  __shared__ double sw[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += partial[i];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (int)(blockDim.x >> 5) ? sw[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) *out = t * scale;
  }
}

__global__ void k_gather_in(int n, int n_pad, int nf, const int* __restrict__ perm, const double* __restrict__ lex,
                            double* internal) {
  const long long tot = (long long)nf * n_pad;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(i / n_pad), p = (int)(i - (long long)f * n_pad);
    const int q = perm[p];   // -1: a row that holds no dof
    internal[i] = q >= 0 ? lex[(size_t)f * n + q] : 0.0;
  }
}

__global__ void k_scatter_out(int n, int n_pad, int nf, const int* __restrict__ perm,
                              const double* __restrict__ internal, double* lex) {
  const long long tot = (long long)nf * n_pad;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(i / n_pad), p = (int)(i - (long long)f * n_pad);
    const int q = perm[p];
    if (q >= 0) lex[(size_t)f * n + q] = internal[i];
  }
}

__global__ void k_combine_field(int n_pad, const double* __restrict__ a, double sa, const double* __restrict__ b,
                                double sb, double* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += gridDim.x * blockDim.x)
    out[i] = sa * a[i] + (b ? sb * b[i] : 0.0);
}

}  // namespace

int step_partials() { return kStepParts; }

cudaError_t upload_quartic(int nl, const double* q, int npairs) {
  const size_t bytes = sizeof(double) * npairs * npairs;
  switch (nl) {
    case 6: return cudaMemcpyToSymbol(c_quart2, q, bytes);
    case 10: return cudaMemcpyToSymbol(c_quart3, q, bytes);
    case 3: return cudaMemcpyToSymbol(c_quart1_2, q, bytes);
    case 4: return cudaMemcpyToSymbol(c_quart1_3, q, bytes);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t upload_pairs(int nl, const int* pair_j, int npairs) {
  const size_t bytes = sizeof(int) * npairs;
  switch (nl) {
    case 6: return cudaMemcpyToSymbol(c_pair_j2, pair_j, bytes);
    case 10: return cudaMemcpyToSymbol(c_pair_j3, pair_j, bytes);
    case 3: return cudaMemcpyToSymbol(c_pair_j1_2, pair_j, bytes);
    case 4: return cudaMemcpyToSymbol(c_pair_j1_3, pair_j, bytes);
    default: return cudaErrorInvalidValue;
  }
}

// the element kernels are instantiated per local node count: 6 / 10 (P2), 3 / 4 (P1)
#define PFC_NL_DISPATCH(nl, KERNEL, GRID, BLOCK, ...)                                   \
  do {                                                                                  \
    switch (nl) {                                                                       \
      case 6: KERNEL<6><<<GRID, BLOCK, 0, st>>>(__VA_ARGS__); break;                    \
      case 10: KERNEL<10><<<GRID, BLOCK, 0, st>>>(__VA_ARGS__); break;                  \
      case 3: KERNEL<3><<<GRID, BLOCK, 0, st>>>(__VA_ARGS__); break;                    \
      case 4: KERNEL<4><<<GRID, BLOCK, 0, st>>>(__VA_ARGS__); break;                    \
      default: return cudaErrorInvalidValue;                                            \
    }                                                                                   \
  } while (0)

cudaError_t launch_elem_mobility(int nl, int E, int ntypes, const int* elem, const double* psi, const double* mu,
                                 double psi_min, const double* mob, double* ebuf, cudaStream_t st) {
  PFC_NL_DISPATCH(nl, k_elem_mobility, blocks_for(E, 128), 128, E, ntypes, elem, psi, mu, psi_min, mob, ebuf);
  return cudaGetLastError();
}

cudaError_t launch_elem_mobload(int nl, int E, int ntypes, const int* elem, const double* psi, const double* mu,
                                double psi_min, const double* mob, double* lbuf, cudaStream_t st) {
  PFC_NL_DISPATCH(nl, k_elem_mobload, blocks_for(E, 128), 128, E, ntypes, elem, psi, mu, psi_min, mob, lbuf);
  return cudaGetLastError();
}

cudaError_t launch_assemble_mob(int nl, long long nnz, const int* cptr, const int* cidx, const int* cols,
                                const int* elem, int E, const double* ebuf, const double* Mv, double tau,
                                double inv_gamma, int with_f, double* A10, double* A11, cudaStream_t st) {
  PFC_NL_DISPATCH(nl, k_assemble_mob, blocks_for(nnz, kBlock), kBlock, nnz, cptr, cidx, cols, elem, E, ebuf, Mv, tau,
                  inv_gamma, with_f, A10, A11);
  return cudaGetLastError();
}

cudaError_t launch_sd_diag_inv(int nslices, const int* sp, const int* cols, const double* Mv, const double* Kv,
                               const int* diag_pos, const double* mdinv, double delta, double* out, float* fout,
                               cudaStream_t st) {
  k_sd_diag_inv<<<blocks_for((long long)nslices * 32, kBlock), kBlock, 0, st>>>(nslices, sp, cols, Mv, Kv, diag_pos,
                                                                               mdinv, delta, out, fout);
  return cudaGetLastError();
}

cudaError_t launch_row_sums(int nslices, const int* sp, const double* vals, double* w, cudaStream_t st) {
  k_row_sums<<<blocks_for((long long)nslices * 32, kBlock), kBlock, 0, st>>>(nslices, sp, vals, w);
  return cudaGetLastError();
}

cudaError_t launch_sum_partials(int nparts, const double* partial, double scale, double* out, cudaStream_t st) {
  k_sum_partials<<<1, 1024, 0, st>>>(nparts, partial, scale, out);
  return cudaGetLastError();
}

cudaError_t launch_dot_partials(int n, const double* a, const double* b, double* partial, int nparts,
                                cudaStream_t st) {
  k_dot_partials<<<nparts, 256, 0, st>>>(n, a, b, partial);
  return cudaGetLastError();
}

cudaError_t launch_assemble_mk(long long nnz, const int* cptr, const int* cidx, int E, int ntypes, int np,
                               const double* mass, const double* stiff, double* Mv, double* Kv, cudaStream_t st) {
  k_assemble_mk<<<blocks_for(nnz, kBlock), kBlock, 0, st>>>(nnz, cptr, cidx, E, ntypes, np, mass, stiff, Mv, Kv);
  return cudaGetLastError();
}

cudaError_t launch_elem_quartic(int nl, int E, const int* elem, const double* psi, double vol, double* ebuf,
                                cudaStream_t st) {
  PFC_NL_DISPATCH(nl, k_elem_quartic, blocks_for(E, 128), 128, E, elem, psi, vol, ebuf);
  return cudaGetLastError();
}

cudaError_t launch_elem_load(int nl, int E, const int* elem, const double* psi, double vol, double* lbuf,
                             cudaStream_t st) {
  PFC_NL_DISPATCH(nl, k_elem_load, blocks_for(E, 128), 128, E, elem, psi, vol, lbuf);
  return cudaGetLastError();
}

cudaError_t launch_assemble_a01(long long nnz, const int* cptr, const int* cidx, const double* ebuf, const double* Mv,
                                const double* Kv, double r, double* Av, cudaStream_t st) {
  k_assemble_a01<<<blocks_for(nnz, kBlock), kBlock, 0, st>>>(nnz, cptr, cidx, ebuf, Mv, Kv, r, Av);
  return cudaGetLastError();
}

cudaError_t launch_inner_mats(int prec, long long nnz, const double* Mv, const double* Kv, double delta, double sdelta,
                              double* MdK, double* MsK, void* iMdK, void* iMsK, cudaStream_t st) {
  const int nb = blocks_for(nnz, kBlock);
  if (prec == 1)
    k_inner_mats<float><<<nb, kBlock, 0, st>>>(nnz, Mv, Kv, delta, sdelta, MdK, MsK, (float*)iMdK, (float*)iMsK);
  else if (prec == 2)
    k_inner_mats<__half><<<nb, kBlock, 0, st>>>(nnz, Mv, Kv, delta, sdelta, MdK, MsK, (__half*)iMdK, (__half*)iMsK);
  else
    k_inner_mats<double><<<nb, kBlock, 0, st>>>(nnz, Mv, Kv, delta, sdelta, MdK, MsK, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_convert(int prec, long long count, const double* src, void* dst, cudaStream_t st) {
  const int nb = blocks_for(count, kBlock);
  if (prec == 1)
    k_convert<float><<<nb, kBlock, 0, st>>>(count, src, (float*)dst);
  else
    k_convert<__half><<<nb, kBlock, 0, st>>>(count, src, (__half*)dst);
  return cudaGetLastError();
}

cudaError_t launch_diag_inv(int n_pad, const int* diag, const double* A, double* dinv, float* fdinv, cudaStream_t st) {
  k_diag_inv<<<blocks_for(n_pad, kBlock), kBlock, 0, st>>>(n_pad, diag, A, dinv, fdinv);
  return cudaGetLastError();
}

cudaError_t launch_rhs(int nslices, const int* sp, const int* cols, const double* Mv, const double* Kv,
                       const int* dptr, const int* didx, const double* lbuf, const double* x, const double* d,
                       double r, double tau, const double* lbuf2, double* b, cudaStream_t st) {
  const int n_pad = nslices * 32;
  k_rhs<<<blocks_for((long long)nslices * 32, kBlock), kBlock, 0, st>>>(nslices, n_pad, sp, cols, Mv, Kv, dptr, didx,
                                                                       lbuf, x, d, r, tau, lbuf2, b);
  return cudaGetLastError();
}

cudaError_t launch_euler_rhs(int nslices, int n_pad, const int* sp, const int* cols, const double* Mv, const int* dptr,
                             const int* didx, const double* lbuf, const double* psi, double* b, cudaStream_t st) {
  k_euler_rhs<<<blocks_for((long long)nslices * 32, kBlock), kBlock, 0, st>>>(nslices, n_pad, sp, cols, Mv, dptr, didx,
                                                                             lbuf, psi, b);
  return cudaGetLastError();
}

cudaError_t launch_dof_gather(int n_pad, const int* dptr, const int* didx, const double* lbuf, double* out,
                              cudaStream_t st) {
  k_dof_gather<<<blocks_for(n_pad, kBlock), kBlock, 0, st>>>(n_pad, dptr, didx, lbuf, out);
  return cudaGetLastError();
}

cudaError_t launch_spmv_combo(int nslices, const int* sp, const int* cols, const double* Mv, const double* Kv,
                              double alpha, const double* u, double beta, const double* v, double gam, const double* w,
                              double delt, const double* l, double* out, cudaStream_t st) {
  k_spmv_combo<<<blocks_for((long long)nslices * 32, kBlock), kBlock, 0, st>>>(nslices, sp, cols, Mv, Kv, alpha, u,
                                                                              beta, v, gam, w, delt, l, out);
  return cudaGetLastError();
}

cudaError_t launch_spmv(int nslices, const int* sp, const int* cols, const double* vals, const double* x, double* y,
                        cudaStream_t st) {
  k_spmv<<<blocks_for((long long)nslices * 32, kBlock), kBlock, 0, st>>>(nslices, sp, cols, vals, x, y);
  return cudaGetLastError();
}

cudaError_t launch_spmv_ar(int nslices, int n_pad, const int* sp, const int* cols, const double* Mv, const double* Kv,
                           const double* Av, double tau, double inv_gamma, const double* A10, const double* A11,
                           const double* z, double* w, cudaStream_t st) {
  k_spmv_ar<<<blocks_for((long long)nslices * 32, kBlock), kBlock, 0, st>>>(nslices, n_pad, sp, cols, Mv, Kv, Av, tau,
                                                                           inv_gamma, A10, A11, z, w);
  return cudaGetLastError();
}

cudaError_t launch_stage_combine(int n_pad, const double* xk, const double* y0, const double* y1, int nprev, double a0,
                                 double a1, double c0, double c1, double* xi, double* d, cudaStream_t st) {
  k_stage_combine<<<blocks_for(3LL * n_pad, kBlock), kBlock, 0, st>>>(n_pad, xk, y0, y1, nprev, a0, a1, c0, c1, xi,
                                                                     d);
  return cudaGetLastError();
}

cudaError_t launch_step_combine(int n_pad, const double* xk, const double* y0, const double* y1, const double* y2,
                                const double m[3], const double e[3], double atol, double rtol, double* xnew,
                                double* partial, int nparts, cudaStream_t st) {
  k_step_combine<<<nparts, kBlock, 0, st>>>(n_pad, xk, y0, y1, y2, m[0], m[1], m[2], e[0], e[1], e[2], atol, rtol,
                                            xnew, partial);
  return cudaGetLastError();
}

cudaError_t launch_reduce_partials(int nparts, const double* partial, double scale, double* out, cudaStream_t st) {
  k_reduce_partials<<<1, 1024, 0, st>>>(nparts, partial, scale, out);
  return cudaGetLastError();
}

cudaError_t launch_gather_in(int n, int n_pad, int nf, const int* perm, const double* lex, double* internal,
                             cudaStream_t st) {
  k_gather_in<<<blocks_for((long long)nf * n_pad, kBlock), kBlock, 0, st>>>(n, n_pad, nf, perm, lex, internal);
  return cudaGetLastError();
}

cudaError_t launch_scatter_out(int n, int n_pad, int nf, const int* perm, const double* internal, double* lex,
                               cudaStream_t st) {
  k_scatter_out<<<blocks_for((long long)nf * n_pad, kBlock), kBlock, 0, st>>>(n, n_pad, nf, perm, internal, lex);
  return cudaGetLastError();
}

cudaError_t launch_combine_field(int n_pad, const double* a, double sa, const double* b, double sb, double* out,
                                 cudaStream_t st) {
  k_combine_field<<<blocks_for(n_pad, kBlock), kBlock, 0, st>>>(n_pad, a, sa, b, sb, out);
  return cudaGetLastError();
}

}  // namespace pfc
