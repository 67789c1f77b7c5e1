// Persistent cooperative kernel for one Rosenbrock stage solve.
//
// One launch runs the whole right-preconditioned FGMRES(restart) with modified
// Gram-Schmidt (Section 4 and Section 6 of Praetorius & Voigt) on
//     A^R = [[M, A01, K], [tau K, M / gamma, 0], [0, K, M]]      (Eq. 3.12, PFC2)
// with the block preconditioner P_CH applied in the steps of Section 4 / 4.2:
//     (1)   M y0 = v0
//     (2)   (M + delta K) y1 = gamma v1 - tau_e K y0
//     (3.1) (M + sqrt(delta) K) w  = M y1
//     (3.2) (M + sqrt(delta) K) x1 = M w
//     (4)   x0 = y0 + (y1 - x1) / delta
//     (5)   M x2 = v2 - K x1
// where tau_e = gamma tau and delta = sqrt(tau_e): the preconditioner of Eq. (4.1)
// is derived for gamma = 1, so the second block row of A^R is scaled by gamma
// and step (2) uses the forward substitution of the lower factor of Eq. (4.1)
// (right-hand side b1 - tau K y0).  Every inner solve is Jacobi-PCG from zero
// to ||r|| <= inner_rtol ||rhs|| (Table 2).
//
// GB300 design.  The grid is co-resident (cooperative launch, a multiple of the
// SM count), every block owns a contiguous, nnz-balanced range of SELL-32 slices
// and the same rows of every vector, and the phases of the algorithm are
// separated by a grid barrier with a bounded spin.  Dot products reduce in a
// fixed order (warp shuffles, then block partials summed identically by every
// block), so all blocks take the same branch decisions and repeated runs are
// bitwise identical.  The scalar Arnoldi/Givens work is done redundantly by
// thread 0 of every block in shared memory.  A vector that another block reads
// (the PCG direction p, the preconditioned basis vector z_j, the iterate y) is
// only read after a barrier; everything else is touched by its owner only.
#include <cuda_fp16.h>

#include "device.cuh"
#include "internal.h"
#include "launch.h"

namespace pfc {
namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kRing = 4;

struct Grid {
  unsigned* arrive;
  int* err;
  double2* part;
  unsigned long long limit_ns;
  int G;
  int expect;      // blocks that arrive at each barrier (G, or more in the timeout self-test)
  unsigned epoch;  // thread 0 only
  int ring;
  int s_lo, s_hi;
};

#define FOR_MY_SLICES(g, s) for (int s = (g).s_lo + (int)(threadIdx.x >> 5); s < (g).s_hi; s += kWarps)

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier: monotone arrival counter; the k-th barrier of a launch
// completes when the counter reaches k * G.  The wait is bounded in time: after
// limit_ns the block sets the timeout bit and the kernel unwinds (false), as it
// does when another block has already flagged a timeout.
__device__ bool grid_sync(Grid& g) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    g.epoch += 1;
    const unsigned target = g.epoch * (unsigned)g.expect;
    __threadfence();
    atomicAdd(g.arrive, 1u);
    unsigned spins = 0;
    unsigned long long t0 = 0;
    int ok = 1;
    while (ld_acquire_u32(g.arrive) < target) {
      if ((++spins & 255u) == 0u) {
        const unsigned long long t = global_ns();
        if (t0 == 0) {
          t0 = t;
        } else if (t - t0 > g.limit_ns) {
          atomicOr(g.err, kErrTimeout);
          ok = 0;
          break;
        }
      }
      __nanosleep(64);
    }
    __threadfence();
    if (ok && (ld_relaxed_i32(g.err) & kErrTimeout)) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Sum of (a, b) over all threads of the grid, identical in every block.
__device__ bool grid_sum2(Grid& g, double a, double b, double2& out) {
  __shared__ double2 s_w[kWarps];
  __shared__ double2 s_res;
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) s_w[w] = make_double2(a, b);
  __syncthreads();
  const int slot = g.ring;
  g.ring = (g.ring + 1) % kRing;
  if (w == 0) {
    double2 t = l < kWarps ? s_w[l] : make_double2(0.0, 0.0);
    t.x = warp_sum(t.x);
    t.y = warp_sum(t.y);
    if (l == 0) __stcg(&g.part[slot * g.G + blockIdx.x], t);
  }
  if (!grid_sync(g)) return false;
  if (w == 0) {
    double2 acc = make_double2(0.0, 0.0);
    for (int i = l; i < g.G; i += 32) {
      const double2 t = __ldcg(&g.part[slot * g.G + i]);
      acc.x += t.x;
      acc.y += t.y;
    }
    acc.x = warp_sum(acc.x);
    acc.y = warp_sum(acc.y);
    if (l == 0) s_res = acc;
  }
  __syncthreads();
  out = s_res;
  return true;
}

__device__ __forceinline__ void flag(Grid& g, int bit) {
  if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(g.err, bit);
}

struct InnerCount {
  long long its = 0;
  int calls = 0;
  int capped = 0;
};

template <class TM, class TV>
struct Ctx {
  using Acc = typename AccOf<TV>::type;
  const SolveArgs& a;
  const TM* iM;
  const TM* iK;
  const TM* iMdK;
  const TM* iMsK;
  const TV* dM;
  const TV* dMdK;
  const TV* dMsK;
  TV *r, *p, *q, *y0, *y1, *wv, *x1, *x2;
  __device__ explicit Ctx(const SolveArgs& args) : a(args) {
    iM = (const TM*)a.iM;
    iK = (const TM*)a.iK;
    iMdK = (const TM*)a.iMdK;
    iMsK = (const TM*)a.iMsK;
    dM = (const TV*)a.dM;
    dMdK = (const TV*)a.dMdK;
    dMsK = (const TV*)a.dMsK;
    TV* base = (TV*)a.ivec;
    const int np = a.n_pad;
    r = base;
    p = base + np;
    q = base + 2 * np;
    y0 = base + 3 * np;
    y1 = base + 4 * np;
    wv = base + 5 * np;
    x1 = base + 6 * np;
    x2 = base + 7 * np;
  }
};

// Jacobi-PCG for A x = rhs, x0 = 0, stop at ||r||_2 <= rtol ||rhs||_2.
// rhs(s, lane, row) is evaluated once per owned row in the first phase (it may
// run a SpMV over vectors completed before the call).
template <class TM, class TV, class RhsF>
__device__ bool pcg(Grid& g, Ctx<TM, TV>& c, const TM* AV, const TV* DI, TV* x, RhsF rhs, double rtol,
                    int maxit, InnerCount& cnt, int& its) {
  using Acc = typename Ctx<TM, TV>::Acc;
  const SolveArgs& a = c.a;
  TV* r = c.r;
  TV* p = c.p;
  TV* q = c.q;
  const int lane = threadIdx.x & 31;
  double pb = 0.0, pz = 0.0;
  FOR_MY_SLICES(g, s) {
    const int row = s * 32 + lane;
    const TV rv = (TV)rhs(s, lane, row);
    const TV z = (TV)((Acc)DI[row] * (Acc)rv);
    x[row] = TV(0);
    r[row] = rv;
    p[row] = z;
    pb += (double)rv * (double)rv;
    pz += (double)rv * (double)z;
  }
  double2 red;
  if (!grid_sum2(g, pb, pz, red)) return false;
  its = 0;
  cnt.calls += 1;
  const double bb = red.x;
  double rz = red.y;
  if (!isfinite(bb)) {
    flag(g, kErrNonfinite);
    return false;
  }
  if (bb == 0.0) return true;
  const double thr = rtol * rtol * bb;
  for (int it = 1; it <= maxit; ++it) {
    double ppq = 0.0;
    FOR_MY_SLICES(g, s) {
      const int row = s * 32 + lane;
      const TV qv = (TV)sell_row<Acc>(a.slice_ptr, a.cols, AV, p, s, lane);
      q[row] = qv;
      ppq += (double)p[row] * (double)qv;
    }
    if (!grid_sum2(g, ppq, 0.0, red)) return false;
    const double pq = red.x;
    if (!isfinite(pq)) {
      flag(g, kErrNonfinite);
      return false;
    }
    if (!(pq > 0.0)) {
      flag(g, kErrBreakdown);
      its = it;
      cnt.its += it;
      return true;
    }
    const Acc alpha = (Acc)(rz / pq);
    double prr = 0.0, prz = 0.0;
    FOR_MY_SLICES(g, s) {
      const int row = s * 32 + lane;
      const Acc xn = (Acc)x[row] + alpha * (Acc)p[row];
      const Acc rn = (Acc)r[row] - alpha * (Acc)q[row];
      x[row] = (TV)xn;
      r[row] = (TV)rn;
      const Acc z = (Acc)DI[row] * rn;
      prr += (double)rn * (double)rn;
      prz += (double)rn * (double)z;
    }
    if (!grid_sum2(g, prr, prz, red)) return false;
    its = it;
    if (!isfinite(red.x)) {
      flag(g, kErrNonfinite);
      return false;
    }
    if (red.x <= thr) {
      cnt.its += it;
      return true;
    }
    const Acc beta = (Acc)(red.y / rz);
    rz = red.y;
    FOR_MY_SLICES(g, s) {
      const int row = s * 32 + lane;
      p[row] = (TV)((Acc)DI[row] * (Acc)r[row] + beta * (Acc)p[row]);
    }
    if (!grid_sync(g)) return false;
  }
  cnt.its += maxit;
  cnt.capped += 1;
  return true;
}

// z = P_CH^{-1} v for 3-field float64 vectors (n_pad per field).  Ends with a
// barrier, so z may be gathered by any block afterwards.
template <class TM, class TV>
__device__ bool apply_pch(Grid& g, Ctx<TM, TV>& c, const double* v, double* z, InnerCount& cnt) {
  using Acc = typename Ctx<TM, TV>::Acc;
  const SolveArgs& a = c.a;
  const int np = a.n_pad;
  const int lane = threadIdx.x & 31;
  const double* v0 = v;
  const double* v1 = v + np;
  const double* v2 = v + 2 * np;
  const double rt = a.inner_rtol;
  const int mi = a.max_inner;
  int its;
  // (1) M y0 = v0
  if (!pcg(g, c, c.iM, c.dM, c.y0, [&](int, int, int row) { return v0[row]; }, rt, mi, cnt, its)) return false;
  // (2) (M + delta K) y1 = gamma v1 - tau_e K y0
  if (!pcg(g, c, c.iMdK, c.dMdK, c.y1,
           [&](int s, int ln, int row) {
             const Acc ky = sell_row<Acc>(a.slice_ptr, a.cols, c.iK, c.y0, s, ln);
             return a.gamma * v1[row] - a.tau_e * (double)ky;
           },
           rt, mi, cnt, its))
    return false;
  // (3.1) (M + sqrt(delta) K) w = M y1
  if (!pcg(g, c, c.iMsK, c.dMsK, c.wv,
           [&](int s, int ln, int) { return (double)sell_row<Acc>(a.slice_ptr, a.cols, c.iM, c.y1, s, ln); }, rt,
           mi, cnt, its))
    return false;
  // (3.2) (M + sqrt(delta) K) x1 = M w
  if (!pcg(g, c, c.iMsK, c.dMsK, c.x1,
           [&](int s, int ln, int) { return (double)sell_row<Acc>(a.slice_ptr, a.cols, c.iM, c.wv, s, ln); }, rt,
           mi, cnt, its))
    return false;
  // (4) x0 = y0 + (y1 - x1) / delta, and z = (x0, x1, .)
  FOR_MY_SLICES(g, s) {
    const int row = s * 32 + lane;
    const double xx1 = (double)c.x1[row];
    z[row] = (double)c.y0[row] + ((double)c.y1[row] - xx1) * a.inv_delta;
    z[np + row] = xx1;
  }
  // (5) M x2 = v2 - K x1
  if (!pcg(g, c, c.iM, c.dM, c.x2,
           [&](int s, int ln, int row) {
             return v2[row] - (double)sell_row<Acc>(a.slice_ptr, a.cols, c.iK, c.x1, s, ln);
           },
           rt, mi, cnt, its))
    return false;
  FOR_MY_SLICES(g, s) {
    const int row = s * 32 + lane;
    z[2 * np + row] = (double)c.x2[row];
  }
  return grid_sync(g);
}

// w = A^R z for one owned row (float64, one column-index stream, three value streams).
__device__ __forceinline__ void block_row(const SolveArgs& a, const double* z, int s, int lane, double& w0,
                                          double& w1, double& w2) {
  const int np = a.n_pad;
  const int beg = __ldg(a.slice_ptr + s) + lane;
  const int end = __ldg(a.slice_ptr + s + 1);
  double m_mu = 0, a_psi = 0, k_om = 0, k_mu = 0, m_psi = 0, k_psi = 0, m_om = 0;
#pragma unroll 2
  for (int idx = beg; idx < end; idx += 32) {
    const int c = __ldg(a.cols + idx);
    const double mv = __ldg(a.Mv + idx), kv = __ldg(a.Kv + idx), av = __ldg(a.Av + idx);
    const double zm = z[c], zp = z[np + c], zo = z[2 * np + c];
    m_mu = fma(mv, zm, m_mu);
    a_psi = fma(av, zp, a_psi);
    k_om = fma(kv, zo, k_om);
    k_mu = fma(kv, zm, k_mu);
    m_psi = fma(mv, zp, m_psi);
    k_psi = fma(kv, zp, k_psi);
    m_om = fma(mv, zo, m_om);
  }
  w0 = m_mu + a_psi + k_om;
  w1 = a.tau * k_mu + a.inv_gamma * m_psi;
  w2 = k_psi + m_om;
}

template <class TM, class TV>
__device__ void write_stats(Grid& g, const SolveArgs& a, int outer, int restarts, const InnerCount& cnt,
                            double rel, double bnorm, int last_its) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    DevStats st;
    st.outer_its = outer;
    st.restarts = restarts;
    st.inner_calls = cnt.calls;
    st.inner_capped = cnt.capped;
    st.inner_its = cnt.its;
    st.rel_residual = rel;
    st.bnorm = bnorm;
    st.err = 0;
    st.last_its = last_its;
    *a.stats = st;
  }
}

template <class TM, class TV>
__device__ void fgmres(Grid& g, Ctx<TM, TV>& c) {
  const SolveArgs& a = c.a;
  __shared__ double H[(kMaxRestart + 1) * kMaxRestart];
  __shared__ double gv[kMaxRestart + 1], cs[kMaxRestart], sn[kMaxRestart], yk[kMaxRestart];
  __shared__ int s_k;
  const int np = a.n_pad, n3 = 3 * np, m = a.restart, ld = m + 1;
  const int lane = threadIdx.x & 31;
  InnerCount cnt;
  double2 red;
  double pb = 0.0;
  FOR_MY_SLICES(g, s) {
    const int row = s * 32 + lane;
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      const double bv = a.b[f * np + row];
      pb += bv * bv;
      a.y[f * np + row] = 0.0;
    }
  }
  if (!grid_sum2(g, pb, 0.0, red)) return;
  const double bnorm = sqrt(red.x);
  if (!isfinite(bnorm)) {
    flag(g, kErrNonfinite);
    return;
  }
  if (bnorm == 0.0) {
    write_stats<TM, TV>(g, a, 0, 0, cnt, 0.0, 0.0, 0);
    return;
  }
  int total = 0, restarts = 0;
  bool first = true;
  while (true) {
    // r = b - A^R y  -> V_0 (y = 0 on the first cycle)
    double* V0 = a.V;
    double pr = 0.0;
    FOR_MY_SLICES(g, s) {
      const int row = s * 32 + lane;
      double w0 = 0.0, w1 = 0.0, w2 = 0.0;
      if (!first) block_row(a, a.y, s, lane, w0, w1, w2);
      const double r0 = a.b[row] - w0, r1 = a.b[np + row] - w1, r2 = a.b[2 * np + row] - w2;
      V0[row] = r0;
      V0[np + row] = r1;
      V0[2 * np + row] = r2;
      pr += r0 * r0 + r1 * r1 + r2 * r2;
    }
    if (!grid_sum2(g, pr, 0.0, red)) return;
    const double beta = sqrt(red.x);
    if (!isfinite(beta)) {
      flag(g, kErrNonfinite);
      return;
    }
    if (beta <= a.tol * bnorm || total >= a.max_outer) {
      if (beta > a.tol * bnorm) flag(g, kErrOuterCap);
      write_stats<TM, TV>(g, a, total, restarts, cnt, beta / bnorm, bnorm, 0);
      return;
    }
    first = false;
    const double ib = 1.0 / beta;
    FOR_MY_SLICES(g, s) {
      const int row = s * 32 + lane;
#pragma unroll
      for (int f = 0; f < 3; ++f) V0[f * np + row] *= ib;
    }
    if (threadIdx.x == 0) {
      gv[0] = beta;
      for (int i = 1; i <= m; ++i) gv[i] = 0.0;
    }
    int k = 0;
    for (int j = 0; j < m; ++j) {
      const double* vj = a.V + (size_t)j * n3;
      double* zj = a.Z + (size_t)j * n3;
      double* w = a.V + (size_t)(j + 1) * n3;
      if (!apply_pch(g, c, vj, zj, cnt)) return;
      // w = A^R z_j, then modified Gram-Schmidt against V_0..V_j
      double ph = 0.0;
      FOR_MY_SLICES(g, s) {
        const int row = s * 32 + lane;
        double w0, w1, w2;
        block_row(a, zj, s, lane, w0, w1, w2);
        w[row] = w0;
        w[np + row] = w1;
        w[2 * np + row] = w2;
        ph += w0 * V0[row] + w1 * V0[np + row] + w2 * V0[2 * np + row];
      }
      if (!grid_sum2(g, ph, 0.0, red)) return;
      double hij = red.x;
      for (int i = 0; i <= j; ++i) {
        if (threadIdx.x == 0) H[i + j * ld] = hij;
        const double* vi = a.V + (size_t)i * n3;
        const double* vn = i < j ? a.V + (size_t)(i + 1) * n3 : nullptr;
        double pn = 0.0;
        FOR_MY_SLICES(g, s) {
          const int row = s * 32 + lane;
#pragma unroll
          for (int f = 0; f < 3; ++f) {
            const double wv = w[f * np + row] - hij * vi[f * np + row];
            w[f * np + row] = wv;
            pn += wv * (vn ? vn[f * np + row] : wv);
          }
        }
        if (!grid_sum2(g, pn, 0.0, red)) return;
        hij = red.x;
      }
      const double hnext = sqrt(hij);
      if (!isfinite(hnext)) {
        flag(g, kErrNonfinite);
        return;
      }
      if (threadIdx.x == 0) {
        for (int i = 0; i < j; ++i) {
          const double t = cs[i] * H[i + j * ld] + sn[i] * H[i + 1 + j * ld];
          H[i + 1 + j * ld] = -sn[i] * H[i + j * ld] + cs[i] * H[i + 1 + j * ld];
          H[i + j * ld] = t;
        }
        const double hjj = H[j + j * ld];
        const double den = hypot(hjj, hnext);
        cs[j] = hjj / den;
        sn[j] = hnext / den;
        H[j + j * ld] = den;
        H[j + 1 + j * ld] = 0.0;
        gv[j + 1] = -sn[j] * gv[j];
        gv[j] = cs[j] * gv[j];
      }
      __syncthreads();
      total += 1;
      k = j + 1;
      if (fabs(gv[j + 1]) <= a.tol * bnorm || hnext == 0.0 || total >= a.max_outer) break;
      const double ih = 1.0 / hnext;
      FOR_MY_SLICES(g, s) {
        const int row = s * 32 + lane;
#pragma unroll
        for (int f = 0; f < 3; ++f) w[f * np + row] *= ih;
      }
    }
    // y += Z_k c, with R c = g (back substitution on the rotated Hessenberg matrix)
    if (threadIdx.x == 0) {
      for (int i = k - 1; i >= 0; --i) {
        double t = gv[i];
        for (int l = i + 1; l < k; ++l) t -= H[i + l * ld] * yk[l];
        yk[i] = t / H[i + i * ld];
      }
      s_k = k;
    }
    __syncthreads();
    const int kk = s_k;
    FOR_MY_SLICES(g, s) {
      const int row = s * 32 + lane;
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        double acc = a.y[f * np + row];
        for (int i = 0; i < kk; ++i) acc = fma(yk[i], a.Z[(size_t)i * n3 + f * np + row], acc);
        a.y[f * np + row] = acc;
      }
    }
    restarts += 1;
    if (!grid_sync(g)) return;
  }
}

template <class TM, class TV>
__global__ void __launch_bounds__(kThreads, 2) solve_kernel(const SolveArgs a) {
  Grid g;
  g.arrive = a.arrive;
  g.err = a.err;
  g.part = a.part;
  g.G = gridDim.x;
  g.expect = gridDim.x + a.barrier_extra;
  g.limit_ns = a.spin_limit_ns;
  g.epoch = 0;
  g.ring = 0;
  g.s_lo = __ldg(a.blk + blockIdx.x);
  g.s_hi = __ldg(a.blk + blockIdx.x + 1);
  Ctx<TM, TV> c(a);
  const int lane = threadIdx.x & 31;
  if (a.mode == 0) {
    fgmres(g, c);
  } else if (a.mode == 1) {
    InnerCount cnt;
    if (apply_pch(g, c, a.b, a.y, cnt)) write_stats<TM, TV>(g, a, 0, 0, cnt, 0.0, 0.0, 0);
  } else {
    InnerCount cnt;
    int its = 0;
    const TM* AV = a.which == 0 ? c.iM : a.which == 1 ? c.iMdK : c.iMsK;
    const TV* DI = a.which == 0 ? c.dM : a.which == 1 ? c.dMdK : c.dMsK;
    const double* b = a.b;
    if (!pcg(g, c, AV, DI, c.y0, [&](int, int, int row) { return b[row]; }, a.inner_rtol, a.max_inner, cnt, its))
      return;
    FOR_MY_SLICES(g, s) {
      const int row = s * 32 + lane;
      a.y[row] = (double)c.y0[row];
    }
    write_stats<TM, TV>(g, a, 0, 0, cnt, 0.0, 0.0, its);
  }
}

template <class TM, class TV>
const void* kernel_ptr() {
  return (const void*)solve_kernel<TM, TV>;
}

const void* kernel_for(int prec) {
  if (prec == 0) return kernel_ptr<double, double>();
  if (prec == 1) return kernel_ptr<float, float>();
  return kernel_ptr<__half, float>();
}

}  // namespace

int solve_threads() { return kThreads; }
int solve_ring() { return kRing; }

cudaError_t solve_occupancy(int prec, int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kernel_for(prec), kThreads, 0);
}

cudaError_t launch_solve(int prec, int grid, const SolveArgs& args, cudaStream_t stream) {
  SolveArgs local = args;
  void* params[] = {&local};
  return cudaLaunchCooperativeKernel(kernel_for(prec), dim3(grid), dim3(kThreads), params, 0, stream);
}

}  // namespace pfc
