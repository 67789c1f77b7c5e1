// Persistent cooperative kernel for one Rosenbrock stage solve.
//
// One launch runs the whole right-preconditioned FGMRES(restart) with modified
// Gram-Schmidt (Section 4 and Section 7 of Praetorius & Voigt) on
//     A^R = [[M, A01, K], [tau K, M / gamma, 0], [0, K, M]]      (Eq. 3.10, PFC2)
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
// (right-hand side b1 - tau K y0).  For PFC1 the second block row of A^R is
// [tau K_+(psi_k), M / gamma + tau F(mu_k), 0] (assembled A10, A11), and P_CH uses
// the constant-mobility approximation K_+ ~ M0 K of Section 4: tau_e = gamma M0 tau.  Every inner solve is Jacobi-PCG from zero
// to ||r|| <= inner_rtol ||rhs|| (Table 2).
//
// GB300 design.  The grid is co-resident (cooperative launch, a multiple of the
// SM count), every block owns a contiguous, nnz-balanced range of SELL-32 slices
// and the same rows of every vector, and the phases of the algorithm are
// separated by a grid barrier with a time-bounded spin.  Inside a phase each warp
// walks its contiguous run of slices (kGroup at a time; 1 by default: wider
// staging spilled registers), and the block ranges are cut by a cost model that
// weights the boundary rows' assembled SELL rows above the stencil rows.
// Dot products reduce in a fixed order (warp shuffles, then block partials
// summed identically by every block), so all blocks take the same branch
// decisions and repeated runs are bitwise identical.  The scalar Arnoldi/Givens
// work is done redundantly by thread 0 of every block in shared memory.  A
// vector that another block reads (the PCG direction, the preconditioned basis
// vector z_j, the iterate y) is only read after a barrier; everything else is
// touched by its owner only.
//
// The inner CG comes in three arithmetically equivalent forms: the textbook
// Jacobi-PCG (three barriers per iteration: after q = A p with p.q, after the
// x/r update with r.z, after the p update); the Chronopoulos-Gear form (two:
// vector recurrences with r.r, then w = A u with both inner products); and the
// pipelined PCG of Ghysels and Vanroose (Parallel Computing 40, 2014), which
// carries w = A u and m = D w as extra recurrences so that one pass does the
// SpMV, every vector update and all partial dot products (one barrier).
#include <cuda_fp16.h>

#include "device.cuh"
#include "internal.h"
#include "launch.h"

namespace pfc {
namespace {

// Launch shape (compile-time): threads per block, minimum resident blocks per SM
// (which caps registers per thread), and the SpMV row form (0: rolled loop
// unrolled by 4; 1: CH loads of a row issued before its gathers).
#ifndef PFC_SOLVER_THREADS
#define PFC_SOLVER_THREADS 1024
#endif
#ifndef PFC_SOLVER_MINBLOCKS
#define PFC_SOLVER_MINBLOCKS 1
#endif
#ifndef PFC_SPMV_WIDE
#define PFC_SPMV_WIDE 1
#endif
#ifndef PFC_GROUP
#define PFC_GROUP 1
#endif
#ifndef PFC_INTERLEAVE
#define PFC_INTERLEAVE 0
#endif
#ifndef PFC_NEIGHBOR_SYNC
#define PFC_NEIGHBOR_SYNC 0
#endif
#ifndef PFC_ST_UNROLL
#define PFC_ST_UNROLL 4
#endif
// the stencil tables are padded to a multiple of 4 entries per type
static_assert(4 % PFC_ST_UNROLL == 0, "PFC_ST_UNROLL must divide 4");

constexpr int kThreads = PFC_SOLVER_THREADS;
constexpr int kWarps = kThreads / 32;
constexpr int kRing = 4;
constexpr int kGroup = PFC_GROUP;   // slices a warp stages at once in vector phases

// phase classes for the optional profile
enum : int { kPhSpmv = 0, kPhVec = 1, kPhOuter = 2, kPhInit = 3 };

struct Grid {
  unsigned* arrive;
  double4_32a* part;
  int* err;
  unsigned long long limit_ns;
  int G;
  int expect;      // blocks that arrive at each barrier (G, or more in the timeout self-test)
  unsigned epoch;  // thread 0 only
  int ring;
  int bid;         // block index inside this solve's grid (its segment in a batched launch)
  int w_lo, w_hi;  // this warp's contiguous slice range (cost balanced on the host)
  int b_lo, b_hi;  // this block's slice range
  int wid;         // warp index in the block
  int sp_lane;     // start slot of this warp's lane-th slice (when sp_reg)
  int sp_end;      // end slot of this warp's lane-th slice (when sp_reg)
  bool sp_reg;     // the slot bounds of all of this warp's slices live in sp_lane / sp_end
  bool prof;       // block 0, thread 0 (accumulators live in shared memory)
  int win_lo, win_n;  // rows [win_lo, win_lo + win_n) of the SpMV source held in s_win
  bool staged;        // stencil SpMVs read the source vector from s_win
  bool ri_smem;       // the block's row-info bytes are in s_rowinfo (row - 32 b_lo)
  // neighbour synchronisation (structured stencils): blocks nb_lo..nb_hi own the rows
  // this block's stencils reach; flags[b] counts block b's published phases
  bool nbsync;
  int nb_lo, nb_hi;
  unsigned nepoch;
  unsigned* flags;
};


__shared__ unsigned long long s_t_last;
__shared__ long long s_prof[8];
// structured-stencil tables, loaded once per block: entry offsets, the start of
// each dof type, and the weights of the four inner operators in the inner type
__shared__ int s_st_start[9];   // first table entry of each dof type (type * stride)
__shared__ int s_st_cnt[9];     // entries of each dof type; the last type is all padding
__shared__ __align__(16) unsigned char s_st_raw[4 * kMaxStencil * 16];

// the row-info bytes of the block's rows (structured stencils), when they fit
constexpr int kRowInfoCap = 16384;
__shared__ __align__(16) unsigned char s_rowinfo[kRowInfoCap];

// Row-info byte of row (one of this block's rows): dof type in bits 0-2, interior bit 3.
__device__ __forceinline__ unsigned row_info(const Grid& g, const SolveArgs& a, int row) {
  return g.ri_smem ? (unsigned)s_rowinfo[row - g.b_lo * 32] : (unsigned)__ldg(a.rowinfo + row);
}

// dynamic shared memory: the block's window of the SpMV source vector (float
// inner vectors, structured stencils; see stage_window)
extern __shared__ __align__(16) float s_win[];

// one stencil entry: column offset and weight, read with a single shared load
template <class Acc> struct StEntry;
template <> struct __align__(8) StEntry<float> { int off; float w; };
template <> struct __align__(16) StEntry<double> { int off; int pad; double w; };

// Slices of a block are dealt to its warps.  Interleaved (default): warp w takes
// the groups of kGroup consecutive slices starting at b_lo + (w + m kWarps) kGroup,
// m = 0, 1, ..., so that every warp gets the same mix of slice kinds (on the
// structured mesh, lattice rows of vertex dofs have longer stencils than rows of
// edge dofs, and a contiguous range would keep a warp inside one lattice row).
// Contiguous: warp w takes the range [w_lo, w_hi) the host cut by cost.  Rows of
// a group: (s0 + u) * 32 + lane, u < nsl.
#if PFC_INTERLEAVE
#define FOR_MY_GROUPS(g, s0, nsl)                                                                 \
  for (int s0 = (g).b_lo + (g).wid * kGroup; s0 < (g).b_hi; s0 += kGroup * kWarps) \
    if (const int nsl = min(kGroup, (g).b_hi - s0); true)
#define FOR_MY_SLICES(g, s) for (int s = (g).b_lo + (g).wid; s < (g).b_hi; s += kWarps)
#else
#define FOR_MY_GROUPS(g, s0, nsl)                                     \
  for (int s0 = (g).w_lo; s0 < (g).w_hi; s0 += kGroup) \
    if (const int nsl = min(kGroup, (g).w_hi - s0); true)
#define FOR_MY_SLICES(g, s) for (int s = (g).w_lo; s < (g).w_hi; ++s)
#endif

#if PFC_INTERLEAVE
#define PFC_WARP_END(g) (g).b_hi
#else
#define PFC_WARP_END(g) (g).w_hi
#endif

// Position of slice s in this warp's list of slices (the order of the loops above).
__device__ __forceinline__ int my_slice_index(const Grid& g, int s) {
#if PFC_INTERLEAVE
  const int d = s - g.b_lo - g.wid * kGroup;
  return (d / (kGroup * kWarps)) * kGroup + d % (kGroup * kWarps);
#else
  return s - g.w_lo;
#endif
}

// The k-th slice of this warp's list (may lie past the block's range).
__device__ __forceinline__ int my_slice(const Grid& g, int k) {
#if PFC_INTERLEAVE
  return g.b_lo + g.wid * kGroup + (k / kGroup) * kGroup * kWarps + k % kGroup;
#else
  return g.w_lo + k;
#endif
}

// First slot and end slot of slice s (one of this warp's slices).  Called by
// all 32 lanes together.
__device__ __forceinline__ int2 slice_bounds(const Grid& g, const int* __restrict__ sp, int s) {
  if (g.sp_reg) {
    const int k = my_slice_index(g, s);
    return make_int2(__shfl_sync(0xffffffffu, g.sp_lane, k), __shfl_sync(0xffffffffu, g.sp_end, k));
  }
  return make_int2(__ldg(sp + s), __ldg(sp + s + 1));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier: monotone arrival counter; the k-th barrier of a launch
// completes when the counter reaches k * G.  The wait is bounded in time: after
// limit_ns the block sets the timeout bit and the kernel unwinds (false), as it
// does when it sees, while waiting, that another block has flagged a timeout.
// The flag is read only inside the wait, so a completed barrier costs no extra
// memory round trip; a block that passes a barrier after another block timed
// out stops at the next one, which the timed-out block never reaches.
// entry_sync = false when the caller has already synchronised the block after
// its last global write (only thread 0's own stores may follow that barrier).
__device__ bool grid_sync(Grid& g, int tag, bool entry_sync = true) {
  __shared__ int s_ok;
  if (entry_sync) __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t_in = 0;
    if (g.prof) {
      t_in = global_ns();
      s_prof[tag] += (long long)(t_in - s_t_last);
    }
    g.epoch += 1;
    const unsigned target = g.epoch * (unsigned)g.expect;
    // release: this block's writes (ordered before by the __syncthreads above) are
    // visible to every block whose acquire load below sees the new count
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" :: "l"(g.arrive) : "memory");
    unsigned spins = 0;
    unsigned long long t0 = 0;
    int ok = 1;
    while (ld_acquire_u32(g.arrive) < target) {
      if ((++spins & 255u) == 0u) {
        if (ld_relaxed_i32(g.err) & kErrTimeout) {
          ok = 0;
          break;
        }
        const unsigned long long t = global_ns();
        if (t0 == 0) {
          t0 = t;
        } else if (t - t0 > g.limit_ns) {
          atomicOr(g.err, kErrTimeout);
          ok = 0;
          break;
        }
      }
    }
    s_ok = ok;
    if (g.prof) {
      s_t_last = global_ns();
      s_prof[4 + tag] += (long long)(s_t_last - t_in);
    }
  }
  __syncthreads();
  return s_ok != 0;
}

// Adds the time since the last mark to the work of phase class tag (profiling only;
// call after a __syncthreads, so that it times the whole block).
__device__ __forceinline__ void prof_mark(const Grid& g, int tag) {
  if (g.prof) {
    const unsigned long long t = global_ns();
    s_prof[tag] += (long long)(t - s_t_last);
    s_t_last = t;
  }
}

// Wait until every block whose rows this block's stencil reaches has finished the
// current phase (a point-to-point replacement for a grid barrier before an SpMV
// whose only cross-block inputs are the source vector's halo rows).  Each block
// publishes its phase count with a release store; thread k waits for neighbour
// nb_lo + k with relaxed loads and one acquire load once it has seen the count.
// The wait is bounded like grid_sync's.
__device__ bool neighbor_sync(Grid& g, int tag) {
  __syncthreads();
  unsigned long long t_in = 0;
  if (g.prof) {
    t_in = global_ns();
    s_prof[tag] += (long long)(t_in - s_t_last);
  }
  g.nepoch += 1;
  const unsigned ep = g.nepoch;
  if (threadIdx.x == 0)
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(g.flags + g.bid), "r"(ep) : "memory");
  const int nb = g.nb_lo + (int)threadIdx.x;
  int bad = 0;
  if (nb <= g.nb_hi && nb != g.bid) {
    unsigned v = 0, spins = 0;
    unsigned long long t0 = 0;
    while (true) {
      asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(g.flags + nb) : "memory");
      if (v >= ep) {
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(g.flags + nb) : "memory");
        break;
      }
      if ((++spins & 255u) == 0u) {
        const unsigned long long t = global_ns();
        if (t0 == 0) {
          t0 = t;
        } else if (t - t0 > g.limit_ns) {
          atomicOr(g.err, kErrTimeout);
          bad = 1;
          break;
        }
        if (ld_relaxed_i32(g.err) & kErrTimeout) {
          bad = 1;
          break;
        }
      }
    }
  }
  bad = __syncthreads_or(bad);
  if (g.prof) {
    s_t_last = global_ns();
    s_prof[4 + tag] += (long long)(s_t_last - t_in);
  }
  return bad == 0;
}

// Result of a grid reduction, in the arithmetic of its tree.
template <class T>
struct alignas(4 * sizeof(T)) Sum4 {
  T x, y, z, w;
};

// A block's partial in its 32-byte ring slot: float4 for a float tree, two
// double2 (the second only when the third value is live) for a double tree.
template <class T, int NV>
__device__ __forceinline__ void store_partial(double4_32a* slot, T x, T y, T z) {
  if constexpr (sizeof(T) == 4) {
    __stcg(reinterpret_cast<float4*>(slot), make_float4(x, y, z, 0.f));
  } else {
    double2* dst = reinterpret_cast<double2*>(slot);
    __stcg(dst, make_double2(x, y));
    if constexpr (NV >= 3) __stcg(dst + 1, make_double2(z, 0.0));
  }
}

template <class T, int NV>
__device__ __forceinline__ void load_partial(const double4_32a* slot, T& x, T& y, T& z) {
  if constexpr (sizeof(T) == 4) {
    const float4 t = __ldcg(reinterpret_cast<const float4*>(slot));
    x = t.x;
    y = t.y;
    z = t.z;
  } else {
    const double2* src = reinterpret_cast<const double2*>(slot);
    const double2 t0 = __ldcg(src);
    x = t0.x;
    y = t0.y;
    if constexpr (NV >= 3) z = __ldcg(src + 1).x;
  }
}

// Sum of up to three values over all threads of the grid, identical in every block.
// Each block publishes its partial in a 32-byte ring slot; after the barrier
// every thread of a block loads at most one partial (the grid has at most
// kThreads blocks), so the read-back is one memory round trip, and the partials
// are summed in a fixed order.
// NV: how many of a, b, c are live (the others are zero and skip their trees).
// T is the arithmetic and the storage of every stage of the tree: float for the
// float32 inner solves, double everywhere else.  Nothing is converted between
// the two on the way: a float64 conversion runs at the scarce float64 rate of
// GB300, and the caller's threads would each pay for one per value.
template <class T, int NV = 3>
__device__ bool grid_sum(Grid& g, T a, T b, T c, Sum4<T>& out, int tag) {
  __shared__ Sum4<T> s_w[kWarps];
  __shared__ Sum4<T> s_res;
  a = warp_sum(a);
  if constexpr (NV >= 2) b = warp_sum(b);
  if constexpr (NV >= 3) c = warp_sum(c);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) s_w[w] = Sum4<T>{a, b, c, T(0)};
  __syncthreads();
  const int slot = g.ring;
  g.ring = (g.ring + 1) % kRing;
  if (w == 0) {
    T tx = T(0), ty = T(0), tz = T(0);
    if (l < kWarps) {
      const Sum4<T> t = s_w[l];
      tx = t.x;
      ty = t.y;
      tz = t.z;
    }
    tx = warp_sum(tx);
    if constexpr (NV >= 2) ty = warp_sum(ty);
    if constexpr (NV >= 3) tz = warp_sum(tz);
    if (l == 0) store_partial<T, NV>(g.part + slot * g.G + g.bid, tx, ty, tz);
  }
  // every thread's writes precede the __syncthreads above; the partial is thread 0's
  if (!grid_sync(g, tag, false)) return false;
  // one partial per thread of the first ceil(G / 32) warps, summed in a fixed order
  if (w * 32 < g.G) {
    T px = T(0), py = T(0), pz = T(0);
    if ((int)threadIdx.x < g.G) load_partial<T, NV>(g.part + slot * g.G + threadIdx.x, px, py, pz);
    px = warp_sum(px);
    if constexpr (NV >= 2) py = warp_sum(py);
    if constexpr (NV >= 3) pz = warp_sum(pz);
    if (l == 0) s_w[w] = Sum4<T>{px, py, pz, T(0)};
  }
  __syncthreads();
  if (w == 0) {
    const int nw = (g.G + 31) >> 5;
    T tx = T(0), ty = T(0), tz = T(0);
    if (l < nw) {
      const Sum4<T> t = s_w[l];
      tx = t.x;
      ty = t.y;
      tz = t.z;
    }
    tx = warp_sum(tx);
    if constexpr (NV >= 2) ty = warp_sum(ty);
    if constexpr (NV >= 3) tz = warp_sum(tz);
    if (l == 0) s_res = Sum4<T>{tx, ty, tz, T(0)};
  }
  __syncthreads();
  out = s_res;
  return true;
}

__device__ __forceinline__ void flag(Grid& g, int bit) {
  if (threadIdx.x == 0 && g.bid == 0) atomicOr(g.err, bit);
}

// One SELL-32 row (lane = row of slice s) times x, loading CH column indices and
// values of the row before any of the CH gathers, so a row of up to CH
// nonzeros costs two dependent memory round trips.
template <class Acc, class TM, class TX>
__device__ __forceinline__ Acc sell_row_wide_impl(int2 se, const int* __restrict__ cols, const TM* __restrict__ vals,
                                                  const TX* x, int lane) {
#ifdef PFC_WIDE_CH
  constexpr int CH = PFC_WIDE_CH;
#else
  constexpr int CH = 10;
#endif
  const int w = (se.y - se.x) >> 5;
  const int beg = se.x + lane;
  Acc acc = Acc(0);
  for (int j0 = 0; j0 < w; j0 += CH) {
    int cc[CH];
    Acc vv[CH];
#pragma unroll
    for (int jj = 0; jj < CH; ++jj) {
      cc[jj] = 0;
      vv[jj] = Acc(0);
      if (j0 + jj < w) {
        const int idx = beg + (j0 + jj) * 32;
        cc[jj] = __ldg(cols + idx);
        vv[jj] = ld_val<Acc>(vals + idx);
      }
    }
    Acc xv[CH];
#pragma unroll
    for (int jj = 0; jj < CH; ++jj) xv[jj] = (j0 + jj < w) ? (Acc)x[cc[jj]] : Acc(0);
#pragma unroll
    for (int jj = 0; jj < CH; ++jj) acc = fma(vv[jj], xv[jj], acc);
  }
  return acc;
}

template <class Acc, class TM, class TX>
__device__ __forceinline__ Acc sell_row_wide(int2 se, const int* __restrict__ cols, const TM* __restrict__ vals,
                                             const TX* x, int lane) {
#if PFC_SPMV_WIDE
  return sell_row_wide_impl<Acc>(se, cols, vals, x, lane);
#else
  Acc acc = Acc(0);
#pragma unroll 4
  for (int idx = se.x + lane; idx < se.y; idx += 32) acc = fma(ld_val<Acc>(vals + idx), (Acc)x[__ldg(cols + idx)], acc);
  return acc;
#endif
}

// Row `row` (slice s, this lane) of inner operator op, whose assembled values are
// vals: interior rows use the structured stencil from shared memory (no matrix
// or index bytes), the others their SELL row.  Called by all 32 lanes together.
template <class Acc, class TM, class TX>
__device__ __forceinline__ Acc inner_row(const Grid& g, const SolveArgs& a, int op, const TM* __restrict__ vals,
                                         const TX* x, int s, int lane) {
  const int2 se = slice_bounds(g, a.slice_ptr, s);
  if (a.stencil) {
    const int row = s * 32 + lane;
    const unsigned info = row_info(g, a, row);
    if (info & 8u) {
      const int t = info & 7u;
      const int k0 = s_st_start[t], k1 = k0 + s_st_cnt[t];
      const StEntry<Acc>* tab = reinterpret_cast<const StEntry<Acc>*>(s_st_raw) + op * kMaxStencil;
      Acc acc = Acc(0);
#pragma unroll 8
      for (int k = k0; k < k1; ++k) {
        const StEntry<Acc> e = tab[k];
        acc = fma(e.w, (Acc)x[row + e.off], acc);
      }
      return acc;
    }
  }
  return sell_row_wide<Acc>(se, a.cols, vals, x, lane);
}

// Copies rows [win_lo, win_lo + win_n) of x into the block's shared window; called
// by all threads of the block, only when g.staged (float vectors).  The window is
// the block's own rows widened by the largest stencil offset on both sides and
// rounded out to multiples of 4 floats, so every interior row's stencil reads
// inside it; x is 16-byte aligned.  The first barrier keeps warps still reading
// the previous window safe, the second publishes the new one.
template <class TX>
__device__ __forceinline__ void stage_window(const Grid& g, const TX* x) {
  __syncthreads();
  if constexpr (sizeof(TX) == 4) {
    const float4* src = reinterpret_cast<const float4*>(x + g.win_lo);
    float4* dst = reinterpret_cast<float4*>(s_win);
    const int n4 = g.win_n >> 2;
    for (int i = threadIdx.x; i < n4; i += kThreads) dst[i] = src[i];
  }
  __syncthreads();
}

// Rows (s0 + u) * 32 + lane, u < nsl, of inner operator op applied to x: the
// group form of inner_row for the SpMV phases.  Each row of the group has its own
// dof type; all lanes loop up to the longest stencil among the warp's rows and
// predicate per row, so lanes of different types (they alternate along x) do not
// serialise, and the loads of all rows of the group are in flight together.  Each
// row accumulates its entries in the same order as inner_row, so the results are
// the same bits.  Rows with a missing element take their SELL row.  Called by all
// 32 lanes together.
template <class Acc, class TM, class TX>
__device__ __forceinline__ void inner_rows(const Grid& g, const SolveArgs& a, int op, const TM* __restrict__ vals,
                                           const TX* x, int s0, int nsl, int lane, Acc (&out)[kGroup],
                                           bool from_win = false) {
  if (!a.stencil) {
#pragma unroll
    for (int uu = 0; uu < kGroup; ++uu)
      if (uu < nsl) out[uu] = sell_row_wide<Acc>(slice_bounds(g, a.slice_ptr, s0 + uu), a.cols, vals, x, lane);
    return;
  }
  const StEntry<Acc>* tab = reinterpret_cast<const StEntry<Acc>*>(s_st_raw) + op * kMaxStencil;
  // every type's entries are padded with (offset 0, weight 0) up to the table
  // stride, and the extra type a.st_types is padding only: rows past the group's
  // end and rows with a missing element run the loop on it, reading x at a valid row
  int base[kGroup], rowc[kGroup];
  bool interior[kGroup];
  int nmax = 0;
#pragma unroll
  for (int uu = 0; uu < kGroup; ++uu) {
    base[uu] = s_st_start[a.st_types];
    rowc[uu] = s0 * 32 + lane;
    interior[uu] = true;
    if (uu < nsl) {
      rowc[uu] = (s0 + uu) * 32 + lane;
      const unsigned info = row_info(g, a, rowc[uu]);
      interior[uu] = (info & 8u) != 0;
      if (interior[uu]) {
        const int t = info & 7u;
        base[uu] = s_st_start[t];
        nmax = max(nmax, s_st_cnt[t]);
      }
    }
  }
  nmax = __reduce_max_sync(0xffffffffu, nmax);
  Acc acc[kGroup];
#pragma unroll
  for (int uu = 0; uu < kGroup; ++uu) acc[uu] = Acc(0);
  if (from_win) {
    // the interior rows' reach lies inside the window (see stage_window)
    for (int k = 0; k < nmax; k += PFC_ST_UNROLL) {
#pragma unroll
      for (int j = 0; j < PFC_ST_UNROLL; ++j) {
#pragma unroll
        for (int uu = 0; uu < kGroup; ++uu) {
          const StEntry<Acc> e = tab[base[uu] + k + j];
          acc[uu] = fma(e.w, (Acc)s_win[rowc[uu] - g.win_lo + e.off], acc[uu]);
        }
      }
    }
  } else {
    for (int k = 0; k < nmax; k += PFC_ST_UNROLL) {
#pragma unroll
      for (int j = 0; j < PFC_ST_UNROLL; ++j) {
#pragma unroll
        for (int uu = 0; uu < kGroup; ++uu) {
          const StEntry<Acc> e = tab[base[uu] + k + j];
          acc[uu] = fma(e.w, (Acc)x[rowc[uu] + e.off], acc[uu]);
        }
      }
    }
  }
#pragma unroll
  for (int uu = 0; uu < kGroup; ++uu) {
    if (uu < nsl) {
      const int2 se = slice_bounds(g, a.slice_ptr, s0 + uu);
      if (!interior[uu]) acc[uu] = sell_row_wide<Acc>(se, a.cols, vals, x, lane);
      out[uu] = acc[uu];
    }
  }
}

// ---------------------------------------------------------------------------
// Chunked stencil SpMV with bulk-copied source windows (float inner vectors).
//
// The block walks its rows in chunks of kChunk consecutive rows, one row per thread.
// Before a chunk is computed, one thread bulk-copies the chunk's source window -
// every lattice line its interior rows' stencils can reach: the chunk's lines and two
// more on each side (2D: one contiguous segment; 3D: that band of lines in each of the
// five planes around the chunk's plane) - from global into shared memory with
// cp.async.bulk, completing on an mbarrier.  Two buffers alternate, so the copy of
// chunk k + 2 runs while chunk k + 1 is computed.  The stencil then reads shared
// memory only: a chunk's 1024 rows share one window, where separate warps each
// gathered their own lines through L1 (in 3D a warp's 32 rows reach ~25 lines of five
// planes, and the reuse of those lines by later slices falls outside L1).
//
// Window index.  With g0 the first copied element and S the stride between plane
// segments (S = plane mod 4, so every segment starts 16-byte aligned), element e of
// plane p sits at  e - g0 - (p - p_lo)(plane - S);  a stencil entry with row offset
// off = dx + lat dy + plane dz therefore sits at a fixed distance
// sdelta = off - dz (plane - S) from its row's own index (2D: plane = 0, sdelta = off).
// Interior rows reach at most two lines (planes) away, inside the window.  A chunk
// whose rows cross a plane boundary, or whose window would not fit, reads global
// memory as before.
constexpr int kChunk = kThreads;

__shared__ __align__(8) unsigned long long s_mbar[2];
__shared__ int s_sdelta[kMaxStencil];   // window offset of each stencil table entry
__shared__ int s_sd_lo[9], s_sd_hi[9];  // smallest and largest window offset of each dof type
__shared__ unsigned s_tma_uses[2];      // copies issued into each buffer (mbarrier phases)

struct ChunkWin {
  int ok;            // the window is staged (else the chunk reads global memory)
  int ncopy;
  int parity;        // mbarrier phase parity of this use of the buffer
  int p_lo;
  long long g0;
  long long src[5];  // first element of each copy (multiple of 4)
  int cnt[5];        // elements of each copy (multiple of 4)
  int dst[5];        // first element of each copy in the buffer (multiple of 4)
};
__shared__ ChunkWin s_cw[2];

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// global -> shared bulk copy (addresses 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Window of the chunk of rows [ra, rb) (see above).  ok = 0 when it cannot be staged.
__device__ __noinline__ ChunkWin chunk_window(const SolveArgs& a, int ra, int rb) {
  ChunkWin w{};
  w.ok = 0;
  const int lat = a.lat;
  if (a.plane == 0) {
    const int ys = max(0, ra / lat - 2), ye = min(lat, (rb - 1) / lat + 3);
    const long long as = ((long long)ys * lat) & ~3LL;
    long long ae = ((long long)ye * lat + 3) & ~3LL;
    if (ae > a.n_pad) ae = a.n_pad;
    if (ae - as > a.tma_cap || ae <= as) return w;
    w.ncopy = 1;
    w.src[0] = as;
    w.cnt[0] = (int)(ae - as);
    w.dst[0] = 0;
    w.g0 = as;
    w.p_lo = 0;
    w.ok = 1;
    return w;
  }
  const int plane = a.plane;
  const int c = ra / plane;
  if ((rb - 1) / plane != c) return w;
  const int ys = max(0, (ra - c * plane) / lat - 2), ye = min(lat, (rb - 1 - c * plane) / lat + 3);
  const int plo = max(0, c - 2), phi = min(lat - 1, c + 2);
  const long long g0 = ((long long)plo * plane + (long long)ys * lat) & ~3LL;
  int prev_end = 0;
  for (int p = plo; p <= phi; ++p) {
    const long long as = ((long long)p * plane + (long long)ys * lat) & ~3LL;
    long long ae = ((long long)p * plane + (long long)ye * lat + 3) & ~3LL;
    if (ae > a.n_pad) ae = a.n_pad;
    const long long d = as - g0 - (long long)(p - plo) * (plane - a.tma_S);
    if (d < prev_end || (d & 3) || ae <= as || d + (ae - as) > a.tma_cap) return w;
    const int k = p - plo;
    w.src[k] = as;
    w.cnt[k] = (int)(ae - as);
    w.dst[k] = (int)d;
    prev_end = (int)(d + (ae - as));
  }
  w.ncopy = phi - plo + 1;
  w.g0 = g0;
  w.p_lo = plo;
  w.ok = 1;
  return w;
}

// Thread 0: plans chunk ck of [R0, R1) into buffer b and issues its copies.
__device__ __noinline__ void issue_chunk(const SolveArgs& a, const float* x, float* buf, int b, int ck, int R0,
                                         int R1) {
  const int ra = R0 + ck * kChunk, rb = min(R1, ra + kChunk);
  ChunkWin w = chunk_window(a, ra, rb);
  if (w.ok) {
    unsigned bytes = 0;
    bool aligned = true;
    for (int k = 0; k < w.ncopy; ++k) {
      bytes += (unsigned)w.cnt[k] * 4u;
      aligned = aligned && ((((unsigned long long)(x + w.src[k])) & 15ull) == 0) &&
                ((smem_u32(buf + w.dst[k]) & 15u) == 0) && ((w.cnt[k] & 3) == 0);
    }
    if (!aligned) w.ok = 0;
    if (w.ok) {
      w.parity = (int)(s_tma_uses[b] & 1u);
      s_tma_uses[b] += 1;
      mbar_expect_tx(&s_mbar[b], bytes);
      for (int k = 0; k < w.ncopy; ++k) bulk_g2s(buf + w.dst[k], x + w.src[k], (unsigned)w.cnt[k] * 4u, &s_mbar[b]);
    }
  }
  s_cw[b] = w;
}

// Bounded wait for buffer b's copies (phase parity).  false: gave up (timeout bit set).
__device__ bool wait_chunk(Grid& g, int b, int parity) {
  unsigned spins = 0;
  unsigned long long t0 = 0;
  while (!mbar_try_wait(&s_mbar[b], (unsigned)parity)) {
    if ((++spins & 255u) == 0u) {
      const unsigned long long t = global_ns();
      if (t0 == 0) {
        t0 = t;
      } else if (t - t0 > g.limit_ns) {
        atomicOr(g.err, kErrTimeout);
        return false;
      }
    }
  }
  return true;
}

// One row of the chunked SpMV: interior rows from the staged window (or global memory),
// the others from their assembled SELL row.
template <class TM>
__device__ __forceinline__ float chunk_row(const Grid& g, const SolveArgs& a, int op, const TM* __restrict__ vals,
                                           const float* x, const ChunkWin& w, const float* buf, int row) {
  const unsigned info = row_info(g, a, row);
  float acc = 0.f;
  if (info & 8u) {
    const int t = info & 7u;
    const int k0 = s_st_start[t], k1 = k0 + s_st_cnt[t];
    const StEntry<float>* tab = reinterpret_cast<const StEntry<float>*>(s_st_raw) + op * kMaxStencil;
    int widx = (int)(row - w.g0);
    if (a.plane) widx -= (row / a.plane - w.p_lo) * (a.plane - a.tma_S);
    // the window holds every interior row's reach by construction; a row whose reach
    // would leave it reads global memory instead
    if (w.ok && widx + s_sd_lo[t] >= 0 && widx + s_sd_hi[t] < a.tma_cap) {
#pragma unroll 4
      for (int k = k0; k < k1; ++k) acc = fma(tab[k].w, buf[widx + s_sdelta[k]], acc);
    } else {
#pragma unroll 4
      for (int k = k0; k < k1; ++k) {
        const StEntry<float> e = tab[k];
        acc = fma(e.w, x[row + e.off], acc);
      }
    }
  } else {
    const int sl = row >> 5;
    acc = sell_row_wide_impl<float>(make_int2(__ldg(a.slice_ptr + sl), __ldg(a.slice_ptr + sl + 1)), a.cols, vals, x,
                                    row & 31);
  }
  return acc;
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
  __device__ explicit Ctx(const SolveArgs& args) : a(args) {}
  __device__ __forceinline__ const TM* iM() const { return (const TM*)a.iM; }
  __device__ __forceinline__ const TM* iK() const { return (const TM*)a.iK; }
  __device__ __forceinline__ const TM* iMdK() const { return (const TM*)a.iMdK; }
  __device__ __forceinline__ const TM* iMsK() const { return (const TM*)a.iMsK; }
  __device__ __forceinline__ const TV* dM() const { return (const TV*)a.dM; }
  __device__ __forceinline__ const TV* dMdK() const { return (const TV*)a.dMdK; }
  __device__ __forceinline__ const TV* dMsK() const { return (const TV*)a.dMsK; }
  // inner vectors: PCG work vectors 0..8 (textbook form uses r, p, q), step outputs 9..13
  __device__ __forceinline__ TV* vec(int k) const { return (TV*)a.ivec + (size_t)k * a.n_pad; }
};

enum : int { kVr = 0, kVp = 1, kVq = 2, kVu = 3, kVw = 4, kVm0 = 5, kVm1 = 6, kVz = 7, kVs = 8,
             kVy0 = 9, kVy1 = 10, kVwv = 11, kVx1 = 12, kVx2 = 13, kVt = 14, kVsd = 15 };

// Right-hand side of an inner solve, per owned row:
//   rhs(row) = alpha vin[row] + beta (mat x vx)[row]   (either term may be absent)
// where vx was completed before the call (a SpMV over other blocks' rows).
template <class TM, class TV>
struct RhsSpec {
  const double* vin;
  double alpha;
  const TM* mat;
  int op;
  const TV* vx;
  double beta;
  __device__ __forceinline__ double operator()(const Grid& g, const SolveArgs& a, int s, int lane, int row) const {
    using Acc = typename AccOf<TV>::type;
    double v = vin ? alpha * vin[row] : 0.0;
    if (mat) v += beta * (double)inner_row<Acc>(g, a, op, mat, vx, s, lane);
    return v;
  }
};

// Textbook Jacobi-PCG for A x = rhs, x0 = 0, stop at ||r||_2 <= rtol ||rhs||_2.
// The right-hand side is evaluated once per owned row in the first phase.
template <class TM, class TV>
__device__ __noinline__ bool pcg_standard(Grid& g, const SolveArgs& a, const TM* AV, int op, const TV* DI, TV* x,
                                          RhsSpec<TM, TV> rhs, double rtol, int maxit, InnerCount& cnt, int& its) {
  Ctx<TM, TV> c(a);
  using Acc = typename Ctx<TM, TV>::Acc;
  TV* r = c.vec(kVr);
  TV* p = c.vec(kVp);
  TV* q = c.vec(kVq);
  const int lane = threadIdx.x & 31;
  // per-thread partial sums stay in the inner type (fp64 throughput is scarce on GB300);
  // the warp, block and grid sums are float64
  Acc pb = Acc(0), pz = Acc(0);
  FOR_MY_GROUPS(g, s0, nsl) {
#pragma unroll
    for (int uu = 0; uu < kGroup; ++uu) {
      if (uu < nsl) {
        const int s = s0 + uu, row = s * 32 + lane;
        const TV rv = (TV)rhs(g, a, s, lane, row);
        const TV zz = (TV)((Acc)DI[row] * (Acc)rv);
        x[row] = TV(0);
        r[row] = rv;
        p[row] = zz;
        pb = fma((Acc)rv, (Acc)rv, pb);
        pz = fma((Acc)rv, (Acc)zz, pz);
      }
    }
  }
  Sum4<Acc> red;
  if (!grid_sum<Acc, 2>(g, pb, pz, Acc(0), red, kPhInit)) return false;
  its = 0;
  cnt.calls += 1;
  const double bb = red.x;
  Acc rz = (Acc)red.y;
  if (!isfinite(bb)) {
    flag(g, kErrNonfinite);
    return false;
  }
  if (bb == 0.0) return true;
  const Acc thr = (Acc)(rtol * rtol * bb);
  for (int it = 1; it <= maxit; ++it) {
    Acc ppq = Acc(0);
    if (g.staged) stage_window(g, p);
    FOR_MY_GROUPS(g, s0, nsl) {
      Acc qa[kGroup];
      inner_rows<Acc>(g, a, op, AV, p, s0, nsl, lane, qa, g.staged);
#pragma unroll
      for (int uu = 0; uu < kGroup; ++uu) {
        if (uu < nsl) {
          const int row = (s0 + uu) * 32 + lane;
          const Acc pr = (Acc)p[row];
          const TV qv = (TV)qa[uu];
          q[row] = qv;
          ppq = fma(pr, (Acc)qv, ppq);
        }
      }
    }
    if (!grid_sum<Acc, 1>(g, ppq, Acc(0), Acc(0), red, kPhSpmv)) return false;
    const Acc pq = (Acc)red.x;
    if (!isfinite(pq)) {
      flag(g, kErrNonfinite);
      return false;
    }
    if (!(pq > Acc(0))) {
      flag(g, kErrBreakdown);
      its = it;
      cnt.its += it;
      return true;
    }
    const Acc alpha = rz / pq;
    Acc prr = Acc(0), prz = Acc(0);
    FOR_MY_GROUPS(g, s0, nsl) {
      TV xv[kGroup], pv[kGroup], qv[kGroup], rv[kGroup], dv[kGroup];
#pragma unroll
      for (int uu = 0; uu < kGroup; ++uu) {
        if (uu < nsl) {
          const int row = (s0 + uu) * 32 + lane;
          xv[uu] = x[row];
          pv[uu] = p[row];
          qv[uu] = q[row];
          rv[uu] = r[row];
          dv[uu] = DI[row];
        }
      }
#pragma unroll
      for (int uu = 0; uu < kGroup; ++uu) {
        if (uu < nsl) {
          const int row = (s0 + uu) * 32 + lane;
          const Acc xn = (Acc)xv[uu] + alpha * (Acc)pv[uu];
          const Acc rn = (Acc)rv[uu] - alpha * (Acc)qv[uu];
          x[row] = (TV)xn;
          r[row] = (TV)rn;
          const Acc zz = (Acc)dv[uu] * rn;
          prr = fma(rn, rn, prr);
          prz = fma(rn, zz, prz);
        }
      }
    }
    if (!grid_sum<Acc, 2>(g, prr, prz, Acc(0), red, kPhVec)) return false;
    its = it;
    if (!isfinite(red.x)) {
      flag(g, kErrNonfinite);
      return false;
    }
    if (red.x <= thr) {
      cnt.its += it;
      return true;
    }
    const Acc rz_new = (Acc)red.y;
    const Acc beta = rz_new / rz;
    rz = rz_new;
    FOR_MY_GROUPS(g, s0, nsl) {
      TV dv[kGroup], rv[kGroup], pv[kGroup];
#pragma unroll
      for (int uu = 0; uu < kGroup; ++uu) {
        if (uu < nsl) {
          const int row = (s0 + uu) * 32 + lane;
          dv[uu] = DI[row];
          rv[uu] = r[row];
          pv[uu] = p[row];
        }
      }
#pragma unroll
      for (int uu = 0; uu < kGroup; ++uu) {
        if (uu < nsl) {
          const int row = (s0 + uu) * 32 + lane;
          p[row] = (TV)((Acc)dv[uu] * (Acc)rv[uu] + beta * (Acc)pv[uu]);
        }
      }
    }
    if (!grid_sync(g, kPhVec)) return false;
  }
  cnt.its += maxit;
  cnt.capped += 1;
  return true;
}

// Step (3) of P(S_D) (Section 4.1): Jacobi-PCG on
//     S_D = M - 2 delta K + delta K M_D^{-1} K,   M_D = diag(M),
// applied without forming K M_D^{-1} K: t = K p and s = M_D^{-1} t on the owned
// rows, a barrier (s is read on halo rows), then q = M p - 2 delta t + delta K s.
// DI is the Jacobi inverse of diag(S_D).  Runs exactly maxit iterations (Table 2:
// a fixed count) unless the residual vanishes or p.S_D p <= 0, which stops it.
template <class TM, class TV>
__device__ __noinline__ bool pcg_sd(Grid& g, const SolveArgs& a, const TV* DI, TV* x, RhsSpec<TM, TV> rhs, int maxit,
                                    InnerCount& cnt, int& its) {
  Ctx<TM, TV> c(a);
  using Acc = typename Ctx<TM, TV>::Acc;
  TV* r = c.vec(kVr);
  TV* p = c.vec(kVp);
  TV* q = c.vec(kVq);
  TV* t = c.vec(kVt);
  TV* sv = c.vec(kVsd);
  const TV* dm = c.dM();
  const Acc delta = (Acc)(1.0 / a.inv_delta);
  const int lane = threadIdx.x & 31;
  Acc pb = Acc(0), pz = Acc(0);
  FOR_MY_GROUPS(g, s0, nsl) {
#pragma unroll
    for (int uu = 0; uu < kGroup; ++uu) {
      if (uu < nsl) {
        const int s = s0 + uu, row = s * 32 + lane;
        const TV rv = (TV)rhs(g, a, s, lane, row);
        const TV zz = (TV)((Acc)DI[row] * (Acc)rv);
        x[row] = TV(0);
        r[row] = rv;
        p[row] = zz;
        pb = fma((Acc)rv, (Acc)rv, pb);
        pz = fma((Acc)rv, (Acc)zz, pz);
      }
    }
  }
  Sum4<Acc> red;
  if (!grid_sum<Acc, 2>(g, pb, pz, Acc(0), red, kPhInit)) return false;
  its = 0;
  cnt.calls += 1;
  const double bb = red.x;
  Acc rz = (Acc)red.y;
  if (!isfinite(bb)) {
    flag(g, kErrNonfinite);
    return false;
  }
  if (bb == 0.0) return true;
  for (int it = 1; it <= maxit; ++it) {
    // t = K p, s = M_D^{-1} t
    FOR_MY_GROUPS(g, s0, nsl) {
      Acc ka[kGroup];
      inner_rows<Acc>(g, a, kOpK, c.iK(), p, s0, nsl, lane, ka);
#pragma unroll
      for (int uu = 0; uu < kGroup; ++uu) {
        if (uu < nsl) {
          const int row = (s0 + uu) * 32 + lane;
          t[row] = (TV)ka[uu];
          sv[row] = (TV)((Acc)dm[row] * ka[uu]);
        }
      }
    }
    if (!grid_sync(g, kPhSpmv)) return false;
    // q = M p - 2 delta t + delta K s
    Acc ppq = Acc(0);
    FOR_MY_GROUPS(g, s0, nsl) {
      Acc ma[kGroup], ks[kGroup];
      inner_rows<Acc>(g, a, kOpM, c.iM(), p, s0, nsl, lane, ma);
      inner_rows<Acc>(g, a, kOpK, c.iK(), sv, s0, nsl, lane, ks);
#pragma unroll
      for (int uu = 0; uu < kGroup; ++uu) {
        if (uu < nsl) {
          const int row = (s0 + uu) * 32 + lane;
          const Acc qv = ma[uu] - Acc(2) * delta * (Acc)t[row] + delta * ks[uu];
          q[row] = (TV)qv;
          ppq = fma((Acc)p[row], qv, ppq);
        }
      }
    }
    if (!grid_sum<Acc, 1>(g, ppq, Acc(0), Acc(0), red, kPhSpmv)) return false;
    const Acc pq = (Acc)red.x;
    if (!isfinite(pq)) {
      flag(g, kErrNonfinite);
      return false;
    }
    if (!(pq > Acc(0))) {
      its = it - 1;
      cnt.its += it - 1;
      return true;
    }
    const Acc alpha = rz / pq;
    Acc prr = Acc(0), prz = Acc(0);
    FOR_MY_GROUPS(g, s0, nsl) {
#pragma unroll
      for (int uu = 0; uu < kGroup; ++uu) {
        if (uu < nsl) {
          const int row = (s0 + uu) * 32 + lane;
          const Acc xn = (Acc)x[row] + alpha * (Acc)p[row];
          const Acc rn = (Acc)r[row] - alpha * (Acc)q[row];
          x[row] = (TV)xn;
          r[row] = (TV)rn;
          const Acc zz = (Acc)DI[row] * rn;
          prr = fma(rn, rn, prr);
          prz = fma(rn, zz, prz);
        }
      }
    }
    if (!grid_sum<Acc, 2>(g, prr, prz, Acc(0), red, kPhVec)) return false;
    its = it;
    if (!isfinite(red.x)) {
      flag(g, kErrNonfinite);
      return false;
    }
    if (red.x == Acc(0)) {
      cnt.its += it;
      return true;
    }
    const Acc rz_new = (Acc)red.y;
    const Acc beta = rz_new / rz;
    rz = rz_new;
    FOR_MY_GROUPS(g, s0, nsl) {
#pragma unroll
      for (int uu = 0; uu < kGroup; ++uu) {
        if (uu < nsl) {
          const int row = (s0 + uu) * 32 + lane;
          p[row] = (TV)((Acc)DI[row] * (Acc)r[row] + beta * (Acc)p[row]);
        }
      }
    }
    if (!grid_sync(g, kPhVec)) return false;
  }
  cnt.its += maxit;
  return true;
}

// Pipelined Jacobi-PCG (Ghysels-Vanroose): the same iterates as pcg_standard in
// exact arithmetic.  Per iteration one pass computes n = A m, the recurrences
//   z = n + b z, q = m + b q, s = w + b s, p = u + b p,
//   x += a p, r -= a s, u -= a q, w -= a z, m' = D w
// and the partial sums of (r, u), (w, u), (r, r); one barrier follows.
template <class TM, class TV>
__device__ __noinline__ bool pcg_pipelined(Grid& g, const SolveArgs& a, const TM* AV, int op, const TV* DI, TV* x,
                                           RhsSpec<TM, TV> rhs, double rtol, int maxit, InnerCount& cnt, int& its) {
  Ctx<TM, TV> c(a);
  using Acc = typename Ctx<TM, TV>::Acc;
  TV* r = c.vec(kVr);
  TV* u = c.vec(kVu);
  TV* w = c.vec(kVw);
  TV* zv = c.vec(kVz);
  TV* qv = c.vec(kVq);
  TV* sv = c.vec(kVs);
  TV* pv = c.vec(kVp);
  TV* mcur = c.vec(kVm0);
  TV* mnext = c.vec(kVm1);
  const int lane = threadIdx.x & 31;
  // r = b, u = D r, x = 0; recurrences start at zero.  Per-thread partial sums
  // stay in the inner type; the warp, block and grid sums are float64.
  Acc pb = Acc(0);
  FOR_MY_GROUPS(g, s0, nsl) {
#pragma unroll
    for (int uu = 0; uu < kGroup; ++uu) {
      if (uu < nsl) {
        const int s = s0 + uu, row = s * 32 + lane;
        const TV rv = (TV)rhs(g, a, s, lane, row);
        x[row] = TV(0);
        r[row] = rv;
        u[row] = (TV)((Acc)DI[row] * (Acc)rv);
        zv[row] = TV(0);
        qv[row] = TV(0);
        sv[row] = TV(0);
        pv[row] = TV(0);
        pb = fma((Acc)rv, (Acc)rv, pb);
      }
    }
  }
  Sum4<Acc> red;
  if (!grid_sum<Acc, 1>(g, pb, Acc(0), Acc(0), red, kPhInit)) return false;
  its = 0;
  cnt.calls += 1;
  const double bb = red.x;
  if (!isfinite(bb)) {
    flag(g, kErrNonfinite);
    return false;
  }
  if (bb == 0.0) return true;
  const double thr = rtol * rtol * bb;
  // w = A u, m = D w, partial (r, u), (w, u)
  Acc pg = Acc(0), pd = Acc(0);
  if (g.staged) stage_window(g, u);
  FOR_MY_GROUPS(g, s0, nsl) {
    Acc wa[kGroup];
    inner_rows<Acc>(g, a, op, AV, u, s0, nsl, lane, wa, g.staged);
#pragma unroll
    for (int uu = 0; uu < kGroup; ++uu) {
      if (uu < nsl) {
        const int row = (s0 + uu) * 32 + lane;
        const TV uvv = u[row];
        const Acc rr0 = (Acc)r[row], dd0 = (Acc)DI[row];
        const TV wvv = (TV)wa[uu];
        w[row] = wvv;
        mcur[row] = (TV)(dd0 * (Acc)wvv);
        pg = fma(rr0, (Acc)uvv, pg);
        pd = fma((Acc)wvv, (Acc)uvv, pd);
      }
    }
  }
  if (!grid_sum<Acc, 2>(g, pg, pd, Acc(0), red, kPhSpmv)) return false;
  double gamma = red.x, delta = red.y, gamma_old = 1.0, alpha_old = 1.0;
  for (int it = 0; it < maxit; ++it) {
    if (!isfinite(gamma) || !isfinite(delta)) {
      flag(g, kErrNonfinite);
      return false;
    }
    double beta, alpha;
    if (it == 0) {
      beta = 0.0;
      alpha = gamma / delta;
    } else {
      beta = gamma / gamma_old;
      alpha = gamma / (delta - beta * gamma / alpha_old);
    }
    if (!(delta > 0.0) || !isfinite(alpha)) {
      flag(g, kErrBreakdown);
      its = it;
      cnt.its += it;
      return true;
    }
    const Acc al = (Acc)alpha, be = (Acc)beta;
    Acc prg = Acc(0), pwd = Acc(0), prr = Acc(0);
    if (g.staged) stage_window(g, mcur);
    FOR_MY_GROUPS(g, s0, nsl) {
      Acc nav[kGroup];
      inner_rows<Acc>(g, a, op, AV, mcur, s0, nsl, lane, nav, g.staged);
#pragma unroll
      for (int uu = 0; uu < kGroup; ++uu) {
      if (uu >= nsl) break;
      const int row = (s0 + uu) * 32 + lane;
      const Acc mv = (Acc)mcur[row], zo = (Acc)zv[row], qo = (Acc)qv[row], so = (Acc)sv[row];
      const Acc po = (Acc)pv[row], xo = (Acc)x[row], ro = (Acc)r[row], uo = (Acc)u[row], wo = (Acc)w[row];
      const Acc dd = (Acc)DI[row];
      const Acc na = nav[uu];
      const Acc z1 = na + be * zo;
      const Acc q1 = mv + be * qo;
      const Acc s1 = wo + be * so;
      const Acc p1 = uo + be * po;
      const Acc x1 = xo + al * p1;
      const Acc r1 = ro - al * s1;
      const Acc u1 = uo - al * q1;
      const Acc w1 = wo - al * z1;
      zv[row] = (TV)z1;
      qv[row] = (TV)q1;
      sv[row] = (TV)s1;
      pv[row] = (TV)p1;
      x[row] = (TV)x1;
      r[row] = (TV)r1;
      u[row] = (TV)u1;
      w[row] = (TV)w1;
      mnext[row] = (TV)(dd * w1);
      prg = fma(r1, u1, prg);
      pwd = fma(w1, u1, pwd);
      prr = fma(r1, r1, prr);
      }
    }
    if (!grid_sum<Acc>(g, prg, pwd, prr, red, kPhSpmv)) return false;
    its = it + 1;
    if (!isfinite(red.z)) {
      flag(g, kErrNonfinite);
      return false;
    }
    if (red.z <= thr) {
      cnt.its += its;
      return true;
    }
    gamma_old = gamma;
    alpha_old = alpha;
    gamma = red.x;
    delta = red.y;
    TV* t = mcur;
    mcur = mnext;
    mnext = t;
  }
  cnt.its += maxit;
  cnt.capped += 1;
  return true;
}

// w = A u with the partial sums (r, u) and (w, u), over this block's rows in chunks of
// kChunk rows whose source windows are bulk-copied into shared memory (see
// chunk_window).  All threads of the block call it; false if a wait gave up.
template <class TM>
__device__ __forceinline__ bool spmv_chunks_cg(Grid& g, const SolveArgs& a, int op, const TM* AV, const float* u,
                                               const float* r, float* w, float& pg, float& pd) {
  const int R0 = g.b_lo * 32, R1 = g.b_hi * 32;
  const int nch = (R1 - R0 + kChunk - 1) / kChunk;
  if (threadIdx.x == 0) {
    // u was written through the generic proxy by every block before the last grid
    // barrier; order those writes before this thread's bulk (async-proxy) reads
    asm volatile("fence.proxy.async.global;" ::: "memory");
    for (int ck = 0; ck < 2 && ck < nch; ++ck) issue_chunk(a, u, s_win + ck * a.tma_cap, ck, ck, R0, R1);
  }
  __syncthreads();
  bool ok = true;
  for (int ck = 0; ck < nch; ++ck) {
    const int b = ck & 1;
    const ChunkWin& cw = s_cw[b];
    if (cw.ok && ok) ok = wait_chunk(g, b, cw.parity);
    const int row = R0 + ck * kChunk + (int)threadIdx.x;
    if (ok && row < R1) {
      const float acc = chunk_row<TM>(g, a, op, AV, u, cw, s_win + b * a.tma_cap, row);
      w[row] = acc;
      const float uo = u[row], ro = r[row];
      pg = fma(ro, uo, pg);
      pd = fma(acc, uo, pd);
    }
    // every thread is done with buffer b (and with s_cw[b]); a wait that gave up stops
    // the whole block, which issues no further copies
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
    if (threadIdx.x == 0 && ok && ck + 2 < nch) issue_chunk(a, u, s_win + b * a.tma_cap, b, ck + 2, R0, R1);
  }
  return ok;
}

// w = A u and the partial sums (r, u), (w, u) of one Chronopoulos-Gear phase: the
// chunked path with staged windows (kChunked, float vectors), else each warp over its
// own slices.
template <class TM, class TV, bool kChunked>
__device__ __forceinline__ bool spmv_cg(Grid& g, const SolveArgs& a, int op, const TM* AV, const TV* u, const TV* r,
                                        TV* w, typename AccOf<TV>::type& pg, typename AccOf<TV>::type& pd) {
  using Acc = typename AccOf<TV>::type;
  if constexpr (kChunked && sizeof(TV) == 4) {
    return spmv_chunks_cg<TM>(g, a, op, AV, u, r, w, pg, pd);
  }
  const int lane = threadIdx.x & 31;
  if (g.staged) stage_window(g, u);
  FOR_MY_GROUPS(g, s0, nsl) {
    Acc wa[kGroup];
    inner_rows<Acc>(g, a, op, AV, u, s0, nsl, lane, wa, g.staged);
#pragma unroll
    for (int uu = 0; uu < kGroup; ++uu) {
      if (uu < nsl) {
        const int row = (s0 + uu) * 32 + lane;
        const Acc uo = (Acc)u[row], ro = (Acc)r[row];
        w[row] = (TV)wa[uu];
        pg = fma(ro, uo, pg);
        pd = fma(wa[uu], uo, pd);
      }
    }
  }
  return true;
}

// Chronopoulos-Gear Jacobi-PCG (Chronopoulos & Gear, J. Comput. Appl. Math. 25,
// 1989): the same iterates as pcg_standard in exact arithmetic with two phases
// per iteration.  It carries w = A u (u = D r) and s = A p as recurrences:
//   phase 1: p = u + b p, s = w + b s, x += a p, r -= a s, u = D r, partial (r, r)
//   phase 2: w = A u, partials (r, u), (w, u);  b = g'/g, a = g' / (d - b g'/a)
template <class TM, class TV, bool kChunked>
__device__ __noinline__ bool pcg_cg(Grid& g, const SolveArgs& a, const TM* AV, int op, const TV* DI, TV* x,
                                    RhsSpec<TM, TV> rhs, double rtol, int maxit, InnerCount& cnt, int& its) {
  Ctx<TM, TV> c(a);
  using Acc = typename Ctx<TM, TV>::Acc;
  TV* r = c.vec(kVr);
  TV* u = c.vec(kVu);
  TV* w = c.vec(kVw);
  TV* sv = c.vec(kVs);
  TV* pv = c.vec(kVp);
  const int lane = threadIdx.x & 31;
  // r = b, u = D r, x = p = s = 0
  Acc pb = Acc(0);
  FOR_MY_GROUPS(g, s0, nsl) {
#pragma unroll
    for (int uu = 0; uu < kGroup; ++uu) {
      if (uu < nsl) {
        const int s = s0 + uu, row = s * 32 + lane;
        const TV rv = (TV)rhs(g, a, s, lane, row);
        x[row] = TV(0);
        r[row] = rv;
        u[row] = (TV)((Acc)DI[row] * (Acc)rv);
        sv[row] = TV(0);
        pv[row] = TV(0);
        pb = fma((Acc)rv, (Acc)rv, pb);
      }
    }
  }
  Sum4<Acc> red;
  if (!grid_sum<Acc, 1>(g, pb, Acc(0), Acc(0), red, kPhInit)) return false;
  its = 0;
  cnt.calls += 1;
  const double bb = red.x;
  if (!isfinite(bb)) {
    flag(g, kErrNonfinite);
    return false;
  }
  if (bb == 0.0) return true;
  const Acc thr = (Acc)(rtol * rtol * bb);
  // w = A u, partials (r, u), (w, u)
  Acc pg = Acc(0), pd = Acc(0);
  if (!spmv_cg<TM, TV, kChunked>(g, a, op, AV, u, r, w, pg, pd)) return false;
  if (!grid_sum<Acc, 2>(g, pg, pd, Acc(0), red, kPhSpmv)) return false;
  Acc gam = (Acc)red.x, del = (Acc)red.y;
  if (!(del > Acc(0))) {
    flag(g, kErrBreakdown);
    return true;
  }
  Acc alpha = gam / del, beta = Acc(0);
  for (int it = 1; it <= maxit; ++it) {
    // phase 1: recurrences and the new residual
    Acc prr = Acc(0);
    FOR_MY_GROUPS(g, s0, nsl) {
      TV uv[kGroup], pvv[kGroup], wv[kGroup], svv[kGroup], xv[kGroup], rv[kGroup], dv[kGroup];
#pragma unroll
      for (int uu = 0; uu < kGroup; ++uu) {
        if (uu < nsl) {
          const int row = (s0 + uu) * 32 + lane;
          uv[uu] = u[row];
          pvv[uu] = pv[row];
          wv[uu] = w[row];
          svv[uu] = sv[row];
          xv[uu] = x[row];
          rv[uu] = r[row];
          dv[uu] = DI[row];
        }
      }
#pragma unroll
      for (int uu = 0; uu < kGroup; ++uu) {
        if (uu < nsl) {
          const int row = (s0 + uu) * 32 + lane;
          const Acc p1 = (Acc)uv[uu] + beta * (Acc)pvv[uu];
          const Acc s1 = (Acc)wv[uu] + beta * (Acc)svv[uu];
          const Acc x1 = (Acc)xv[uu] + alpha * p1;
          const Acc r1 = (Acc)rv[uu] - alpha * s1;
          pv[row] = (TV)p1;
          sv[row] = (TV)s1;
          x[row] = (TV)x1;
          r[row] = (TV)r1;
          u[row] = (TV)((Acc)dv[uu] * r1);
          prr = fma(r1, r1, prr);
        }
      }
    }
    if (g.nbsync) {
      // the next phase needs only the halo of u: wait for the neighbours, and
      // reduce (r, r) together with the phase-2 products (the test follows them)
      if (!neighbor_sync(g, kPhVec)) return false;
    } else {
      if (!grid_sum<Acc, 1>(g, prr, Acc(0), Acc(0), red, kPhVec)) return false;
      its = it;
      if (!isfinite(red.x)) {
        flag(g, kErrNonfinite);
        return false;
      }
      if ((Acc)red.x <= thr) {
        cnt.its += it;
        return true;
      }
    }
    // phase 2: w = A u and the two inner products
    pg = Acc(0);
    pd = Acc(0);
    if (!spmv_cg<TM, TV, kChunked>(g, a, op, AV, u, r, w, pg, pd)) return false;
    if (!grid_sum<Acc>(g, pg, pd, g.nbsync ? prr : Acc(0), red, kPhSpmv)) return false;
    if (g.nbsync) {
      its = it;
      if (!isfinite(red.z)) {
        flag(g, kErrNonfinite);
        return false;
      }
      if ((Acc)red.z <= thr) {
        cnt.its += it;
        return true;
      }
    }
    const Acc gnew = (Acc)red.x, dnew = (Acc)red.y;
    beta = gnew / gam;
    const Acc den = dnew - beta * gnew / alpha;
    if (!(den > Acc(0)) || !isfinite(den)) {
      flag(g, kErrBreakdown);
      cnt.its += it;
      return true;
    }
    alpha = gnew / den;
    gam = gnew;
  }
  cnt.its += maxit;
  cnt.capped += 1;
  return true;
}

// ---------------------------------------------------------------------------
// Cell kernels: Chronopoulos-Gear Jacobi-PCG with one grid barrier per iteration
// (P2 rows in cell-major order, float inner vectors; cell2d.h, cell3d.h).
//
// A cell is 2 x 2 (2D) or 2 x 2 x 2 (3D) lattice points, its rows consecutive, so a
// vector is read and written one float4 "unit" (four rows) at a time: U = 1 unit per
// cell in 2D, 2 in 3D.  For these phases the cell grid (cell_S cells per axis) is cut
// into cell_gx x cell_gy (x cell_gz) boxes, tile (b % gx, (b / gx) % gy, b / (gx gy))
// owned by block b (blocks past gx gy gz own none).  A block keeps the preconditioned
// residual u of its tile and of the ring of cells around it (every cell its rows'
// stencils reach) in a shared-memory window, so the product w = A u reads no global
// memory.  Instead of a grid barrier that would publish u before the product, the
// block recomputes u on the ring itself from the owners' r, s and w of the previous
// iteration with the same arithmetic the owners use (so the values agree bit for
// bit); r, s and w alternate between two buffers, so that an owner writing iteration
// k + 1 never overwrites what a neighbour still reads for iteration k.  One iteration:
//   phase A, tile: p = u + b p, s' = w + b s, x += a p, r' = r - a s', u' = D r'
//           (partials (r', r'), (r', u')); ring: s', r', u' as above, u' only kept
//   phase B, tile: w' = A u' from the window (partial (w', u'))
//   one grid sum of the three partials: stop test on (r', r'), then
//   b = g' / g, a = g' / (d' - b g' / a)
// The iterates are those of pcg_cg; its separate (r, r) barrier is gone (the test
// comes one product later, after the same iterate x).  Every cell runs the couplings
// of cell2d.h / cell3d.h with the weights of its cell class (interior cells: class 0;
// a coupling a row lacks has weight 0).  The set-up before the loop (r = b etc.) and
// the caller's use of x go by the block's slices as everywhere else; the grid barriers
// in between order the two ownerships.

template <int DIM> struct CellDim;
template <> struct CellDim<2> {
  static constexpr int U = 1, E = kCell2dEntries, stride = 48;
};
template <> struct CellDim<3> {
  static constexpr int U = 2, E = kCell3dEntries, stride = 232;
};
__host__ __device__ constexpr int cell_stride(int dim) { return dim == 2 ? 48 : 232; }

// This block's tile: cells (x0 + i, y0 + j, z0 + l), i < tw, j < th, l < td (td = 1,
// z0 = 0 in 2D).  Window coordinates (lx, ly, lz) = (i + 1, j + 1, l + wz) with wz = 1
// in 3D, 0 in 2D; window cell index lx + ly sx + lz sxy.  The walk over the tile cells
// k = threadIdx.x, + kThreads, ... steps by (dx, dy, dz) with kThreads = (dz th + dy) tw
// + dx; inv_tw, inv_th are the float reciprocals for the first quotients.
struct CellTile {
  int x0, y0, z0, tw, th, td, wz, sx, sxy, own, win, ring, dx, dy, dz;
  float inv_tw, inv_th;
};
__shared__ CellTile s_tile;   // set once per launch (cell_tables)
__shared__ int s_ring_n;
__device__ __forceinline__ const CellTile& cell_tile() { return s_tile; }

__device__ __forceinline__ CellTile cell_tile_of(const Grid& g, const SolveArgs& a) {
  CellTile t;
  const int gx = a.cell_gx, gy = a.cell_gy, gz = a.cell_dim == 3 ? a.cell_gz : 1, S = a.cell_S;
  const bool has = g.bid < gx * gy * gz;
  const int ix = has ? g.bid % gx : 0, iy = has ? (g.bid / gx) % gy : 0, iz = has ? g.bid / (gx * gy) : 0;
  t.x0 = (int)((long long)ix * S / gx);
  t.y0 = (int)((long long)iy * S / gy);
  t.z0 = a.cell_dim == 3 ? (int)((long long)iz * S / gz) : 0;
  t.tw = has ? (int)((long long)(ix + 1) * S / gx) - t.x0 : 0;
  t.th = has ? (int)((long long)(iy + 1) * S / gy) - t.y0 : 0;
  t.td = !has ? 0 : a.cell_dim == 3 ? (int)((long long)(iz + 1) * S / gz) - t.z0 : 1;
  t.wz = a.cell_dim == 3 ? 1 : 0;
  t.sx = t.tw + 2;
  t.sxy = (t.tw + 2) * (t.th + 2);
  t.own = t.tw * t.th * t.td;
  t.win = t.own > 0 ? t.sxy * (t.td + 2 * t.wz) : 0;
  t.ring = t.win - t.own;
  const int plane = t.tw * t.th;
  t.dz = plane > 0 ? kThreads / plane : 0;
  const int rem = plane > 0 ? kThreads - t.dz * plane : 0;
  t.dy = t.tw > 0 ? rem / t.tw : 0;
  t.dx = t.tw > 0 ? rem - t.dy * t.tw : 0;
  t.inv_tw = t.tw > 0 ? 1.0f / (float)t.tw : 0.f;
  t.inv_th = t.th > 0 ? 1.0f / (float)t.th : 0.f;
  return t;
}

// Walks the tile cells k = threadIdx.x, + kThreads, ... of the block's tile without a
// division per cell.  The first quotients come from float reciprocals: (k + 1/2) / n
// lies at least 1/(2n) from an integer and k < 2^10, so the rounding of one float
// product cannot cross one.  In 2D a tile cell never needs the z carry (k < tw th).
template <int DIM>
struct TileWalk {
  int lx, ly, lz;
  __device__ __forceinline__ explicit TileWalk(const CellTile& t) {
    const int k0 = threadIdx.x;
    const int q1 = __float2int_rz(((float)k0 + 0.5f) * t.inv_tw);
    lx = k0 - q1 * t.tw + 1;
    if constexpr (DIM == 3) {
      const int q2 = __float2int_rz(((float)q1 + 0.5f) * t.inv_th);
      ly = q1 - q2 * t.th + 1;
      lz = q2 + 1;
    } else {
      ly = q1 + 1;
      lz = 0;
    }
  }
  __device__ __forceinline__ void next(const CellTile& t) {
    if constexpr (DIM == 3) {
      lx += t.dx;
      if (lx > t.tw) {
        lx -= t.tw;
        ly += 1;
      }
      ly += t.dy;
      if (ly > t.th) {
        ly -= t.th;
        lz += 1;
      }
      lz += t.dz;
    } else {
      // kThreads = q tw + r with q = dz th + dy, r = dx
      lx += t.dx;
      ly += t.dz * t.th + t.dy;
      if (lx > t.tw) {
        lx -= t.tw;
        ly += 1;
      }
    }
  }
  __device__ __forceinline__ int wi(const CellTile& t) const {
    return DIM == 3 ? lx + ly * t.sx + lz * t.sxy : lx + ly * t.sx;
  }
  __device__ __forceinline__ int cell(const CellTile& t, int S) const {
    return DIM == 3 ? ((t.z0 - 1 + lz) * S + (t.y0 - 1 + ly)) * S + (t.x0 - 1 + lx) : (t.y0 - 1 + ly) * S + (t.x0 - 1 + lx);
  }
};

// Dynamic shared memory of the cell kernels (layout: cell_smem_bytes).
struct CellMem {
  float4* win;               // u: unit h of window cell j at h cell_wcap + j (planes of units,
                             //   so that lanes reading consecutive cells read consecutive float4)
  const int2* ring;          // ring cell j: {window cell, cell index or -1 outside the grid}
  float* wts;                // the current operator's coupling weights, one row per cell class
  const unsigned char* cc;   // class of each tile cell, tile order
};
__device__ __forceinline__ CellMem cell_mem(const SolveArgs& a) {
  char* base = reinterpret_cast<char*>(s_win);
  const int U = a.cell_dim == 3 ? 2 : 1;
  CellMem m;
  m.win = reinterpret_cast<float4*>(base);
  m.ring = reinterpret_cast<const int2*>(base + cell_off_ring(a.cell_wcap, U));
  m.wts = reinterpret_cast<float*>(base + cell_off_weights(a.cell_wcap, U, a.cell_rcap));
  m.cc = reinterpret_cast<const unsigned char*>(
      base + cell_off_classes(a.cell_wcap, U, a.cell_rcap, a.ccls_n, cell_stride(a.cell_dim)));
  return m;
}

// Fills the tile record, the ring list and the tile's cell classes, and zeroes the
// window cells outside the cell grid (read with weight 0 by the cells on its edges,
// never written); called by all threads at the start of a launch.
__device__ void cell_tables(const Grid& g, const SolveArgs& a) {
  char* base = reinterpret_cast<char*>(s_win);
  const int U = a.cell_dim == 3 ? 2 : 1;
  int2* ring = reinterpret_cast<int2*>(base + cell_off_ring(a.cell_wcap, U));
  unsigned char* cc = reinterpret_cast<unsigned char*>(
      base + cell_off_classes(a.cell_wcap, U, a.cell_rcap, a.ccls_n, cell_stride(a.cell_dim)));
  const CellTile t = cell_tile_of(g, a);
  if (threadIdx.x == 0) {
    s_tile = t;
    s_ring_n = 0;
  }
  __syncthreads();
  const int S = a.cell_S;
  float4* win = reinterpret_cast<float4*>(base);
  for (int k = threadIdx.x; k < t.win; k += kThreads) {
    const int lx = k % t.sx, ly = (k / t.sx) % (t.th + 2), lz = k / t.sxy;
    const int cx = t.x0 - 1 + lx, cy = t.y0 - 1 + ly, cz = t.z0 - t.wz + lz;
    const bool inside_tile = lx >= 1 && lx <= t.tw && ly >= 1 && ly <= t.th && lz >= t.wz && lz < t.wz + t.td;
    const bool in_grid = cx >= 0 && cx < S && cy >= 0 && cy < S && cz >= 0 && cz < (t.wz ? S : 1);
    if (!in_grid)
      for (int h = 0; h < U; ++h) win[h * a.cell_wcap + k] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!inside_tile) {
      // the order of the ring list does not matter: each ring cell is computed alone
      const int j = atomicAdd(&s_ring_n, 1);
      ring[j] = make_int2(k, in_grid ? (cz * S + cy) * S + cx : -1);
    }
  }
  if (a.cell_dim == 3) {
    TileWalk<3> tk(t);
    for (int k = threadIdx.x; k < t.own; k += kThreads, tk.next(t)) cc[k] = __ldg(a.cellclass + tk.cell(t, S));
  } else {
    TileWalk<2> tk(t);
    for (int k = threadIdx.x; k < t.own; k += kThreads, tk.next(t)) cc[k] = __ldg(a.cellclass + tk.cell(t, S));
  }
}

__device__ __forceinline__ float dot4(float4 a, float4 b, float acc) {
  acc = fmaf(a.x, b.x, acc);
  acc = fmaf(a.y, b.y, acc);
  acc = fmaf(a.z, b.z, acc);
  return fmaf(a.w, b.w, acc);
}
template <int K>
__device__ __forceinline__ float comp4(float4 v) {
  return K == 0 ? v.x : K == 1 ? v.y : K == 2 ? v.z : v.w;
}
template <int K>
__device__ __forceinline__ float comp8(float4 lo, float4 hi) {
  return K < 4 ? comp4<K & 3>(lo) : comp4<K & 3>(hi);
}

// s' = w + b s, r' = r - a s', u' = D r' on one unit: the one formula the owner and
// the blocks that hold the cell in their ring both evaluate.
__device__ __forceinline__ void cell_rsu(float4 w, float4 sv, float4 r, float4 d, float al, float be, float4& s1,
                                         float4& r1, float4& u1) {
  s1 = make_float4(fmaf(be, sv.x, w.x), fmaf(be, sv.y, w.y), fmaf(be, sv.z, w.z), fmaf(be, sv.w, w.w));
  r1 = make_float4(fmaf(-al, s1.x, r.x), fmaf(-al, s1.y, r.y), fmaf(-al, s1.z, r.z), fmaf(-al, s1.w, r.w));
  u1 = make_float4(d.x * r1.x, d.y * r1.y, d.z * r1.z, d.w * r1.w);
}

// Inner vector k of the cell kernels (float4 units).  r, s and w alternate between two
// buffers: iteration parity cur reads buffer cur and writes buffer !cur.
__device__ __forceinline__ float4* cvec(const SolveArgs& a, int k) {
  return reinterpret_cast<float4*>((float*)a.ivec + (size_t)k * a.n_pad);
}
__device__ __forceinline__ int cell_r(int cur) { return cur ? kVu : kVr; }
__device__ __forceinline__ int cell_s(int cur) { return cur ? kVq : kVs; }
__device__ __forceinline__ int cell_w(int cur) { return cur ? kVm0 : kVw; }

// The current operator's coupling weights for every cell class into shared memory
// (one row of cell_stride floats per class); called by all threads before the first
// product of an inner solve.
__device__ __forceinline__ void cell_weights(const SolveArgs& a, int op) {
  const CellMem m = cell_mem(a);
  const int stride = cell_stride(a.cell_dim), E = a.cell_dim == 3 ? kCell3dEntries : kCell2dEntries;
  const double cM = a.op_cM[op], cK = a.op_cK[op];
  for (int k = threadIdx.x; k < a.ccls_n * stride; k += kThreads) {
    const int cls = k / stride, e = k - cls * stride;
    float w = 0.f;
    if (e < E) w = (float)(cM * __ldg(a.ccls_wM + cls * E + e) + cK * __ldg(a.ccls_wK + cls * E + e));
    m.wts[k] = w;
  }
}

// Jacobi inverse of unit h of cell c of class cls: the interior types' values for class
// 0 (the rule owner and ring both apply; d0, d1 for units 0 and 1), else the cell's own.
__device__ __forceinline__ float4 cell_d(int cls, const float4* di, float4 d0, float4 d1, int unit, int h) {
  return cls == 0 ? (h == 0 ? d0 : d1) : di[unit];
}

// u = D r on the tile and its ring (the window); partial (r, u) on the tile.
template <int DIM>
__device__ __forceinline__ void cell_fill(const SolveArgs& a, const float4* r, const float4* di, float4 d0, float4 d1,
                                          float& pg) {
  const CellMem m = cell_mem(a);
  const CellTile& t = cell_tile();
  constexpr int U = CellDim<DIM>::U;
  const int S = a.cell_S;
  TileWalk<DIM> tk(t);
  for (int k = threadIdx.x; k < t.own + t.ring; k += kThreads, tk.next(t)) {
    int wi, c, cls;
    if (k < t.own) {
      wi = tk.wi(t);
      c = tk.cell(t, S);
      cls = m.cc[k];
    } else {
      const int2 rg = m.ring[k - t.own];
      wi = rg.x;
      c = rg.y;
      if (c < 0) continue;
      cls = __ldg(a.cellclass + c);
    }
#pragma unroll
    for (int h = 0; h < U; ++h) {
      const float4 rv = r[U * c + h], d = cell_d(cls, di, d0, d1, U * c + h, h);
      const float4 u = make_float4(d.x * rv.x, d.y * rv.y, d.z * rv.z, d.w * rv.w);
      m.win[h * a.cell_wcap + wi] = u;
      if (k < t.own) pg = dot4(rv, u, pg);
    }
  }
}

// Phase A of one iteration (see above): reads r, s, w of parity cur, writes those of
// !cur, updates p and x, keeps u' in the window.
template <int DIM>
__device__ __forceinline__ void cell_phase_a(const SolveArgs& a, float al, float be, int cur, float4* x,
                                             const float4* di, float4 d0, float4 d1, float& prr, float& pg) {
  const CellMem m = cell_mem(a);
  const CellTile& t = cell_tile();
  constexpr int U = CellDim<DIM>::U;
  const int S = a.cell_S;
  float4* const pv = cvec(a, kVp);
  const float4* const rc = cvec(a, cell_r(cur));
  const float4* const sc = cvec(a, cell_s(cur));
  const float4* const wc = cvec(a, cell_w(cur));
  float4* const rn = cvec(a, cell_r(cur ^ 1));
  float4* const sn = cvec(a, cell_s(cur ^ 1));
  TileWalk<DIM> tk(t);
  for (int k = threadIdx.x; k < t.own + t.ring; k += kThreads, tk.next(t)) {
    if (k < t.own) {
      const int c = tk.cell(t, S), wi = tk.wi(t), cls = m.cc[k];
#pragma unroll 1
      for (int h = 0; h < U; ++h) {
        const int un = U * c + h, wu = h * a.cell_wcap + wi;
        const float4 u = m.win[wu];
        const float4 p = pv[un], w = wc[un], sv = sc[un], r = rc[un], xx = x[un];
        // a cell of interior rows (class 0) has the Jacobi inverses of the interior dof types
        const float4 d = cell_d(cls, di, d0, d1, un, h);
        float4 s1, r1, u1;
        cell_rsu(w, sv, r, d, al, be, s1, r1, u1);
        const float4 p1 = make_float4(fmaf(be, p.x, u.x), fmaf(be, p.y, u.y), fmaf(be, p.z, u.z), fmaf(be, p.w, u.w));
        pv[un] = p1;
        sn[un] = s1;
        rn[un] = r1;
        x[un] = make_float4(fmaf(al, p1.x, xx.x), fmaf(al, p1.y, xx.y), fmaf(al, p1.z, xx.z), fmaf(al, p1.w, xx.w));
        m.win[wu] = u1;
        prr = dot4(r1, r1, prr);
        pg = dot4(r1, u1, pg);
      }
    } else {
      const int2 rg = m.ring[k - t.own];
      const int c = rg.y;
      if (c < 0) continue;
      const int cls = __ldg(a.cellclass + c);
#pragma unroll 1
      for (int h = 0; h < U; ++h) {
        const int un = U * c + h;
        const float4 w = wc[un], sv = sc[un], r = rc[un], d = cell_d(cls, di, d0, d1, un, h);
        float4 s1, r1, u1;
        cell_rsu(w, sv, r, d, al, be, s1, r1, u1);
        m.win[h * a.cell_wcap + rg.x] = u1;
      }
    }
  }
}

// Phase B: w = A_op u on the tile from the window; partial (w, u).  Every cell runs
// the couplings of cell2d.h / cell3d.h with the weights of its class (interior cells
// all read the class-0 row, a broadcast); the window cells outside the cell grid hold
// zeros.
template <int DIM>
__device__ __forceinline__ void cell_phase_b(const SolveArgs& a, float4* wn, float& pd) {
  const CellMem m = cell_mem(a);
  const CellTile& t = cell_tile();
  const int S = a.cell_S;
  TileWalk<DIM> tk(t);
  for (int k = threadIdx.x; k < t.own; k += kThreads, tk.next(t)) {
    const int c = tk.cell(t, S), wi = tk.wi(t);
    const float* fw = m.wts + m.cc[k] * CellDim<DIM>::stride;
    int e = 0;
    if constexpr (DIM == 2) {
      constexpr int DX[kCell2dSrc] = PFC_CELL2D_DX, DY[kCell2dSrc] = PFC_CELL2D_DY;
      const int sx = t.sx;
      float4 v[kCell2dSrc];
#pragma unroll
      for (int q = 0; q < kCell2dSrc; ++q) v[q] = m.win[wi + DY[q] * sx + DX[q]];
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#define PFC_CELL_FMA(t, q, sub)                   \
  acc[t] = fmaf(fw[e], comp4<sub>(v[q]), acc[t]); \
  ++e;
      PFC_CELL2D_ENTRIES(PFC_CELL_FMA)
#undef PFC_CELL_FMA
      const float4 w1 = make_float4(acc[0], acc[1], acc[2], acc[3]);
      wn[c] = w1;
      pd = dot4(w1, v[3], pd);
    } else {
      constexpr int DX[kCell3dSrc] = PFC_CELL3D_DX, DY[kCell3dSrc] = PFC_CELL3D_DY, DZ[kCell3dSrc] = PFC_CELL3D_DZ;
      const int sx = t.sx, sxy = t.sxy, wcap = a.cell_wcap;
      float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      float4 lo, hi;
#define PFC_CELL_LOAD(q)                                        \
  {                                                             \
    const int wq = wi + DZ[q] * sxy + DY[q] * sx + DX[q];       \
    lo = m.win[wq];                                             \
    hi = m.win[wcap + wq];                                      \
  }
#define PFC_CELL_FMA(t, q, sub)                       \
  acc[t] = fmaf(fw[e], comp8<sub>(lo, hi), acc[t]);   \
  ++e;
      PFC_CELL3D_ENTRIES(PFC_CELL_FMA, PFC_CELL_LOAD)
#undef PFC_CELL_FMA
#undef PFC_CELL_LOAD
      const float4 w0 = make_float4(acc[0], acc[1], acc[2], acc[3]), w1 = make_float4(acc[4], acc[5], acc[6], acc[7]);
      wn[2 * c] = w0;
      wn[2 * c + 1] = w1;
      pd = dot4(w0, m.win[wi], pd);
      pd = dot4(w1, m.win[wcap + wi], pd);
    }
  }
}


// Chronopoulos-Gear Jacobi-PCG on the cell kernels (see above); same contract as pcg_cg.
template <class TM, int DIM>
__device__ __noinline__ bool pcg_cell(Grid& g, const SolveArgs& a, int op, const float* DI, float* x,
                                      RhsSpec<TM, float> rhs, double rtol, int maxit, InnerCount& cnt, int& its) {
  float* const rb0 = (float*)cvec(a, kVr);
  float* const sb0 = (float*)cvec(a, kVs);
  float* const pv = (float*)cvec(a, kVp);
  const int lane = threadIdx.x & 31;
  // this operator's weights (read after the grid sum below)
  cell_weights(a, op);
  // r = b, x = p = s = 0 on the block's rows
  float pb = 0.f;
  FOR_MY_GROUPS(g, s0, nsl) {
#pragma unroll
    for (int uu = 0; uu < kGroup; ++uu) {
      if (uu < nsl) {
        const int s = s0 + uu, row = s * 32 + lane;
        const float rv = (float)rhs(g, a, s, lane, row);
        x[row] = 0.f;
        rb0[row] = rv;
        sb0[row] = 0.f;
        pv[row] = 0.f;
        pb = fmaf(rv, rv, pb);
      }
    }
  }
  Sum4<float> red;
  if (!grid_sum<float, 1>(g, pb, 0.f, 0.f, red, kPhInit)) return false;
  its = 0;
  cnt.calls += 1;
  const double bb = red.x;
  if (!isfinite(bb)) {
    flag(g, kErrNonfinite);
    return false;
  }
  if (bb == 0.0) return true;
  const float thr = (float)(rtol * rtol * bb);
  float4* const x4 = reinterpret_cast<float4*>(x);
  const float4* const d4 = reinterpret_cast<const float4*>(DI);
  // the Jacobi inverse of an interior row depends only on its dof type: read it at an
  // interior row of each type, and use it for every cell of class 0 (owner and ring)
  const float4 d0 = make_float4(DI[a.cell_rep[0]], DI[a.cell_rep[1]], DI[a.cell_rep[2]], DI[a.cell_rep[3]]);
  const float4 d1 = DIM == 3 ? make_float4(DI[a.cell_rep[4]], DI[a.cell_rep[5]], DI[a.cell_rep[6]], DI[a.cell_rep[7]])
                             : d0;
  float pg = 0.f, pd = 0.f;
  cell_fill<DIM>(a, cvec(a, kVr), d4, d0, d1, pg);
  __syncthreads();
  cell_phase_b<DIM>(a, cvec(a, cell_w(0)), pd);
  if (!grid_sum<float, 2>(g, pg, pd, 0.f, red, kPhSpmv)) return false;
  float gam = red.x, del = red.y;
  if (!(del > 0.f)) {
    flag(g, kErrBreakdown);
    return true;
  }
  float alpha = gam / del, beta = 0.f;
  int cur = 0;
  for (int it = 1; it <= maxit; ++it) {
    float prr = 0.f;
    pg = 0.f;
    pd = 0.f;
    cell_phase_a<DIM>(a, alpha, beta, cur, x4, d4, d0, d1, prr, pg);
    __syncthreads();
    prof_mark(g, kPhVec);
    cell_phase_b<DIM>(a, cvec(a, cell_w(cur ^ 1)), pd);
    if (!grid_sum<float, 3>(g, prr, pg, pd, red, kPhSpmv)) return false;
    its = it;
    if (!isfinite(red.x)) {
      flag(g, kErrNonfinite);
      return false;
    }
    if (red.x <= thr) {
      cnt.its += it;
      return true;
    }
    const float gnew = red.y, dnew = red.z;
    beta = gnew / gam;
    const float den = dnew - beta * gnew / alpha;
    if (!(den > 0.f) || !isfinite(den)) {
      flag(g, kErrBreakdown);
      cnt.its += it;
      return true;
    }
    alpha = gnew / den;
    gam = gnew;
    cur ^= 1;
  }
  cnt.its += maxit;
  cnt.capped += 1;
  return true;
}

template <class TM, class TV>
__device__ __forceinline__ bool pcg(Grid& g, Ctx<TM, TV>& c, const TM* AV, int op, const TV* DI, TV* x,
                                    RhsSpec<TM, TV> rhs, double rtol, int maxit, InnerCount& cnt, int& its) {
  if (c.a.pcg_variant == 1) return pcg_pipelined<TM, TV>(g, c.a, AV, op, DI, x, rhs, rtol, maxit, cnt, its);
  if (c.a.pcg_variant == 3) {
    if constexpr (sizeof(TV) == 4) {
      if (c.a.cells) {
        if (c.a.cell_dim == 3) return pcg_cell<TM, 3>(g, c.a, op, DI, x, rhs, rtol, maxit, cnt, its);
        return pcg_cell<TM, 2>(g, c.a, op, DI, x, rhs, rtol, maxit, cnt, its);
      }
      if (c.a.tma) return pcg_cg<TM, TV, true>(g, c.a, AV, op, DI, x, rhs, rtol, maxit, cnt, its);
    }
    return pcg_cg<TM, TV, false>(g, c.a, AV, op, DI, x, rhs, rtol, maxit, cnt, its);
  }
  return pcg_standard<TM, TV>(g, c.a, AV, op, DI, x, rhs, rtol, maxit, cnt, its);
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
  using R = RhsSpec<TM, TV>;
  // (1) M y0 = v0
  if (!pcg(g, c, c.iM(), kOpM, c.dM(), c.vec(kVy0), R{v0, 1.0, nullptr, 0, nullptr, 0.0}, rt, mi, cnt, its))
    return false;
  // (2) (M + delta K) y1 = gamma v1 - tau_e K y0
  if (!pcg(g, c, c.iMdK(), kOpMdK, c.dMdK(), c.vec(kVy1), R{v1, a.gamma, c.iK(), kOpK, c.vec(kVy0), -a.tau_e}, rt,
           mi, cnt, its))
    return false;
  if (a.schur == 1) {
    // (3) S_D x1 = M y1, a fixed number of Jacobi-PCG iterations (Section 4.1, Table 2)
    if (!pcg_sd<TM, TV>(g, a, (const TV*)a.dSD, c.vec(kVx1), R{nullptr, 0.0, c.iM(), kOpM, c.vec(kVy1), 1.0},
                        a.schur_its, cnt, its))
      return false;
  } else {
    // (3.1) (M + sqrt(delta) K) w = M y1
    if (!pcg(g, c, c.iMsK(), kOpMsK, c.dMsK(), c.vec(kVwv), R{nullptr, 0.0, c.iM(), kOpM, c.vec(kVy1), 1.0}, rt, mi,
             cnt, its))
      return false;
    // (3.2) (M + sqrt(delta) K) x1 = M w
    if (!pcg(g, c, c.iMsK(), kOpMsK, c.dMsK(), c.vec(kVx1), R{nullptr, 0.0, c.iM(), kOpM, c.vec(kVwv), 1.0}, rt, mi,
             cnt, its))
      return false;
  }
  // (4) x0 = y0 + (y1 - x1) / delta, and z = (x0, x1, .)
  FOR_MY_GROUPS(g, s0, nsl) {
#pragma unroll
    for (int uu = 0; uu < kGroup; ++uu) {
      if (uu < nsl) {
        const int row = (s0 + uu) * 32 + lane;
        const double xx1 = (double)c.vec(kVx1)[row];
        z[row] = (double)c.vec(kVy0)[row] + ((double)c.vec(kVy1)[row] - xx1) * a.inv_delta;
        z[np + row] = xx1;
      }
    }
  }
  // (5) M x2 = v2 - K x1
  if (!pcg(g, c, c.iM(), kOpM, c.dM(), c.vec(kVx2), R{v2, 1.0, c.iK(), kOpK, c.vec(kVx1), -1.0}, rt, mi, cnt, its))
    return false;
  FOR_MY_GROUPS(g, s0, nsl) {
#pragma unroll
    for (int uu = 0; uu < kGroup; ++uu) {
      if (uu < nsl) {
        const int row = (s0 + uu) * 32 + lane;
        z[2 * np + row] = (double)c.vec(kVx2)[row];
      }
    }
  }
  return grid_sync(g, kPhVec);
}

// w = A^R z for one owned row (float64, one column-index stream, three value streams).
__device__ __forceinline__ void block_row(const SolveArgs& a, const double* z, int s, int lane, double& w0,
                                          double& w1, double& w2) {
  const int np = a.n_pad;
  const int beg = __ldg(a.slice_ptr + s) + lane;
  const int end = __ldg(a.slice_ptr + s + 1);
  double m_mu = 0, a_psi = 0, k_om = 0, k_mu = 0, m_psi = 0, k_psi = 0, m_om = 0;
#pragma unroll 4
  for (int idx = beg; idx < end; idx += 32) {
    const int c = __ldg(a.cols + idx);
    const double mv = __ldg(a.Mv + idx), kv = __ldg(a.Kv + idx), av = __ldg(a.Av + idx);
    const double zm = z[c], zp = z[np + c], zo = z[2 * np + c];
    m_mu = fma(mv, zm, m_mu);
    a_psi = fma(av, zp, a_psi);
    k_om = fma(kv, zo, k_om);
    k_mu = fma(a.A10 ? __ldg(a.A10 + idx) : kv, zm, k_mu);
    m_psi = fma(a.A11 ? __ldg(a.A11 + idx) : mv, zp, m_psi);
    k_psi = fma(kv, zp, k_psi);
    m_om = fma(mv, zo, m_om);
  }
  w0 = m_mu + a_psi + k_om;
  // PFC1: the second block row is [tau K_+(psi_k), M / gamma + tau F(mu_k)], stored
  w1 = a.A10 ? k_mu + m_psi : a.tau * k_mu + a.inv_gamma * m_psi;
  w2 = k_psi + m_om;
}

constexpr double kNaN = __builtin_nan("");
constexpr double kInf = __builtin_inf();

__device__ void write_stats(Grid& g, const SolveArgs& a, int outer, int restarts, const InnerCount& cnt, double rel,
                            double bnorm, int last_its, double err_est = kNaN, double sigma = kInf) {
  if (g.bid == 0 && threadIdx.x == 0) {
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
    for (int k = 0; k < 8; ++k) st.prof_ns[k] = s_prof[k];
    st.err_est = err_est;
    st.sigma = sigma;
    *a.stats = st;
  }
}

// Inverse iterations on R^T R for the solution-error estimate of fgmres.
constexpr int kSigmaIts = 16;

// Smallest singular value of the k x k upper triangle R (R_il = H[i + l ld], i <= l,
// k <= 64): inverse iteration on R^T R from the constant vector, kSigmaIts steps,
// with the Rayleigh quotient x^T (R^T R)^{-1} x as the estimate of 1 / sigma^2
// (so the result is >= sigma_min and converges to it).  Run by the 32 lanes of
// one warp together; lane L holds entries L and L + 32, and the triangular solves
// sweep by columns (one broadcast per row).  Every block computes the same value.
__device__ double tri_sigma_min(const double* H, int ld, int k) {
  const int lane = threadIdx.x & 31;
  for (int i = 0; i < k; ++i)
    if (!(H[i + i * ld] != 0.0)) return 0.0;
  const double x_init = 1.0 / sqrt((double)k);
  double x0 = lane < k ? x_init : 0.0, x1 = lane + 32 < k ? x_init : 0.0;
  double lam = 0.0;
  for (int it = 0; it < kSigmaIts; ++it) {
    double u0 = x0, u1 = x1;
    // R^T u = x: u_i = x_i / R_ii, then x_l -= R_il u_i for l > i
    for (int i = 0; i < k; ++i) {
      const double ui = __shfl_sync(0xffffffffu, (i < 32 ? u0 : u1) / H[i + i * ld], i & 31);
      if (lane == (i & 31)) {
        if (i < 32) u0 = ui;
        else u1 = ui;
      }
      if (lane > i && lane < k) u0 = fma(-H[i + lane * ld], ui, u0);
      if (lane + 32 > i && lane + 32 < k) u1 = fma(-H[i + (lane + 32) * ld], ui, u1);
    }
    // R v = u: v_i = u_i / R_ii, then u_l -= R_li v_i for l < i
    for (int i = k - 1; i >= 0; --i) {
      const double vi = __shfl_sync(0xffffffffu, (i < 32 ? u0 : u1) / H[i + i * ld], i & 31);
      if (lane == (i & 31)) {
        if (i < 32) u0 = vi;
        else u1 = vi;
      }
      if (lane < i) u0 = fma(-H[lane + i * ld], vi, u0);
      if (lane + 32 < i) u1 = fma(-H[lane + 32 + i * ld], vi, u1);
    }
    lam = warp_sum(fma(x0, u0, x1 * u1));
    const double inv = 1.0 / sqrt(warp_sum(fma(u0, u0, u1 * u1)));
    x0 = u0 * inv;
    x1 = u1 * inv;
  }
  return lam > 0.0 ? 1.0 / sqrt(lam) : 0.0;
}

// FGMRES(restart) with modified Gram-Schmidt, right preconditioner P_CH, zero
// initial guess; the true residual is recomputed in float64 at every restart.
//
// Stop rule.  The residual test ||b - A^R y|| <= tol_r ||b|| (tol_r = a.tol) ends a
// solve when a.err_tol = 0.  With a.err_tol > 0 the solution error must be small
// too: e = (A^R)^{-1} r = P^{-1} (A^R P^{-1})^{-1} r, so once the residual test passes
// the kernel estimates
//     E = ||P^{-1} r|| / (||y|| sigma),
// sigma = the smallest singular value of the cycles' Hessenberg matrices seen so far
// (they represent A^R P^{-1} on the Krylov spaces), and stops only if E <= err_tol.
// Otherwise it tightens tol_r to (||r|| / ||b||)(err_tol / E) / 2 and goes on; the
// P^{-1} r / ||r|| it computed is the first preconditioned vector of the next cycle,
// so a failed test wastes nothing.  The ratio E / (||r|| / ||b||) of the last tested
// solve is kept in a.kappa with its tau; the next solve starts from the residual
// target that ratio (scaled by tau / tau_kappa) predicts, so that the test usually
// passes the first time.
template <class TM, class TV>
__device__ void fgmres(Grid& g, Ctx<TM, TV>& c) {
  const SolveArgs& a = c.a;
  __shared__ double H[(kMaxRestart + 1) * kMaxRestart];
  __shared__ double gv[kMaxRestart + 1], cs[kMaxRestart], sn[kMaxRestart], yk[kMaxRestart];
  __shared__ int s_k;
  __shared__ double s_sigma;
  const int np = a.n_pad, n3 = 3 * np, m = a.restart, ld = m + 1;
  const int lane = threadIdx.x & 31;
  const bool err_test = a.err_tol > 0.0;
  InnerCount cnt;
  Sum4<double> red;
  double tol_r = a.tol;
  if (err_test && a.kappa) {
    const double k0 = a.kappa[0], t0 = a.kappa[1];
    if (k0 > 0.0 && t0 > 0.0 && isfinite(k0))
      tol_r = fmin(a.tol, fmax(1e-16, 0.5 * a.err_tol / (k0 * (a.tau / t0))));
  }
  if (threadIdx.x == 0) s_sigma = kInf;
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
  if (!grid_sum<double, 1>(g, pb, 0.0, 0.0, red, kPhOuter)) return;
  const double bnorm = sqrt(red.x);
  if (!isfinite(bnorm)) {
    flag(g, kErrNonfinite);
    return;
  }
  if (bnorm == 0.0) {
    write_stats(g, a, 0, 0, cnt, 0.0, 0.0, 0);
    return;
  }
  int total = 0, restarts = 0;
  bool first = true;
  double ynorm = 0.0, err_est = kNaN;
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
    if (!grid_sum<double, 1>(g, pr, 0.0, 0.0, red, kPhOuter)) return;
    const double beta = sqrt(red.x);
    if (!isfinite(beta)) {
      flag(g, kErrNonfinite);
      return;
    }
    const bool res_ok = beta <= tol_r * bnorm;
    // the error test needs an iterate (not the first pass) and one more P^{-1}
    bool checking = res_ok && err_test && !first && beta > 0.0 && total < a.max_outer;
    if (!checking && (res_ok || total >= a.max_outer)) {
      // a passing residual whose error test is still owed at the cap is not converged
      if (!res_ok || (err_test && beta > 0.0 && !first)) flag(g, kErrOuterCap);
      write_stats(g, a, total, restarts, cnt, beta / bnorm, bnorm, 0, err_est, s_sigma);
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
      // w = A^R z_j, then modified Gram-Schmidt against V_0..V_j; during an error
      // test also ||z_0||^2 = ||P^{-1} r||^2 / beta^2
      const bool test_now = checking && j == 0;
      double ph = 0.0, pz = 0.0;
      FOR_MY_SLICES(g, s) {
        const int row = s * 32 + lane;
        double w0, w1, w2;
        block_row(a, zj, s, lane, w0, w1, w2);
        w[row] = w0;
        w[np + row] = w1;
        w[2 * np + row] = w2;
        ph += w0 * V0[row] + w1 * V0[np + row] + w2 * V0[2 * np + row];
        if (test_now) {
          const double z0 = zj[row], z1 = zj[np + row], z2 = zj[2 * np + row];
          pz += z0 * z0 + z1 * z1 + z2 * z2;
        }
      }
      if (test_now) {
        if (!grid_sum<double, 2>(g, ph, pz, 0.0, red, kPhOuter)) return;
        err_est = beta * sqrt(red.y) / (ynorm * s_sigma);
        if (!(err_est > a.err_tol)) {
          if (!isfinite(err_est)) {
            flag(g, kErrNonfinite);
            return;
          }
          if (a.kappa && g.bid == 0 && threadIdx.x == 0) {
            a.kappa[0] = err_est * bnorm / beta;
            a.kappa[1] = a.tau;
          }
          write_stats(g, a, total, restarts, cnt, beta / bnorm, bnorm, 0, err_est, s_sigma);
          return;
        }
        tol_r = fmax(1e-16, 0.5 * (beta / bnorm) * (a.err_tol / err_est));
        checking = false;
      } else {
        if (!grid_sum<double, 1>(g, ph, 0.0, 0.0, red, kPhOuter)) return;
      }
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
        if (!grid_sum<double, 1>(g, pn, 0.0, 0.0, red, kPhOuter)) return;
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
      if (fabs(gv[j + 1]) <= tol_r * bnorm || hnext == 0.0 || total >= a.max_outer) break;
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
    // warp 0 finds the cycle's smallest singular value (the rotated k x k triangle
    // has those of the Hessenberg matrix) while the other warps update y
    if (err_test && threadIdx.x < 32) {
      const double sg = tri_sigma_min(H, ld, kk);
      if (threadIdx.x == 0) s_sigma = fmin(s_sigma, sg);
    }
    double py = 0.0;
    FOR_MY_SLICES(g, s) {
      const int row = s * 32 + lane;
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        double acc = a.y[f * np + row];
        for (int i = 0; i < kk; ++i) acc = fma(yk[i], a.Z[(size_t)i * n3 + f * np + row], acc);
        a.y[f * np + row] = acc;
        py = fma(acc, acc, py);
      }
    }
    restarts += 1;
    if (err_test) {
      if (!grid_sum<double, 1>(g, py, 0.0, 0.0, red, kPhOuter)) return;
      ynorm = sqrt(red.x);
    } else {
      if (!grid_sync(g, kPhOuter)) return;
    }
  }
}

// One solve (FGMRES stage solve, one P_CH application or one PCG solve) run by
// the G blocks bid = 0..G-1 of a grid or of a segment of a batched grid.
template <class TM, class TV>
__device__ __forceinline__ void solve_body(const SolveArgs& a, int bid, int G) {
  Grid g;
  g.arrive = a.arrive;
  g.err = a.err;
  g.part = a.part;
  g.bid = bid;
  g.G = G;
  g.expect = G + a.barrier_extra;
  g.limit_ns = a.spin_limit_ns;
  g.epoch = 0;
  g.ring = 0;
  {
    const int wi = bid * kWarps + (int)(threadIdx.x >> 5);
    g.w_lo = __ldg(a.blk + wi);
    g.w_hi = __ldg(a.blk + wi + 1);
    g.b_lo = __ldg(a.blk + bid * kWarps);
    g.b_hi = __ldg(a.blk + (bid + 1) * kWarps);
    g.wid = (int)(threadIdx.x >> 5);
    // slot bounds of this warp's slices in registers when it has at most 32
    g.sp_reg = my_slice(g, 32) >= PFC_WARP_END(g);
    const int sl = my_slice(g, (int)(threadIdx.x & 31));
    const bool have = g.sp_reg && sl < PFC_WARP_END(g);
    g.sp_lane = have ? __ldg(a.slice_ptr + sl) : 0;
    g.sp_end = have ? __ldg(a.slice_ptr + sl + 1) : 0;
  }
  g.prof = a.prof && bid == 0 && threadIdx.x == 0;
  {
    const int rs = __ldg(a.blk + bid * kWarps) * 32, re = __ldg(a.blk + (bid + 1) * kWarps) * 32;
    g.win_lo = max(0, rs - a.st_halo) & ~3;
    g.win_n = min(a.n_pad, (re + a.st_halo + 3) & ~3) - g.win_lo;
    g.staged = sizeof(TV) == 4 && a.stencil && a.win_cap > 0 && re > rs && g.win_n <= a.win_cap;
    g.ri_smem = false;
    // neighbour range: blocks whose rows meet [rs - halo, re + halo)
    g.nbsync = PFC_NEIGHBOR_SYNC && !PFC_INTERLEAVE && a.stencil && a.st_halo > 0 && a.barrier_extra == 0;
    g.nepoch = 0;
    g.flags = a.arrive + 4;
    g.nb_lo = g.nb_hi = bid;
    if (g.nbsync) {
      while (g.nb_lo > 0 && __ldg(a.blk + g.nb_lo * kWarps) * 32 > rs - a.st_halo) --g.nb_lo;
      while (g.nb_hi + 1 < G && __ldg(a.blk + (g.nb_hi + 1) * kWarps) * 32 < re + a.st_halo) ++g.nb_hi;
      g.nbsync = g.nb_hi - g.nb_lo < kThreads;
    }
  }
  if (threadIdx.x == 0) {
    for (int k = 0; k < 8; ++k) s_prof[k] = 0;
    s_t_last = global_ns();
  }
  if (a.stencil) {
    using Acc = typename AccOf<TV>::type;
    // table stride: the longest type stencil rounded up to a multiple of 4 (the
    // host checks (types + 1) * stride <= kMaxStencil); entries past a type's
    // length and the whole extra type a.st_types are (offset 0, weight 0)
    int L = 0;
    for (int t = 0; t < a.st_types; ++t) L = max(L, __ldg(a.st_start + t + 1) - __ldg(a.st_start + t));
    L = (L + 3) & ~3;
    const int total = (a.st_types + 1) * L;
    StEntry<Acc>* tab = reinterpret_cast<StEntry<Acc>*>(s_st_raw);
    for (int k = threadIdx.x; k < total; k += blockDim.x) {
      const int t = k / L, j = k - t * L;
      const int len = t < a.st_types ? __ldg(a.st_start + t + 1) - __ldg(a.st_start + t) : 0;
      int off = 0;
      double wm = 0.0, wk = 0.0;
      if (j < len) {
        const int src = __ldg(a.st_start + t) + j;
        off = __ldg(a.st_off + src);
        wm = __ldg(a.st_wM + src);
        wk = __ldg(a.st_wK + src);
      }
      if (a.tma) {
        // staged window offset of the entry: off - dz (plane - S), dz its plane offset
        int sd = off;
        if (a.plane) {
          const int half = a.plane / 2;
          const int dz = off >= 0 ? (off + half) / a.plane : -((-off + half) / a.plane);
          sd = off - dz * (a.plane - a.tma_S);
        }
        s_sdelta[k] = sd;
      }
#pragma unroll
      for (int op = 0; op < 4; ++op) {
        StEntry<Acc> e{};
        e.off = off;
        e.w = (Acc)(a.op_cM[op] * wm + a.op_cK[op] * wk);
        tab[op * kMaxStencil + k] = e;
      }
    }
    if ((int)threadIdx.x <= a.st_types) {
      const int t = threadIdx.x;
      s_st_start[t] = t * L;
      s_st_cnt[t] = t < a.st_types ? __ldg(a.st_start + t + 1) - __ldg(a.st_start + t) : 0;
    }
    if (a.tma) {
      __syncthreads();   // s_sdelta complete
      if ((int)threadIdx.x < a.st_types) {
        const int t = threadIdx.x;
        int lo = 0, hi = 0;
        for (int k = t * L; k < t * L + (__ldg(a.st_start + t + 1) - __ldg(a.st_start + t)); ++k) {
          lo = min(lo, s_sdelta[k]);
          hi = max(hi, s_sdelta[k]);
        }
        s_sd_lo[t] = lo;
        s_sd_hi[t] = hi;
      }
    }
    if (a.tma && threadIdx.x == 0) {
      mbar_init(&s_mbar[0], 1);
      mbar_init(&s_mbar[1], 1);
      s_tma_uses[0] = s_tma_uses[1] = 0;
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (sizeof(TV) == 4 && a.cells) cell_tables(g, a);
    // this block's row-info bytes, 16 at a time (the row ranges start at multiples of 32)
    const int nrow = (g.b_hi - g.b_lo) * 32;
    g.ri_smem = nrow <= kRowInfoCap;
    if (g.ri_smem) {
      const uint4* src = reinterpret_cast<const uint4*>(a.rowinfo + g.b_lo * 32);
      uint4* dst = reinterpret_cast<uint4*>(s_rowinfo);
      for (int i = threadIdx.x; i < nrow / 16; i += kThreads) dst[i] = __ldg(src + i);
    }
    __syncthreads();
  }
  Ctx<TM, TV> c(a);
  const int lane = threadIdx.x & 31;
  if (a.mode == 0) {
    fgmres(g, c);
  } else if (a.mode == 1) {
    InnerCount cnt;
    if (apply_pch(g, c, a.b, a.y, cnt)) write_stats(g, a, 0, 0, cnt, 0.0, 0.0, 0);
  } else {
    InnerCount cnt;
    int its = 0;
    const TM* AV = a.which == 0 ? c.iM() : a.which == 1 ? c.iMdK() : c.iMsK();
    const int op = a.which == 0 ? kOpM : a.which == 1 ? kOpMdK : kOpMsK;
    const TV* DI = a.which == 0 ? c.dM() : a.which == 1 ? c.dMdK() : c.dMsK();
    const double* b = a.b;
    if (!pcg(g, c, AV, op, DI, c.vec(kVy0), RhsSpec<TM, TV>{b, 1.0, nullptr, 0, nullptr, 0.0}, a.inner_rtol,
             a.max_inner, cnt, its))
      return;
    FOR_MY_SLICES(g, s) {
      const int row = s * 32 + lane;
      a.y[row] = (double)c.vec(kVy0)[row];
    }
    write_stats(g, a, 0, 0, cnt, 0.0, 0.0, its);
  }
}

template <class TM, class TV>
__global__ void __launch_bounds__(kThreads, PFC_SOLVER_MINBLOCKS) solve_kernel(const __grid_constant__ SolveArgs a) {
  solve_body<TM, TV>(a, blockIdx.x, gridDim.x);
}

// Batched launch: instance k owns the blocks seg[k] .. seg[k+1]-1 of the grid and
// solves its own stage system with them (its own barrier counter, partial sums,
// error word and statistics).  Segments never wait for one another.
template <class TM, class TV>
__global__ void __launch_bounds__(kThreads, PFC_SOLVER_MINBLOCKS) solve_batch_kernel(const __grid_constant__ BatchArgs b) {
  int lo = 0, hi = b.count;  // find k with seg[k] <= blockIdx.x < seg[k+1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(b.seg + mid) <= (int)blockIdx.x) lo = mid;
    else hi = mid;
  }
  const int s0 = __ldg(b.seg + lo), s1 = __ldg(b.seg + lo + 1);
  solve_body<TM, TV>(b.inst[lo], (int)blockIdx.x - s0, s1 - s0);
}

template <class TM, class TV>
const void* kernel_ptr(bool batch) {
  return batch ? (const void*)solve_batch_kernel<TM, TV> : (const void*)solve_kernel<TM, TV>;
}

const void* kernel_for(int prec, bool batch = false) {
  if (prec == 0) return kernel_ptr<double, double>(batch);
  if (prec == 1) return kernel_ptr<float, float>(batch);
  return kernel_ptr<__half, float>(batch);
}

}  // namespace

int solve_threads() { return kThreads; }
int solve_ring() { return kRing; }

// Allows dyn_smem bytes of dynamic shared memory for the kernel (above the 48 KiB
// default a kernel must opt in).
cudaError_t allow_dyn_smem(const void* fn, size_t dyn_smem) {
  if (dyn_smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem);
}

cudaError_t solve_occupancy(int prec, int* blocks_per_sm, size_t dyn_smem) {
  cudaError_t e = allow_dyn_smem(kernel_for(prec), dyn_smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kernel_for(prec), kThreads, dyn_smem);
}

cudaError_t launch_solve(int prec, int grid, const SolveArgs& args, cudaStream_t stream) {
  SolveArgs local = args;
  void* params[] = {&local};
  size_t dyn = (prec != 0 && args.win_cap > 0) ? (size_t)args.win_cap * sizeof(float) : 0;
  if (prec != 0 && args.tma) dyn = 2 * (size_t)args.tma_cap * sizeof(float);
  if (prec != 0 && args.cells)
    dyn = cell_smem_bytes(args.cell_wcap, args.cell_dim == 3 ? 2 : 1, args.cell_rcap, args.ccls_n,
                          args.cell_dim == 3 ? 232 : 48, args.cell_ccap);
  cudaError_t e = allow_dyn_smem(kernel_for(prec), dyn);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel(kernel_for(prec), dim3(grid), dim3(kThreads), params, dyn, stream);
}

cudaError_t batch_occupancy(int prec, int* blocks_per_sm, size_t dyn_smem) {
  cudaError_t e = allow_dyn_smem(kernel_for(prec, true), dyn_smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kernel_for(prec, true), kThreads, dyn_smem);
}

cudaError_t launch_solve_batch(int prec, int grid, const BatchArgs& args, cudaStream_t stream, size_t dyn_smem) {
  BatchArgs local = args;
  void* params[] = {&local};
  cudaError_t e = allow_dyn_smem(kernel_for(prec, true), dyn_smem);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel(kernel_for(prec, true), dim3(grid), dim3(kThreads), params, dyn_smem, stream);
}

}  // namespace pfc
