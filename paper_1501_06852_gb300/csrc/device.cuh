// Device helpers shared by the kernels of the PFC stage solver.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "cell2d.h"
#include "cell3d.h"

namespace pfc {

// Device error bits (DevStats::err and the context error word).
enum : int {
  kErrTimeout = 1,     // a grid barrier stopped waiting
  kErrNonfinite = 2,   // NaN/Inf in a reduction
  kErrOuterCap = 4,    // FGMRES hit max_outer
  kErrBreakdown = 8    // p^T A p <= 0 in PCG (matrix not SPD or underflow)
};

struct DevStats {
  int outer_its;
  int restarts;
  int inner_calls;
  int inner_capped;
  long long inner_its;
  double rel_residual;
  double bnorm;
  int err;
  int last_its;        // iterations of a single PCG solve (pcg mode)
  long long prof_ns[8];  // block 0: work / barrier-wait time per phase class (when profiling)
  double err_est;      // last solution-error estimate E (err_tol > 0; NaN when never tested)
  double sigma;        // smallest singular value of the cycles' Hessenberg matrices (inf: none)
};

// Arguments of the persistent solver kernel.  Inner arrays are typed by the
// kernel instantiation (TM for matrix values, TV for inner vectors).
struct SolveArgs {
  int n_pad;
  const int* slice_ptr;
  const int* cols;
  const int* blk;          // gridDim.x * warps + 1 slice boundaries, one range per warp
  const double* Mv;        // float64 M, K, A01 values (outer operator A^R)
  const double* Kv;
  const double* Av;
  const double* A10;       // PFC1: tau K_+(psi_k) and M / gamma + tau F(mu_k) (second block row); PFC2: null
  const double* A11;
  const void* iM;          // inner values M, K, M + delta K, M + sqrt(delta) K
  const void* iK;
  const void* iMdK;
  const void* iMsK;
  const void* dM;          // inner Jacobi inverses of M, M + delta K, M + sqrt(delta) K
  const void* dMdK;
  const void* dMsK;
  double tau, gamma, inv_gamma, tau_e, inv_delta;
  double tol, inner_rtol;
  double err_tol;          // > 0: FGMRES also stops only once its solution-error estimate is <= err_tol
  double* kappa;           // err_tol > 0: {error / residual ratio, tau} of the context's last tested
                           //   solve (read at the start to set the residual target, written at the end)
  int restart, max_outer, max_inner;
  int mode;                // 0 FGMRES stage solve, 1 one P_CH application, 2 one PCG solve
  int which;               // mode 2: 0 M, 1 M + delta K, 2 M + sqrt(delta) K
  const double* b;         // 3 n_pad (modes 0, 1) or n_pad (mode 2)
  double* y;
  double* V;               // (restart + 1) x 3 n_pad
  double* Z;               // restart x 3 n_pad
  void* ivec;              // kInnerVecs inner vectors of n_pad TV each
  unsigned* arrive;        // grid barrier counter (zeroed before each launch)
  int* err;                // error word (zeroed before each launch)
  double4_32a* part;           // reduction partials, kRing x gridDim.x
  DevStats* stats;
  unsigned long long spin_limit_ns;  // a barrier wait gives up after this long
  int barrier_extra;       // 0; > 0 only in the timeout self-test (waits cannot complete)
  int pcg_variant;         // 0 standard PCG (3 grid barriers per iteration), 1 pipelined PCG (1)
  int prof;                // 1: block 0 records per-phase work and wait times
  // structured-stencil inner operators (lexicographic internal order only)
  int stencil;             // 1: interior rows of M, K, M + delta K, M + sqrt(delta) K use the stencils
  const unsigned char* rowinfo;  // bits 0-2 dof type, bit 3 interior
  const int* st_start;     // ntypes + 1
  const int* st_off;       // column offset of each stencil entry
  const double* st_wM;     // M and K weights of each entry
  const double* st_wK;
  int st_types;
  int schur;               // 0: S_CH (steps 3.1, 3.2); 1: S_D (step 3, schur_its Jacobi-PCG iterations)
  int schur_its;
  const void* dSD;         // inner-type Jacobi inverse of diag(S_D) (schur == 1)
  int st_halo;             // largest |column offset| of a stencil entry
  int win_cap;             // > 0: floats of dynamic shared memory per block for the window of
                           //   the SpMV source vector (float inner vectors only); 0: no window
  double op_cK[4];         // inner operator op = M, K, M + delta K, M + sqrt(delta) K:
  double op_cM[4];         //   weights op_cM[op] * wM + op_cK[op] * wK
  // chunked stencil SpMV with bulk-copied source windows (float inner vectors, structured
  // stencils, lexicographic rows; see spmv_chunks in solver.cu)
  int tma;                 // 1: on
  int lat;                 // lattice points per axis
  int plane;               // rows per lattice plane (3D: lat^2); 0 in 2D (one window segment)
  int tma_S;               // 3D: shared-memory stride between plane segments (S = plane mod 4)
  int tma_cap;             // floats of one window buffer (two buffers in dynamic shared memory)
  // cell kernels of the Chronopoulos-Gear inner solves (P2 rows in cell-major order,
  // float inner vectors; pcg_cell in solver.cu): the block keeps u on its tile of cells
  // and the ring around it in dynamic shared memory (cell_smem_bytes)
  int cells;               // 1: on (the host checked the stencils and the shared memory)
  int cell_dim;            // 2 or 3
  int cell_S;              // cells per lattice axis (side + 1)
  int cell_gx, cell_gy, cell_gz;  // tiles of the cell grid per axis (block b owns tile
                                  // (b % gx, (b / gx) % gy, b / (gx gy)))
  int cell_ccap;           // largest tile, in cells
  int cell_wcap;           // largest tile with its ring, in cells
  int cell_rcap;           // largest ring, in cells
  int ccls_n;              // cell classes: distinct stencils of a cell's rows (class 0: all interior)
  const double* ccls_wM;   // ccls_n x couplings (46 in 2D, 230 in 3D): M and K weights of the
  const double* ccls_wK;   //   couplings of cell2d.h / cell3d.h (0 where a row lacks one)
  const unsigned char* cellclass;  // n_pad / 2^dim: class of each cell
  int cell_rep[8];         // an interior row of each dof type (its Jacobi inverse is the type's)
};

// Dynamic shared memory of the cell kernels, in this order: the window of u (U planes
// of one float4 per cell of the tile and its ring; U = 1 in 2D, 2 in 3D), the ring cells {window
// cell, cell or -1}, the current operator's coupling weights for every cell class
// (stride floats per class: 48 in 2D, 232 in 3D), the classes of the tile's cells.
__host__ __device__ inline size_t cell_off_ring(int wcap, int U) { return (size_t)wcap * U * 16; }
__host__ __device__ inline size_t cell_off_weights(int wcap, int U, int rcap) {
  return cell_off_ring(wcap, U) + (((size_t)rcap * 8 + 15) & ~(size_t)15);
}
__host__ __device__ inline size_t cell_off_classes(int wcap, int U, int rcap, int ncc, int stride) {
  return cell_off_weights(wcap, U, rcap) + (size_t)ncc * stride * 4;
}
__host__ __device__ inline size_t cell_smem_bytes(int wcap, int U, int rcap, int ncc, int stride, int ccap) {
  return cell_off_classes(wcap, U, rcap, ncc, stride) + (((size_t)ccap + 15) & ~(size_t)15);
}

// A batched launch: instance k (arguments inst[k], in device memory) owns the
// blocks seg[k] .. seg[k+1]-1 of the grid.
struct BatchArgs {
  const SolveArgs* inst;
  const int* seg;
  int count;
};

constexpr int kMaxStencil = 640;   // stencil entries over all dof types
enum : int { kOpM = 0, kOpK = 1, kOpMdK = 2, kOpMsK = 3 };

constexpr int kInnerVecs = 16;

template <class T> struct AccOf { using type = float; };
template <> struct AccOf<double> { using type = double; };

template <class A> __device__ __forceinline__ A ld_val(const double* p) { return (A)__ldg(p); }
template <class A> __device__ __forceinline__ A ld_val(const float* p) { return (A)__ldg(p); }
template <class A> __device__ __forceinline__ A ld_val(const __half* p) { return (A)__half2float(__ldg(p)); }

template <class T> __device__ __forceinline__ T from_acc(double v) { return (T)v; }
template <class T> __device__ __forceinline__ T from_acc(float v) { return (T)v; }

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed_i32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// y_row = sum_j vals[j] x[cols[j]] over one SELL-32 row (slot stride 32).
// Matrix data is read-only for the kernel lifetime (__ldg); x is written by
// other blocks during persistent kernels, so it is read with plain loads.
template <class Acc, class TM, class TX>
__device__ __forceinline__ Acc sell_row(const int* __restrict__ slice_ptr, const int* __restrict__ cols,
                                        const TM* __restrict__ vals, const TX* x, int s, int lane) {
  const int beg = __ldg(slice_ptr + s) + lane;
  const int end = __ldg(slice_ptr + s + 1);
  Acc acc = Acc(0);
#pragma unroll 4
  for (int idx = beg; idx < end; idx += 32) {
    const int c = __ldg(cols + idx);
    acc = fma(ld_val<Acc>(vals + idx), (Acc)x[c], acc);
  }
  return acc;
}

}  // namespace pfc
