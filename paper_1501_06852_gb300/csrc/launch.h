// Host-side launchers of the device kernels (one translation unit each).
#pragma once

#include <cuda_runtime.h>

#include "device.cuh"

namespace pfc {

// persistent solver (solver.cu); prec: 0 float64, 1 float32, 2 float16 values
int solve_threads();
int solve_ring();
cudaError_t solve_occupancy(int prec, int* blocks_per_sm, size_t dyn_smem = 0);
cudaError_t launch_solve(int prec, int grid, const SolveArgs& args, cudaStream_t stream);
cudaError_t batch_occupancy(int prec, int* blocks_per_sm, size_t dyn_smem = 0);
// dyn_smem: dynamic shared memory per block (the cell kernels' window and tables)
cudaError_t launch_solve_batch(int prec, int grid, const BatchArgs& args, cudaStream_t stream, size_t dyn_smem = 0);

// element and vector kernels (kernels.cu)
// element kernels take the local node count nl: 6 / 10 (P2 triangles / tetrahedra), 3 / 4 (P1)
cudaError_t upload_quartic(int nl, const double* unit_quartic, int npairs);
cudaError_t launch_assemble_mk(long long nnz_sell, const int* cptr, const int* cidx, int E, int ntypes, int np,
                               const double* mass_tab, const double* stiff_tab, double* Mv, double* Kv,
                               cudaStream_t st);
cudaError_t launch_elem_quartic(int nl, int E, const int* elem, const double* psi, double vol, double* ebuf,
                                cudaStream_t st);
cudaError_t launch_elem_load(int nl, int E, const int* elem, const double* psi, double vol, double* lbuf,
                             cudaStream_t st);
cudaError_t launch_assemble_a01(long long nnz_sell, const int* cptr, const int* cidx, const double* ebuf,
                                const double* Mv, const double* Kv, double r, double* Av, cudaStream_t st);
cudaError_t launch_inner_mats(int prec, long long nnz_sell, const double* Mv, const double* Kv, double delta,
                              double sdelta, double* MdK, double* MsK, void* iMdK, void* iMsK, cudaStream_t st);
cudaError_t launch_convert(int prec, long long count, const double* src, void* dst, cudaStream_t st);
cudaError_t launch_diag_inv(int n_pad, const int* diag_pos, const double* A, double* dinv, float* fdinv,
                            cudaStream_t st);
cudaError_t launch_rhs(int nslices, const int* slice_ptr, const int* cols, const double* Mv, const double* Kv,
                       const int* dptr, const int* didx, const double* lbuf, const double* x, const double* d,
                       double r, double tau, const double* lbuf2, double* b, cudaStream_t st);
// PFC1 mobility (Eq. 3.10): element values of K_+(psi) and F(mu), element loads
// (psi^+ grad mu, grad phi), slot assembly of A10 = tau K_+ and A11 = M / gamma + tau F
cudaError_t upload_pairs(int nl, const int* pair_j, int npairs);
cudaError_t launch_elem_mobility(int nl, int E, int ntypes, const int* elem, const double* psi, const double* mu,
                                 double psi_min, const double* mob, double* ebuf, cudaStream_t st);
cudaError_t launch_elem_mobload(int nl, int E, int ntypes, const int* elem, const double* psi, const double* mu,
                                double psi_min, const double* mob, double* lbuf, cudaStream_t st);
cudaError_t launch_assemble_mob(int nl, long long nnz, const int* cptr, const int* cidx, const int* cols,
                                const int* elem, int E, const double* ebuf, const double* Mv, double tau,
                                double inv_gamma, int with_f, double* A10, double* A11, cudaStream_t st);
cudaError_t launch_sd_diag_inv(int nslices, const int* sp, const int* cols, const double* Mv, const double* Kv,
                               const int* diag_pos, const double* mdinv, double delta, double* out, float* fout,
                               cudaStream_t st);
cudaError_t launch_row_sums(int nslices, const int* sp, const double* vals, double* w, cudaStream_t st);
cudaError_t launch_sum_partials(int nparts, const double* partial, double scale, double* out, cudaStream_t st);
cudaError_t launch_dot_partials(int n, const double* a, const double* b, double* partial, int nparts,
                                cudaStream_t st);
cudaError_t launch_euler_rhs(int nslices, int n_pad, const int* slice_ptr, const int* cols, const double* Mv,
                             const int* dptr, const int* didx, const double* lbuf, const double* psi, double* b,
                             cudaStream_t st);
cudaError_t launch_dof_gather(int n_pad, const int* dptr, const int* didx, const double* lbuf, double* out,
                              cudaStream_t st);
cudaError_t launch_spmv_combo(int nslices, const int* slice_ptr, const int* cols, const double* Mv,
                              const double* Kv, double alpha, const double* u, double beta, const double* v,
                              double gam, const double* w, double delt, const double* l, double* out,
                              cudaStream_t st);
cudaError_t launch_spmv(int nslices, const int* slice_ptr, const int* cols, const double* vals, const double* x,
                        double* y, cudaStream_t st);
cudaError_t launch_spmv_ar(int nslices, int n_pad, const int* slice_ptr, const int* cols, const double* Mv,
                           const double* Kv, const double* Av, double tau, double inv_gamma, const double* A10,
                           const double* A11, const double* z, double* w, cudaStream_t st);
cudaError_t launch_stage_combine(int n_pad, const double* xk, const double* y0, const double* y1, int nprev,
                                 double a0, double a1, double c0, double c1, double* xi, double* d,
                                 cudaStream_t st);
cudaError_t launch_step_combine(int n_pad, const double* xk, const double* y0, const double* y1,
                                const double* y2, const double m[3], const double e[3], double atol, double rtol,
                                double* xnew, double* partial, int nparts, cudaStream_t st);
cudaError_t launch_reduce_partials(int nparts, const double* partial, double scale, double* out, cudaStream_t st);
cudaError_t launch_gather_in(int n, int n_pad, int nf, const int* perm, const double* lex, double* internal,
                             cudaStream_t st);
cudaError_t launch_scatter_out(int n, int n_pad, int nf, const int* perm, const double* internal, double* lex,
                               cudaStream_t st);
cudaError_t launch_combine_field(int n_pad, const double* a, double sa, const double* b, double sb, double* out,
                                 cudaStream_t st);
int step_partials();

}  // namespace pfc
