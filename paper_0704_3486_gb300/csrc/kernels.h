// Host-side launchers of the library's kernels (internal interface).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace ovs {

struct Geom;

enum { PREC_F64 = 0, PREC_F32 = 1 };

// Opt a kernel in to `bytes` of dynamic shared memory on the current device
// (once per kernel, device and size; thread safe).
cudaError_t ensure_dyn_smem(const void* kernel, size_t bytes);

// ---- K1 / K7 (dslash.cu)
// Shape of a stencil launch: `rt` right-hand sides per thread (1 or 2), a
// block of `sites` sites (threadIdx.x) times `rb` right-hand-side tiles
// (threadIdx.y). Every shape gives bit-identical results (each output entry
// is summed by one thread in the same order).
struct StencilShape {
    int rt = 1;
    int sites = 128;
    int rb = 1;
};
constexpr int kNumStencilShapes = 18;
constexpr StencilShape kStencilShapes[kNumStencilShapes] = {
    {1, 32, 1}, {1, 32, 2}, {1, 32, 4}, {1, 32, 8}, {1, 64, 1}, {1, 64, 2}, {1, 64, 4}, {1, 128, 1}, {1, 128, 2},
    {2, 32, 1}, {2, 32, 2}, {2, 32, 4}, {2, 32, 8}, {2, 64, 1}, {2, 64, 2}, {2, 64, 4}, {2, 128, 1}, {2, 128, 2}};
cudaError_t launch_wilson(int prec, bool gamma5, const void* links, const void* in, size_t in_stride, void* out,
                          size_t out_stride, const Geom& g, int nrhs, double kappa, double mu, const int* active,
                          cudaStream_t st, StencilShape shape = StencilShape{});
// out = ah * H_w in + bx * X + by * Y (fused Chebyshev-recurrence step)
cudaError_t launch_wilson_axpy(int prec, const void* links, const void* in, size_t in_stride, void* out,
                               size_t out_stride, const void* X, size_t xs, double bx, const void* Y, size_t ys,
                               double by, double ah, const Geom& g, int nrhs, double kappa, double mu,
                               cudaStream_t st, StencilShape shape = StencilShape{});
// flat complex128 <-> complex64 conversion of internal fields (to_prec = target)
cudaError_t launch_convert(int to_prec, const void* in, void* out, long long ncplx, cudaStream_t st);
// uniform (-1,1) complex entries from a hash of (seed, index)
cudaError_t launch_random_fill(void* q, long long ncplx, uint64_t seed, cudaStream_t st);
cudaError_t launch_to_internal(int prec, const void* canon, size_t canon_stride_cplx, void* out, size_t out_stride,
                               int V, int nrhs, cudaStream_t st);
cudaError_t launch_to_canonical(int prec, const void* in, size_t in_stride, void* canon, size_t canon_stride_cplx,
                                int V, int nrhs, cudaStream_t st);
// canon = x + gamma5 * in (in: internal complex128 planes): D_ov's last step
cudaError_t launch_to_canonical_overlap(const void* in, size_t in_stride, const void* x, size_t x_stride_cplx,
                                        void* canon, size_t canon_stride_cplx, int V, int nrhs, cudaStream_t st);
cudaError_t launch_links_to_internal(const void* canon, void* u64, void* u32, int V, cudaStream_t st);
cudaError_t launch_links_to_canonical(const void* u64, void* canon, int V, cudaStream_t st);

// ---- K2 / K4 / K5 (blas.cu)
// A "field" is a flat array of 16-byte units: one complex128 (F64) or two
// complex64 (F32). nunits = N (F64) or N/2 (F32).
struct BlasPlan {
    int nblk;        // row blocks per right-hand side
    long long chunk; // units per row block
};
BlasPlan blas_plan(long long nunits, int nrhs, int num_sms);

// Inner products of one sweep over J basis vectors (K2 / K5):
// partial[r][b][S], S = gdots_stride(nw, J) = nw*J + 2, holds for row
// block b: s_i = V_i^H u (i < J), then (nw == 2) t_i = V_i^H z, then
// (u^H u, 0) and u^H z if extras. Basis of rhs r at basis + r*basis_rhs_stride
// units (0: shared by all rhs), vector i at + i*vec_stride units.
int gdots_stride(int nw, int J);
cudaError_t launch_gdots(int prec, int nw, const void* basis, long long basis_rhs_stride, long long vec_stride,
                         int J, const void* u, long long u_rhs_stride, const void* z, long long z_rhs_stride,
                         bool extras, long long nunits, const BlasPlan& plan, int nrhs, void* partial,
                         const int* active, cudaStream_t st);

// out_r = in_r + alpha * sum_{i<J_r} V_r,i c_r,i   (coef: complex128 [r][coef_stride])
// J_r = J (host) or Jdev[r] (device, if Jdev != nullptr, clamped to J).
// out precision: prec_out (F64: complex128 units, F32: complex64 pairs). in may
// be nullptr (zero) or equal to out. If norm_partial != nullptr, also
// writes sum |out|^2 per block to norm_partial[r][b].
cudaError_t launch_update(int prec_v, int prec_out, const void* basis, long long basis_rhs_stride,
                          long long vec_stride, int J, const int* Jdev, const void* coef, long long coef_stride,
                          double alpha, const void* in, long long in_rhs_stride, void* out, long long out_rhs_stride,
                          long long nunits_v, const BlasPlan& plan, int nrhs, double* norm_partial,
                          const int* active, cudaStream_t st);

// out_r = [in_r] + alpha * sum_{i < m} R_i c_{r,i} for a complex64 basis R
// shared by all right-hand sides (m <= 1536); out complex128 (prec_out = F64,
// strides in complex128 entries) or complex64 (F32, strides in complex64
// entries); in may be nullptr or equal to out
cudaError_t launch_shared_combine(int prec_out, const void* R, long long vec_stride, int m, const void* coef,
                                  long long coef_stride, double alpha, const void* in, long long in_rhs_stride,
                                  void* out, long long out_rhs_stride, long long nunits, int nrhs, cudaStream_t st);
// inner products against a complex64 basis S shared by all right-hand sides,
// read once per call: partial[r][b][i] (row stride pstride) for the nblk
// chunks b, i < m; nblk from shared_dots_blocks (0: not applicable)
int shared_dots_blocks(int m, int nrhs, long long nunits, int num_sms, int max_blocks);
cudaError_t launch_shared_dots(const void* S, long long svec, int m, const void* Z, long long zstride, int nrhs,
                               long long nunits, int nblk, void* partial, int pstride, const int* active,
                               cudaStream_t st);
// sum partial[r][b][i] (row stride pstride) over b -> out[r*out_stride + i], i < J
cudaError_t launch_reduce(const void* partial, int nblk, int pstride, int J, int nrhs, void* out,
                          long long out_stride, bool accumulate, const int* active, cudaStream_t st);

// Arnoldi step j of CGS2 with delayed reorthogonalisation (see blas.cu).
cudaError_t launch_arnoldi_step(const void* red, long long red_stride, int j, void* H, long long h_rhs, int ldh,
                                double* beta0, double* inv_beta, void* dcoef, double* hnorm2, int* active,
                                int* k_used, int nrhs, cudaStream_t st);
// column j of H (the O(j^2) part of the step), after launch_arnoldi_step
cudaError_t launch_arnoldi_column(const void* red, long long red_stride, int j, void* H, long long h_rhs, int ldh,
                                  const double* inv_beta, const void* dcoef, const int* active, int nrhs,
                                  cudaStream_t st);
// v_j = (u - V s)/beta -> slot J; u <- (z - V t)/beta - v_j d
cudaError_t launch_arnoldi_update(int prec, void* basis, long long basis_rhs_stride, long long vec_stride, int J,
                                  const void* red, long long red_stride, const double* inv_beta, const void* dcoef,
                                  void* u, long long u_rhs_stride, const void* z, long long z_rhs_stride,
                                  long long nunits, const BlasPlan& plan, int nrhs, const int* active,
                                  cudaStream_t st);
// last column: H[:k][k-1] += s, H[k][k-1] = ||u - V s||
// red[r]: s at [0, k), u^H u at entry uu_at
cudaError_t launch_arnoldi_final(const void* red, long long red_stride, int k, int uu_at, void* H, long long h_rhs,
                                 int ldh, const int* active, int nrhs, cudaStream_t st);

// TMA-pipelined complex64 form of the Arnoldi update sweep (tma_sweeps.cu);
// *err receives OVS_ETIMEOUT if a bounded wait gives up.
bool tma_update_fits(int J);
// persistent TMA inner-product sweep (complex64, NW = 2): one block per SM
// over row chunks of 2048 units; partial[r][slot][2J + 2] for
// slot < gdots_chunk_slots(nunits, nrhs, num_sms)
bool gdots_chunk_fits(int J);
int gdots_chunk_slots(long long nunits, int nrhs, int num_sms);
cudaError_t launch_gdots2_chunk(const void* basis, long long basis_rhs_stride, long long vec_stride, int J,
                                const void* u, long long u_rhs_stride, const void* z, long long z_rhs_stride,
                                long long nunits, int nrhs, int num_sms, int nslot, void* partial, const int* active,
                                int* err, cudaStream_t st);
// y += alpha * sum_{i < min(J, Jdev[r])} V_i c_i: complex64 basis, complex128
// y (internal layout, updated in place, y_rhs_stride in complex128 entries)
bool recombine_tma_fits(int J);
cudaError_t launch_recombine_tma(const void* basis, long long basis_rhs_stride, long long vec_stride, int J,
                                 const int* Jdev, const void* coef, long long coef_stride, double alpha, void* y,
                                 long long y_rhs_stride, long long nunits, int nrhs, int num_sms, const int* active,
                                 int* err, cudaStream_t st);
// self-check: a bounded mbarrier wait that can never complete; *code gets
// the error word it left (OVS_ETIMEOUT when the bound works)
cudaError_t check_wait_timeout(cudaStream_t st, int* code);
cudaError_t launch_arnoldi_update_tma(void* basis, long long basis_rhs_stride, long long vec_stride, int J,
                                      const void* red, long long red_stride, const double* inv_beta,
                                      const void* dcoef, void* u, long long u_rhs_stride, const void* z,
                                      long long z_rhs_stride, long long nunits, int nrhs, int num_sms,
                                      const int* active, int* err, cudaStream_t st);

// c'_r,i = sgn(Re lambda_i) * c_r,i
cudaError_t launch_sign_scale(const void* c, const double* sgn, int m, int nrhs, void* out, cudaStream_t st);

// ---- K3 (newton.cu)
// coeff_r = beta_r * sgn(H_r[0:k,0:k]) e_1 with k = k_used[r], by Roberts'
// iteration in FP64. work: 2 * nrhs * kmax * kmax complex128.
// n_fixed > 0: use H[0:n_fixed, 0:n_fixed] instead of k_used[r]; right-hand
// sides with active[r] == 0 are skipped when active != nullptr.
cudaError_t launch_newton(const void* H, long long h_rhs_stride, int ldh, const int* k_used, const double* beta,
                          void* coeff, long long coeff_stride, void* work, int kmax, int nrhs, int* iters,
                          int* status, cudaStream_t st, const int* active = nullptr, int n_fixed = 0,
                          int k_bound = 0);
// harmonic variant: H_r[:, k-1] += |h_(k+1,k)|^2 H_k^-H e_k (k = k_used[r]);
// work as for launch_newton (used as scratch before it)
cudaError_t launch_harmonic(void* H, long long h_rhs_stride, int ldh, const int* k_used, void* work, int kmax,
                            int nrhs, cudaStream_t st);
// ---- Schur deflation (schur.cu)
// X[:, j] = (X[:, j] - X[:, <j] s) / beta_j, s = red[r][0..j)
cudaError_t launch_schur_xcol(void* X, long long x_rhs, int m, int j, const void* red, long long red_stride,
                              const double* inv_beta, const int* active, int nrhs, cudaStream_t st);
// cS_r = sgn(T) c_r + beta_r Y_r e_1, Y_r from T Y - Y H_k = sgn(T) X - X sgn(H_k)
bool schur_coeff_fits(int kmax);
long long schur_scratch_per_rhs(int m);
cudaError_t launch_schur_coeff(const void* T, const void* fT, int m, const void* X, long long x_rhs, const void* H,
                               long long h_rhs, int ldh, const void* fH, long long fh_rhs, const int* k_used,
                               const int* status, const double* beta, const void* c, long long c_stride,
                               void* scratch, void* cS, long long cs_stride, int nrhs, int kmax, cudaStream_t st);
// ---- outer GMRES of the overlap solve (solve.cu); canonical complex128
int norm_blocks();  // partials per right-hand side of the norm kernels
// norm[r] = ||v_r||, inv[r] = 1/norm[r] (inv may be nullptr); partial: nrhs x norm_blocks()
cudaError_t launch_norms(const void* v, long long n, long long stride, int nrhs, double* partial, double* norm,
                         double* inv, cudaStream_t st);
cudaError_t launch_norm_partials(const void* v, long long n, long long stride, int nrhs, double* partial,
                                 cudaStream_t st);
cudaError_t launch_scale(const void* in, long long in_stride, void* out, long long out_stride, const double* s,
                         long long n, int nrhs, cudaStream_t st);
cudaError_t launch_sub(const void* a, const void* b, void* out, long long n, int nrhs, cudaStream_t st);
cudaError_t launch_gmres_start(const double* beta, void* gv, int restart, int nrhs, cudaStream_t st);
cudaError_t launch_gmres_col(const void* red1, const void* red2, long long red_stride, const double* npart, int j,
                             int restart, void* R, void* rot, void* gv, double* est, double* inv_hn, int nrhs,
                             cudaStream_t st);
cudaError_t launch_gmres_backsub(const void* R, const void* gv, int jj, int restart, void* y, int nrhs,
                                 cudaStream_t st);
// A7 convergence checks: per right-hand side state of the check schedule
// (jl: j of the coefficients kept for comparison; (j0, e0), (j1, e1): the
// last two one-interval estimates; next: j of the next check)
struct CheckState {
    int jl, j0, j1, next;
    double e0, e1;
};
cudaError_t launch_check_init(CheckState* cs, int every, int nrhs, cudaStream_t st);
// after the last step: due[r] = 0 for a right-hand side stopped by a check
// (its coefficients, kept in cold, copied to coeff), else 1
cudaError_t launch_check_final(const CheckState* cs, const void* cold, void* coeff, long long stride,
                               const int* k_used, int* due, int nrhs, cudaStream_t st);
// due[r] = active[r] and cs[r].next == j
cudaError_t launch_check_due(const int* active, const CheckState* cs, int j, int* due, int nrhs, cudaStream_t st);
// for the due right-hand sides: the estimate ||cnew - cold|| / ||cnew|| over
// the first n entries, the stop (active = 0, k_used = n) below tol, else cold
// = cnew and the next check (skip: the skip-ahead schedule; cap: the last
// check j the schedule may aim at)
cudaError_t launch_conv_check(const void* cnew, void* cold, long long stride, int n, double tol, int* active,
                              int* k_used, double* est, const int* due, CheckState* cs, int every, int cap,
                              bool skip, int nrhs, cudaStream_t st);

}  // namespace ovs
