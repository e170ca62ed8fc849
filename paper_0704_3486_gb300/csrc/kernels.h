// Host-side launchers of the library's kernels (internal interface).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace ovs {

struct Geom;

enum { PREC_F64 = 0, PREC_F32 = 1 };

// ---- K1 / K7 (dslash.cu)
cudaError_t launch_wilson(int prec, bool gamma5, const void* links, const void* in, size_t in_stride, void* out,
                          size_t out_stride, const Geom& g, int nrhs, double kappa, double mu, const int* active,
                          cudaStream_t st);
cudaError_t launch_to_internal(int prec, const void* canon, size_t canon_stride_cplx, void* out, size_t out_stride,
                               int V, int nrhs, cudaStream_t st);
cudaError_t launch_to_canonical(int prec, const void* in, size_t in_stride, void* canon, size_t canon_stride_cplx,
                                int V, int nrhs, cudaStream_t st);
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

// partial[r][b][i] = sum over block b of conj(V_r,i) . w_r, i < J
// (basis of rhs r at basis + r*basis_rhs_stride units, vector i at
// + i*vec_stride units).
cudaError_t launch_dots(int prec, const void* basis, long long basis_rhs_stride, long long vec_stride, int J,
                        const void* w, long long w_rhs_stride, long long nunits, const BlasPlan& plan, int nrhs,
                        void* partial, const int* active, cudaStream_t st);

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

// sum partial[r][b][i] over b -> out[r*out_stride + i] (= or +=)
cudaError_t launch_reduce(const void* partial, int nblk, int J, int nrhs, void* out, long long out_stride,
                          bool accumulate, const int* active, cudaStream_t st);

// After the second Gram-Schmidt update of Arnoldi step j (0-based): beta =
// sqrt(sum norm_partial), H[j+1][j] = beta (H column-major, leading dim ldh),
// breakdown test, inv_beta, k_used, active.
cudaError_t launch_finalize(const double* norm_partial, int nblk, int nrhs, void* H, long long h_rhs_stride,
                            int ldh, int j, double* hnorm2, double* inv_beta, int* active, int* k_used,
                            cudaStream_t st);

// Start of Arnoldi: beta0 = sqrt(sum norm_partial); inv_beta; active = beta0 > 0.
cudaError_t launch_init_beta(const double* norm_partial, int nblk, int nrhs, double* beta, double* inv_beta,
                             double* hnorm2, int* active, int* k_used, cudaStream_t st);

// out_r = in_r * inv_beta[r] (units of precision prec)
cudaError_t launch_scale(int prec, const void* in, long long in_rhs_stride, void* out, long long out_rhs_stride,
                         long long nunits, const double* inv_beta, int nrhs, const int* active, cudaStream_t st);

// c'_r,i = sgn(Re lambda_i) * c_r,i
cudaError_t launch_sign_scale(const void* c, const double* sgn, int m, int nrhs, void* out, cudaStream_t st);

// ---- K3 (newton.cu)
// coeff_r = beta_r * sgn(H_r[0:k,0:k]) e_1 with k = k_used[r], by Roberts'
// iteration in FP64. work: 2 * nrhs * kmax * kmax complex128.
cudaError_t launch_newton(const void* H, long long h_rhs_stride, int ldh, const int* k_used, const double* beta,
                          void* coeff, long long coeff_stride, void* work, int kmax, int nrhs, int* iters,
                          int* status, cudaStream_t st);

}  // namespace ovs
