// Schur deflation (Sec. 5.2): set-up of the partial Schur form and the
// per-application kernels that the LR form does not have.
//
// Set-up (Sec. 5.2 steps i-ii): S_m, an orthonormal basis of the span of m
// right eigenvectors R_m in their order (two passes of Cholesky QR: G =
// S^H S = U^H U, S <- S U^-1, U upper triangular, so the leading columns of
// S span the leading eigenvectors), T_m = S_m^H H_w S_m (Eq. pSd; its
// strictly lower part, at the level of the eigenvectors' residual, is
// dropped) and sgn(T_m) by Roberts' iteration on the device (K3).
//
// Application (Sec. 5.2 steps iii-vi), built on the LR form's kernels:
//  - c = S^H x and x_perp = x - S c, twice (classical Gram-Schmidt applied
//    twice against S);
//  - modified Arnoldi (Eq. modArnoldi): after every matvec z = H_w u the
//    Schur directions are projected out of z, twice, and xz = S^H z is kept;
//    the Arnoldi sweeps over V then run on z as in the LR form. u is the
//    first-pass residual of the delayed-reorthogonalisation form, v_j =
//    (u - V_{<j} s) / beta_j, so column j of X = S^H H_w V_k follows as
//    X[:, j] = (xz - X[:, <j] s) / beta_j (k_schur_xcol);
//  - after K3 has formed the full sgn(H_k): C = sgn(T) X - X sgn(H_k), the
//    Sylvester equation T Y - Y H_k = C solved row by row from the bottom by
//    the recurrences of App. A (Eqs. SolveRow, xij, abij; the sums over H
//    end at row min(j+1, n), H being Hessenberg), and the Schur coefficients
//    sgn(T) c + beta Y e_1 (Eq. formula, k_schur_coeff);
//  - y = S (sgn(T) c + beta Y e_1) + V_k (beta sgn(H_k) e_1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <vector>

#include "common.cuh"
#include "handle.h"
#include "kernels.h"

namespace ovs {

// X[:, j] = (X[:, j] - X[:, <j] s) / beta_j per right-hand side; X is
// column-major m x kmax (x_rhs per right-hand side), s = red[r][0..j),
// 1/beta_j = inv_beta[r]. One warp per row, grid (rows / 8, nrhs).
__global__ void __launch_bounds__(256) k_schur_xcol(double2* __restrict__ X, long long x_rhs, int m, int j,
                                                    const double2* __restrict__ red, long long red_stride,
                                                    const double* __restrict__ inv_beta,
                                                    const int* __restrict__ active) {
    const int r = blockIdx.y, lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= m || active[r] == 0) return;
    double2* Xr = X + r * x_rhs;
    const double2* s = red + r * red_stride;
    double gr = 0.0, gi = 0.0;
    for (int l = lane; l < j; l += 32) {
        const double2 x = Xr[i + (long long)l * m], sl = s[l];
        gr += x.x * sl.x - x.y * sl.y;
        gi += x.x * sl.y + x.y * sl.x;
    }
    for (int off = 16; off > 0; off >>= 1) {
        gr += __shfl_xor_sync(0xffffffffu, gr, off);
        gi += __shfl_xor_sync(0xffffffffu, gi, off);
    }
    if (lane == 0) {
        const double ib = inv_beta[r];
        const double2 xz = Xr[i + (long long)j * m];
        Xr[i + (long long)j * m] = make_double2((xz.x - gr) * ib, (xz.y - gi) * ib);
    }
}

__device__ __forceinline__ void warp_dot2(const cd* a, const cd* b, const double2* h, int cnt, cd& sa, cd& sb) {
    const int lane = threadIdx.x & 31;
    double ar = 0.0, ai = 0.0, br = 0.0, bi = 0.0;
    for (int l = lane; l < cnt; l += 32) {
        const double2 hl = h[l];
        const cd al = a[l], bl = b[l];
        ar += al.re * hl.x - al.im * hl.y;
        ai += al.re * hl.y + al.im * hl.x;
        br += bl.re * hl.x - bl.im * hl.y;
        bi += bl.re * hl.y + bl.im * hl.x;
    }
    for (int off = 16; off > 0; off >>= 1) {
        ar += __shfl_xor_sync(0xffffffffu, ar, off);
        ai += __shfl_xor_sync(0xffffffffu, ai, off);
        br += __shfl_xor_sync(0xffffffffu, br, off);
        bi += __shfl_xor_sync(0xffffffffu, bi, off);
    }
    sa = {ar, ai};
    sb = {br, bi};
}

__device__ __forceinline__ cd cdiv(cd a, cd b) {
    const double den = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / den, (a.im * b.re - a.re * b.im) / den};
}

constexpr int kSylvMaxK = 800;

// Schur coefficients of one right-hand side per block (Sec. 5.2 steps v-vi,
// App. A): cS = sgn(T) c + beta Y e_1. T, fT = sgn(T): column-major m x m;
// X: column-major m x kmax; fH = sgn(H_k): row-major n x n (the K3 work
// space), n = k_used[r]; scratch: 2 m kmax complex128 per right-hand side
// (C, then Y, both row-major m x n). A right-hand side without Krylov part
// (n = 0) or whose sgn(H_k) failed (status OVS_ESIGN) gets cS = sgn(T) c.
__global__ void __launch_bounds__(256) k_schur_coeff(
    const double2* __restrict__ T, const double2* __restrict__ fT, int m, const double2* __restrict__ X,
    long long x_rhs, const double2* __restrict__ H, long long h_rhs, int ldh, const double2* __restrict__ fH,
    long long fh_rhs, const int* __restrict__ k_used, const int* __restrict__ status, const double* __restrict__ beta,
    const double2* __restrict__ c, long long c_stride, double2* __restrict__ scratch, long long scr_rhs,
    double2* __restrict__ cS, long long cs_stride) {
    __shared__ cd ct[kSylvMaxK], av[kSylvMaxK], bv[kSylvMaxK];
    __shared__ cd s_y1;
    const int r = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int n = k_used[r];
    const bool krylov = n > 0 && status[r] >= 0;
    const double2* cr = c + r * c_stride;
    const double2* Xr = X + r * x_rhs;
    const double2* Hr = H + r * h_rhs;
    const cd* F = reinterpret_cast<const cd*>(fH) + r * fh_rhs;
    cd* C = reinterpret_cast<cd*>(scratch) + r * scr_rhs;
    cd* Y = C + (size_t)m * kSylvMaxK;
    (void)Xr;
    (void)F;
    if (krylov) {
        // C = sgn(T) X - X sgn(H_k) was formed by k_schur_cmat
        for (int i = m - 1; i >= 0; --i) {
            // c~_ij = c_ij - sum_{l > i} T_il y_lj
            for (int j = tid; j < n; j += nt) {
                cd v = C[(size_t)i * n + j];
                for (int l = i + 1; l < m; ++l) {
                    const double2 t = T[i + (long long)l * m];
                    const cd y = Y[(size_t)l * n + j];
                    v.re -= t.x * y.re - t.y * y.im;
                    v.im -= t.x * y.im + t.y * y.re;
                }
                ct[j] = v;
            }
            __syncthreads();
            if (tid < 32) {
                const double2 tt = T[i + (long long)i * m];
                const cd tii = {tt.x, tt.y};
                if (tid == 0) {
                    av[0] = {1.0, 0.0};
                    bv[0] = {0.0, 0.0};
                }
                __syncwarp();
                for (int j = 0; j + 1 < n; ++j) {
                    cd sa, sb;
                    warp_dot2(av, bv, Hr + (long long)j * ldh, j + 1, sa, sb);
                    if (tid == 0) {
                        const double2 hs = Hr[j + 1 + (long long)j * ldh];
                        const cd hsub = {hs.x, hs.y};
                        const cd ta = cmul(tii, av[j]), tb = cmul(tii, bv[j]);
                        // a_{j+1} = -(-T_ii a_j + sum_l a_l H_lj) / H_{j+1,j}
                        // b_{j+1} = -(c~_ij - T_ii b_j + sum_l b_l H_lj) / H_{j+1,j}
                        av[j + 1] = cdiv(ta - sa, hsub);
                        bv[j + 1] = cdiv(tb - sb - ct[j], hsub);
                    }
                    __syncwarp();
                }
                cd sa, sb;
                warp_dot2(av, bv, Hr + (long long)(n - 1) * ldh, n, sa, sb);
                if (tid == 0) {
                    const cd num = ct[n - 1] - cmul(tii, bv[n - 1]) + sb;
                    const cd den = cmul(tii, av[n - 1]) - sa;
                    s_y1 = cdiv(num, den);
                }
            }
            __syncthreads();
            const cd y1 = s_y1;
            for (int j = tid; j < n; j += nt) Y[(size_t)i * n + j] = cmul(av[j], y1) + bv[j];
            __syncthreads();
        }
    }
    const double bt = krylov ? beta[r] : 0.0;
    for (int i = tid; i < m; i += nt) {
        double re = 0.0, im = 0.0;
        for (int l = i; l < m; ++l) {
            const double2 a = fT[i + (long long)l * m], b = cr[l];
            re += a.x * b.x - a.y * b.y;
            im += a.x * b.y + a.y * b.x;
        }
        if (krylov) {
            const cd y = Y[(size_t)i * n];
            re += bt * y.re;
            im += bt * y.im;
        }
        cS[r * cs_stride + i] = make_double2(re, im);
    }
}

cudaError_t launch_schur_xcol(void* X, long long x_rhs, int m, int j, const void* red, long long red_stride,
                              const double* inv_beta, const int* active, int nrhs, cudaStream_t st) {
    const dim3 grid((m + 7) / 8, nrhs);
    k_schur_xcol<<<grid, 256, 0, st>>>((double2*)X, x_rhs, m, j, (const double2*)red, red_stride, inv_beta, active);
    return cudaGetLastError();
}

bool schur_coeff_fits(int kmax) { return kmax <= kSylvMaxK; }
long long schur_scratch_per_rhs(int m) { return 2LL * m * kSylvMaxK; }

// C = sgn(T) X - X sgn(H_k) for every right-hand side (row-major m x n,
// n = k_used[r], at the start of its scratch): a tiled complex product, one
// 16 x 16 tile of C per block, the factors staged in shared memory 16 terms
// at a time. Grid (column tiles, row tiles, right-hand sides) over the
// largest n; tiles beyond a right-hand side's n do nothing.
constexpr int TC = 16;
__global__ void __launch_bounds__(TC * TC) k_schur_cmat(const double2* __restrict__ fT, int m,
                                                        const double2* __restrict__ X, long long x_rhs,
                                                        const double2* __restrict__ fH, long long fh_rhs,
                                                        const int* __restrict__ k_used,
                                                        const int* __restrict__ status,
                                                        double2* __restrict__ scratch, long long scr_rhs) {
    __shared__ double2 As[TC][TC + 1], Bs[TC][TC + 1];
    const int r = blockIdx.z;
    const int n = k_used[r];
    if (n <= 0 || status[r] < 0) return;  // uniform over the block
    const int i0 = blockIdx.y * TC, j0 = blockIdx.x * TC;
    if (i0 >= m || j0 >= n) return;       // uniform over the block
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = i0 + ty, j = j0 + tx;
    const double2* Xr = X + r * x_rhs;
    const double2* F = fH + r * fh_rhs;  // row-major n x n
    double re = 0.0, im = 0.0;
    // sgn(T) X: A[i][l] = fT[i + l m], B[l][j] = X[l + j m], l < m
    for (int k0 = 0; k0 < m; k0 += TC) {
        const int la = k0 + tx, lb = k0 + ty;
        As[ty][tx] = (i < m && la < m) ? fT[i + (long long)la * m] : make_double2(0.0, 0.0);
        Bs[ty][tx] = (lb < m && j < n) ? Xr[lb + (long long)j * m] : make_double2(0.0, 0.0);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < TC; ++q) {
            const double2 a = As[ty][q], b = Bs[q][tx];
            re = fma(a.x, b.x, re);
            re = fma(-a.y, b.y, re);
            im = fma(a.x, b.y, im);
            im = fma(a.y, b.x, im);
        }
        __syncthreads();
    }
    // - X sgn(H_k): A[i][l] = X[i + l m], B[l][j] = F[l n + j], l < n
    for (int k0 = 0; k0 < n; k0 += TC) {
        const int la = k0 + tx, lb = k0 + ty;
        As[ty][tx] = (i < m && la < n) ? Xr[i + (long long)la * m] : make_double2(0.0, 0.0);
        Bs[ty][tx] = (lb < n && j < n) ? F[(size_t)lb * n + j] : make_double2(0.0, 0.0);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < TC; ++q) {
            const double2 a = As[ty][q], b = Bs[q][tx];
            re = fma(-a.x, b.x, re);
            re = fma(a.y, b.y, re);
            im = fma(-a.x, b.y, im);
            im = fma(-a.y, b.x, im);
        }
        __syncthreads();
    }
    if (i < m && j < n) scratch[r * scr_rhs + (size_t)i * n + j] = make_double2(re, im);
}

cudaError_t launch_schur_coeff(const void* T, const void* fT, int m, const void* X, long long x_rhs, const void* H,
                               long long h_rhs, int ldh, const void* fH, long long fh_rhs, const int* k_used,
                               const int* status, const double* beta, const void* c, long long c_stride,
                               void* scratch, void* cS, long long cs_stride, int nrhs, int kmax, cudaStream_t st) {
    const dim3 grid((kmax + TC - 1) / TC, (m + TC - 1) / TC, nrhs);
    k_schur_cmat<<<grid, dim3(TC, TC), 0, st>>>((const double2*)fT, m, (const double2*)X, x_rhs, (const double2*)fH,
                                                fh_rhs, k_used, status, (double2*)scratch, schur_scratch_per_rhs(m));
    k_schur_coeff<<<nrhs, 256, 0, st>>>((const double2*)T, (const double2*)fT, m, (const double2*)X, x_rhs,
                                        (const double2*)H, h_rhs, ldh, (const double2*)fH, fh_rhs, k_used, status,
                                        beta, (const double2*)c, c_stride, (double2*)scratch,
                                        schur_scratch_per_rhs(m), (double2*)cS, cs_stride);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ set-up
namespace {

// Cholesky A = U^H U of a Hermitian positive definite m x m matrix (row-major
// a[i*m + j] = A_ij), then U^-1 (upper triangular), row-major.
bool chol_inv_upper(std::vector<std::complex<double>>& a, int m, std::vector<std::complex<double>>& uinv) {
    std::vector<std::complex<double>> u((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) {
        std::complex<double> d = a[(size_t)i * m + i];
        for (int k = 0; k < i; ++k) d -= std::conj(u[(size_t)k * m + i]) * u[(size_t)k * m + i];
        if (!(d.real() > 0.0)) return false;
        const double uii = std::sqrt(d.real());
        u[(size_t)i * m + i] = uii;
        for (int j = i + 1; j < m; ++j) {
            std::complex<double> v = a[(size_t)i * m + j];
            for (int k = 0; k < i; ++k) v -= std::conj(u[(size_t)k * m + i]) * u[(size_t)k * m + j];
            u[(size_t)i * m + j] = v / uii;
        }
    }
    uinv.assign((size_t)m * m, 0.0);
    for (int j = 0; j < m; ++j) {  // solve U w = e_j by back substitution
        for (int i = j; i >= 0; --i) {
            std::complex<double> v = (i == j) ? 1.0 : 0.0;
            for (int k = i + 1; k <= j; ++k) v -= u[(size_t)i * m + k] * uinv[(size_t)k * m + j];
            uinv[(size_t)i * m + j] = v / u[(size_t)i * m + i];
        }
    }
    return true;
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

}  // namespace

#define SCK(call)                                                                                            \
    do {                                                                                                     \
        cudaError_t e_ = (call);                                                                             \
        if (e_ != cudaSuccess) {                                                                             \
            char msg_[256];                                                                                  \
            snprintf(msg_, sizeof(msg_), "Schur set-up: %s: %s", #call, cudaGetErrorString(e_));            \
            cudaGetLastError();                                                                              \
            return lib_fail(e_ == cudaErrorMemoryAllocation ? OVS_ENOMEM : OVS_ECUDA, msg_);                 \
        }                                                                                                    \
    } while (0)

int install_schur(ovs_gauge_s* g, int m, const void* Rc) {
    cudaStream_t st = 0;
    free_deflation(g);
    if (m == 0) return OVS_OK;
    const long long N = g->N;
    const int V = (int)g->V;
    const size_t f64 = (size_t)N * 16;
    DevBuf a, b, G, part, Tdev, work, kused, beta, coeff, iters, status;
    SCK(cudaMalloc(&a.p, f64 * m));
    SCK(cudaMalloc(&b.p, f64 * m));
    SCK(cudaMalloc(&G.p, sizeof(double2) * (size_t)m * m));
    const BlasPlan plan = blas_plan(N, m, g->num_sms);
    const int S = gdots_stride(1, m);
    SCK(cudaMalloc(&part.p, sizeof(double2) * (size_t)plan.nblk * S * m));
    SCK(launch_to_internal(PREC_F64, Rc, N, a.p, f64, V, m, st));
    std::vector<std::complex<double>> gh((size_t)m * m), am((size_t)m * m), uinv, cf((size_t)m * m);
    // two passes of Cholesky QR: S <- S U^-1 with S^H S = U^H U
    for (int pass = 0; pass < 2; ++pass) {
        SCK(launch_gdots(PREC_F64, 1, a.p, 0, N, m, a.p, N, nullptr, 0, false, N, plan, m, part.p, nullptr, st));
        SCK(launch_reduce(part.p, plan.nblk, S, m, m, G.p, m, false, nullptr, st));
        SCK(cudaMemcpy(gh.data(), G.p, sizeof(double2) * (size_t)m * m, cudaMemcpyDeviceToHost));
        // gh[r*m + i] = S_i^H S_r = A_ir
        for (int r = 0; r < m; ++r)
            for (int i = 0; i < m; ++i) am[(size_t)i * m + r] = gh[(size_t)r * m + i];
        if (!chol_inv_upper(am, m, uinv))
            return lib_fail(OVS_EINVAL, "Schur set-up: the right vectors are linearly dependent");
        // new S_r = sum_i S_i (U^-1)_ir: coefficient [r][i]
        for (int r = 0; r < m; ++r)
            for (int i = 0; i < m; ++i) cf[(size_t)r * m + i] = uinv[(size_t)i * m + r];
        SCK(cudaMemcpy(G.p, cf.data(), sizeof(double2) * (size_t)m * m, cudaMemcpyHostToDevice));
        SCK(launch_update(PREC_F64, PREC_F64, a.p, 0, N, m, nullptr, G.p, m, 1.0, nullptr, 0, b.p, N, N, plan, m,
                          nullptr, nullptr, st));
        std::swap(a.p, b.p);
    }
    // T = S^H H_w S (column r = S^H H_w S_r), strictly lower part dropped
    const StencilShape sh = stencil_shape(g, PREC_F64, m, a.p, f64, b.p, f64, st);
    SCK(launch_wilson(PREC_F64, true, g->links64, a.p, f64, b.p, f64, g->geom, m, g->kappa, g->mu, nullptr, st, sh));
    SCK(launch_gdots(PREC_F64, 1, a.p, 0, N, m, b.p, N, nullptr, 0, false, N, plan, m, part.p, nullptr, st));
    SCK(launch_reduce(part.p, plan.nblk, S, m, m, G.p, m, false, nullptr, st));
    SCK(cudaMemcpy(gh.data(), G.p, sizeof(double2) * (size_t)m * m, cudaMemcpyDeviceToHost));
    std::vector<std::complex<double>> tcm((size_t)m * m, 0.0);  // column-major T
    std::vector<double> lam(2 * m);
    double lmax = 0.0;
    for (int r = 0; r < m; ++r)
        for (int i = 0; i <= r; ++i) tcm[i + (size_t)r * m] = gh[(size_t)r * m + i];
    for (int i = 0; i < m; ++i) {
        lam[2 * i] = tcm[i + (size_t)i * m].real();
        lam[2 * i + 1] = tcm[i + (size_t)i * m].imag();
        lmax = std::max(lmax, std::abs(tcm[i + (size_t)i * m]));
    }
    for (int i = 0; i < m; ++i)
        if (!(std::fabs(lam[2 * i]) > 1e-12 * lmax)) {
            char msg[160];
            snprintf(msg, sizeof(msg), "Schur set-up: eigenvalue %d has Re lambda = %g: sign undefined", i, lam[2 * i]);
            return lib_fail(OVS_ESIGN, msg);
        }
    // sgn(T) by Roberts' iteration (K3) on the device
    SCK(cudaMalloc(&Tdev.p, sizeof(double2) * (size_t)m * m));
    SCK(cudaMemcpy(Tdev.p, tcm.data(), sizeof(double2) * (size_t)m * m, cudaMemcpyHostToDevice));
    SCK(cudaMalloc(&work.p, sizeof(double2) * 2 * (size_t)m * m));
    SCK(cudaMalloc(&kused.p, sizeof(int)));
    SCK(cudaMalloc(&beta.p, sizeof(double)));
    SCK(cudaMalloc(&coeff.p, sizeof(double2) * m));
    SCK(cudaMalloc(&iters.p, sizeof(int)));
    SCK(cudaMalloc(&status.p, sizeof(int)));
    const double one = 1.0;
    SCK(cudaMemcpy(kused.p, &m, sizeof(int), cudaMemcpyHostToDevice));
    SCK(cudaMemcpy(beta.p, &one, sizeof(double), cudaMemcpyHostToDevice));
    SCK(launch_newton(Tdev.p, 0, m, (const int*)kused.p, (const double*)beta.p, coeff.p, 0, work.p, m, 1,
                      (int*)iters.p, (int*)status.p, st, nullptr, m));
    int nst = 0;
    SCK(cudaMemcpy(&nst, status.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (nst != OVS_OK) return lib_fail(OVS_ESIGN, "Schur set-up: Roberts' iteration on T_m did not converge");
    std::vector<std::complex<double>> srm((size_t)m * m), fcm((size_t)m * m);
    SCK(cudaMemcpy(srm.data(), work.p, sizeof(double2) * (size_t)m * m, cudaMemcpyDeviceToHost));
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) fcm[i + (size_t)j * m] = (i <= j) ? srm[(size_t)i * m + j] : 0.0;
    // install
    SCK(cudaMalloc(&g->schurT, sizeof(double2) * (size_t)m * m));
    SCK(cudaMalloc(&g->schurFT, sizeof(double2) * (size_t)m * m));
    SCK(cudaMemcpy(g->schurT, tcm.data(), sizeof(double2) * (size_t)m * m, cudaMemcpyHostToDevice));
    SCK(cudaMemcpy(g->schurFT, fcm.data(), sizeof(double2) * (size_t)m * m, cudaMemcpyHostToDevice));
    g->R64 = a.p;
    a.p = nullptr;
    if (g->prec == OVS_MIXED) {
        const size_t f32 = (size_t)N * 8;
        SCK(cudaMalloc(&g->R32, f32 * m));
        SCK(launch_to_canonical(PREC_F64, g->R64, f64, b.p, N, V, m, st));
        SCK(launch_to_internal(PREC_F32, b.p, N, g->R32, f32, V, m, st));
    }
    SCK(cudaDeviceSynchronize());
    g->m = m;
    g->scheme = DEFL_SCHUR;
    g->lambda = lam;
    return OVS_OK;
}

}  // namespace ovs
