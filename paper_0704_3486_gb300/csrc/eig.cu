// K6: critical eigenpairs of H_w(mu) for LR deflation (Sec. 5.3 step i;
// Sec. 6) -- the set-up, done once per operator and timed separately.
//
// The paper finds the eigenvalues of smallest magnitude of H_w through
// H_w^2, whose smallest eigenvalues lie on the edge of the spectrum (Sec. 6).
// Here a block of p > m vectors is driven towards them by Chebyshev-filtered
// subspace iteration on H_w^2:
//   1. filter:   Q <- T_d(H^2) Q, the scaled three-term Chebyshev
//                recurrence that damps [a, b] (b >= spectral radius of H^2,
//                a = the largest Ritz value of H^2 in the block), fused into
//                the stencil's epilogue; complex64 while the residuals are
//                far above FP32 rounding, complex128 afterwards;
//   2. orthonormalise Q twice by SVQB (Gram matrix Q^H Q, Hermitian
//      eigen-decomposition, Q <- Q U Lambda^-1/2);
//   3. Rayleigh-Ritz with H_w itself: G = Q^H H Q, G Y = Y Theta, Ritz
//      vectors X = Q Y and residuals ||H x - theta x|| (complex128);
//   4. stop when the m Ritz pairs of smallest |theta| have relative residual
//      <= tol; otherwise Q <- X and pick the next degree d so that the
//      filter gains a factor ~1e3 between the m-th Ritz value and the cut.
// Left eigenvectors are right eigenvectors of H_w(mu)^+ = H_w(-mu)
// (gamma5-hermiticity) with eigenvalues conj(lambda): the same iteration at
// -mu, matched to the right pairs by eigenvalue. Of the converged pairs the m
// with smallest |Re lambda| are installed (L biorthonormalised against R).
// Dense algebra of the set-up (block Gram matrices, Ritz vectors, the small
// Hermitian and non-Hermitian eigenproblems) uses cuBLAS and cuSOLVER.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "handle.h"
#include "kernels.h"

namespace ovs {

// ||Z_i - theta_i X_i|| for each column i (one block per column)
__global__ void k_ritz_resid(const double2* __restrict__ Z, const double2* __restrict__ X,
                             const double2* __restrict__ theta, long long N, double* __restrict__ out) {
    __shared__ double sh[32];
    const int i = blockIdx.x;
    const double2 t = theta[i];
    const double2* z = Z + (size_t)i * N;
    const double2* x = X + (size_t)i * N;
    double s = 0.0;
    for (long long n = threadIdx.x; n < N; n += blockDim.x) {
        const double2 a = z[n], b = x[n];
        const double rx = a.x - (t.x * b.x - t.y * b.y);
        const double ry = a.y - (t.x * b.y + t.y * b.x);
        s += rx * rx + ry * ry;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w];
        out[i] = sqrt(tot);
    }
}

// the same for complex64 blocks, accumulated in FP64
__global__ void k_ritz_resid32(const float2* __restrict__ Z, const float2* __restrict__ X,
                               const double2* __restrict__ theta, long long N, double* __restrict__ out) {
    __shared__ double sh[32];
    const int i = blockIdx.x;
    const double2 t = theta[i];
    const float2* z = Z + (size_t)i * N;
    const float2* x = X + (size_t)i * N;
    double s = 0.0;
    for (long long n = threadIdx.x; n < N; n += blockDim.x) {
        const float2 a = z[n], b = x[n];
        const double rx = (double)a.x - (t.x * b.x - t.y * b.y);
        const double ry = (double)a.y - (t.x * b.y + t.y * b.x);
        s += rx * rx + ry * ry;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w];
        out[i] = sqrt(tot);
    }
}

// Per column i of Q (complex128): Rayleigh quotient theta_i = q^H w / q^H q
// and residual ||w - theta_i q|| / ||q|| with W = H Q (one block per column).
__global__ void k_rq_resid(const double2* __restrict__ W, const double2* __restrict__ Q, long long N,
                           double2* __restrict__ theta, double* __restrict__ out) {
    __shared__ double sh[4][32];
    __shared__ double2 s_t;
    const int i = blockIdx.x;
    const double2* w = W + (size_t)i * N;
    const double2* q = Q + (size_t)i * N;
    double ar = 0.0, ai = 0.0, qq = 0.0;
    for (long long n = threadIdx.x; n < N; n += blockDim.x) {
        const double2 a = q[n], b = w[n];
        ar += a.x * b.x + a.y * b.y;
        ai += a.x * b.y - a.y * b.x;
        qq += a.x * a.x + a.y * a.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        ar += __shfl_xor_sync(0xffffffffu, ar, o);
        ai += __shfl_xor_sync(0xffffffffu, ai, o);
        qq += __shfl_xor_sync(0xffffffffu, qq, o);
    }
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    if (lane == 0) { sh[0][wp] = ar; sh[1][wp] = ai; sh[2][wp] = qq; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tr = 0.0, ti = 0.0, tq = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { tr += sh[0][k]; ti += sh[1][k]; tq += sh[2][k]; }
        s_t = tq > 0.0 ? make_double2(tr / tq, ti / tq) : make_double2(0.0, 0.0);
        sh[3][0] = tq;
        theta[i] = s_t;
    }
    __syncthreads();
    const double2 t = s_t;
    double s = 0.0;
    for (long long n = threadIdx.x; n < N; n += blockDim.x) {
        const double2 a = q[n], b = w[n];
        const double rx = b.x - (t.x * a.x - t.y * a.y);
        const double ry = b.y - (t.x * a.y + t.y * a.x);
        s += rx * rx + ry * ry;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __syncthreads();
    if (lane == 0) sh[0][wp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tot += sh[0][k];
        out[i] = sh[3][0] > 0.0 ? sqrt(tot / sh[3][0]) : 0.0;
    }
}

// U[:, j] *= 1/sqrt(max(lam_j, floor)) (column-major p x p)
__global__ void k_scale_cols(double2* __restrict__ U, const double* __restrict__ lam, int p, double floor_) {
    const int j = blockIdx.x;
    const double l = lam[j] > floor_ ? lam[j] : floor_;
    const double s = 1.0 / sqrt(l);
    for (int i = threadIdx.x; i < p; i += blockDim.x) {
        double2 v = U[(size_t)j * p + i];
        U[(size_t)j * p + i] = make_double2(v.x * s, v.y * s);
    }
}

namespace {

struct Ctx {
    ovs_gauge_s* g = nullptr;
    cudaStream_t st = 0;
    cublasHandle_t cb = nullptr;
    cusolverDnHandle_t cs = nullptr;
    cusolverDnParams_t params = nullptr;
    long long N = 0;
    int p = 0;
    double2 *Q = nullptr, *W = nullptr, *A1 = nullptr, *A2 = nullptr;  // [p][N] complex128
    void* F[3] = {nullptr, nullptr, nullptr};                            // [p][N] complex64 filter buffers
    double2 *G = nullptr, *G2 = nullptr, *Y = nullptr, *theta = nullptr;
    float2 *G32 = nullptr, *Y32 = nullptr;  // p x p complex64 copies for the complex64 block algebra
    double* lam = nullptr;
    double* resid = nullptr;
    int* info = nullptr;
    void* dwork = nullptr;
    size_t dwork_bytes = 0;
    std::vector<char> hwork;
    char err[256] = {0};
    ~Ctx() {
        for (void* q : {(void*)Q, (void*)W, (void*)A1, (void*)A2, F[0], F[1], F[2], (void*)G, (void*)G2, (void*)Y,
                        (void*)theta, (void*)lam, (void*)resid, (void*)info, dwork, (void*)G32, (void*)Y32})
            if (q) cudaFree(q);
        if (params) cusolverDnDestroyParams(params);
        if (cs) cusolverDnDestroy(cs);
        if (cb) cublasDestroy(cb);
    }
};

#define ECK(call)                                                                        \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            snprintf(c.err, sizeof(c.err), "%s: %s", #call, cudaGetErrorString(e_));     \
            cudaGetLastError(); /* clear a non-sticky error for later launches */       \
            return e_ == cudaErrorMemoryAllocation ? OVS_ENOMEM : OVS_ECUDA;             \
        }                                                                                \
    } while (0)
#define BCK(call)                                                                        \
    do {                                                                                 \
        int s_ = (int)(call);                                                            \
        if (s_ != 0) {                                                                   \
            snprintf(c.err, sizeof(c.err), "%s failed with status %d", #call, s_);       \
            return OVS_ECUDA;                                                            \
        }                                                                                \
    } while (0)

const cuDoubleComplex kOne = {1.0, 0.0}, kZero = {0.0, 0.0};

// out = H_w(mu) in for the p vectors of a block
int apply_h(Ctx& c, int prec, const void* in, void* out, double mu) {
    ovs_gauge_s* g = c.g;
    const size_t fb = (size_t)c.N * (prec == PREC_F64 ? 16 : 8);
    const void* L = prec == PREC_F64 ? g->links64 : g->links32;
    const StencilShape sh = stencil_shape(g, prec, c.p, in, fb, out, fb, c.st);
    ECK(launch_wilson(prec, true, L, in, fb, out, fb, g->geom, c.p, g->kappa, mu, nullptr, c.st, sh));
    return OVS_OK;
}

// Scaled Chebyshev filter of degree deg in H^2: T_deg((z - cc)/e) normalised
// to 1 at z = 0, which damps the ellipses with foci cc +/- e. Buffers b0
// (input), b1, bt of precision prec; *out_idx receives the buffer index
// holding the result.
int cheb_filter(Ctx& c, int prec, void* bufs[3], int deg, double cc, double e, double mu, int* out_idx) {
    ovs_gauge_s* g = c.g;
    const size_t fb = (size_t)c.N * (prec == PREC_F64 ? 16 : 8);
    const void* L = prec == PREC_F64 ? g->links64 : g->links32;
    const double sigma1 = e / (0.0 - cc);
    double sigma = sigma1;
    void* prev = bufs[0];
    void* cur = bufs[1];
    void* tmp = bufs[2];
    const StencilShape sh = stencil_shape(g, prec, c.p, prev, fb, tmp, fb, c.st);
    // Y1 = (sigma1/e) (H^2 - c) Y0
    {
        int rc = apply_h(c, prec, prev, tmp, mu);
        if (rc) return rc;
        ECK(launch_wilson_axpy(prec, L, tmp, fb, cur, fb, prev, fb, -sigma1 * cc / e, prev, fb, 0.0, sigma1 / e,
                               g->geom, c.p, g->kappa, mu, c.st, sh));
    }
    for (int k = 1; k < deg; ++k) {
        const double sn = 1.0 / (2.0 / sigma1 - sigma);
        int rc = apply_h(c, prec, cur, tmp, mu);
        if (rc) return rc;
        // Y_{k+1} = (2 sn/e)(H^2 - c) Y_k - sigma sn Y_{k-1}, written over Y_{k-1}
        ECK(launch_wilson_axpy(prec, L, tmp, fb, prev, fb, cur, fb, -2.0 * sn * cc / e, prev, fb, -sigma * sn,
                               2.0 * sn / e, g->geom, c.p, g->kappa, mu, c.st, sh));
        std::swap(prev, cur);
        sigma = sn;
    }
    *out_idx = (cur == bufs[0]) ? 0 : (cur == bufs[1] ? 1 : 2);
    return OVS_OK;
}

// Q <- Q U diag(lam)^-1/2 with G = Q^H Q = U diag(lam) U^H (twice)
int svqb(Ctx& c) {
    const int p = c.p;
    const long long N = c.N;
    for (int pass = 0; pass < 2; ++pass) {
        BCK(cublasZgemm(c.cb, CUBLAS_OP_C, CUBLAS_OP_N, p, p, (int)N, &kOne, (const cuDoubleComplex*)c.Q, (int)N,
                        (const cuDoubleComplex*)c.Q, (int)N, &kZero, (cuDoubleComplex*)c.G, p));
        int lwork = 0;
        BCK(cusolverDnZheevd_bufferSize(c.cs, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, p,
                                        (cuDoubleComplex*)c.G, p, c.lam, &lwork));
        if ((size_t)lwork * 16 > c.dwork_bytes) {
            if (c.dwork) cudaFree(c.dwork);
            c.dwork_bytes = (size_t)lwork * 16;
            ECK(cudaMalloc(&c.dwork, c.dwork_bytes));
        }
        BCK(cusolverDnZheevd(c.cs, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, p, (cuDoubleComplex*)c.G, p,
                             c.lam, (cuDoubleComplex*)c.dwork, lwork, c.info));
        std::vector<double> lam(p);
        ECK(cudaMemcpyAsync(lam.data(), c.lam, sizeof(double) * p, cudaMemcpyDeviceToHost, c.st));
        ECK(cudaStreamSynchronize(c.st));
        const double floor_ = std::max(lam[p - 1], 1e-300) * 1e-28;
        k_scale_cols<<<p, 128, 0, c.st>>>(c.G, c.lam, p, floor_);
        ECK(cudaGetLastError());
        BCK(cublasZgemm(c.cb, CUBLAS_OP_N, CUBLAS_OP_N, (int)N, p, p, &kOne, (const cuDoubleComplex*)c.Q, (int)N,
                        (const cuDoubleComplex*)c.G, p, &kZero, (cuDoubleComplex*)c.A1, (int)N));
        std::swap(c.Q, c.A1);
    }
    return OVS_OK;
}

// Rayleigh-Ritz of H_w(mu) on span(Q): Ritz values theta (host), Ritz
// vectors in A1 (unit norm), residual norms (host).
int rayleigh_ritz(Ctx& c, double mu, std::vector<std::complex<double>>& theta, std::vector<double>& resid) {
    const int p = c.p;
    const long long N = c.N;
    int rc = apply_h(c, PREC_F64, c.Q, c.W, mu);
    if (rc) return rc;
    BCK(cublasZgemm(c.cb, CUBLAS_OP_C, CUBLAS_OP_N, p, p, (int)N, &kOne, (const cuDoubleComplex*)c.Q, (int)N,
                    (const cuDoubleComplex*)c.W, (int)N, &kZero, (cuDoubleComplex*)c.G, p));
    size_t dbytes = 0, hbytes = 0;
    BCK(cusolverDnXgeev_bufferSize(c.cs, c.params, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_VECTOR, p,
                                   CUDA_C_64F, c.G, p, CUDA_C_64F, c.theta, CUDA_C_64F, nullptr, p, CUDA_C_64F, c.Y,
                                   p, CUDA_C_64F, &dbytes, &hbytes));
    if (dbytes > c.dwork_bytes) {
        if (c.dwork) cudaFree(c.dwork);
        c.dwork_bytes = dbytes;
        ECK(cudaMalloc(&c.dwork, c.dwork_bytes));
    }
    if (hbytes > c.hwork.size()) c.hwork.resize(hbytes);
    BCK(cusolverDnXgeev(c.cs, c.params, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_VECTOR, p, CUDA_C_64F, c.G, p,
                        CUDA_C_64F, c.theta, CUDA_C_64F, nullptr, p, CUDA_C_64F, c.Y, p, CUDA_C_64F, c.dwork,
                        c.dwork_bytes, c.hwork.empty() ? nullptr : c.hwork.data(), c.hwork.size(), c.info));
    int info = 0;
    ECK(cudaMemcpyAsync(&info, c.info, sizeof(int), cudaMemcpyDeviceToHost, c.st));
    // X = Q Y, Z = W Y
    BCK(cublasZgemm(c.cb, CUBLAS_OP_N, CUBLAS_OP_N, (int)N, p, p, &kOne, (const cuDoubleComplex*)c.Q, (int)N,
                    (const cuDoubleComplex*)c.Y, p, &kZero, (cuDoubleComplex*)c.A1, (int)N));
    BCK(cublasZgemm(c.cb, CUBLAS_OP_N, CUBLAS_OP_N, (int)N, p, p, &kOne, (const cuDoubleComplex*)c.W, (int)N,
                    (const cuDoubleComplex*)c.Y, p, &kZero, (cuDoubleComplex*)c.A2, (int)N));
    k_ritz_resid<<<p, 256, 0, c.st>>>(c.A2, c.A1, c.theta, N, c.resid);
    ECK(cudaGetLastError());
    theta.resize(p);
    resid.resize(p);
    ECK(cudaMemcpyAsync(theta.data(), c.theta, sizeof(double2) * p, cudaMemcpyDeviceToHost, c.st));
    ECK(cudaMemcpyAsync(resid.data(), c.resid, sizeof(double) * p, cudaMemcpyDeviceToHost, c.st));
    ECK(cudaStreamSynchronize(c.st));
    if (info != 0) {
        snprintf(c.err, sizeof(c.err), "geev info = %d", info);
        return OVS_EEIG;
    }
    return OVS_OK;
}

const cuComplex kOneF = {1.0f, 0.0f}, kZeroF = {0.0f, 0.0f};

// SVQB of a complex64 block, twice: G = Q^H Q by CGEMM, its eigen-
// decomposition in complex128, Q <- Q U diag(lam)^-1/2 by CGEMM. Q and tmp
// are swapped as needed; on return Q points at the orthonormal block.
int svqb32(Ctx& c, void*& Q, void*& tmp) {
    const int p = c.p;
    const long long N = c.N;
    for (int pass = 0; pass < 2; ++pass) {
        BCK(cublasCgemm(c.cb, CUBLAS_OP_C, CUBLAS_OP_N, p, p, (int)N, &kOneF, (const cuComplex*)Q, (int)N,
                        (const cuComplex*)Q, (int)N, &kZeroF, (cuComplex*)c.G32, p));
        ECK(launch_convert(PREC_F64, c.G32, c.G, (long long)p * p, c.st));
        int lwork = 0;
        BCK(cusolverDnZheevd_bufferSize(c.cs, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, p,
                                        (cuDoubleComplex*)c.G, p, c.lam, &lwork));
        if ((size_t)lwork * 16 > c.dwork_bytes) {
            if (c.dwork) cudaFree(c.dwork);
            c.dwork_bytes = (size_t)lwork * 16;
            ECK(cudaMalloc(&c.dwork, c.dwork_bytes));
        }
        BCK(cusolverDnZheevd(c.cs, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, p, (cuDoubleComplex*)c.G, p,
                             c.lam, (cuDoubleComplex*)c.dwork, lwork, c.info));
        std::vector<double> lam(p);
        ECK(cudaMemcpyAsync(lam.data(), c.lam, sizeof(double) * p, cudaMemcpyDeviceToHost, c.st));
        ECK(cudaStreamSynchronize(c.st));
        const double floor_ = std::max(lam[p - 1], 1e-300) * 1e-12;
        k_scale_cols<<<p, 128, 0, c.st>>>(c.G, c.lam, p, floor_);
        ECK(cudaGetLastError());
        ECK(launch_convert(PREC_F32, c.G, c.G32, (long long)p * p, c.st));
        BCK(cublasCgemm(c.cb, CUBLAS_OP_N, CUBLAS_OP_N, (int)N, p, p, &kOneF, (const cuComplex*)Q, (int)N,
                        (const cuComplex*)c.G32, p, &kZeroF, (cuComplex*)tmp, (int)N));
        std::swap(Q, tmp);
    }
    return OVS_OK;
}

// Rayleigh-Ritz of H_w(mu) on the complex64 orthonormal block Q: Z = H Q
// (complex64 stencil), G = Q^H Z (CGEMM), the p x p eigenproblem in
// complex128, Ritz vectors X = Q Y and Z Y (CGEMM), residual norms
// ||Z y - theta Q y|| summed in FP64. Buffers Z, X, ZX: p x N complex64.
int rayleigh_ritz32(Ctx& c, double mu, void* Q, void* Z, void* X, void* ZX,
                    std::vector<std::complex<double>>& theta, std::vector<double>& resid) {
    const int p = c.p;
    const long long N = c.N;
    int rc = apply_h(c, PREC_F32, Q, Z, mu);
    if (rc) return rc;
    BCK(cublasCgemm(c.cb, CUBLAS_OP_C, CUBLAS_OP_N, p, p, (int)N, &kOneF, (const cuComplex*)Q, (int)N,
                    (const cuComplex*)Z, (int)N, &kZeroF, (cuComplex*)c.G32, p));
    ECK(launch_convert(PREC_F64, c.G32, c.G, (long long)p * p, c.st));
    size_t dbytes = 0, hbytes = 0;
    BCK(cusolverDnXgeev_bufferSize(c.cs, c.params, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_VECTOR, p,
                                   CUDA_C_64F, c.G, p, CUDA_C_64F, c.theta, CUDA_C_64F, nullptr, p, CUDA_C_64F, c.Y,
                                   p, CUDA_C_64F, &dbytes, &hbytes));
    if (dbytes > c.dwork_bytes) {
        if (c.dwork) cudaFree(c.dwork);
        c.dwork_bytes = dbytes;
        ECK(cudaMalloc(&c.dwork, c.dwork_bytes));
    }
    if (hbytes > c.hwork.size()) c.hwork.resize(hbytes);
    BCK(cusolverDnXgeev(c.cs, c.params, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_VECTOR, p, CUDA_C_64F, c.G, p,
                        CUDA_C_64F, c.theta, CUDA_C_64F, nullptr, p, CUDA_C_64F, c.Y, p, CUDA_C_64F, c.dwork,
                        c.dwork_bytes, c.hwork.empty() ? nullptr : c.hwork.data(), c.hwork.size(), c.info));
    int info = 0;
    ECK(cudaMemcpyAsync(&info, c.info, sizeof(int), cudaMemcpyDeviceToHost, c.st));
    ECK(launch_convert(PREC_F32, c.Y, c.Y32, (long long)p * p, c.st));
    BCK(cublasCgemm(c.cb, CUBLAS_OP_N, CUBLAS_OP_N, (int)N, p, p, &kOneF, (const cuComplex*)Q, (int)N,
                    (const cuComplex*)c.Y32, p, &kZeroF, (cuComplex*)X, (int)N));
    BCK(cublasCgemm(c.cb, CUBLAS_OP_N, CUBLAS_OP_N, (int)N, p, p, &kOneF, (const cuComplex*)Z, (int)N,
                    (const cuComplex*)c.Y32, p, &kZeroF, (cuComplex*)ZX, (int)N));
    k_ritz_resid32<<<p, 256, 0, c.st>>>((const float2*)ZX, (const float2*)X, c.theta, N, c.resid);
    ECK(cudaGetLastError());
    theta.resize(p);
    resid.resize(p);
    ECK(cudaMemcpyAsync(theta.data(), c.theta, sizeof(double2) * p, cudaMemcpyDeviceToHost, c.st));
    ECK(cudaMemcpyAsync(resid.data(), c.resid, sizeof(double) * p, cudaMemcpyDeviceToHost, c.st));
    ECK(cudaStreamSynchronize(c.st));
    if (info != 0) {
        snprintf(c.err, sizeof(c.err), "geev info = %d", info);
        return OVS_EEIG;
    }
    return OVS_OK;
}

// Complex128 residuals of the Ritz pairs in Q (complex128, the vectors of a
// complex64 Rayleigh-Ritz): W = H Q in complex128, then per vector its
// Rayleigh quotient and residual (k_rq_resid). No block algebra: each pair
// is certified on its own, at the cost of one complex128 stencil.
int pair_residuals64(Ctx& c, double mu, std::vector<std::complex<double>>& theta, std::vector<double>& resid) {
    const int p = c.p;
    const long long N = c.N;
    int rc = apply_h(c, PREC_F64, c.Q, c.W, mu);
    if (rc) return rc;
    k_rq_resid<<<p, 256, 0, c.st>>>(c.W, c.Q, N, c.theta, c.resid);
    ECK(cudaGetLastError());
    theta.resize(p);
    resid.resize(p);
    ECK(cudaMemcpyAsync(theta.data(), c.theta, sizeof(double2) * p, cudaMemcpyDeviceToHost, c.st));
    ECK(cudaMemcpyAsync(resid.data(), c.resid, sizeof(double) * p, cudaMemcpyDeviceToHost, c.st));
    ECK(cudaStreamSynchronize(c.st));
    return OVS_OK;
}

struct SideResult {
    std::vector<std::complex<double>> theta;
    std::vector<double> resid;
    double* X = nullptr;  // device [p][N] complex128 (owned by caller after return)
    int iters = 0;
    long long matvecs = 0;
    bool converged = false;
};

// Spectral radius bound of H^2 from a short power iteration on one vector.
int spectral_bound(Ctx& c, double mu, double* b_out) {
    const long long N = c.N;
    ovs_gauge_s* g = c.g;
    const size_t fb = (size_t)N * 16;
    double2* v = c.A1;
    double2* w = c.A2;
    ECK(launch_random_fill(v, N, 977, c.st));
    double rho = 0.0;
    for (int it = 0; it < 40; ++it) {
        ECK(launch_wilson(PREC_F64, true, g->links64, v, fb, w, fb, g->geom, 1, g->kappa, mu, nullptr, c.st));
        ECK(launch_wilson(PREC_F64, true, g->links64, w, fb, v, fb, g->geom, 1, g->kappa, mu, nullptr, c.st));
        double nv = 0.0;
        BCK(cublasDznrm2(c.cb, (int)N, (const cuDoubleComplex*)v, 1, &nv));
        ECK(cudaStreamSynchronize(c.st));
        if (!(nv > 0.0)) break;
        const double inv = 1.0 / nv;
        BCK(cublasZdscal(c.cb, (int)N, &inv, (cuDoubleComplex*)v, 1));
        rho = nv;  // ||H^2 v|| with ||v|| = 1 from the previous step
    }
    *b_out = 1.15 * rho;
    return OVS_OK;
}

// Chebyshev filter for the non-Hermitian H^2. The eigenvalues z = lambda^2
// of H_w(mu) lie near the positive real axis: |Im lambda| <= eta with
// eta = ||(H - H^+)/2|| <= 4 kappa sinh|mu| (H - H^+ = H(mu) - H(-mu) has
// only temporal hops, 2 kappa |e^mu - e^-mu| each, through a rank-2
// projector), so |Im z| <= Y(x) = 2 eta sqrt(x + eta^2) at Re z = x. Near
// the cut the bound is replaced by 1.5 x the largest |Im theta| of the
// block's Ritz values (the small eigenvalues of the bow-tie are far closer
// to the real axis than the bound), growing linearly to the bound at the
// top of the spectrum. The
// unwanted part {a <= Re z <= b, |Im z| <= Y} is enclosed in an ellipse
// with left vertex aE = (lm + a)/2, right vertex 1.5 b and semi-axis B
// high enough to contain the region; the filter is the Chebyshev polynomial
// for the foci of that ellipse. Its per-degree gain at the wanted Ritz value
// lm over the ellipse fixes the degree (gain 1e3 per application).
struct FilterPlan {
    double c, e;
    int deg;
};

// lmin: the smallest |theta|^2 of the block; range: the largest ratio of
// the filter's gains at lmin and at lm that the working precision keeps
// (the filter damps a wanted vector relative to the smallest one by that
// ratio; beyond the precision's range the wanted vector is lost to
// rounding); dmax: a cap on the degree.
FilterPlan plan_filter(double b, double lm, double a, double kappa, double mu, double eta_near, double lmin,
                       double range, int dmax) {
    const double eta_glob = 4.0 * kappa * std::sinh(std::fabs(mu));
    eta_near = std::min(eta_near, eta_glob);
    const double aE = 0.5 * (lm + a);
    const double bE = 1.5 * b;
    const double A = 0.5 * (bE - aE), cc = 0.5 * (bE + aE);
    double B = 0.0;
    for (int i = 0; i <= 400; ++i) {
        // sample Re z on [a, b], densely near a
        const double t = i / 400.0;
        const double x = a + (b - a) * t * t;
        // near the cut the Ritz values show the imaginary parts; towards the
        // top of the spectrum the rigorous bound takes over linearly
        const double eta = eta_near + (eta_glob - eta_near) * std::min(1.0, x / b);
        const double y = 2.0 * eta * std::sqrt(x + eta * eta);
        const double q = (x - cc) / A;
        const double room = 1.0 - q * q;
        if (room > 1e-14) B = std::max(B, y / std::sqrt(room));
    }
    B = std::min(B, 0.95 * A);
    FilterPlan fp;
    fp.c = cc;
    fp.e = std::sqrt(A * A - B * B);
    const double rho_ell = (A + B) / fp.e;
    const double w = (cc - lm) / fp.e;
    const double rho_w = w > 1.0 ? w + std::sqrt(w * w - 1.0) : 1.0;
    const double gain = rho_w / rho_ell;
    double d = gain > 1.0 + 1e-9 ? std::log(1e3) / std::log(gain) : (double)dmax;
    const double w0 = (cc - lmin) / fp.e;
    const double rho_0 = w0 > 1.0 ? w0 + std::sqrt(w0 * w0 - 1.0) : 1.0;
    if (rho_0 > rho_w * (1.0 + 1e-12)) d = std::min(d, std::log(range) / std::log(rho_0 / rho_w));
    fp.deg = (int)std::min(std::max(d, 16.0), (double)dmax);
    return fp;
}

// OVS_SETUP_LOG=1 in the environment prints one line per iteration of the
// set-up to stderr (degree, precision, residuals, time): a diagnosis aid.
bool setup_log() {
    const char* v = std::getenv("OVS_SETUP_LOG");
    return v != nullptr && v[0] == '1';
}

// start: a device block of p complex128 vectors (internal layout) to start
// from, or null for a seeded random block. want: eigenvalues in order of
// preference, of which m (all, if fewer) must find partners, Ritz pairs at
// tol at relative distance <= 1e-6 (matched greedily, nearest first, as the
// final selection does), before the side counts as converged; or null.
int run_side(Ctx& c, int m, double tol, double mu, uint64_t seed, double deadline_s, SideResult& res,
             const double2* start = nullptr, const std::vector<std::complex<double>>* want = nullptr) {
    const auto t_start = std::chrono::steady_clock::now();
    const bool log = setup_log();
    const int p = c.p;
    const long long N = c.N;
    ovs_gauge_s* g = c.g;
    double b = 0.0;
    int rc = spectral_bound(c, mu, &b);
    if (rc) return rc;
    const double hnorm = std::sqrt(b);
    if (start)
        ECK(cudaMemcpyAsync(c.Q, start, sizeof(double2) * (size_t)p * N, cudaMemcpyDeviceToDevice, c.st));
    else
        ECK(launch_random_fill(c.Q, (long long)p * N, seed, c.st));
    rc = svqb(c);
    if (rc) return rc;
    // complex64 phase: filter, orthonormalisation and Rayleigh-Ritz all in
    // complex64 (CGEMM on the CUDA cores; GB300's FP64 rate is 1/58 of its
    // FP32 rate), with a complex128 Rayleigh-Ritz to certify the pairs;
    // complex128 filtering only if complex64 stops making progress
    bool c64 = (g->prec == OVS_MIXED && g->links32 != nullptr);
    const double kRange32 = 1e4, kRange64 = 1e9;
    const int kDmax32 = 800, kDmax64 = 3000;
    FilterPlan fp = plan_filter(b, 0.01 * b, 0.02 * b, g->kappa, mu, 1e300, 0.0, c64 ? kRange32 : kRange64,
                                c64 ? kDmax32 : kDmax64);
    const long long budget = 400000LL * std::max(1, (int)std::ceil(8.0e6 / (double)N)) + 200LL * p * 3000;
    double last_rmax = 1e300, last_rmax32 = 1e300;
    int last_deg = fp.deg;
    const int max_iter = 60;
    std::vector<int> order(p);
    double last_iter_s = 0.0;
    bool have64 = false;  // the last pairs come from a complex128 Rayleigh-Ritz (Q holds them)
    bool switched = false;  // this iteration left complex64
    int last_nconv = 0;     // most wanted pairs at tol so far (complex64 residuals)
    if (c64) ECK(launch_convert(PREC_F32, c.Q, c.F[0], (long long)p * N, c.st));
    auto sort_order = [&]() {
        std::iota(order.begin(), order.end(), 0);
        std::sort(order.begin(), order.end(),
                  [&](int x, int y) { return std::abs(res.theta[x]) < std::abs(res.theta[y]); });
    };
    auto max_resid = [&]() {
        double r = 0.0;
        for (int i = 0; i < m; ++i) r = std::max(r, res.resid[order[i]] / hnorm);
        return r;
    };
    // convergence measure: the m-th smallest residual over the whole block,
    // i.e. m pairs at tol. The pairs installed are the m of smallest
    // |Re theta| among those at tol. Ritz values of unresolved directions
    // (residuals stuck at ~1e-2 while their |theta| wanders from one
    // iteration to the next) may sit among the smallest |theta|; they are
    // not eigenvalues and are not installed.
    auto mth_resid = [&]() {
        std::vector<double> rr(p);
        for (int i = 0; i < p; ++i) rr[i] = res.resid[i] / hnorm;
        std::nth_element(rr.begin(), rr.begin() + (m - 1), rr.end());
        return rr[m - 1];
    };
    // m of the wanted eigenvalues (all of them, if fewer) have partners: the
    // final selection will find as many matched pairs as it can
    auto partners_ok = [&]() {
        if (!want) return true;
        const int need = std::min<int>(m, (int)want->size());
        if (need == 0) return true;
        std::vector<char> taken(p, 0);
        int matched = 0;
        for (const auto& w : *want) {
            int best = -1;
            double bd = 1e300;
            for (int i = 0; i < p; ++i) {
                if (taken[i] || !(res.resid[i] / hnorm <= tol)) continue;
                const double d = std::abs(res.theta[i] - w);
                if (d < bd) { bd = d; best = i; }
            }
            if (best < 0 || bd > 1e-6 * std::abs(w)) continue;
            taken[best] = 1;
            if (++matched == need) return true;
        }
        return false;
    };
    auto count_at_tol = [&]() {
        int n = 0;
        for (int i = 0; i < p; ++i) n += res.resid[i] / hnorm <= tol;
        return n;
    };
    // progress measure: the median residual of the m wanted pairs (the
    // largest one, at the edge of the wanted set, converges slowest)
    auto median_resid = [&]() {
        std::vector<double> rr(m);
        for (int i = 0; i < m; ++i) rr[i] = res.resid[order[i]] / hnorm;
        std::nth_element(rr.begin(), rr.begin() + m / 2, rr.end());
        return rr[m / 2];
    };
    auto report = [&](int it, const char* what, double rmax) {
        if (!log) return;
        std::vector<double> rr(m);
        for (int i = 0; i < m; ++i) rr[i] = res.resid[order[i]] / hnorm;
        std::sort(rr.begin(), rr.end());
        int nconv = 0;
        for (int i = 0; i < m; ++i) nconv += rr[i] <= tol;
        std::fprintf(stderr,
                     "[setup] mu=%+.3f it=%d deg=%d %s |theta| min=%.4e m-th=%.4e p-th=%.4e resid max=%.3e "
                     "median=%.3e converged=%d/%d elapsed=%.2fs\n",
                     mu, it + 1, fp.deg, what, std::abs(res.theta[order[0]]), std::abs(res.theta[order[m - 1]]),
                     std::abs(res.theta[order[p - 1]]), rmax, rr[m / 2], nconv, m,
                     std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count());
    };
    // complex128 Rayleigh-Ritz of the block in Q (orthonormalised first);
    // Q then holds the Ritz vectors
    // complex128 residuals of the complex64 Ritz pairs now in Q, pair by pair
    auto certify_pairs = [&](int it) -> int {
        int r2 = pair_residuals64(c, mu, res.theta, res.resid);
        if (r2) return r2;
        res.matvecs += p;
        sort_order();
        have64 = true;
        report(it, "c128 residuals", max_resid());
        return OVS_OK;
    };
    auto certify = [&](int it) -> int {
        int r2 = svqb(c);
        if (r2) return r2;
        r2 = rayleigh_ritz(c, mu, res.theta, res.resid);
        if (r2) return r2;
        res.matvecs += p;
        std::swap(c.Q, c.A1);
        sort_order();
        have64 = true;
        const double rmax = max_resid();
        report(it, "c128 Rayleigh-Ritz", rmax);
        return OVS_OK;
    };
    for (int it = 0; it < max_iter; ++it) {
        const auto t_iter = std::chrono::steady_clock::now();
        // stop before an iteration that would overrun the deadline (the
        // first iteration always runs, so a basis is always produced)
        if (it > 0 && deadline_s > 0.0) {
            const double el = std::chrono::duration<double>(t_iter - t_start).count();
            if (el + last_iter_s > deadline_s) break;
        }
        double rmax = 0.0;
        if (c64) {
            // 1. filter (complex64), F[0] -> F[idx]
            void* bufs[3] = {c.F[0], c.F[1], c.F[2]};
            int idx = 0;
            rc = cheb_filter(c, PREC_F32, bufs, fp.deg, fp.c, fp.e, mu, &idx);
            if (rc) return rc;
            res.matvecs += 2LL * fp.deg * p;
            // 2. orthonormalise, 3. Rayleigh-Ritz, all complex64
            void* q = bufs[idx];
            void* tmp = bufs[(idx + 1) % 3];
            rc = svqb32(c, q, tmp);
            if (rc) return rc;
            rc = rayleigh_ritz32(c, mu, q, c.W, c.A1, c.A2, res.theta, res.resid);
            if (rc) return rc;
            res.matvecs += p;
            ECK(cudaMemcpyAsync(c.F[0], c.A1, sizeof(float2) * p * N, cudaMemcpyDeviceToDevice, c.st));
            have64 = false;
            sort_order();
            report(it, "c64", max_resid());
            const double r32 = mth_resid();
            // progress: more pairs at tol, or a falling median
            const double med = median_resid();
            const int nconv = count_at_tol();
            const bool stalled = it > 0 && med > 0.7 * last_rmax32 && nconv <= last_nconv;
            last_rmax32 = std::min(last_rmax32, med);
            last_nconv = std::max(last_nconv, nconv);
            rmax = r32;
            if (r32 <= tol || stalled) {
                // certify in complex128, pair by pair (one complex128 stencil)
                ECK(launch_convert(PREC_F64, c.F[0], c.Q, (long long)p * N, c.st));
                rc = certify_pairs(it);
                if (rc) return rc;
                rmax = mth_resid();
                if (rmax > tol && (rmax < 100.0 * tol || rmax < 1e-5)) {
                    // close to tol: a complex128 Rayleigh-Ritz on the block
                    rc = certify(it);
                    if (rc) return rc;
                    rmax = mth_resid();
                    if (rmax > tol && stalled) {
                        // complex64 rounding is what keeps the pairs from
                        // tol: complex128 filtering from here, whose stencil
                        // is FP64-ALU bound and ~20x slower per degree
                        c64 = false;
                        switched = true;
                    } else if (rmax > tol) {
                        ECK(launch_convert(PREC_F32, c.Q, c.F[0], (long long)p * N, c.st));
                    }
                }
                // far from tol: the slow pairs need more filtering, not more
                // precision; the complex64 block in F[0] carries on
            }
        } else {
            void* bufs[3] = {c.Q, c.A1, c.A2};
            int idx = 0;
            rc = cheb_filter(c, PREC_F64, bufs, fp.deg, fp.c, fp.e, mu, &idx);
            if (rc) return rc;
            if (idx != 0) ECK(cudaMemcpyAsync(c.Q, bufs[idx], sizeof(double2) * p * N, cudaMemcpyDeviceToDevice, c.st));
            res.matvecs += 2LL * fp.deg * p;
            rc = certify(it);
            if (rc) return rc;
            rmax = mth_resid();
        }
        res.iters = it + 1;
        if (rmax <= tol && have64 && partners_ok()) {
            res.converged = true;
            break;
        }
        // 4. next filter: cut between the m-th and the last Ritz value of H^2
        const double lm2 = std::abs(res.theta[order[m - 1]] * res.theta[order[m - 1]]);
        const double ap2 = std::abs(res.theta[order[p - 1]] * res.theta[order[p - 1]]);
        const double l02 = std::abs(res.theta[order[0]] * res.theta[order[0]]);
        double eta_near = 0.0;
        for (int i = 0; i < p; ++i) eta_near = std::max(eta_near, std::fabs(res.theta[i].imag()));
        fp = plan_filter(b, lm2, std::max(ap2, 1.2 * lm2), g->kappa, mu, 1.5 * eta_near + 1e-12, l02,
                         c64 ? kRange32 : kRange64, c64 ? kDmax32 : kDmax64);
        if (res.matvecs + 2LL * fp.deg * p > budget) break;
        // cost of the next iteration, scaled by its degree
        last_iter_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_iter).count() *
                      std::max(1.0, (double)fp.deg / std::max(1, last_deg));
        if (switched) last_iter_s *= 20.0;
        switched = false;
        last_deg = fp.deg;
        last_rmax = rmax;
    }
    if (!have64) {  // the last pairs are complex64 ones: certify them
        ECK(launch_convert(PREC_F64, c.F[0], c.Q, (long long)p * N, c.st));
        rc = certify_pairs(res.iters);
        if (rc) return rc;
        res.converged = mth_resid() <= tol && partners_ok();
    }
    // hand the Ritz vectors (now in Q) to the caller, sorted by |theta|
    std::vector<std::complex<double>> th(p);
    std::vector<double> rs(p);
    for (int i = 0; i < p; ++i) {
        ECK(cudaMemcpyAsync(c.A1 + (size_t)i * N, c.Q + (size_t)order[i] * N, sizeof(double2) * N,
                            cudaMemcpyDeviceToDevice, c.st));
        th[i] = res.theta[order[i]];
        rs[i] = res.resid[order[i]] / hnorm;
    }
    res.theta = th;
    res.resid = rs;
    std::swap(c.Q, c.A1);
    ECK(cudaStreamSynchronize(c.st));
    return OVS_OK;
}

// Schur deflation needs the right vectors only (Sec. 5.2 step i; Sec. 5.4):
// the m converged pairs of smallest |Re lambda| (all m if fewer converged)
// become the Schur basis, in that order.
int finish_schur(Ctx& c, ovs_gauge_s* g, int m, double tol, const SideResult& right, double* eig_out) {
    const int p = c.p;
    const long long N = c.N;
    std::vector<int> cand;
    for (int i = 0; i < p; ++i)
        if (right.resid[i] <= tol) cand.push_back(i);
    bool ok = right.converged;
    if ((int)cand.size() < m) {
        cand.clear();
        for (int i = 0; i < m; ++i) cand.push_back(i);
        ok = false;
    }
    std::stable_sort(cand.begin(), cand.end(), [&](int x, int y) {
        return std::fabs(right.theta[x].real()) < std::fabs(right.theta[y].real());
    });
    cand.resize(m);
    const size_t fv = sizeof(double2) * (size_t)N;
    double2 *Rc = nullptr, *tmp = nullptr;
    cudaError_t e = cudaMalloc((void**)&Rc, fv * m);
    if (e == cudaSuccess) e = cudaMalloc((void**)&tmp, fv * m);
    for (int i = 0; i < m && e == cudaSuccess; ++i)
        e = cudaMemcpy(tmp + (size_t)i * N, c.Q + (size_t)cand[i] * N, fv, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = launch_to_canonical(PREC_F64, tmp, fv, Rc, N, (int)g->V, m, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) {
        if (Rc) cudaFree(Rc);
        cudaGetLastError();
        return lib_fail(OVS_ECUDA, "deflate_setup_schur: gathering eigenvectors failed");
    }
    int rc = install_schur(g, m, Rc);
    cudaFree(Rc);
    if (rc < 0) return rc;
    if (eig_out)
        for (int i = 0; i < 2 * m; ++i) eig_out[i] = g->lambda[i];
    double rmax = 0.0;
    for (int i = 0; i < m; ++i) rmax = std::max(rmax, right.resid[cand[i]]);
    g->setup_resid = rmax;
    g->setup_iters[0] = right.iters;
    g->setup_iters[1] = 0;
    g->setup_matvecs = right.matvecs;
    if (!ok) {
        char msg[200];
        snprintf(msg, sizeof(msg),
                 "deflate_setup_schur: pairs did not all reach tol (%s after %d iterations, worst residual %.2e); "
                 "basis installed", right.converged ? "converged" : "not converged", right.iters, rmax);
        return lib_fail(OVS_EEIG, msg);
    }
    return OVS_OK;
}

}  // namespace

int eig_setup(ovs_gauge_s* g, int m, double tol, double* eig_out, bool schur) {
    Ctx c;
    c.g = g;
    c.st = 0;
    c.N = g->N;
    // block size p > m: the cut of the filter sits at the p-th Ritz value.
    // OVS_SETUP_BLOCK=<p> in the environment overrides it (a diagnosis aid).
    // For m >= 64 the block is 2.5 m: the wanted edge of such a set lies in
    // a dense part of the spectrum, where a cut at 1.5 m sits only a few per
    // cent above it (at 16^3 x 32, m = 100: |lambda| 0.0454 vs 0.0479) and
    // the filter separates the two slowly; with the cut at 2.5 m (0.054)
    // the median residual fell ~10x per iteration instead of ~4x.
    long long pb = m < 64 ? m + std::max(8, (m + 1) / 2) : m + (3LL * m + 1) / 2;
    if (const char* ev = std::getenv("OVS_SETUP_BLOCK")) {
        const long long v = std::atoll(ev);
        if (v > m) pb = v;
    }
    c.p = (int)std::min<long long>(pb, g->N / 2);
    if (c.p > 65535) return lib_fail(OVS_EINVAL, "m too large for the set-up block");
    const int p = c.p;
    const long long N = c.N;
    char msg[320];
#define SETUP_FAIL(code)                                                                        \
    do {                                                                                        \
        snprintf(msg, sizeof(msg), "deflate_setup: %s", c.err[0] ? c.err : "CUDA error");       \
        return lib_fail((code), msg);                                                           \
    } while (0)
    if (cublasCreate(&c.cb) != CUBLAS_STATUS_SUCCESS || cusolverDnCreate(&c.cs) != CUSOLVER_STATUS_SUCCESS ||
        cusolverDnCreateParams(&c.params) != CUSOLVER_STATUS_SUCCESS)
        return lib_fail(OVS_ECUDA, "deflate_setup: cannot create cuBLAS/cuSOLVER handles");
    cublasSetStream(c.cb, c.st);
    cusolverDnSetStream(c.cs, c.st);
    const size_t blk = sizeof(double2) * (size_t)p * N;
    cudaError_t e = cudaSuccess;
    for (double2** q : {&c.Q, &c.W, &c.A1, &c.A2})
        if (e == cudaSuccess) e = cudaMalloc((void**)q, blk);
    if (g->prec == OVS_MIXED)
        for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaMalloc(&c.F[i], blk / 2);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c.G, sizeof(double2) * p * p);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c.G2, sizeof(double2) * p * p);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c.Y, sizeof(double2) * p * p);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c.G32, sizeof(float2) * p * p);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c.Y32, sizeof(float2) * p * p);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c.theta, sizeof(double2) * p);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c.lam, sizeof(double) * p);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c.resid, sizeof(double) * p);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c.info, sizeof(int));
    if (e != cudaSuccess) return lib_fail(OVS_ENOMEM, "deflate_setup: device memory for the set-up block");

    // right eigenvectors of H_w(mu)
    SideResult right, left;
    // time budget: the right side gets half of it (all of it for Schur), the
    // left side what the right side left over
    const auto t_setup = std::chrono::steady_clock::now();
    const double side_s = g->setup_budget_s > 0.0 ? (schur ? 1.0 : 0.5) * g->setup_budget_s : 0.0;
    int rc = run_side(c, m, tol, g->mu, 12345, side_s, right);
    if (rc) SETUP_FAIL(rc);
    if (schur) return finish_schur(c, g, m, tol, right, eig_out);
    double2* Rblk = nullptr;
    if (cudaMalloc((void**)&Rblk, blk) != cudaSuccess) return lib_fail(OVS_ENOMEM, "deflate_setup: right block");
    cudaMemcpy(Rblk, c.Q, blk, cudaMemcpyDeviceToDevice);
    // left eigenvectors: right eigenvectors of H_w(-mu), eigenvalues
    // conj(lambda). The iteration starts from the right side's Ritz vectors
    // (H_w(-mu) = H_w(mu)^H differs from H_w(mu) only in the temporal hops,
    // so left and right eigenvectors are close), and it runs until m of the
    // right pairs at tol (in the order of the selection below: smallest
    // |Re lambda| first) have partners at tol: two independent runs would
    // converge on different fringes of the wanted set and leave pairs
    // unmatched.
    std::vector<std::complex<double>> want;
    {
        std::vector<int> at;
        for (int i = 0; i < p; ++i)
            if (right.resid[i] <= tol) at.push_back(i);
        std::stable_sort(at.begin(), at.end(), [&](int x, int y) {
            return std::fabs(right.theta[x].real()) < std::fabs(right.theta[y].real());
        });
        for (int i : at) want.push_back(std::conj(right.theta[i]));
    }
    double left_s = 0.0;
    if (g->setup_budget_s > 0.0)
        left_s = std::max(0.5 * g->setup_budget_s,
                          g->setup_budget_s -
                              std::chrono::duration<double>(std::chrono::steady_clock::now() - t_setup).count());
    rc = run_side(c, m, tol, -g->mu, 54321, left_s, left, Rblk, &want);
    if (rc) {
        cudaFree(Rblk);
        SETUP_FAIL(rc);
    }
    // choose the m right pairs of smallest |Re lambda| that are at tol and
    // have a left partner at tol (eigenvalue conj(lambda), relative distance
    // <= 1e-6); if fewer than m qualify, fill up with the nearest pairs in
    // the same order and report OVS_EEIG
    std::vector<int> order_r(p);
    std::iota(order_r.begin(), order_r.end(), 0);
    std::stable_sort(order_r.begin(), order_r.end(), [&](int x, int y) {
        const bool cx = right.resid[x] <= tol, cy = right.resid[y] <= tol;
        if (cx != cy) return cx;  // pairs at tol first
        return std::fabs(right.theta[x].real()) < std::fabs(right.theta[y].real());
    });
    std::vector<int> cand, lsel;
    std::vector<char> used(p, 0);
    double worst_match = 0.0;
    auto nearest_left = [&](int ri, bool at_tol, double* dist) {
        const std::complex<double> want = std::conj(right.theta[ri]);
        int best = -1;
        double bd = 1e300;
        for (int j = 0; j < p; ++j) {
            if (used[j] || (at_tol && !(left.resid[j] <= tol))) continue;
            const double d = std::abs(left.theta[j] - want);
            if (d < bd) { bd = d; best = j; }
        }
        *dist = bd / std::max(std::abs(want), 1e-300);
        return best;
    };
    for (int q = 0; q < p && (int)cand.size() < m; ++q) {  // both sides at tol, matched
        const int ri = order_r[q];
        if (!(right.resid[ri] <= tol)) break;
        double d = 0.0;
        const int lj = nearest_left(ri, true, &d);
        if (lj < 0 || d > 1e-6) continue;
        used[lj] = 1;
        cand.push_back(ri);
        lsel.push_back(lj);
    }
    bool ok = (int)cand.size() == m;
    for (int q = 0; q < p && (int)cand.size() < m; ++q) {  // fill up
        const int ri = order_r[q];
        if (std::find(cand.begin(), cand.end(), ri) != cand.end()) continue;
        double d = 0.0;
        const int lj = nearest_left(ri, false, &d);
        used[lj] = 1;
        cand.push_back(ri);
        lsel.push_back(lj);
        worst_match = std::max(worst_match, d);
    }
    // canonical copies of the chosen vectors, then install (biorthonormalises L)
    double2 *Rc = nullptr, *Lc = nullptr, *tmp = nullptr;
    const size_t fv = sizeof(double2) * (size_t)N;
    e = cudaMalloc((void**)&Rc, fv * m);
    if (e == cudaSuccess) e = cudaMalloc((void**)&Lc, fv * m);
    if (e == cudaSuccess) e = cudaMalloc((void**)&tmp, fv * m);
    std::vector<double> lambda(2 * m);
    for (int i = 0; i < m && e == cudaSuccess; ++i) {
        e = cudaMemcpy(tmp + (size_t)i * N, Rblk + (size_t)cand[i] * N, fv, cudaMemcpyDeviceToDevice);
        lambda[2 * i] = right.theta[cand[i]].real();
        lambda[2 * i + 1] = right.theta[cand[i]].imag();
    }
    if (e == cudaSuccess) e = launch_to_canonical(PREC_F64, tmp, fv, Rc, N, (int)g->V, m, 0);
    for (int i = 0; i < m && e == cudaSuccess; ++i)
        e = cudaMemcpy(tmp + (size_t)i * N, c.Q + (size_t)lsel[i] * N, fv, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = launch_to_canonical(PREC_F64, tmp, fv, Lc, N, (int)g->V, m, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(Rblk);
    if (e != cudaSuccess) {
        cudaFree(Rc); cudaFree(Lc); cudaFree(tmp);
        return lib_fail(OVS_ECUDA, "deflate_setup: gathering eigenvectors failed");
    }
    rc = install_deflation(g, m, Rc, Lc, lambda.data());
    cudaFree(Rc);
    cudaFree(Lc);
    cudaFree(tmp);
    if (rc < 0) return rc;
    if (eig_out)
        for (int i = 0; i < 2 * m; ++i) eig_out[i] = lambda[i];
    double rmax = 0.0;
    for (int i = 0; i < m; ++i) rmax = std::max(rmax, right.resid[cand[i]]);
    g->setup_resid = rmax;
    g->setup_iters[0] = right.iters;
    g->setup_iters[1] = left.iters;
    g->setup_matvecs = right.matvecs + left.matvecs;
    if (!ok) {
        snprintf(msg, sizeof(msg),
                 "deflate_setup: pairs did not all reach tol (right %s after %d iterations, left %s after %d, "
                 "worst left/right eigenvalue mismatch %.2e); basis installed",
                 right.converged ? "converged" : "not converged", right.iters,
                 left.converged ? "converged" : "not converged", left.iters, worst_match);
        return lib_fail(OVS_EEIG, msg);
    }
    return OVS_OK;
}

}  // namespace ovs
