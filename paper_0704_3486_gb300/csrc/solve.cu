// Nested inversion of the overlap operator: restarted GMRES for
// D_ov(mu) x = b, every outer iteration one application of D_ov(mu) =
// 1 + gamma5 sgn(H_w(mu)) through the deflated Arnoldi method (the use the
// paper names for its method, Secs. 6 and 7; the outer method is not fixed
// there). Small kernels of the outer iteration, all right-hand sides at
// once: norms, the Hessenberg column with its Givens rotation (the small
// least-squares problem min ||beta e_1 - Hbar y|| is kept in triangular
// form as the columns arrive), scaling, the triangular solve for y.
// Vectors are canonical complex128; the outer basis is [restart+1][nrhs][N],
// so that basis vector j of all right-hand sides is one contiguous block.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace ovs {

constexpr int kNormBlocks = 64;

// partial[r][b] = sum over block b's slice of |v_r|^2
__global__ void __launch_bounds__(256) k_norm2_partial(const double2* __restrict__ v, long long n, long long stride,
                                                       double* __restrict__ partial) {
    __shared__ double sh[8];
    const int r = blockIdx.y, b = blockIdx.x;
    const double2* vr = v + r * stride;
    double s = 0.0;
    for (long long i = (long long)b * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double2 a = vr[i];
        s = fma(a.x, a.x, s);
        s = fma(a.y, a.y, s);
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sh[w];
        partial[r * gridDim.x + b] = t;
    }
}

// norm[r] = sqrt(sum_b partial[r][b]); inv[r] = 1/norm[r] (0 if norm is 0)
__global__ void k_norm_finish(const double* __restrict__ partial, int nblk, int nrhs, double* __restrict__ norm,
                              double* __restrict__ inv) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs) return;
    double t = 0.0;
    for (int b = 0; b < nblk; ++b) t += partial[r * nblk + b];
    const double nv = sqrt(t);
    norm[r] = nv;
    if (inv) inv[r] = nv > 0.0 ? 1.0 / nv : 0.0;
}

// out_r = s_r * in_r (s real, per right-hand side)
__global__ void k_scale(const double2* __restrict__ in, long long in_stride, double2* __restrict__ out,
                        long long out_stride, const double* __restrict__ s, long long n) {
    const int r = blockIdx.y;
    const double f = s[r];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double2 a = in[r * in_stride + i];
        out[r * out_stride + i] = make_double2(a.x * f, a.y * f);
    }
}

// out_r = a_r - b_r
__global__ void k_sub(const double2* __restrict__ a, const double2* __restrict__ b, double2* __restrict__ out,
                      long long n) {
    const int r = blockIdx.y;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double2 x = a[r * n + i], y = b[r * n + i];
        out[r * n + i] = make_double2(x.x - y.x, x.y - y.y);
    }
}

// Column j of the outer Arnoldi process, one thread per right-hand side:
// h = h1 + h2 (the two Gram-Schmidt passes, red1/red2[r][0..j]), h_(j+1,j) =
// ||z|| (from the norm partials of the second update); the previous
// rotations are applied to the column, a new rotation G_j = [[conj(c),
// conj(s)], [-s, c]] (c = a/rho, s = b/rho) annihilates h_(j+1,j), and the
// right-hand side g of the least-squares problem is rotated with it.
// R: [nrhs][restart][restart] column-major triangular factor; rot: [nrhs]
// [restart][2] (c, s); gv: [nrhs][restart+1]; est[r] = |g_(j+1)|;
// inv_hn[r] = 1/h_(j+1,j) (0 at a breakdown: the Krylov space is invariant).
__global__ void k_gmres_col(const double2* __restrict__ red1, const double2* __restrict__ red2, long long red_stride,
                            const double* __restrict__ npart, int nblk, int j, int restart, double2* __restrict__ R,
                            double2* __restrict__ rot, double2* __restrict__ gv, double* __restrict__ est,
                            double* __restrict__ inv_hn, int nrhs) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs) return;
    double t = 0.0;
    for (int b = 0; b < nblk; ++b) t += npart[r * nblk + b];
    const double hn = sqrt(t);
    cd* col = reinterpret_cast<cd*>(R) + ((size_t)r * restart + j) * restart;
    cd* ro = reinterpret_cast<cd*>(rot) + (size_t)r * restart * 2;
    cd* g = reinterpret_cast<cd*>(gv) + (size_t)r * (restart + 1);
    for (int i = 0; i <= j; ++i) {
        const double2 a = red1[r * red_stride + i], b = red2[r * red_stride + i];
        col[i] = {a.x + b.x, a.y + b.y};
    }
    for (int i = 0; i < j; ++i) {  // previous rotations on rows i, i+1
        const cd c = ro[2 * i], s = ro[2 * i + 1];
        const cd w1 = col[i], w2 = (i + 1 < j + 1) ? col[i + 1] : cd{0.0, 0.0};
        col[i] = cmulc(c, w1) + cmulc(s, w2);
        col[i + 1] = cmul(c, w2) - cmul(s, w1);
    }
    const cd a = col[j];
    const double rho = sqrt(a.re * a.re + a.im * a.im + hn * hn);
    cd c = {1.0, 0.0}, s = {0.0, 0.0};
    if (rho > 0.0) {
        c = {a.re / rho, a.im / rho};
        s = {hn / rho, 0.0};
    }
    ro[2 * j] = c;
    ro[2 * j + 1] = s;
    col[j] = {rho, 0.0};  // conj(c) a + conj(s) hn = rho
    const cd gj = g[j];
    g[j] = cmulc(c, gj);
    g[j + 1] = -cmul(s, gj);
    est[r] = sqrt(g[j + 1].re * g[j + 1].re + g[j + 1].im * g[j + 1].im);
    inv_hn[r] = hn > 0.0 ? 1.0 / hn : 0.0;
}

// g = (beta_r, 0, ...): start of a cycle
__global__ void k_gmres_start(const double* __restrict__ beta, double2* __restrict__ gv, int restart, int nrhs) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs) return;
    double2* g = gv + (size_t)r * (restart + 1);
    g[0] = make_double2(beta[r], 0.0);
    for (int i = 1; i <= restart; ++i) g[i] = make_double2(0.0, 0.0);
}

// y = R^-1 g over the first jj columns (back substitution), one thread per
// right-hand side; y: [nrhs][restart] (also the coefficients of x += W y)
__global__ void k_gmres_backsub(const double2* __restrict__ R, const double2* __restrict__ gv, int jj, int restart,
                                double2* __restrict__ y, int nrhs) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs) return;
    const cd* Rr = reinterpret_cast<const cd*>(R) + (size_t)r * restart * restart;
    const cd* g = reinterpret_cast<const cd*>(gv) + (size_t)r * (restart + 1);
    cd* yr = reinterpret_cast<cd*>(y) + (size_t)r * restart;
    for (int i = jj - 1; i >= 0; --i) {
        cd v = g[i];
        for (int l = i + 1; l < jj; ++l) v = v - cmul(Rr[(size_t)l * restart + i], yr[l]);
        const cd d = Rr[(size_t)i * restart + i];
        const double den = d.re * d.re + d.im * d.im;
        yr[i] = den > 0.0 ? cd{(v.re * d.re + v.im * d.im) / den, (v.im * d.re - v.re * d.im) / den} : cd{0.0, 0.0};
    }
    for (int i = jj; i < restart; ++i) yr[i] = {0.0, 0.0};
}

static dim3 vec_grid(long long n, int nrhs) {
    long long b = (n + 255) / 256;
    if (b > 1024) b = 1024;
    return dim3((unsigned)b, nrhs);
}

int norm_blocks() { return kNormBlocks; }

cudaError_t launch_norms(const void* v, long long n, long long stride, int nrhs, double* partial, double* norm,
                         double* inv, cudaStream_t st) {
    k_norm2_partial<<<dim3(kNormBlocks, nrhs), 256, 0, st>>>((const double2*)v, n, stride, partial);
    k_norm_finish<<<(nrhs + 127) / 128, 128, 0, st>>>(partial, kNormBlocks, nrhs, norm, inv);
    return cudaGetLastError();
}

cudaError_t launch_norm_partials(const void* v, long long n, long long stride, int nrhs, double* partial,
                                 cudaStream_t st) {
    k_norm2_partial<<<dim3(kNormBlocks, nrhs), 256, 0, st>>>((const double2*)v, n, stride, partial);
    return cudaGetLastError();
}

cudaError_t launch_scale(const void* in, long long in_stride, void* out, long long out_stride, const double* s,
                         long long n, int nrhs, cudaStream_t st) {
    k_scale<<<vec_grid(n, nrhs), 256, 0, st>>>((const double2*)in, in_stride, (double2*)out, out_stride, s, n);
    return cudaGetLastError();
}

cudaError_t launch_sub(const void* a, const void* b, void* out, long long n, int nrhs, cudaStream_t st) {
    k_sub<<<vec_grid(n, nrhs), 256, 0, st>>>((const double2*)a, (const double2*)b, (double2*)out, n);
    return cudaGetLastError();
}

cudaError_t launch_gmres_start(const double* beta, void* gv, int restart, int nrhs, cudaStream_t st) {
    k_gmres_start<<<(nrhs + 127) / 128, 128, 0, st>>>(beta, (double2*)gv, restart, nrhs);
    return cudaGetLastError();
}

cudaError_t launch_gmres_col(const void* red1, const void* red2, long long red_stride, const double* npart, int j,
                             int restart, void* R, void* rot, void* gv, double* est, double* inv_hn, int nrhs,
                             cudaStream_t st) {
    k_gmres_col<<<(nrhs + 127) / 128, 128, 0, st>>>((const double2*)red1, (const double2*)red2, red_stride, npart,
                                                    kNormBlocks, j, restart, (double2*)R, (double2*)rot,
                                                    (double2*)gv, est, inv_hn, nrhs);
    return cudaGetLastError();
}

cudaError_t launch_gmres_backsub(const void* R, const void* gv, int jj, int restart, void* y, int nrhs,
                                 cudaStream_t st) {
    k_gmres_backsub<<<(nrhs + 127) / 128, 128, 0, st>>>((const double2*)R, (const double2*)gv, jj, restart,
                                                        (double2*)y, nrhs);
    return cudaGetLastError();
}

}  // namespace ovs
