// K3: sgn(H_k) e_1 by Roberts' iteration S <- (S + S^-1)/2, S^0 = H_k
// (Sec. 5.2, Eq. Roberts; used for H_k in Sec. 5.3 step v), in FP64 on the
// device, one thread block per right-hand side.
//
// The inverse is an in-place Gauss-Jordan elimination with partial (row)
// pivoting; the row interchanges are undone as column interchanges at the
// end. Stopping rule: after the first iterate whose relative change
// ||S^(n+1) - S^n||_F / ||S^(n+1)||_F is <= 1e-9, one more iteration (the
// quadratic convergence then reaches rounding level); at most 50 iterations.
// A zero or non-finite pivot (an eigenvalue on or numerically at the
// imaginary axis makes S singular) ends with status OVS_ESIGN; no
// convergence within 50 iterations gives OVS_NOT_CONVERGED.
#include "common.cuh"
#include "kernels.h"

namespace ovs {

constexpr int NT = 1024;
constexpr double kSwitchTol = 1e-9;
constexpr int kExtra = 1;
constexpr int kMaxIter = 50;
enum { ST_OK = 0, ST_NOT_CONVERGED = 1, ST_ESIGN = -6 };

__device__ __forceinline__ double blk_sum(double v, double* sh) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (threadIdx.x == 0) sh[32] = s;
    }
    __syncthreads();
    return sh[32];
}

// In-place inverse of the n x n row-major matrix A. Returns false if a
// pivot is zero or not finite.
__device__ bool gauss_jordan(cd* A, int n, int* perm, cd* colp, cd* rowp, double* sval, int* sidx) {
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    __shared__ int s_ok;
    if (tid == 0) s_ok = 1;
    for (int p = 0; p < n; ++p) {
        // pivot: argmax_{i >= p} |A[i][p]|
        double best = -1.0;
        int bi = p;
        for (int i = p + tid; i < n; i += NT) {
            const cd a = A[(size_t)i * n + p];
            const double v = a.re * a.re + a.im * a.im;
            if (v > best) { best = v; bi = i; }
        }
        for (int off = 16; off > 0; off >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, off);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { sval[w] = best; sidx[w] = bi; }
        __syncthreads();
        if (tid == 0) {
            double b = sval[0];
            int ib = sidx[0];
            for (int q = 1; q < NT / 32; ++q)
                if (sval[q] > b || (sval[q] == b && sidx[q] < ib)) { b = sval[q]; ib = sidx[q]; }
            perm[p] = ib;
            if (!(b > 0.0) || !isfinite(b)) s_ok = 0;
        }
        __syncthreads();
        if (!s_ok) return false;
        const int piv = perm[p];
        if (piv != p) {
            for (int j = tid; j < n; j += NT) {
                const cd t = A[(size_t)p * n + j];
                A[(size_t)p * n + j] = A[(size_t)piv * n + j];
                A[(size_t)piv * n + j] = t;
            }
            __syncthreads();
        }
        const cd a = A[(size_t)p * n + p];
        const double den = a.re * a.re + a.im * a.im;
        const cd inv = {a.re / den, -a.im / den};
        for (int i = tid; i < n; i += NT) {
            colp[i] = A[(size_t)i * n + p];
            rowp[i] = (i == p) ? inv : cmul(A[(size_t)p * n + i], inv);
        }
        __syncthreads();
        for (int idx = tid; idx < n * n; idx += NT) {
            const int i = idx / n, j = idx - i * n;
            if (i == p) {
                A[idx] = rowp[j];
            } else if (j == p) {
                A[idx] = -cmul(colp[i], inv);
            } else {
                cd v = A[idx];
                const cd f = colp[i], g = rowp[j];
                v.re -= f.re * g.re - f.im * g.im;
                v.im -= f.re * g.im + f.im * g.re;
                A[idx] = v;
            }
        }
        __syncthreads();
    }
    // undo the row interchanges as column interchanges, last first
    for (int p = n - 1; p >= 0; --p) {
        const int q = perm[p];
        if (q != p) {
            for (int i = tid; i < n; i += NT) {
                const cd t = A[(size_t)i * n + p];
                A[(size_t)i * n + p] = A[(size_t)i * n + q];
                A[(size_t)i * n + q] = t;
            }
            __syncthreads();
        }
    }
    return true;
}

__global__ void __launch_bounds__(NT) k_newton(const double2* __restrict__ H, long long h_rhs_stride, int ldh,
                                               const int* __restrict__ k_used, const double* __restrict__ beta,
                                               double2* __restrict__ coeff, long long coeff_stride,
                                               double2* __restrict__ work, int kmax, int* __restrict__ iters,
                                               int* __restrict__ status) {
    extern __shared__ unsigned char smem_raw[];
    const int r = blockIdx.x, tid = threadIdx.x;
    const int n = k_used[r];
    cd* S = reinterpret_cast<cd*>(work) + (size_t)r * 2 * kmax * kmax;
    cd* T = S + (size_t)kmax * kmax;
    cd* colp = reinterpret_cast<cd*>(smem_raw);
    cd* rowp = colp + kmax;
    int* perm = reinterpret_cast<int*>(rowp + kmax);
    __shared__ double sval[NT / 32 + 1];
    __shared__ int sidx[NT / 32];
    double2* cr = coeff + r * coeff_stride;
    if (n <= 0) {
        for (int i = tid; i < kmax; i += NT) cr[i] = make_double2(0.0, 0.0);
        if (tid == 0) { iters[r] = 0; status[r] = ST_OK; }
        return;
    }
    const double2* Hr = H + r * h_rhs_stride;
    for (int idx = tid; idx < n * n; idx += NT) {
        const int i = idx / n, j = idx - i * n;
        const double2 h = Hr[i + (long long)j * ldh];
        S[idx] = {h.x, h.y};
    }
    __syncthreads();
    int st = ST_NOT_CONVERGED, it_done = 0, remaining = -1;
    for (int it = 1; it <= kMaxIter; ++it) {
        for (int idx = tid; idx < n * n; idx += NT) T[idx] = S[idx];
        __syncthreads();
        if (!gauss_jordan(T, n, perm, colp, rowp, sval, sidx)) {
            st = ST_ESIGN;
            it_done = it;
            break;
        }
        double d2 = 0.0, s2 = 0.0;
        for (int idx = tid; idx < n * n; idx += NT) {
            const cd a = S[idx], b = T[idx];
            const cd v = {0.5 * (a.re + b.re), 0.5 * (a.im + b.im)};
            const double dx = v.re - a.re, dy = v.im - a.im;
            d2 += dx * dx + dy * dy;
            s2 += v.re * v.re + v.im * v.im;
            S[idx] = v;
        }
        d2 = blk_sum(d2, sval);
        s2 = blk_sum(s2, sval);
        it_done = it;
        const double change = sqrt(d2 / s2);
        if (!isfinite(change)) {
            st = ST_ESIGN;
            break;
        }
        if (remaining < 0 && change <= kSwitchTol) remaining = kExtra;
        if (remaining >= 0) {
            if (remaining == 0) {
                st = ST_OK;
                break;
            }
            --remaining;
        }
    }
    const double b = beta[r];
    for (int i = tid; i < kmax; i += NT) {
        if (i < n && st != ST_ESIGN) {
            const cd s = S[(size_t)i * n];
            cr[i] = make_double2(b * s.re, b * s.im);
        } else {
            cr[i] = make_double2(0.0, 0.0);
        }
    }
    if (tid == 0) {
        iters[r] = it_done;
        status[r] = st;
    }
}

cudaError_t launch_newton(const void* H, long long h_rhs_stride, int ldh, const int* k_used, const double* beta,
                          void* coeff, long long coeff_stride, void* work, int kmax, int nrhs, int* iters,
                          int* status, cudaStream_t st) {
    const size_t smem = (size_t)kmax * 2 * sizeof(cd) + (size_t)kmax * sizeof(int);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_newton, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    k_newton<<<nrhs, NT, smem, st>>>((const double2*)H, h_rhs_stride, ldh, k_used, beta, (double2*)coeff,
                                     coeff_stride, (double2*)work, kmax, iters, status);
    return cudaGetLastError();
}

}  // namespace ovs
