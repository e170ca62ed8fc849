// K2 (classical Gram-Schmidt sweeps of the Arnoldi recurrence, Sec. 4
// Eq. Arnoldi), K4 (recombination y += V_k c, Eq. yproj3 / fAxLRArn) and
// K5 (LR projection c = L^+ x, x_ominus = x - R c, Sec. 5.3 Eq. xdec).
//
// A field is a flat array of 16-byte units (one complex128, or two
// complex64). Each right-hand side r owns its Krylov basis; a block of 256
// threads covers one row block of one right-hand side and streams every
// basis vector through it, so the basis is read once per sweep with fully
// coalesced 16-byte loads.
//
// Precision: in the complex64 form the products and the partial sums of a
// thread (2*E terms) and of a warp (a 32-lane tree) are FP32; every warp
// partial is then added into FP64, so inner products, norms and Hessenberg
// entries are accumulated in FP64 over the rest of the vector.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace ovs {

constexpr int BT = 256;  // threads per block
constexpr int NWARP = BT / 32;

template <typename R> __device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// ----------------------------------------------------------------- dots
template <typename R, int E, int IU>
__global__ void __launch_bounds__(BT) k_dots(const typename Unit<R>::vec* __restrict__ basis,
                                             long long basis_rhs_stride, long long vec_stride, int J,
                                             const typename Unit<R>::vec* __restrict__ w, long long w_rhs_stride,
                                             long long nunits, long long chunk, int nblk,
                                             double2* __restrict__ partial, const int* __restrict__ active) {
    using vec = typename Unit<R>::vec;
    constexpr int NC = Unit<R>::ncplx;
    extern __shared__ double2 sacc[];  // [NWARP][J]
    const int r = blockIdx.y, b = blockIdx.x;
    if (active != nullptr && active[r] == 0) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < NWARP * J; i += BT) sacc[i] = make_double2(0.0, 0.0);
    __syncthreads();
    const vec* Vr = basis + r * basis_rhs_stride;
    const vec* wr = w + r * w_rhs_stride;
    const long long u0 = (long long)b * chunk;
    const long long u1 = min(u0 + chunk, nunits);
    for (long long base = u0; base < u1; base += (long long)BT * E) {
        cplx<R> wv[E][NC];
        bool ok[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const long long u = base + tid + (long long)BT * e;
            ok[e] = u < u1;
            if (ok[e]) {
                Unit<R>::split(__ldg(wr + u), wv[e]);
            } else {
#pragma unroll
                for (int c = 0; c < NC; ++c) wv[e][c] = {R(0), R(0)};
            }
        }
        for (int i0 = 0; i0 < J; i0 += IU) {
            cplx<R> acc[IU];
#pragma unroll
            for (int ii = 0; ii < IU; ++ii) acc[ii] = {R(0), R(0)};
#pragma unroll
            for (int ii = 0; ii < IU; ++ii) {
                if (i0 + ii < J) {
                    const vec* vi = Vr + (long long)(i0 + ii) * vec_stride;
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        if (ok[e]) {
                            cplx<R> vc[NC];
                            Unit<R>::split(__ldcs(vi + base + tid + (long long)BT * e), vc);
#pragma unroll
                            for (int c = 0; c < NC; ++c) cfmac(acc[ii], vc[c], wv[e][c]);
                        }
                    }
                }
            }
#pragma unroll
            for (int ii = 0; ii < IU; ++ii) {
                acc[ii].re = warp_sum(acc[ii].re);
                acc[ii].im = warp_sum(acc[ii].im);
            }
            if (lane == 0) {
#pragma unroll
                for (int ii = 0; ii < IU; ++ii) {
                    if (i0 + ii < J) {
                        double2& s = sacc[warp * J + i0 + ii];
                        s.x += double(acc[ii].re);
                        s.y += double(acc[ii].im);
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < J; i += BT) {
        double sx = 0.0, sy = 0.0;
#pragma unroll
        for (int q = 0; q < NWARP; ++q) {
            sx += sacc[q * J + i].x;
            sy += sacc[q * J + i].y;
        }
        partial[((size_t)r * nblk + b) * J + i] = make_double2(sx, sy);
    }
}

// --------------------------------------------------------------- update
// Out element type per basis unit: NC complex numbers of precision RO.
template <typename RO, int NC> struct OutIO;
template <> struct OutIO<double, 1> {
    __device__ __forceinline__ static void load(const void* p, long long u, cd* o) {
        double2 v = static_cast<const double2*>(p)[u];
        o[0] = {v.x, v.y};
    }
    __device__ __forceinline__ static void store(void* p, long long u, const cd* o) {
        static_cast<double2*>(p)[u] = make_double2(o[0].re, o[0].im);
    }
};
template <> struct OutIO<double, 2> {
    __device__ __forceinline__ static void load(const void* p, long long u, cd* o) {
        const double2* q = static_cast<const double2*>(p) + 2 * u;
        double2 a = q[0], b = q[1];
        o[0] = {a.x, a.y};
        o[1] = {b.x, b.y};
    }
    __device__ __forceinline__ static void store(void* p, long long u, const cd* o) {
        double2* q = static_cast<double2*>(p) + 2 * u;
        q[0] = make_double2(o[0].re, o[0].im);
        q[1] = make_double2(o[1].re, o[1].im);
    }
};
template <> struct OutIO<float, 2> {
    __device__ __forceinline__ static void load(const void* p, long long u, cf* o) {
        float4 v = static_cast<const float4*>(p)[u];
        o[0] = {v.x, v.y};
        o[1] = {v.z, v.w};
    }
    __device__ __forceinline__ static void store(void* p, long long u, const cf* o) {
        static_cast<float4*>(p)[u] = make_float4(o[0].re, o[0].im, o[1].re, o[1].im);
    }
};

// out_r = in_r + sum_{i<J_r} V_r,i * (alpha c_r,i). Strides of in/out are in
// complex numbers of precision RO; basis strides in units.
template <typename RV, typename RO, int E>
__global__ void __launch_bounds__(BT) k_update(const typename Unit<RV>::vec* __restrict__ basis,
                                               long long basis_rhs_stride, long long vec_stride, int J,
                                               const int* __restrict__ Jdev, const double2* __restrict__ coef,
                                               long long coef_stride, double alpha, const cplx<RO>* in,
                                               long long in_rhs_stride, cplx<RO>* out, long long out_rhs_stride,
                                               long long nunits, long long chunk, int nblk,
                                               double* __restrict__ norm_partial, const int* __restrict__ active) {
    using vec = typename Unit<RV>::vec;
    constexpr int NC = Unit<RV>::ncplx;
    extern __shared__ double2 scoef[];
    __shared__ double sred[NWARP];
    const int r = blockIdx.y, b = blockIdx.x;
    if (active != nullptr && active[r] == 0) return;
    int Jr = J;
    if (Jdev != nullptr) Jr = min(J, Jdev[r]);
    const int tid = threadIdx.x;
    for (int i = tid; i < Jr; i += BT) {
        double2 c = coef[r * coef_stride + i];
        scoef[i] = make_double2(alpha * c.x, alpha * c.y);
    }
    __syncthreads();
    const vec* Vr = basis + r * basis_rhs_stride;
    const cplx<RO>* inr = in ? in + r * in_rhs_stride : nullptr;
    cplx<RO>* outr = out + r * out_rhs_stride;
    const long long u0 = (long long)b * chunk;
    const long long u1 = min(u0 + chunk, nunits);
    double nrm = 0.0;
    for (long long base = u0; base < u1; base += (long long)BT * E) {
        cplx<RO> o[E][NC];
        cplx<RV> acc[E][NC];
        bool ok[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const long long u = base + tid + (long long)BT * e;
            ok[e] = u < u1;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                o[e][c] = {RO(0), RO(0)};
                acc[e][c] = {RV(0), RV(0)};
            }
            if (ok[e] && inr != nullptr) OutIO<RO, NC>::load(inr, u, o[e]);
        }
        int since_flush = 0;
        for (int i = 0; i < Jr; ++i) {
            const double2 cd_ = scoef[i];
            const cplx<RV> ci = {RV(cd_.x), RV(cd_.y)};
            const vec* vi = Vr + (long long)i * vec_stride;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                if (ok[e]) {
                    cplx<RV> vc[NC];
                    Unit<RV>::split(__ldcs(vi + base + tid + (long long)BT * e), vc);
#pragma unroll
                    for (int c = 0; c < NC; ++c) cfma(acc[e][c], vc[c], ci);
                }
            }
            // Wider output than basis: flush the FP32 partial sums every 16 terms.
            if (sizeof(RO) > sizeof(RV) && ++since_flush == 16) {
                since_flush = 0;
#pragma unroll
                for (int e = 0; e < E; ++e)
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        o[e][c].re += RO(acc[e][c].re);
                        o[e][c].im += RO(acc[e][c].im);
                        acc[e][c] = {RV(0), RV(0)};
                    }
            }
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
            if (!ok[e]) continue;
            RV pn = RV(0);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                o[e][c].re += RO(acc[e][c].re);
                o[e][c].im += RO(acc[e][c].im);
                pn += RV(o[e][c].re) * RV(o[e][c].re) + RV(o[e][c].im) * RV(o[e][c].im);
            }
            nrm += double(pn);
            OutIO<RO, NC>::store(outr, base + tid + (long long)BT * e, o[e]);
        }
    }
    if (norm_partial != nullptr) {
        nrm = warp_sum(nrm);
        if ((tid & 31) == 0) sred[tid >> 5] = nrm;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < NWARP; ++q) s += sred[q];
            norm_partial[(size_t)r * nblk + b] = s;
        }
    }
}

// --------------------------------------------------------------- small ops
__global__ void k_reduce(const double2* __restrict__ partial, int nblk, int J, int nrhs, double2* __restrict__ out,
                         long long out_stride, int accumulate, const int* __restrict__ active) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= J * nrhs) return;
    const int r = idx / J, i = idx % J;
    if (active != nullptr && active[r] == 0) return;
    double sx = 0.0, sy = 0.0;
    for (int b = 0; b < nblk; ++b) {
        double2 p = partial[((size_t)r * nblk + b) * J + i];
        sx += p.x;
        sy += p.y;
    }
    double2* o = out + r * out_stride + i;
    if (accumulate) {
        double2 v = *o;
        *o = make_double2(v.x + sx, v.y + sy);
    } else {
        *o = make_double2(sx, sy);
    }
}

constexpr double kBreakdownTol = 1e-12;  // relative to ||H_j||_F; rounding of an exactly
                                         // invariant space is ~100 eps at N ~ 1e5

__global__ void k_finalize(const double* __restrict__ norm_partial, int nblk, int nrhs, double2* __restrict__ H,
                           long long h_rhs_stride, int ldh, int j, double* __restrict__ hnorm2,
                           double* __restrict__ inv_beta, int* __restrict__ active, int* __restrict__ k_used) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs || active[r] == 0) return;
    double b2 = 0.0;
    for (int b = 0; b < nblk; ++b) b2 += norm_partial[(size_t)r * nblk + b];
    const double beta = sqrt(b2);
    double2* col = H + r * h_rhs_stride + (long long)j * ldh;
    double c2 = 0.0;
    for (int i = 0; i <= j; ++i) c2 += col[i].x * col[i].x + col[i].y * col[i].y;
    const double hn2 = hnorm2[r] + c2 + b2;
    hnorm2[r] = hn2;
    k_used[r] = j + 1;
    if (!(beta > kBreakdownTol * sqrt(hn2))) {
        // invariant Krylov space (or NaN): stop this right-hand side here
        col[j + 1] = make_double2(0.0, 0.0);
        inv_beta[r] = 0.0;
        active[r] = 0;
    } else {
        col[j + 1] = make_double2(beta, 0.0);
        inv_beta[r] = 1.0 / beta;
    }
}

__global__ void k_init_beta(const double* __restrict__ norm_partial, int nblk, int nrhs, double* __restrict__ beta,
                            double* __restrict__ inv_beta, double* __restrict__ hnorm2, int* __restrict__ active,
                            int* __restrict__ k_used) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs) return;
    double b2 = 0.0;
    for (int b = 0; b < nblk; ++b) b2 += norm_partial[(size_t)r * nblk + b];
    const double bt = sqrt(b2);
    beta[r] = bt;
    hnorm2[r] = 0.0;
    k_used[r] = 0;
    if (bt > 0.0 && bt == bt) {
        inv_beta[r] = 1.0 / bt;
        active[r] = 1;
    } else {
        inv_beta[r] = 0.0;
        active[r] = 0;
    }
}

template <typename R>
__global__ void k_scale(const typename Unit<R>::vec* __restrict__ in, long long in_rhs_stride,
                        typename Unit<R>::vec* __restrict__ out, long long out_rhs_stride, long long nunits,
                        const double* __restrict__ inv_beta, const int* __restrict__ active) {
    const int r = blockIdx.y;
    if (active != nullptr && active[r] == 0) return;
    const R s = R(inv_beta[r]);
    const typename Unit<R>::vec* a = in + r * in_rhs_stride;
    typename Unit<R>::vec* o = out + r * out_rhs_stride;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < nunits;
         u += (long long)gridDim.x * blockDim.x) {
        typename Unit<R>::vec v = a[u];
        if constexpr (Unit<R>::ncplx == 1) {
            v.x *= s; v.y *= s;
        } else {
            v.x *= s; v.y *= s; v.z *= s; v.w *= s;
        }
        o[u] = v;
    }
}

__global__ void k_sign_scale(const double2* __restrict__ c, const double* __restrict__ sgn, int m, int nrhs,
                             double2* __restrict__ out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m * nrhs) return;
    const int i = idx % m;
    double2 v = c[idx];
    out[idx] = make_double2(sgn[i] * v.x, sgn[i] * v.y);
}

// ------------------------------------------------------------------ launch
BlasPlan blas_plan(long long nunits, int nrhs, int num_sms) {
    BlasPlan p;
    long long want = std::max<long long>(1, (8LL * num_sms + nrhs - 1) / nrhs);
    long long chunk = (nunits + want - 1) / want;
    chunk = ((chunk + BT - 1) / BT) * BT;  // whole warps per block
    if (chunk < BT) chunk = BT;
    p.chunk = chunk;
    p.nblk = (int)((nunits + chunk - 1) / chunk);
    return p;
}

static bool g_attr_done = false;
static void set_smem_attrs() {
    if (g_attr_done) return;
    const int big = 200 * 1024;
    cudaFuncSetAttribute(k_dots<double, 2, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_dots<float, 2, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_update<double, double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_update<float, float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_update<float, double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    g_attr_done = true;
}

cudaError_t launch_dots(int prec, const void* basis, long long basis_rhs_stride, long long vec_stride, int J,
                        const void* w, long long w_rhs_stride, long long nunits, const BlasPlan& plan, int nrhs,
                        void* partial, const int* active, cudaStream_t st) {
    if (J <= 0) return cudaSuccess;
    set_smem_attrs();
    dim3 grid(plan.nblk, nrhs);
    size_t smem = (size_t)NWARP * J * sizeof(double2);
    if (prec == PREC_F64)
        k_dots<double, 2, 4><<<grid, BT, smem, st>>>((const double2*)basis, basis_rhs_stride, vec_stride, J,
                                                     (const double2*)w, w_rhs_stride, nunits, plan.chunk, plan.nblk,
                                                     (double2*)partial, active);
    else
        k_dots<float, 2, 4><<<grid, BT, smem, st>>>((const float4*)basis, basis_rhs_stride, vec_stride, J,
                                                    (const float4*)w, w_rhs_stride, nunits, plan.chunk, plan.nblk,
                                                    (double2*)partial, active);
    return cudaGetLastError();
}

cudaError_t launch_update(int prec_v, int prec_out, const void* basis, long long basis_rhs_stride,
                          long long vec_stride, int J, const int* Jdev, const void* coef, long long coef_stride,
                          double alpha, const void* in, long long in_rhs_stride, void* out, long long out_rhs_stride,
                          long long nunits_v, const BlasPlan& plan, int nrhs, double* norm_partial,
                          const int* active, cudaStream_t st) {
    set_smem_attrs();
    dim3 grid(plan.nblk, nrhs);
    size_t smem = (size_t)std::max(J, 1) * sizeof(double2);
    if (prec_v == PREC_F64 && prec_out == PREC_F64) {
        k_update<double, double, 2><<<grid, BT, smem, st>>>(
            (const double2*)basis, basis_rhs_stride, vec_stride, J, Jdev, (const double2*)coef, coef_stride, alpha,
            (const cd*)in, in_rhs_stride, (cd*)out, out_rhs_stride, nunits_v, plan.chunk, plan.nblk, norm_partial,
            active);
    } else if (prec_v == PREC_F32 && prec_out == PREC_F32) {
        k_update<float, float, 2><<<grid, BT, smem, st>>>(
            (const float4*)basis, basis_rhs_stride, vec_stride, J, Jdev, (const double2*)coef, coef_stride, alpha,
            (const cf*)in, in_rhs_stride, (cf*)out, out_rhs_stride, nunits_v, plan.chunk, plan.nblk, norm_partial,
            active);
    } else if (prec_v == PREC_F32 && prec_out == PREC_F64) {
        k_update<float, double, 2><<<grid, BT, smem, st>>>(
            (const float4*)basis, basis_rhs_stride, vec_stride, J, Jdev, (const double2*)coef, coef_stride, alpha,
            (const cd*)in, in_rhs_stride, (cd*)out, out_rhs_stride, nunits_v, plan.chunk, plan.nblk, norm_partial,
            active);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_reduce(const void* partial, int nblk, int J, int nrhs, void* out, long long out_stride,
                          bool accumulate, const int* active, cudaStream_t st) {
    if (J <= 0) return cudaSuccess;
    const int n = J * nrhs;
    k_reduce<<<(n + 127) / 128, 128, 0, st>>>((const double2*)partial, nblk, J, nrhs, (double2*)out, out_stride,
                                              accumulate ? 1 : 0, active);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const double* norm_partial, int nblk, int nrhs, void* H, long long h_rhs_stride,
                            int ldh, int j, double* hnorm2, double* inv_beta, int* active, int* k_used,
                            cudaStream_t st) {
    k_finalize<<<(nrhs + 63) / 64, 64, 0, st>>>(norm_partial, nblk, nrhs, (double2*)H, h_rhs_stride, ldh, j, hnorm2,
                                                inv_beta, active, k_used);
    return cudaGetLastError();
}

cudaError_t launch_init_beta(const double* norm_partial, int nblk, int nrhs, double* beta, double* inv_beta,
                             double* hnorm2, int* active, int* k_used, cudaStream_t st) {
    k_init_beta<<<(nrhs + 63) / 64, 64, 0, st>>>(norm_partial, nblk, nrhs, beta, inv_beta, hnorm2, active, k_used);
    return cudaGetLastError();
}

cudaError_t launch_scale(int prec, const void* in, long long in_rhs_stride, void* out, long long out_rhs_stride,
                         long long nunits, const double* inv_beta, int nrhs, const int* active, cudaStream_t st) {
    long long blocks = std::min<long long>((nunits + 255) / 256, 4096);
    dim3 grid((unsigned)std::max<long long>(blocks, 1), nrhs);
    if (prec == PREC_F64)
        k_scale<double><<<grid, 256, 0, st>>>((const double2*)in, in_rhs_stride, (double2*)out, out_rhs_stride,
                                              nunits, inv_beta, active);
    else
        k_scale<float><<<grid, 256, 0, st>>>((const float4*)in, in_rhs_stride, (float4*)out, out_rhs_stride, nunits,
                                             inv_beta, active);
    return cudaGetLastError();
}

cudaError_t launch_sign_scale(const void* c, const double* sgn, int m, int nrhs, void* out, cudaStream_t st) {
    const int n = m * nrhs;
    if (n == 0) return cudaSuccess;
    k_sign_scale<<<(n + 127) / 128, 128, 0, st>>>((const double2*)c, sgn, m, nrhs, (double2*)out);
    return cudaGetLastError();
}

}  // namespace ovs
