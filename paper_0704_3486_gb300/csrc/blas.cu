// K2 (classical Gram-Schmidt sweeps of the Arnoldi recurrence, Sec. 4
// Eq. Arnoldi), K4 (recombination y += V_k c, Eq. yproj3 / fAxLRArn) and
// K5 (LR projection c = L^+ x, x_ominus = x - R c, Sec. 5.3 Eq. xdec).
//
// A field is a flat array of 16-byte units (one complex128, or two
// complex64). Each right-hand side r owns its Krylov basis; in the register
// sweeps here a block of 256 threads covers one row block of one
// right-hand side and streams every basis vector through it, so the basis
// is read once per sweep with fully coalesced 16-byte loads. They serve the
// complex128 form and the shared-basis projections; the complex64 form's
// Arnoldi sweeps and recombination are the TMA kernels of tma_sweeps.cu.
// Also here: the shared-basis combination of the deflated part
// (k_shared_combine) and the small kernels of each Arnoldi step (partial
// sums, Hessenberg column, final pass).
//
// Precision: in the complex64 form the products and the partial sums of a
// thread (2*E terms) and of a warp (a 32-lane tree) are FP32; every warp
// partial is then added into FP64, so inner products, norms and Hessenberg
// entries are accumulated in FP64 over the rest of the vector.
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

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
// Warp transpose-reduction: every lane holds M values; after five halving
// exchanges lane l holds, in v[0 .. M/32), the warp sums of the values
// with index l*(M/32) + q. Each shuffle moves one useful value, so 32
// vectors cost 31 shuffles instead of 5 x 32.
template <int CUR, int O, typename R, int M>
__device__ __forceinline__ void tr_step(R (&v)[M], bool upper) {
#pragma unroll
    for (int i = 0; i < CUR / 2; ++i) {
        const R send = upper ? v[i] : v[i + CUR / 2];
        const R keep = upper ? v[i + CUR / 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
    }
}
template <typename R, int M> __device__ __forceinline__ void transpose_reduce(R (&v)[M], int lane) {
    static_assert(M % 32 == 0, "M must be a multiple of 32");
    tr_step<M, 16>(v, (lane & 16) != 0);
    tr_step<M / 2, 8>(v, (lane & 8) != 0);
    tr_step<M / 4, 4>(v, (lane & 4) != 0);
    tr_step<M / 8, 2>(v, (lane & 2) != 0);
    tr_step<M / 16, 1>(v, (lane & 1) != 0);
}

// Gram-Schmidt inner products of one basis sweep, per right-hand side r and
// row block b: s_i = V_i^H u, and if NW == 2 also t_i = V_i^H z (i < J);
// if `extras`, also u^H u and u^H z. Output partial[r][b][S],
// S = NW*J + 2: s_0..s_{J-1}, t_0..t_{J-1}, (u^H u, 0), u^H z.
// A lane keeps E 16-byte units of u (and z) in registers (a tile of 256*E
// units per block); G basis vectors are then streamed past them. Each lane
// accumulates its E*NC products per vector in FP32 (FP64 for complex128
// fields), a warp transpose-reduction finishes the partial over the 32
// lanes (at most 32*E*NC = 512 terms in FP32), and the warp partials are
// accumulated in FP64 in shared memory.
template <typename R, int NW, int G, int E>
__global__ void __launch_bounds__(BT, sizeof(R) == 4 ? 2 : 1) k_gdots(const typename Unit<R>::vec* __restrict__ basis,
                                              long long basis_rhs_stride, long long vec_stride, int J,
                                              const typename Unit<R>::vec* __restrict__ u, long long u_rhs_stride,
                                              const typename Unit<R>::vec* __restrict__ z, long long z_rhs_stride,
                                              int extras, long long nunits, long long chunk, int nblk,
                                              double2* __restrict__ partial, const int* __restrict__ active) {
    using vec = typename Unit<R>::vec;
    constexpr int NC = Unit<R>::ncplx;
    constexpr int M = 2 * NW * G;
    constexpr int PER = M / 32;
    extern __shared__ double2 sacc2[];  // [NWARP][S]
    double* sacc = reinterpret_cast<double*>(sacc2);
    const int r = blockIdx.x, b = blockIdx.y;
    if (active != nullptr && active[r] == 0) return;
    const int S = NW * J + 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < NWARP * S * 2; i += BT) sacc[i] = 0.0;
    __syncthreads();
    const vec* Vr = basis + r * basis_rhs_stride;
    const vec* ur = u + r * u_rhs_stride;
    const vec* zr = (NW == 2) ? z + r * z_rhs_stride : nullptr;
    double* myacc = sacc + (size_t)warp * S * 2;
    const long long u0 = (long long)b * chunk;
    const long long u1 = min(u0 + chunk, nunits);
    double uu = 0.0, uzr = 0.0, uzi = 0.0;
    for (long long base = u0; base < u1; base += (long long)BT * E) {
        cplx<R> uc[E][NC], zc[E][NC];
        bool ok[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const long long q = base + tid + (long long)BT * e;
            ok[e] = q < u1;
#pragma unroll
            for (int c = 0; c < NC; ++c) uc[e][c] = zc[e][c] = {R(0), R(0)};
            if (ok[e]) {
                Unit<R>::split(__ldg(ur + q), uc[e]);
                if (NW == 2) Unit<R>::split(__ldg(zr + q), zc[e]);
            }
        }
        if (extras) {
            cplx<R> a = {R(0), R(0)}, bz = {R(0), R(0)};
#pragma unroll
            for (int e = 0; e < E; ++e)
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    cfmac(a, uc[e][c], uc[e][c]);
                    if (NW == 2) cfmac(bz, uc[e][c], zc[e][c]);
                }
            uu += double(a.re);
            uzr += double(bz.re);
            uzi += double(bz.im);
        }
        for (int i0 = 0; i0 < J; i0 += G) {
            R v[M];
#pragma unroll
            for (int q = 0; q < M; ++q) v[q] = R(0);
#pragma unroll
            for (int gi = 0; gi < G; ++gi) {
                if (i0 + gi < J) {
                    const vec* vi = Vr + (long long)(i0 + gi) * vec_stride;
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        if (ok[e]) {
                            cplx<R> vc[NC];
                            Unit<R>::split(__ldcs(vi + base + tid + (long long)BT * e), vc);
#pragma unroll
                            for (int c = 0; c < NC; ++c) {
                                cplx<R> acc = {v[2 * gi], v[2 * gi + 1]};
                                cfmac(acc, vc[c], uc[e][c]);
                                v[2 * gi] = acc.re;
                                v[2 * gi + 1] = acc.im;
                                if (NW == 2) {
                                    cplx<R> acz = {v[2 * (G + gi)], v[2 * (G + gi) + 1]};
                                    cfmac(acz, vc[c], zc[e][c]);
                                    v[2 * (G + gi)] = acz.re;
                                    v[2 * (G + gi) + 1] = acz.im;
                                }
                            }
                        }
                    }
                }
            }
            transpose_reduce(v, lane);
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int idx = lane * PER + q;
                const int item = idx >> 1, comp = idx & 1;
                const int which = item / G, gi = item - which * G;
                if (i0 + gi < J) myacc[(which * J + i0 + gi) * 2 + comp] += double(v[q]);
            }
        }
    }
    if (extras) {
        uu = warp_sum(uu);
        uzr = warp_sum(uzr);
        uzi = warp_sum(uzi);
        if (lane == 0) {
            myacc[NW * J * 2] += uu;
            myacc[(NW * J + 1) * 2] += uzr;
            myacc[(NW * J + 1) * 2 + 1] += uzi;
        }
    }
    __syncthreads();
    for (int i = tid; i < 2 * S; i += BT) {
        double sum = 0.0;
#pragma unroll
        for (int q = 0; q < NWARP; ++q) sum += sacc[(size_t)q * S * 2 + i];
        reinterpret_cast<double*>(partial + ((size_t)r * nblk + b) * S)[i] = sum;
    }
}

// Arnoldi update sweep of the delayed-reorthogonalisation form of CGS2:
//   v_j    = (u - sum_{i<J} V_i s_i) / beta          -> basis slot J
//   u_next = (z - sum_{i<J} V_i t_i) / beta - v_j d  -> u (in place)
// s, t are read from red[r] (s at 0, t at J), 1/beta from inv_beta[r] and
// d from dcoef[r].
template <typename R, int E>
__global__ void __launch_bounds__(BT) k_arnoldi_update(typename Unit<R>::vec* __restrict__ basis,
                                                       long long basis_rhs_stride, long long vec_stride, int J,
                                                       const double2* __restrict__ red, long long red_stride,
                                                       const double* __restrict__ inv_beta,
                                                       const double2* __restrict__ dcoef,
                                                       typename Unit<R>::vec* __restrict__ u, long long u_rhs_stride,
                                                       const typename Unit<R>::vec* __restrict__ z,
                                                       long long z_rhs_stride, long long nunits, long long chunk,
                                                       const int* __restrict__ active) {
    using vec = typename Unit<R>::vec;
    constexpr int NC = Unit<R>::ncplx;
    extern __shared__ double2 scf[];
    cplx<R>* sc = reinterpret_cast<cplx<R>*>(scf);  // s at [0, J), t at [J, 2J)
    const int r = blockIdx.x, b = blockIdx.y;
    if (active != nullptr && active[r] == 0) return;
    const int tid = threadIdx.x;
    for (int i = tid; i < 2 * J; i += BT) {
        const double2 c = red[r * red_stride + i];
        sc[i] = {R(c.x), R(c.y)};
    }
    __syncthreads();
    const R ib = R(inv_beta[r]);
    const double2 dd = dcoef[r];
    const cplx<R> d = {R(dd.x), R(dd.y)};
    vec* Vr = basis + r * basis_rhs_stride;
    vec* vout = Vr + (long long)J * vec_stride;
    vec* ur = u + r * u_rhs_stride;
    const vec* zr = z + r * z_rhs_stride;
    const long long u0 = (long long)b * chunk;
    const long long u1 = min(u0 + chunk, nunits);
    for (long long base = u0; base < u1; base += (long long)BT * E) {
        cplx<R> a[E][NC], bb[E][NC];
        bool ok[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            ok[e] = base + tid + (long long)BT * e < u1;
#pragma unroll
            for (int c = 0; c < NC; ++c) a[e][c] = bb[e][c] = {R(0), R(0)};
        }
        for (int i = 0; i < J; ++i) {
            const cplx<R> si = sc[i], ti = sc[J + i];
            const vec* vi = Vr + (long long)i * vec_stride;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                if (ok[e]) {
                    cplx<R> vc[NC];
                    Unit<R>::split(__ldcs(vi + base + tid + (long long)BT * e), vc);
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        cfma(a[e][c], vc[c], si);
                        cfma(bb[e][c], vc[c], ti);
                    }
                }
            }
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
            if (!ok[e]) continue;
            const long long q = base + tid + (long long)BT * e;
            cplx<R> uc[NC], zc[NC], vo[NC], un[NC];
            Unit<R>::split(ur[q], uc);
            Unit<R>::split(__ldg(zr + q), zc);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                vo[c] = (uc[c] - a[e][c]) * ib;
                un[c] = (zc[c] - bb[e][c]) * ib;
                cplx<R> dv = cmul(vo[c], d);
                un[c] = un[c] - dv;
            }
            vout[q] = Unit<R>::join(vo);
            ur[q] = Unit<R>::join(un);
        }
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
    extern __shared__ double2 scoef2[];
    cplx<RV>* scoef = reinterpret_cast<cplx<RV>*>(scoef2);  // alpha*c, converted once per block
    __shared__ double sred[NWARP];
    const int r = blockIdx.x, b = blockIdx.y;
    if (active != nullptr && active[r] == 0) return;
    int Jr = J;
    if (Jdev != nullptr) Jr = min(J, Jdev[r]);
    const int tid = threadIdx.x;
    for (int i = tid; i < Jr; i += BT) {
        double2 c = coef[r * coef_stride + i];
        scoef[i] = {RV(alpha * c.x), RV(alpha * c.y)};
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
            const cplx<RV> ci = scoef[i];
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
__global__ void k_reduce(const double2* __restrict__ partial, int nblk, int pstride, int J, int nrhs,
                         double2* __restrict__ out, long long out_stride, int accumulate,
                         const int* __restrict__ active) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= J * nrhs) return;
    const int r = idx / J, i = idx % J;
    if (active != nullptr && active[r] == 0) return;
    double sx = 0.0, sy = 0.0;
    for (int b = 0; b < nblk; ++b) {
        double2 p = partial[((size_t)r * nblk + b) * pstride + i];
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

__device__ __forceinline__ void block_sum3(double& a, double& b, double& c, double* sh) {
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) {
        sh[3 * w] = a;
        sh[3 * w + 1] = b;
        sh[3 * w + 2] = c;
    }
    __syncthreads();
    a = b = c = 0.0;
    for (int q = 0; q < nw; ++q) {
        a += sh[3 * q];
        b += sh[3 * q + 1];
        c += sh[3 * q + 2];
    }
    __syncthreads();
}

// One Arnoldi step in the delayed-reorthogonalisation form of CGS2 (one
// block per right-hand side). Input red[r] = (s, t, u^H u, u^H z) from the
// sweep over V_0..V_{j-1} (s = V^H u, t = V^H z, z = A u), where u is the
// first-pass Gram-Schmidt residual of the previous step (x_ominus at j=0).
//  - beta = ||u - V s|| = sqrt(u^H u - ||s||^2) (V orthonormal);
//  - j > 0: column j-1 of H gets its second-pass correction s and
//    H[j][j-1] = beta; breakdown if beta <= 1e-12 ||H_j||_F (k_used = j);
//  - j = 0: beta is ||x_ominus|| (kept in beta0 for the result);
//  - column j, first pass: with g = Hbar_{j-1} s (Arnoldi relation
//    A V_{j-1} = V_j Hbar_{j-1}), H[i][j] = (t_i - g_i)/beta for i < j and
//    H[j][j] = (u^H z - s^H t)/beta^2 - g_j/beta (k_arnoldi_column, the
//    O(j^2) part, spread over many blocks);
//  - the update sweep then needs 1/beta and d = (u^H z - s^H t)/beta^2.
__global__ void __launch_bounds__(256) k_arnoldi_step(const double2* __restrict__ red, long long red_stride, int j,
                                                      double2* __restrict__ H, long long h_rhs, int ldh,
                                                      double* __restrict__ beta0, double* __restrict__ inv_beta,
                                                      double2* __restrict__ dcoef, double* __restrict__ hnorm2,
                                                      int* __restrict__ active, int* __restrict__ k_used) {
    __shared__ double sh[3 * 8];
    const int r = blockIdx.x, tid = threadIdx.x;
    if (active[r] == 0) return;
    const double2* rr = red + r * red_stride;
    double2* Hr = H + r * h_rhs;
    double ss = 0.0, shr = 0.0, shi = 0.0;
    for (int i = tid; i < j; i += blockDim.x) {
        const double2 si = rr[i], ti = rr[j + i];
        ss += si.x * si.x + si.y * si.y;
        shr += si.x * ti.x + si.y * ti.y;
        shi += si.x * ti.y - si.y * ti.x;
    }
    block_sum3(ss, shr, shi, sh);
    const double uu = rr[2 * j].x;
    const double2 uz = rr[2 * j + 1];
    const double b2 = uu - ss;
    // a NaN (from a non-finite source) stays NaN, so that it is reported
    const double beta = (b2 > 0.0 || isnan(b2)) ? sqrt(b2) : 0.0;
    if (j == 0) {
        if (tid == 0) {
            beta0[r] = beta;
            hnorm2[r] = 0.0;
        }
        if (!(beta > 0.0) || !isfinite(beta)) {
            if (tid == 0) {
                active[r] = 0;
                k_used[r] = 0;
                inv_beta[r] = 0.0;
            }
            return;
        }
    } else {
        for (int i = tid; i < j; i += blockDim.x) {
            double2 h = Hr[i + (long long)(j - 1) * ldh];
            const double2 si = rr[i];
            Hr[i + (long long)(j - 1) * ldh] = make_double2(h.x + si.x, h.y + si.y);
        }
        __syncthreads();
        double c2 = 0.0, z1 = 0.0, z2 = 0.0;
        for (int i = tid; i < j; i += blockDim.x) {
            const double2 h = Hr[i + (long long)(j - 1) * ldh];
            c2 += h.x * h.x + h.y * h.y;
        }
        block_sum3(c2, z1, z2, sh);
        const double hn2 = hnorm2[r] + c2 + beta * beta;
        const bool brk = !(beta > kBreakdownTol * sqrt(hn2)) || !isfinite(beta);
        if (tid == 0) {
            hnorm2[r] = hn2;
            Hr[j + (long long)(j - 1) * ldh] = make_double2(brk ? 0.0 : beta, 0.0);
            if (brk) {
                active[r] = 0;
                k_used[r] = j;
                inv_beta[r] = 0.0;
            }
        }
        if (brk) return;
        __syncthreads();
    }
    const double ib = 1.0 / beta;
    const double dr = (uz.x - shr) * ib * ib, di = (uz.y - shi) * ib * ib;
    if (tid == 0) {
        inv_beta[r] = ib;
        dcoef[r] = make_double2(dr, di);
        k_used[r] = j + 1;
    }
}

// Column j of H, first pass (after k_arnoldi_step of the same j): with
// g = Hbar_{j-1} s, H[l][j] = (t_l - g_l)/beta for l < j and
// H[j][j] = d - g_j/beta. One warp per row l: the lanes split the terms of
// g_l (H is upper Hessenberg, so i >= l - 1) and reduce with shuffles.
// Grid: x = groups of 8 rows, y = right-hand side.
__global__ void __launch_bounds__(256) k_arnoldi_column(const double2* __restrict__ red, long long red_stride, int j,
                                                        double2* __restrict__ H, long long h_rhs, int ldh,
                                                        const double* __restrict__ inv_beta,
                                                        const double2* __restrict__ dcoef,
                                                        const int* __restrict__ active) {
    const int r = blockIdx.y, lane = threadIdx.x & 31;
    const int l = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (active[r] == 0 || l > j) return;  // stopped (breakdown, zero source) or past the column
    const double2* rr = red + r * red_stride;
    double2* Hr = H + r * h_rhs;
    double gr = 0.0, gi = 0.0;
    for (int i = (l > 0 ? l - 1 : 0) + lane; i < j; i += 32) {
        const double2 h = Hr[l + (long long)i * ldh];
        const double2 si = rr[i];
        gr += h.x * si.x - h.y * si.y;
        gi += h.x * si.y + h.y * si.x;
    }
    for (int off = 16; off > 0; off >>= 1) {
        gr += __shfl_xor_sync(0xffffffffu, gr, off);
        gi += __shfl_xor_sync(0xffffffffu, gi, off);
    }
    if (lane != 0) return;
    const double ib = inv_beta[r];
    if (l < j) {
        const double2 ti = rr[j + l];
        Hr[l + (long long)j * ldh] = make_double2((ti.x - gr) * ib, (ti.y - gi) * ib);
    } else {
        const double2 d = dcoef[r];
        Hr[j + (long long)j * ldh] = make_double2(d.x - gr * ib, d.y - gi * ib);
    }
}

// Second Gram-Schmidt pass of the last column: red[r] holds s at [0, k) and
// u^H u at entry uu_at, from a sweep over V_0..V_{k-1};
// H[:k][k-1] += s, H[k][k-1] = ||u - V s||.
__global__ void __launch_bounds__(256) k_arnoldi_final(const double2* __restrict__ red, long long red_stride, int k,
                                                       int uu_at, double2* __restrict__ H, long long h_rhs, int ldh,
                                                       const int* __restrict__ active) {
    __shared__ double sh[3 * 8];
    const int r = blockIdx.x, tid = threadIdx.x;
    if (active[r] == 0) return;
    const double2* rr = red + r * red_stride;
    double2* Hr = H + r * h_rhs;
    double ss = 0.0, z1 = 0.0, z2 = 0.0;
    for (int i = tid; i < k; i += blockDim.x) {
        const double2 si = rr[i];
        const double2 h = Hr[i + (long long)(k - 1) * ldh];
        Hr[i + (long long)(k - 1) * ldh] = make_double2(h.x + si.x, h.y + si.y);
        ss += si.x * si.x + si.y * si.y;
    }
    block_sum3(ss, z1, z2, sh);
    if (tid == 0) {
        const double b2 = rr[uu_at].x - ss;
        Hr[k + (long long)(k - 1) * ldh] = make_double2(b2 > 0.0 ? sqrt(b2) : 0.0, 0.0);
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

// ------------------------------------------------------- shared-basis dots
// Inner products against a complex64 basis shared by all right-hand sides
// (the LR projection L^+ x, the Schur projections S^H z of every Arnoldi
// step): partial[(r*nblk + b)*pstride + i] = sum over the units of chunk b
// of S_i^H z_r, i < m, r < nrhs. A block takes one chunk of units and stages
// it KD units at a time, every S_i and every z_r, in shared memory by
// asynchronous 16-byte copies (cp.async), two stages deep: the copies of
// tile t+1 are in flight while tile t is multiplied, so a block keeps
// (m + nrhs) KD 16-byte units in flight without registers. Stage layout
// vector-major with a row pitch of KD+1 units: the copies write consecutive
// units, and the threads of a quarter warp, reading 8 consecutive vectors
// at one unit, fall on 8 distinct 4-bank groups. Each thread accumulates a
// tile of 4 basis vectors x 2 right-hand sides: FP32 over one staged tile
// (2 KD complex terms), FP64 across tiles. Each element of the basis is
// read from memory once per call, not once per right-hand side.
constexpr int KD = 32;
constexpr int KP = KD + 1;  // row pitch of a staged vector, in units

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int n = valid ? 16 : 0;  // 0: nothing is read, the 16 bytes are zero-filled
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__global__ void __launch_bounds__(BT) k_shared_dots(const float4* __restrict__ S, long long svec, int m,
                                                    const float4* __restrict__ Z, long long zstride, int nrhs,
                                                    long long nunits, long long chunk, int nblk,
                                                    double2* __restrict__ partial, int pstride,
                                                    const int* __restrict__ active) {
    extern __shared__ float4 sd_smem[];
    const int rows = m + nrhs;  // staged vectors: S_0 .. S_(m-1), then z_0 .. z_(nrhs-1)
    const size_t stage = (size_t)rows * KP;
    const int b = blockIdx.x, tid = threadIdx.x;
    const long long u0 = (long long)b * chunk;
    const long long u1 = min(u0 + chunk, nunits);
    const int itiles = (m + 3) / 4, rtiles = (nrhs + 1) / 2;
    const int ti = tid % itiles, tr = tid / itiles;
    const bool work = tr < rtiles;
    double acc[4][2][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 2; ++c) acc[a][c][0] = acc[a][c][1] = 0.0;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    // copies of the tile at unit t0 into stage buffer st (zero beyond u1)
    auto issue = [&](long long t0, int st) {
        float4* dst = sd_smem + st * stage;
        for (int idx = tid; idx < rows * KD; idx += BT) {
            const int row = idx / KD, u = idx - row * KD;
            const bool valid = t0 + u < u1;
            const float4* src = row < m ? S + (size_t)row * svec : Z + (size_t)(row - m) * zstride;
            cp_async16(dst + (size_t)row * KP + u, valid ? src + t0 + u : S, valid);
        }
        cp_async_commit();
    };
    const long long ntile = (u1 - u0 + KD - 1) / KD;
    if (ntile > 0) issue(u0, 0);
    for (long long t = 0; t < ntile; ++t) {
        if (t + 1 < ntile) {
            issue(u0 + (t + 1) * KD, (int)((t + 1) & 1));
            cp_async_wait<1>();  // tile t has landed (tile t+1 may still be in flight)
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const float4* sS = sd_smem + (t & 1) * stage;
        const float4* sZ = sS + (size_t)m * KP;
        const int cnt = (int)min((long long)KD, u1 - (u0 + t * KD));
        if (work) {
            float a32[4][2][2];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 2; ++c) a32[a][c][0] = a32[a][c][1] = 0.f;
            for (int u = 0; u < cnt; ++u) {
                float4 sv[4], zv[2];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int i = ti + q * itiles;
                    sv[q] = (i < m) ? sS[(size_t)i * KP + u] : zero;
                }
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int r = tr + q * rtiles;
                    zv[q] = (r < nrhs) ? sZ[(size_t)r * KP + u] : zero;
                }
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 2; ++c) {  // conj(s) z for the two complex numbers of the unit
                        float re = a32[a][c][0], im = a32[a][c][1];
                        re = fmaf(sv[a].x, zv[c].x, re);
                        re = fmaf(sv[a].y, zv[c].y, re);
                        re = fmaf(sv[a].z, zv[c].z, re);
                        re = fmaf(sv[a].w, zv[c].w, re);
                        im = fmaf(sv[a].x, zv[c].y, im);
                        im = fmaf(-sv[a].y, zv[c].x, im);
                        im = fmaf(sv[a].z, zv[c].w, im);
                        im = fmaf(-sv[a].w, zv[c].z, im);
                        a32[a][c][0] = re;
                        a32[a][c][1] = im;
                    }
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    acc[a][c][0] += (double)a32[a][c][0];
                    acc[a][c][1] += (double)a32[a][c][1];
                }
        }
        __syncthreads();  // stage (t & 1) is refilled by the copies issued in the next iteration
    }
    if (!work) return;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int i = ti + a * itiles, r = tr + c * rtiles;
            if (i >= m || r >= nrhs) continue;
            if (active != nullptr && active[r] == 0) continue;
            partial[((size_t)r * nblk + b) * pstride + i] = make_double2(acc[a][c][0], acc[a][c][1]);
        }
}

static size_t shared_dots_smem(int m, int nrhs) { return 2 * (size_t)(m + nrhs) * KP * sizeof(float4); }

// Blocks of the shared-basis dots for nunits within the partial slots
// available: as many per SM as their two stages fit (at most 4); 0 when the
// tile does not fit (the register sweep k_gdots serves then).
int shared_dots_blocks(int m, int nrhs, long long nunits, int num_sms, int max_blocks) {
    const int itiles = (m + 3) / 4, rtiles = (nrhs + 1) / 2;
    if (m < 1 || nrhs < 1 || (long long)itiles * rtiles > BT) return 0;
    const size_t smem = shared_dots_smem(m, nrhs);
    if (smem > 200 * 1024) return 0;
    const long long per_sm = std::max<long long>(1, std::min<long long>(4, (long long)(220 * 1024) / (long long)smem));
    long long want = per_sm * num_sms;
    want = std::min<long long>(want, std::max<long long>(1, nunits / KD));
    want = std::min<long long>(want, max_blocks);
    return want < 1 ? 0 : (int)want;
}

cudaError_t launch_shared_dots(const void* S, long long svec, int m, const void* Z, long long zstride, int nrhs,
                               long long nunits, int nblk, void* partial, int pstride, const int* active,
                               cudaStream_t st) {
    const size_t smem = shared_dots_smem(m, nrhs);
    cudaError_t e = ensure_dyn_smem((const void*)k_shared_dots, 200 * 1024);
    if (e != cudaSuccess) return e;
    long long chunk = (nunits + nblk - 1) / nblk;
    chunk = ((chunk + KD - 1) / KD) * KD;
    k_shared_dots<<<nblk, BT, smem, st>>>((const float4*)S, svec, m, (const float4*)Z, zstride, nrhs, nunits, chunk,
                                         nblk, (double2*)partial, pstride, active);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ launch
BlasPlan blas_plan(long long nunits, int nrhs, int num_sms) {
    BlasPlan p;
    long long want = std::max<long long>(1, (8LL * num_sms + nrhs - 1) / nrhs);
    long long chunk = (nunits + want - 1) / want;
    const long long tile = (long long)BT * 8;  // one inner-product tile of 8 units per thread
    chunk = ((chunk + tile - 1) / tile) * tile;
    p.chunk = chunk;
    p.nblk = (int)((nunits + chunk - 1) / chunk);
    return p;
}

cudaError_t ensure_dyn_smem(const void* kernel, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> granted;  // (kernel, device) -> bytes
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = granted[std::make_pair(kernel, dev)];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

// the register sweeps keep their reduction buffers (up to 200 KB) in
// dynamic shared memory
static void set_smem_attrs() {
    const size_t big = 200 * 1024;
    ensure_dyn_smem((const void*)k_gdots<double, 1, 16, 4>, big);
    ensure_dyn_smem((const void*)k_gdots<double, 2, 8, 4>, big);
    ensure_dyn_smem((const void*)k_gdots<float, 1, 16, 4>, big);
    ensure_dyn_smem((const void*)k_gdots<float, 2, 8, 4>, big);
    ensure_dyn_smem((const void*)k_arnoldi_update<double, 2>, big);
    ensure_dyn_smem((const void*)k_arnoldi_update<float, 2>, big);
    ensure_dyn_smem((const void*)k_update<double, double, 2>, big);
    ensure_dyn_smem((const void*)k_update<float, float, 2>, big);
    ensure_dyn_smem((const void*)k_update<float, double, 2>, big);
}

int gdots_stride(int nw, int J) { return nw * J + 2; }

cudaError_t launch_gdots(int prec, int nw, const void* basis, long long basis_rhs_stride, long long vec_stride,
                         int J, const void* u, long long u_rhs_stride, const void* z, long long z_rhs_stride,
                         bool extras, long long nunits, const BlasPlan& plan, int nrhs, void* partial,
                         const int* active, cudaStream_t st) {
    set_smem_attrs();
    dim3 grid(nrhs, plan.nblk);  // right-hand side fastest: a shared basis is re-read from L2
    const size_t smem = (size_t)NWARP * gdots_stride(nw, J) * sizeof(double2);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    const int ex = extras ? 1 : 0;
    if (prec == PREC_F64) {
        if (nw == 1)
            k_gdots<double, 1, 16, 4><<<grid, BT, smem, st>>>((const double2*)basis, basis_rhs_stride, vec_stride, J,
                                                              (const double2*)u, u_rhs_stride, nullptr, 0, ex, nunits,
                                                              plan.chunk, plan.nblk, (double2*)partial, active);
        else
            k_gdots<double, 2, 8, 4><<<grid, BT, smem, st>>>((const double2*)basis, basis_rhs_stride, vec_stride, J,
                                                             (const double2*)u, u_rhs_stride, (const double2*)z,
                                                             z_rhs_stride, ex, nunits, plan.chunk, plan.nblk,
                                                             (double2*)partial, active);
    } else {
        if (nw == 1)
            k_gdots<float, 1, 16, 4><<<grid, BT, smem, st>>>((const float4*)basis, basis_rhs_stride, vec_stride, J,
                                                             (const float4*)u, u_rhs_stride, nullptr, 0, ex, nunits,
                                                             plan.chunk, plan.nblk, (double2*)partial, active);
        else
            k_gdots<float, 2, 8, 4><<<grid, BT, smem, st>>>((const float4*)basis, basis_rhs_stride, vec_stride, J,
                                                             (const float4*)u, u_rhs_stride, (const float4*)z,
                                                             z_rhs_stride, ex, nunits, plan.chunk, plan.nblk,
                                                             (double2*)partial, active);
    }
    return cudaGetLastError();
}

cudaError_t launch_arnoldi_update(int prec, void* basis, long long basis_rhs_stride, long long vec_stride, int J,
                                  const void* red, long long red_stride, const double* inv_beta, const void* dcoef,
                                  void* u, long long u_rhs_stride, const void* z, long long z_rhs_stride,
                                  long long nunits, const BlasPlan& plan, int nrhs, const int* active,
                                  cudaStream_t st) {
    set_smem_attrs();
    dim3 grid(nrhs, plan.nblk);  // right-hand side fastest: a shared basis is re-read from L2
    const size_t smem = (size_t)std::max(2 * J, 1) * sizeof(double2);
    if (prec == PREC_F64)
        k_arnoldi_update<double, 2><<<grid, BT, smem, st>>>((double2*)basis, basis_rhs_stride, vec_stride, J,
                                                            (const double2*)red, red_stride, inv_beta,
                                                            (const double2*)dcoef, (double2*)u, u_rhs_stride,
                                                            (const double2*)z, z_rhs_stride, nunits, plan.chunk,
                                                            active);
    else
        k_arnoldi_update<float, 2><<<grid, BT, smem, st>>>((float4*)basis, basis_rhs_stride, vec_stride, J,
                                                           (const double2*)red, red_stride, inv_beta,
                                                           (const double2*)dcoef, (float4*)u, u_rhs_stride,
                                                           (const float4*)z, z_rhs_stride, nunits, plan.chunk,
                                                           active);
    return cudaGetLastError();
}

cudaError_t launch_arnoldi_step(const void* red, long long red_stride, int j, void* H, long long h_rhs, int ldh,
                                double* beta0, double* inv_beta, void* dcoef, double* hnorm2, int* active,
                                int* k_used, int nrhs, cudaStream_t st) {
    k_arnoldi_step<<<nrhs, 256, 0, st>>>((const double2*)red, red_stride, j, (double2*)H, h_rhs, ldh, beta0, inv_beta,
                                         (double2*)dcoef, hnorm2, active, k_used);
    return cudaGetLastError();
}

cudaError_t launch_arnoldi_column(const void* red, long long red_stride, int j, void* H, long long h_rhs, int ldh,
                                  const double* inv_beta, const void* dcoef, const int* active, int nrhs,
                                  cudaStream_t st) {
    const dim3 grid((j + 1 + 7) / 8, nrhs);
    k_arnoldi_column<<<grid, 256, 0, st>>>((const double2*)red, red_stride, j, (double2*)H, h_rhs, ldh, inv_beta,
                                           (const double2*)dcoef, active);
    return cudaGetLastError();
}

cudaError_t launch_arnoldi_final(const void* red, long long red_stride, int k, int uu_at, void* H, long long h_rhs,
                                 int ldh, const int* active, int nrhs, cudaStream_t st) {
    k_arnoldi_final<<<nrhs, 256, 0, st>>>((const double2*)red, red_stride, k, uu_at, (double2*)H, h_rhs, ldh, active);
    return cudaGetLastError();
}

cudaError_t launch_update(int prec_v, int prec_out, const void* basis, long long basis_rhs_stride,
                          long long vec_stride, int J, const int* Jdev, const void* coef, long long coef_stride,
                          double alpha, const void* in, long long in_rhs_stride, void* out, long long out_rhs_stride,
                          long long nunits_v, const BlasPlan& plan, int nrhs, double* norm_partial,
                          const int* active, cudaStream_t st) {
    set_smem_attrs();
    dim3 grid(nrhs, plan.nblk);  // right-hand side fastest: a shared basis is re-read from L2
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

// Shared-basis combination for all right-hand sides (the deflation part of
// Sec. 5.3: x - R c and R sgn(Lambda) c, with R the complex64 copy of the
// deflation basis): out_r = [in_r] + alpha * sum_{i < m} R_i c_{r,i}.
// A block takes a tile of BT*2 units and a group of SG right-hand sides;
// blocks are numbered with the group fastest, so the SG-groups of a tile
// run together and R is read from DRAM once and from L2 by the other
// groups. The vector loop is unrolled by 4 (8 loads in flight per thread);
// products are FP32, and for a complex128 output the FP32 partial sums are
// added into FP64 accumulators every 16 vectors.
constexpr int SG = 4;
template <typename RO>
__global__ void __launch_bounds__(BT) k_shared_combine(const float4* __restrict__ R, long long vec_stride, int m,
                                                       const double2* __restrict__ coef, long long coef_stride,
                                                       double alpha, const cplx<RO>* in, long long in_rhs_stride,
                                                       cplx<RO>* out, long long out_rhs_stride, long long nunits,
                                                       int nrhs, int ngroups) {
    extern __shared__ double2 smc[];
    cf* sc = reinterpret_cast<cf*>(smc);  // [SG][m] alpha * c
    const int grp = blockIdx.x % ngroups;
    const long long tile = blockIdx.x / ngroups;
    const int r0 = grp * SG;
    const int nr = min(SG, nrhs - r0);
    const int tid = threadIdx.x;
    for (int i = tid; i < SG * m; i += BT) {
        const int q = i / m, v = i - q * m;
        const double2 c = q < nr ? coef[(long long)(r0 + q) * coef_stride + v] : make_double2(0.0, 0.0);
        sc[i] = {float(alpha * c.x), float(alpha * c.y)};
    }
    __syncthreads();
    long long u[2];
    bool ok[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        u[e] = tile * (2 * BT) + tid + (long long)BT * e;
        ok[e] = u[e] < nunits;
    }
    cplx<RO> o[SG][2][2];
    cf acc[SG][2][2];
#pragma unroll
    for (int q = 0; q < SG; ++q)
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                o[q][e][c] = {RO(0), RO(0)};
                acc[q][e][c] = {0.f, 0.f};
            }
    auto flush = [&]() {
#pragma unroll
        for (int q = 0; q < SG; ++q)
#pragma unroll
            for (int e = 0; e < 2; ++e)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    o[q][e][c].re += RO(acc[q][e][c].re);
                    o[q][e][c].im += RO(acc[q][e][c].im);
                    acc[q][e][c] = {0.f, 0.f};
                }
    };
    int i = 0;
    for (; i + 4 <= m; i += 4) {
        float4 v[4][2];
#pragma unroll
        for (int d = 0; d < 4; ++d)
#pragma unroll
            for (int e = 0; e < 2; ++e)
                v[d][e] = ok[e] ? __ldg(R + (long long)(i + d) * vec_stride + u[e]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int d = 0; d < 4; ++d)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                cf vc[2];
                Unit<float>::split(v[d][e], vc);
#pragma unroll
                for (int q = 0; q < SG; ++q) {
                    const cf cq = sc[q * m + i + d];
#pragma unroll
                    for (int c = 0; c < 2; ++c) cfma(acc[q][e][c], vc[c], cq);
                }
            }
        if (sizeof(RO) > 4 && ((i + 4) & 15) == 0) flush();
    }
    for (; i < m; ++i) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const float4 v = ok[e] ? __ldg(R + (long long)i * vec_stride + u[e]) : make_float4(0.f, 0.f, 0.f, 0.f);
            cf vc[2];
            Unit<float>::split(v, vc);
#pragma unroll
            for (int q = 0; q < SG; ++q) {
                const cf cq = sc[q * m + i];
#pragma unroll
                for (int c = 0; c < 2; ++c) cfma(acc[q][e][c], vc[c], cq);
            }
        }
    }
    flush();
#pragma unroll
    for (int q = 0; q < SG; ++q) {
        if (q >= nr) break;
        const int r = r0 + q;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            if (!ok[e]) continue;
            cplx<RO> res[2];
            if (in != nullptr) OutIO<RO, 2>::load(in + (long long)r * in_rhs_stride, u[e], res);
            else res[0] = res[1] = {RO(0), RO(0)};
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                res[c].re += o[q][e][c].re;
                res[c].im += o[q][e][c].im;
            }
            OutIO<RO, 2>::store(out + (long long)r * out_rhs_stride, u[e], res);
        }
    }
}

cudaError_t launch_shared_combine(int prec_out, const void* R, long long vec_stride, int m, const void* coef,
                                  long long coef_stride, double alpha, const void* in, long long in_rhs_stride,
                                  void* out, long long out_rhs_stride, long long nunits, int nrhs, cudaStream_t st) {
    if (m < 1 || nrhs < 1) return cudaErrorInvalidValue;
    const int ngroups = (nrhs + SG - 1) / SG;
    const long long tiles = (nunits + 2 * BT - 1) / (2 * BT);
    const long long blocks = tiles * ngroups;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const size_t smem = (size_t)SG * m * sizeof(cf);
    if (smem > 48 * 1024) return cudaErrorInvalidValue;
    if (prec_out == PREC_F64)
        k_shared_combine<double><<<(unsigned)blocks, BT, smem, st>>>(
            (const float4*)R, vec_stride, m, (const double2*)coef, coef_stride, alpha, (const cd*)in, in_rhs_stride,
            (cd*)out, out_rhs_stride, nunits, nrhs, ngroups);
    else
        k_shared_combine<float><<<(unsigned)blocks, BT, smem, st>>>(
            (const float4*)R, vec_stride, m, (const double2*)coef, coef_stride, alpha, (const cf*)in, in_rhs_stride,
            (cf*)out, out_rhs_stride, nunits, nrhs, ngroups);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const void* partial, int nblk, int pstride, int J, int nrhs, void* out,
                          long long out_stride, bool accumulate, const int* active, cudaStream_t st) {
    if (J <= 0) return cudaSuccess;
    const int n = J * nrhs;
    k_reduce<<<(n + 127) / 128, 128, 0, st>>>((const double2*)partial, nblk, pstride, J, nrhs, (double2*)out,
                                              out_stride, accumulate ? 1 : 0, active);
    return cudaGetLastError();
}

cudaError_t launch_sign_scale(const void* c, const double* sgn, int m, int nrhs, void* out, cudaStream_t st) {
    const int n = m * nrhs;
    if (n == 0) return cudaSuccess;
    k_sign_scale<<<(n + 127) / 128, 128, 0, st>>>((const double2*)c, sgn, m, nrhs, (double2*)out);
    return cudaGetLastError();
}

}  // namespace ovs
