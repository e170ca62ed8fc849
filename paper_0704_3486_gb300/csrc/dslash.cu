// K1: the Wilson-Dirac stencil at chemical potential, H_w(mu) = gamma5 D_w(mu)
// (Sec. 2, Eqs. Dov and Dw), and K7: field layout conversions.
//
// A thread block is a tile of sites (threadIdx.x) times a tile of
// right-hand sides (threadIdx.y): the warps of one block work on the same
// sites for different right-hand sides, so a link reaches shared L1 once per
// block and not once per right-hand side. A thread may in addition take RT
// right-hand sides (RT = 1 or 2), loading each link once for them. Each of
// the eight hops projects
// the neighbour's 4-spinor onto the rank-2 subspace of (1 -/+ gamma_nu)
// (a 2 x 3 half spinor), multiplies the two colour vectors by U (forward)
// or U^+ (backward), scales by kappa-independent factors (e^{+/-mu} on
// temporal hops, -1 on hops that wrap in t) and adds the reconstructed
// 4-spinor. The diagonal term and gamma5 are applied in the store.
//
// Chiral basis: gamma_k = [[0, -i s_k], [i s_k, 0]], gamma_4 = [[0,1],[1,0]],
// so with upper = spins (0,1) and lower = spins (2,3):
//   (1 - gamma_k) psi = [h; -i s_k h],   h = psi_up + i s_k psi_dn
//   (1 + gamma_k) psi = [h;  i s_k h],   h = psi_up - i s_k psi_dn
//   (1 - gamma_4) psi = [h; -h],         h = psi_up - psi_dn
//   (1 + gamma_4) psi = [h;  h],         h = psi_up + psi_dn
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace ovs {

// ------------------------------------------------------------- field access
template <typename R> struct Field;
template <> struct Field<double> {
    __device__ __forceinline__ static void load(const void* f, int V, int s, cd (&p)[12]) {
        const double2* d = static_cast<const double2*>(f);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const double2* u = d + 2 * ((size_t)q * V + s);
            double2 a = __ldg(u), b = __ldg(u + 1);
            p[2 * q] = {a.x, a.y};
            p[2 * q + 1] = {b.x, b.y};
        }
    }
    __device__ __forceinline__ static void store(void* f, int V, int s, const cd (&p)[12]) {
        double2* d = static_cast<double2*>(f);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            double2* u = d + 2 * ((size_t)q * V + s);
            u[0] = make_double2(p[2 * q].re, p[2 * q].im);
            u[1] = make_double2(p[2 * q + 1].re, p[2 * q + 1].im);
        }
    }
    __device__ __forceinline__ static void link(const void* u, int V, int nu, int s, cd (&m)[9]) {
        const double2* d = static_cast<const double2*>(u) + (size_t)nu * 9 * V;
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            double2 v = __ldg(d + (size_t)e * V + s);
            m[e] = {v.x, v.y};
        }
    }
};
template <> struct Field<float> {
    __device__ __forceinline__ static void load(const void* f, int V, int s, cf (&p)[12]) {
        const float4* d = static_cast<const float4*>(f);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            float4 v = __ldg(d + (size_t)q * V + s);
            p[2 * q] = {v.x, v.y};
            p[2 * q + 1] = {v.z, v.w};
        }
    }
    __device__ __forceinline__ static void store(void* f, int V, int s, const cf (&p)[12]) {
        float4* d = static_cast<float4*>(f);
#pragma unroll
        for (int q = 0; q < 6; ++q)
            d[(size_t)q * V + s] = make_float4(p[2 * q].re, p[2 * q].im, p[2 * q + 1].re, p[2 * q + 1].im);
    }
    // complex64 links: per direction four float4 planes holding the entries
    // (0,1) (2,3) (4,5) (6,7) of U (row-major 3x3), at float4 plane 4 nu + q;
    // the ninth entry of every direction in float2 planes after those 16
    // planes (float2 plane 32 + nu). Five loads per link instead of nine.
    __device__ __forceinline__ static void link(const void* u, int V, int nu, int s, cf (&m)[9]) {
        const float4* d = static_cast<const float4*>(u) + (size_t)nu * 4 * V;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 v = __ldg(d + (size_t)q * V + s);
            m[2 * q] = {v.x, v.y};
            m[2 * q + 1] = {v.z, v.w};
        }
        const float2 w = __ldg(static_cast<const float2*>(u) + (size_t)(32 + nu) * V + s);
        m[8] = {w.x, w.y};
    }
};

// --------------------------------------------------------------------- hops
// Forward hop: acc += (1 - gamma_NU) * fac * U * psi
template <int NU, typename R>
__device__ __forceinline__ void hop_fwd(const cplx<R> (&p)[12], const cplx<R> (&U)[9], R fac, cplx<R> (&acc)[12]) {
    cplx<R> h0[3], h1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cplx<R> a0 = p[c], a1 = p[3 + c], a2 = p[6 + c], a3 = p[9 + c];
        if (NU == 0) { h0[c] = a0 + ti(a3); h1[c] = a1 + ti(a2); }
        if (NU == 1) { h0[c] = a0 + a3;     h1[c] = a1 - a2; }
        if (NU == 2) { h0[c] = a0 + ti(a2); h1[c] = a1 - ti(a3); }
        if (NU == 3) { h0[c] = a0 - a2;     h1[c] = a1 - a3; }
        h0[c] = h0[c] * fac;
        h1[c] = h1[c] * fac;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        cplx<R> u0 = {R(0), R(0)}, u1 = {R(0), R(0)};
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            cfma(u0, U[3 * a + b], h0[b]);
            cfma(u1, U[3 * a + b], h1[b]);
        }
        acc[a] = acc[a] + u0;
        acc[3 + a] = acc[3 + a] + u1;
        if (NU == 0) { acc[6 + a] = acc[6 + a] + tmi(u1); acc[9 + a] = acc[9 + a] + tmi(u0); }
        if (NU == 1) { acc[6 + a] = acc[6 + a] - u1;      acc[9 + a] = acc[9 + a] + u0; }
        if (NU == 2) { acc[6 + a] = acc[6 + a] + tmi(u0); acc[9 + a] = acc[9 + a] + ti(u1); }
        if (NU == 3) { acc[6 + a] = acc[6 + a] - u0;      acc[9 + a] = acc[9 + a] - u1; }
    }
}

// Backward hop: acc += (1 + gamma_NU) * fac * U^+ * psi, U the link of the
// backward neighbour in direction NU.
template <int NU, typename R>
__device__ __forceinline__ void hop_bwd(const cplx<R> (&p)[12], const cplx<R> (&U)[9], R fac, cplx<R> (&acc)[12]) {
    cplx<R> h0[3], h1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cplx<R> a0 = p[c], a1 = p[3 + c], a2 = p[6 + c], a3 = p[9 + c];
        if (NU == 0) { h0[c] = a0 + tmi(a3); h1[c] = a1 + tmi(a2); }
        if (NU == 1) { h0[c] = a0 - a3;      h1[c] = a1 + a2; }
        if (NU == 2) { h0[c] = a0 + tmi(a2); h1[c] = a1 + ti(a3); }
        if (NU == 3) { h0[c] = a0 + a2;      h1[c] = a1 + a3; }
        h0[c] = h0[c] * fac;
        h1[c] = h1[c] * fac;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        cplx<R> u0 = {R(0), R(0)}, u1 = {R(0), R(0)};
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            cfmac(u0, U[3 * b + a], h0[b]);
            cfmac(u1, U[3 * b + a], h1[b]);
        }
        acc[a] = acc[a] + u0;
        acc[3 + a] = acc[3 + a] + u1;
        if (NU == 0) { acc[6 + a] = acc[6 + a] + ti(u1); acc[9 + a] = acc[9 + a] + ti(u0); }
        if (NU == 1) { acc[6 + a] = acc[6 + a] + u1;     acc[9 + a] = acc[9 + a] - u0; }
        if (NU == 2) { acc[6 + a] = acc[6 + a] + ti(u0); acc[9 + a] = acc[9 + a] + tmi(u1); }
        if (NU == 3) { acc[6 + a] = acc[6 + a] + u0;     acc[9 + a] = acc[9 + a] + u1; }
    }
}

// Operands of one hop: the link and the neighbour spinors of the tile.
template <typename R, int RT> struct HopData {
    cplx<R> U[9];
    cplx<R> p[RT][12];
    R fac;
};

// Load the operands of the forward (FWD) or backward hop in direction NU:
// U_NU(s) and psi(s + NU), or U_NU(s - NU) and psi(s - NU); the factor is
// e^{+mu} / e^{-mu} on temporal hops (efwd / ebwd) and -1 on hops that
// wrap in time (antiperiodic).
template <int NU, bool FWD, typename R, int RT>
__device__ __forceinline__ void hop_load(const void* links, const char* in, size_t in_stride, int r0,
                                         const bool (&live)[RT], const Geom& g, int s, int coord, R efwd, R ebwd,
                                         HopData<R, RT>& d) {
    const int L = g.L[NU], st = g.stride[NU];
    int sn;
    if (FWD) {
        sn = (coord == L - 1) ? s - (L - 1) * st : s + st;
        d.fac = (NU == 3 && coord == L - 1) ? -efwd : efwd;
        Field<R>::link(links, g.V, NU, s, d.U);
    } else {
        sn = (coord == 0) ? s + (L - 1) * st : s - st;
        d.fac = (NU == 3 && coord == 0) ? -ebwd : ebwd;
        Field<R>::link(links, g.V, NU, sn, d.U);
    }
#pragma unroll
    for (int i = 0; i < RT; ++i)
        if (live[i]) Field<R>::load(in + (size_t)(r0 + i) * in_stride, g.V, sn, d.p[i]);
}

template <int NU, bool FWD, typename R, int RT>
__device__ __forceinline__ void hop_apply(const HopData<R, RT>& d, const bool (&live)[RT], cplx<R> (&acc)[RT][12]) {
#pragma unroll
    for (int i = 0; i < RT; ++i) {
        if (!live[i]) continue;
        if (FWD)
            hop_fwd<NU>(d.p[i], d.U, d.fac, acc[i]);
        else
            hop_bwd<NU>(d.p[i], d.U, d.fac, acc[i]);
    }
}

// Optional epilogue of the stencil: out = ah * (stencil result) + bx * X + by * Y
// (used by the Chebyshev filter of the eigensolver set-up).
struct Axpy {
    const char* X;
    size_t xs;
    double bx;
    const char* Y;
    size_t ys;
    double by;
    double ah;
};

// out_r = [gamma5] (in_r - kappa * hops(in_r)) for the right-hand sides r
// of the thread. in/out strides are in bytes between right-hand sides.
// Blocks are numbered with the right-hand-side tile fastest, so the blocks
// of all tiles that share a tile of sites (and of links) run back to back.
template <typename R, bool G5, int RT, bool AX = false>
__global__ void __launch_bounds__(256) k_wilson(const void* __restrict__ links, const char* __restrict__ in,
                                                char* out, size_t in_stride, size_t out_stride, Geom g,
                                                R kappa, R emu, R emmu, int nrhs, int ntiles,
                                                const int* __restrict__ active, Axpy ax = Axpy{}) {
    const int tile = blockIdx.x % ntiles;
    const int s = (blockIdx.x / ntiles) * blockDim.x + threadIdx.x;
    const int r0 = (tile * blockDim.y + threadIdx.y) * RT;
    if (s >= g.V || r0 >= nrhs) return;
    bool live[RT];
    bool any = false;
#pragma unroll
    for (int i = 0; i < RT; ++i) {
        live[i] = (r0 + i < nrhs) && (active == nullptr || active[r0 + i] != 0);
        any = any || live[i];
    }
    if (!any) return;
    int c = s;
    const int x = c % g.L[0]; c /= g.L[0];
    const int y = c % g.L[1]; c /= g.L[1];
    const int z = c % g.L[2];
    const int t = c / g.L[2];
    cplx<R> acc[RT][12];
#pragma unroll
    for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int q = 0; q < 12; ++q) acc[i][q] = {R(0), R(0)};
    // the eight hops in a two-deep pipeline (RT = 1): the operands of the next
    // hop are loaded before the current one is computed
    HopData<R, RT> A, B;
    const R one = R(1);
    if (RT > 1) {  // registers of two RT-tiles in flight would spill: one hop at a time
        hop_load<0, true>(links, in, in_stride, r0, live, g, s, x, one, one, A);
        hop_apply<0, true>(A, live, acc);
        hop_load<0, false>(links, in, in_stride, r0, live, g, s, x, one, one, A);
        hop_apply<0, false>(A, live, acc);
        hop_load<1, true>(links, in, in_stride, r0, live, g, s, y, one, one, A);
        hop_apply<1, true>(A, live, acc);
        hop_load<1, false>(links, in, in_stride, r0, live, g, s, y, one, one, A);
        hop_apply<1, false>(A, live, acc);
        hop_load<2, true>(links, in, in_stride, r0, live, g, s, z, one, one, A);
        hop_apply<2, true>(A, live, acc);
        hop_load<2, false>(links, in, in_stride, r0, live, g, s, z, one, one, A);
        hop_apply<2, false>(A, live, acc);
        hop_load<3, true>(links, in, in_stride, r0, live, g, s, t, emu, emmu, A);
        hop_apply<3, true>(A, live, acc);
        hop_load<3, false>(links, in, in_stride, r0, live, g, s, t, emu, emmu, A);
        hop_apply<3, false>(A, live, acc);
    } else {
    hop_load<0, true>(links, in, in_stride, r0, live, g, s, x, one, one, A);
    hop_load<0, false>(links, in, in_stride, r0, live, g, s, x, one, one, B);
    hop_apply<0, true>(A, live, acc);
    hop_load<1, true>(links, in, in_stride, r0, live, g, s, y, one, one, A);
    hop_apply<0, false>(B, live, acc);
    hop_load<1, false>(links, in, in_stride, r0, live, g, s, y, one, one, B);
    hop_apply<1, true>(A, live, acc);
    hop_load<2, true>(links, in, in_stride, r0, live, g, s, z, one, one, A);
    hop_apply<1, false>(B, live, acc);
    hop_load<2, false>(links, in, in_stride, r0, live, g, s, z, one, one, B);
    hop_apply<2, true>(A, live, acc);
    hop_load<3, true>(links, in, in_stride, r0, live, g, s, t, emu, emmu, A);
    hop_apply<2, false>(B, live, acc);
    hop_load<3, false>(links, in, in_stride, r0, live, g, s, t, emu, emmu, B);
    hop_apply<3, true>(A, live, acc);
    hop_apply<3, false>(B, live, acc);
    }
#pragma unroll
    for (int i = 0; i < RT; ++i) {
        if (!live[i]) continue;
        const int r = r0 + i;
        cplx<R> p[12];
        Field<R>::load(in + (size_t)r * in_stride, g.V, s, p);
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            cplx<R> v = p[q] - acc[i][q] * kappa;
            if (G5 && q >= 6) v = -v;
            p[q] = v;
        }
        if (AX) {
            cplx<R> xv[12], yv[12];
            Field<R>::load(ax.X + (size_t)r * ax.xs, g.V, s, xv);
            Field<R>::load(ax.Y + (size_t)r * ax.ys, g.V, s, yv);
            const R ah = R(ax.ah), bx = R(ax.bx), by = R(ax.by);
#pragma unroll
            for (int q = 0; q < 12; ++q) p[q] = p[q] * ah + xv[q] * bx + yv[q] * by;
        }
        Field<R>::store(out + (size_t)r * out_stride, g.V, s, p);
    }
}

// Flat precision conversion of internal fields (the two layouts pair up).
__global__ void k_f64_to_f32(const double2* __restrict__ a, float2* __restrict__ b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double2 v = a[i];
        b[i] = make_float2(float(v.x), float(v.y));
    }
}
__global__ void k_f32_to_f64(const float2* __restrict__ a, double2* __restrict__ b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float2 v = a[i];
        b[i] = make_double2(double(v.x), double(v.y));
    }
}

// Uniform (-1, 1) real and imaginary parts from a 64-bit mixing hash of
// (seed, index) (splitmix64 finaliser); used for random starting blocks.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__global__ void k_random_fill(double2* __restrict__ q, long long n, uint64_t seed) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const uint64_t a = mix64(seed * 0x9E3779B97F4A7C15ULL + 2 * (uint64_t)i + 1);
        const uint64_t b = mix64(a + 0x632BE59BD9B4E019ULL);
        q[i] = make_double2(((a >> 11) + 0.5) * 0x1p-52 - 1.0, ((b >> 11) + 0.5) * 0x1p-52 - 1.0);
    }
}

// ------------------------------------------------------------ layouts (K7)
// canonical complex128 [nrhs][V][12]  ->  internal planes of precision R
template <typename R>
__global__ void k_to_internal(const double2* __restrict__ canon, size_t canon_stride, char* __restrict__ out,
                              size_t out_stride, int V) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (s >= V) return;
    const double2* src = canon + r * canon_stride + (size_t)s * 12;
    cplx<R> p[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        double2 v = src[q];
        p[q] = {R(v.x), R(v.y)};
    }
    Field<R>::store(out + r * out_stride, V, s, p);
}

// internal planes of precision R -> canonical complex128
template <typename R>
__global__ void k_to_canonical(const char* __restrict__ in, size_t in_stride, double2* __restrict__ canon,
                               size_t canon_stride, int V) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (s >= V) return;
    cplx<R> p[12];
    Field<R>::load(in + r * in_stride, V, s, p);
    double2* dst = canon + r * canon_stride + (size_t)s * 12;
#pragma unroll
    for (int q = 0; q < 12; ++q) dst[q] = make_double2(double(p[q].re), double(p[q].im));
}

// D_ov(mu) y = x + gamma5 sgn(H_w) x (Sec. 2, Eq. Dov) fused into the last
// layout pass: in holds sgn(H_w) x in internal complex128 planes, x is the
// canonical source; gamma5 = diag(1, 1, -1, -1) flips the entries of spin
// 2 and 3 (spin*3 + colour >= 6).
__global__ void k_to_canonical_overlap(const char* __restrict__ in, size_t in_stride,
                                       const double2* __restrict__ x, size_t x_stride, double2* __restrict__ canon,
                                       size_t canon_stride, int V) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (s >= V) return;
    cplx<double> p[12];
    Field<double>::load(in + r * in_stride, V, s, p);
    const double2* xs = x + r * x_stride + (size_t)s * 12;
    double2* dst = canon + r * canon_stride + (size_t)s * 12;
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        const double2 xv = xs[q];
        const double g = q < 6 ? 1.0 : -1.0;
        dst[q] = make_double2(fma(g, p[q].re, xv.x), fma(g, p[q].im, xv.y));
    }
}

// canonical links complex128 [V][4][3][3] -> planes [nu][e][V] (complex128 and,
// if u32 != nullptr, complex64)
__global__ void k_links_to_internal(const double2* __restrict__ canon, double2* __restrict__ u64,
                                    float2* __restrict__ u32, int V) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
#pragma unroll
    for (int nu = 0; nu < 4; ++nu)
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            double2 v = canon[((size_t)s * 4 + nu) * 9 + e];
            u64[((size_t)nu * 9 + e) * V + s] = v;
            if (u32 != nullptr) {  // complex64 layout of Field<float>::link
                const size_t i = e < 8 ? ((size_t)(nu * 4 + e / 2) * V + s) * 2 + (e & 1) : (size_t)(32 + nu) * V + s;
                u32[i] = make_float2(float(v.x), float(v.y));
            }
        }
}

__global__ void k_links_to_canonical(const double2* __restrict__ u64, double2* __restrict__ canon, int V) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
#pragma unroll
    for (int nu = 0; nu < 4; ++nu)
#pragma unroll
        for (int e = 0; e < 9; ++e) canon[((size_t)s * 4 + nu) * 9 + e] = u64[((size_t)nu * 9 + e) * V + s];
}

// ------------------------------------------------------------- host launch
static inline dim3 site_grid(int V, int nrhs, int threads) { return dim3((V + threads - 1) / threads, nrhs); }

static bool valid_shape(const StencilShape& sh) {
    for (int i = 0; i < kNumStencilShapes; ++i)
        if (kStencilShapes[i].rt == sh.rt && kStencilShapes[i].sites == sh.sites && kStencilShapes[i].rb == sh.rb)
            return true;
    return false;
}

template <typename R, bool G5, bool AX>
static void wilson_dispatch(const StencilShape& sh, unsigned blocks, int ntiles, cudaStream_t st, const void* links,
                            const void* in, size_t in_stride, void* out, size_t out_stride, const Geom& g,
                            double kappa, double emu, double emmu, int nrhs, const int* active, const Axpy& ax) {
    const R k = (R)kappa, e1 = (R)emu, e2 = (R)emmu;
    const char* i = (const char*)in;
    char* o = (char*)out;
    const dim3 block(sh.sites, sh.rb);
    if (sh.rt == 1)
        k_wilson<R, G5, 1, AX><<<blocks, block, 0, st>>>(links, i, o, in_stride, out_stride, g, k, e1, e2, nrhs, ntiles,
                                                           active, ax);
    else
        k_wilson<R, G5, 2, AX><<<blocks, block, 0, st>>>(links, i, o, in_stride, out_stride, g, k, e1, e2, nrhs, ntiles,
                                                           active, ax);
}

cudaError_t launch_wilson(int prec, bool gamma5, const void* links, const void* in, size_t in_stride, void* out,
                          size_t out_stride, const Geom& g, int nrhs, double kappa, double mu, const int* active,
                          cudaStream_t st, StencilShape sh) {
    if (!valid_shape(sh)) return cudaErrorInvalidValue;
    const int ntiles = (nrhs + sh.rt * sh.rb - 1) / (sh.rt * sh.rb);
    const long long blocks = (long long)ntiles * ((g.V + sh.sites - 1) / sh.sites);
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const double emu = exp(mu), emmu = exp(-mu);
    const Axpy ax{};
    if (prec == PREC_F64) {
        if (gamma5)
            wilson_dispatch<double, true, false>(sh, (unsigned)blocks, ntiles, st, links, in, in_stride, out,
                                                 out_stride, g, kappa, emu, emmu, nrhs, active, ax);
        else
            wilson_dispatch<double, false, false>(sh, (unsigned)blocks, ntiles, st, links, in, in_stride, out,
                                                  out_stride, g, kappa, emu, emmu, nrhs, active, ax);
    } else {
        if (gamma5)
            wilson_dispatch<float, true, false>(sh, (unsigned)blocks, ntiles, st, links, in, in_stride, out,
                                                out_stride, g, kappa, emu, emmu, nrhs, active, ax);
        else
            wilson_dispatch<float, false, false>(sh, (unsigned)blocks, ntiles, st, links, in, in_stride, out,
                                                 out_stride, g, kappa, emu, emmu, nrhs, active, ax);
    }
    return cudaGetLastError();
}

cudaError_t launch_wilson_axpy(int prec, const void* links, const void* in, size_t in_stride, void* out,
                               size_t out_stride, const void* X, size_t xs, double bx, const void* Y, size_t ys,
                               double by, double ah, const Geom& g, int nrhs, double kappa, double mu,
                               cudaStream_t st, StencilShape sh) {
    if (!valid_shape(sh)) return cudaErrorInvalidValue;
    const int ntiles = (nrhs + sh.rt * sh.rb - 1) / (sh.rt * sh.rb);
    const long long blocks = (long long)ntiles * ((g.V + sh.sites - 1) / sh.sites);
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const double emu = exp(mu), emmu = exp(-mu);
    const Axpy ax{(const char*)X, xs, bx, (const char*)Y, ys, by, ah};
    if (prec == PREC_F64)
        wilson_dispatch<double, true, true>(sh, (unsigned)blocks, ntiles, st, links, in, in_stride, out, out_stride,
                                            g, kappa, emu, emmu, nrhs, nullptr, ax);
    else
        wilson_dispatch<float, true, true>(sh, (unsigned)blocks, ntiles, st, links, in, in_stride, out, out_stride,
                                           g, kappa, emu, emmu, nrhs, nullptr, ax);
    return cudaGetLastError();
}

cudaError_t launch_convert(int to_prec, const void* in, void* out, long long ncplx, cudaStream_t st) {
    const int blocks = (int)std::min<long long>((ncplx + 255) / 256, 8192);
    if (to_prec == PREC_F32)
        k_f64_to_f32<<<blocks, 256, 0, st>>>((const double2*)in, (float2*)out, ncplx);
    else
        k_f32_to_f64<<<blocks, 256, 0, st>>>((const float2*)in, (double2*)out, ncplx);
    return cudaGetLastError();
}

cudaError_t launch_random_fill(void* q, long long ncplx, uint64_t seed, cudaStream_t st) {
    const int blocks = (int)std::min<long long>((ncplx + 255) / 256, 8192);
    k_random_fill<<<blocks, 256, 0, st>>>((double2*)q, ncplx, seed);
    return cudaGetLastError();
}

cudaError_t launch_to_internal(int prec, const void* canon, size_t canon_stride_cplx, void* out, size_t out_stride,
                               int V, int nrhs, cudaStream_t st) {
    dim3 grid = site_grid(V, nrhs, 128);
    if (prec == PREC_F64)
        k_to_internal<double><<<grid, 128, 0, st>>>((const double2*)canon, canon_stride_cplx, (char*)out, out_stride, V);
    else
        k_to_internal<float><<<grid, 128, 0, st>>>((const double2*)canon, canon_stride_cplx, (char*)out, out_stride, V);
    return cudaGetLastError();
}

cudaError_t launch_to_canonical(int prec, const void* in, size_t in_stride, void* canon, size_t canon_stride_cplx,
                                int V, int nrhs, cudaStream_t st) {
    dim3 grid = site_grid(V, nrhs, 128);
    if (prec == PREC_F64)
        k_to_canonical<double><<<grid, 128, 0, st>>>((const char*)in, in_stride, (double2*)canon, canon_stride_cplx, V);
    else
        k_to_canonical<float><<<grid, 128, 0, st>>>((const char*)in, in_stride, (double2*)canon, canon_stride_cplx, V);
    return cudaGetLastError();
}

cudaError_t launch_to_canonical_overlap(const void* in, size_t in_stride, const void* x, size_t x_stride_cplx,
                                        void* canon, size_t canon_stride_cplx, int V, int nrhs, cudaStream_t st) {
    dim3 grid = site_grid(V, nrhs, 128);
    k_to_canonical_overlap<<<grid, 128, 0, st>>>((const char*)in, in_stride, (const double2*)x, x_stride_cplx,
                                                 (double2*)canon, canon_stride_cplx, V);
    return cudaGetLastError();
}

cudaError_t launch_links_to_internal(const void* canon, void* u64, void* u32, int V, cudaStream_t st) {
    k_links_to_internal<<<(V + 127) / 128, 128, 0, st>>>((const double2*)canon, (double2*)u64, (float2*)u32, V);
    return cudaGetLastError();
}

cudaError_t launch_links_to_canonical(const void* u64, void* canon, int V, cudaStream_t st) {
    k_links_to_canonical<<<(V + 127) / 128, 128, 0, st>>>((const double2*)u64, (double2*)canon, V);
    return cudaGetLastError();
}

}  // namespace ovs
