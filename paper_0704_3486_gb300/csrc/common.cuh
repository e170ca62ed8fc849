// Shared device helpers: complex arithmetic, internal field layouts, errors.
//
// Internal layouts (device only; the ABI uses the canonical site-major one):
//  - spinor field: 6 planes of V sites; plane q of site s holds the two
//    complex numbers with spin*3+colour = 2q and 2q+1, as one float4
//    (complex64) or two consecutive double2 (complex128). The 16-byte unit u
//    of a complex64 field thus holds the same two entries as units 2u and
//    2u+1 of a complex128 field, so mixed-precision sweeps line up;
//  - links, complex128: [nu][row*3+col] planes of V double2;
//  - links, complex64:  [nu][row*3+col] planes of V float2.
// A plane-major layout makes the 32 sites of a warp read 32 consecutive
// 16-byte (or 8-byte) words, so stencil loads are fully coalesced. For the
// Gram-Schmidt kernels a field is a flat array of 16-byte units
// (one complex128 or two complex64), whatever the order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ovs {

// ------------------------------------------------------------------ complex
template <typename R> struct cplx { R re, im; };
using cd = cplx<double>;
using cf = cplx<float>;

template <typename R> __host__ __device__ __forceinline__ cplx<R> mk(R a, R b) { return {a, b}; }
template <typename R> __device__ __forceinline__ cplx<R> operator+(cplx<R> a, cplx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R> __device__ __forceinline__ cplx<R> operator-(cplx<R> a, cplx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R> __device__ __forceinline__ cplx<R> operator-(cplx<R> a) { return {-a.re, -a.im}; }
template <typename R> __device__ __forceinline__ cplx<R> operator*(cplx<R> a, R s) { return {a.re * s, a.im * s}; }
template <typename R> __device__ __forceinline__ cplx<R> cmul(cplx<R> a, cplx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// conj(a) * b
template <typename R> __device__ __forceinline__ cplx<R> cmulc(cplx<R> a, cplx<R> b) {
    return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
// i * a
template <typename R> __device__ __forceinline__ cplx<R> ti(cplx<R> a) { return {-a.im, a.re}; }
// -i * a
template <typename R> __device__ __forceinline__ cplx<R> tmi(cplx<R> a) { return {a.im, -a.re}; }
// acc += a * b
template <typename R> __device__ __forceinline__ void cfma(cplx<R>& acc, cplx<R> a, cplx<R> b) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <typename R> __device__ __forceinline__ void cfmac(cplx<R>& acc, cplx<R> a, cplx<R> b) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(-a.im, b.re, acc.im);
}

// ------------------------------------------------------- 16-byte field units
// Unit<T>: one 16-byte load/store holding U complex numbers of precision R.
template <typename R> struct Unit;
template <> struct Unit<double> {
    using vec = double2;
    static constexpr int ncplx = 1;
    __device__ __forceinline__ static void split(const double2& v, cd* c) { c[0] = {v.x, v.y}; }
    __device__ __forceinline__ static double2 join(const cd* c) { return make_double2(c[0].re, c[0].im); }
};
template <> struct Unit<float> {
    using vec = float4;
    static constexpr int ncplx = 2;
    __device__ __forceinline__ static void split(const float4& v, cf* c) { c[0] = {v.x, v.y}; c[1] = {v.z, v.w}; }
    __device__ __forceinline__ static float4 join(const cf* c) { return make_float4(c[0].re, c[0].im, c[1].re, c[1].im); }
};

template <typename T> __device__ __forceinline__ T ldg_stream(const T* p) { return __ldcs(p); }

// ----------------------------------------------------------- lattice geometry
struct Geom {
    int L[4];    // Lx, Ly, Lz, Lt
    int V;
    int stride[4];  // site stride of each direction: 1, Lx, Lx*Ly, Lx*Ly*Lz
};

__host__ inline Geom make_geom(const int32_t dims[4]) {
    Geom g;
    for (int i = 0; i < 4; ++i) g.L[i] = dims[i];
    g.stride[0] = 1;
    g.stride[1] = dims[0];
    g.stride[2] = dims[0] * dims[1];
    g.stride[3] = dims[0] * dims[1] * dims[2];
    g.V = g.stride[3] * dims[3];
    return g;
}

// Status words kept on the device per right-hand side.
enum : int { RHS_ACTIVE = 1, RHS_DONE = 0 };

}  // namespace ovs
