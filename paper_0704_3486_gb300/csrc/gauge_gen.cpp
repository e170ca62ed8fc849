// Host generator of the seeded synthetic SU(3) field behind ovs_create_gauge.
//
// Per link l = 4 s + nu: nine Philox4x32-10 calls (Salmon et al., SC'11) with
// counter (l mod 2^32, l div 2^32, j, 0), j = 0..8, and key (seed mod 2^32,
// seed div 2^32). Call j yields two uniforms u = (floor(w / 2^12) + 1/2) 2^-52
// from the 64-bit words (w1:w0) and (w3:w2), and the Box-Muller pair
// r cos(2 pi u1), r sin(2 pi u1), r = sqrt(-2 ln u0): normals 2j, 2j+1.
// A[a][b] = n[2(3a+b)] + i n[2(3a+b)+1]; X = traceless Hermitian part of A;
// U = exp(i eps X) by a degree-18 Taylor series with scaling and squaring
// (scale so that the Frobenius norm is <= 1/2); then rows are reunitarised
// and row 2 is set to conj(row0 x row1), which makes det U = 1.
#include <cmath>
#include <complex>
#include <cstdint>
#include <thread>
#include <vector>

namespace ovs {

using cdouble = std::complex<double>;

static inline void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    for (int round = 0; round < 10; ++round) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c[1] ^ k0;
        const uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

static inline double uniform52(uint32_t lo, uint32_t hi) {
    const uint64_t w = ((uint64_t)hi << 32) | (uint64_t)lo;
    return ((double)(w >> 12) + 0.5) * 0x1p-52;
}

struct M3 {
    cdouble a[3][3];
};

static inline M3 mul(const M3& x, const M3& y) {
    M3 z;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cdouble s = 0.0;
            for (int k = 0; k < 3; ++k) s += x.a[i][k] * y.a[k][j];
            z.a[i][j] = s;
        }
    return z;
}

static M3 expm_taylor(const M3& m) {
    double nrm2 = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) nrm2 += std::norm(m.a[i][j]);
    const double nrm = std::sqrt(nrm2);
    int s = 0;
    if (nrm > 0.5) s = (int)std::ceil(std::log2(nrm / 0.5));
    while (nrm / std::ldexp(1.0, s) > 0.5) ++s;
    const double scale = std::ldexp(1.0, s);
    M3 ms;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) ms.a[i][j] = m.a[i][j] / scale;
    M3 result, term;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) result.a[i][j] = term.a[i][j] = (i == j) ? 1.0 : 0.0;
    for (int n = 1; n <= 18; ++n) {
        term = mul(term, ms);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                term.a[i][j] /= (double)n;
                result.a[i][j] += term.a[i][j];
            }
    }
    for (int q = 0; q < s; ++q) result = mul(result, result);
    return result;
}

static M3 reunitarise(const M3& u) {
    cdouble r0[3], r1[3], r2[3];
    double n0 = 0.0;
    for (int j = 0; j < 3; ++j) n0 += std::norm(u.a[0][j]);
    n0 = std::sqrt(n0);
    for (int j = 0; j < 3; ++j) r0[j] = u.a[0][j] / n0;
    cdouble d = 0.0;
    for (int j = 0; j < 3; ++j) d += std::conj(r0[j]) * u.a[1][j];
    for (int j = 0; j < 3; ++j) r1[j] = u.a[1][j] - d * r0[j];
    double n1 = 0.0;
    for (int j = 0; j < 3; ++j) n1 += std::norm(r1[j]);
    n1 = std::sqrt(n1);
    for (int j = 0; j < 3; ++j) r1[j] /= n1;
    r2[0] = std::conj(r0[1] * r1[2] - r0[2] * r1[1]);
    r2[1] = std::conj(r0[2] * r1[0] - r0[0] * r1[2]);
    r2[2] = std::conj(r0[0] * r1[1] - r0[1] * r1[0]);
    M3 o;
    for (int j = 0; j < 3; ++j) {
        o.a[0][j] = r0[j];
        o.a[1][j] = r1[j];
        o.a[2][j] = r2[j];
    }
    return o;
}

static void one_link(uint64_t l, uint64_t seed, double eps, double* out) {
    double n[18];
    const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu), k1 = (uint32_t)(seed >> 32);
    for (uint32_t j = 0; j < 9; ++j) {
        uint32_t c[4] = {(uint32_t)(l & 0xFFFFFFFFu), (uint32_t)(l >> 32), j, 0u};
        philox4x32_10(c, k0, k1);
        const double u0 = uniform52(c[0], c[1]);
        const double u1 = uniform52(c[2], c[3]);
        const double r = std::sqrt(-2.0 * std::log(u0));
        n[2 * j] = r * std::cos(6.283185307179586 * u1);
        n[2 * j + 1] = r * std::sin(6.283185307179586 * u1);
    }
    M3 a, x;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) a.a[i][j] = cdouble(n[2 * (3 * i + j)], n[2 * (3 * i + j) + 1]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) x.a[i][j] = 0.5 * (a.a[i][j] + std::conj(a.a[j][i]));
    const cdouble tr = (x.a[0][0] + x.a[1][1] + x.a[2][2]) / 3.0;
    for (int i = 0; i < 3; ++i) x.a[i][i] -= tr;
    M3 m;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) m.a[i][j] = cdouble(0.0, eps) * x.a[i][j];
    const M3 u = reunitarise(expm_taylor(m));
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            out[2 * (3 * i + j)] = u.a[i][j].real();
            out[2 * (3 * i + j) + 1] = u.a[i][j].imag();
        }
}

// links: 72 * V doubles, canonical [V][4][3][3] complex128.
void generate_links(long long V, uint64_t seed, double eps, double* links) {
    const long long nl = 4 * V;
    unsigned nt = std::thread::hardware_concurrency();
    if (nt == 0) nt = 1;
    if (nt > 64) nt = 64;
    if (nl < 4096) nt = 1;
    std::vector<std::thread> pool;
    for (unsigned t = 0; t < nt; ++t) {
        pool.emplace_back([=]() {
            for (long long l = t; l < nl; l += nt) one_link((uint64_t)l, seed, eps, links + 18 * l);
        });
    }
    for (auto& th : pool) th.join();
}

}  // namespace ovs
