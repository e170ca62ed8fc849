// TMA-pipelined sweeps over the complex64 Arnoldi basis: the inner products
// and the update of the delayed-reorthogonalisation step (K2), and the
// recombination y += V_k c (K4); also the self-check of the bounded waits.
//
// The sweeps stream the whole basis of every right-hand side, so they are
// bound by HBM bandwidth. All three are persistent
// (one block per SM) and warp-specialised: one producer lane moves basis
// tiles into shared memory with 1D bulk asynchronous copies (cp.async.bulk,
// completion counted in bytes on an mbarrier), 3 stages of 8 vectors x 512
// 16-byte units (64 KB each, 192 KB in flight per SM), and 8 consumer warps
// read them and hand each stage back through a second mbarrier. The
// producer refills a stage as soon as all consumer warps have released it
// (after a proxy fence, since generic loads read the buffer before the
// asynchronous copy overwrites it), so the consumers never wait for the
// copy issue and may run up to 3 stages apart.
//
// Every wait is bounded. A consumer whose wait runs out records OVS_ETIMEOUT
// in *err and raises a shared abort flag; the other waits then give up at
// once, the consumers leave together at their next common barrier, and the
// producer waits (bounded) for the copies it still has in flight before the
// block exits.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace ovs {

namespace {

constexpr int TB = 256;       // threads per block
constexpr int TW = TB / 32;   // warps
constexpr int TG = 8;         // basis vectors per stage
// update sweep: 2 units per thread per tile, 3 stages of 64 KB
constexpr int TE = 2;
constexpr int TU = TB * TE;
constexpr int TNS = 3;
constexpr size_t kStageBytes = (size_t)TG * TU * 16;
constexpr unsigned long long kWaitNs = 1000000000ull;  // a wait gives up after 1 s
constexpr int OVS_ETIMEOUT_CODE = -7;        // OVS_ETIMEOUT

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// try_wait until the phase completes or kWaitNs have passed (the clock is
// read only once the first try has failed)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > kWaitNs) return false;
    }
}
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

}  // namespace

// Inner products of the delayed-reorthogonalisation Arnoldi step, complex64
// basis: s_i = V_i^H u, t_i = V_i^H z (i < J), u^H u and u^H z.
//
// Persistent, warp-specialised form, one block per SM: 8 consumer warps and
// one producer warp. The work items are the row chunks of CU = 2048 units of
// every right-hand side, flattened as (r, c) and split into one contiguous
// range per block. For each chunk a consumer thread holds its 8 units of u
// and of z in registers; the basis streams through DS = 3 stages (192 KB in
// flight) of 8 vectors x 512 units, groups of 8 vectors in the outer order
// and the 4 tiles of the chunk inside, so a thread keeps its products of one
// group in registers across the 4 stages (16 complex terms per vector,
// FP32). A warp transpose-reduction then leaves one (item, component) per
// lane; the 8 warps' partials (512 terms each) are summed in FP64 into the
// block's accumulators.
//
// Stage hand-off uses mbarriers only: `full[s]` completes when the copies of
// stage s have landed (transaction bytes), `empty[s]` when all 8 consumer
// warps have read it. The producer (one lane) refills a stage as soon as it
// is released, so consumer warps run up to DS stages apart and none of them
// waits for the copy issue. The consumers meet on a named barrier once per
// group of 8 vectors, where they also agree on any timed-out wait.
//
// Output: the partial sums of right-hand side r go to partial[r][slot][2J+2]
// (layout of k_gdots with NW = 2, slot = block - first block of r); a block
// that starts r also zeroes r's slots beyond its last one, so every one of
// the `nslot` slots is defined.
namespace {
constexpr int CU = 2048;                     // units per row chunk
constexpr int DU = 512;                      // units per tile
constexpr int DE = DU / TB;                  // units per consumer thread per tile
constexpr int DNT = CU / DU;                 // tiles per chunk
constexpr int DS = 3;                        // stages
constexpr int DTHREADS = TB + 32;            // consumer warps + producer warp
constexpr size_t kDStage = (size_t)TG * DU * 16;

template <int CUR, int O>
__device__ __forceinline__ void tstep32(float (&v)[32], bool upper) {
#pragma unroll
    for (int i = 0; i < CUR / 2; ++i) {
        const float send = upper ? v[i] : v[i + CUR / 2];
        const float keep = upper ? v[i + CUR / 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
    }
}
__device__ __forceinline__ double wsum_d(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// named barrier 1 over the TB consumer threads; the OR of `p` over them
__device__ __forceinline__ bool consumers_sync_or(bool p) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred a, b;\n setp.ne.u32 a, %1, 0;\n bar.red.or.pred b, 1, %2, a;\n selp.u32 %0, 1, 0, b;\n}"
        : "=r"(r)
        : "r"((uint32_t)p), "n"(TB)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void consumers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(TB) : "memory"); }
// bounded wait that also gives up once another thread has raised `abort`
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort || global_ns() - t0 > kWaitNs) return false;
    }
}
// block that owns flattened item i under the contiguous split of T items
// over G blocks (block q owns [floor(qT/G), floor((q+1)T/G)))
__host__ __device__ inline int owner_of(long long i, long long T, int G) {
    return (int)(((i + 1) * G - 1) / T);
}
__host__ __device__ inline long long range_lo(int q, long long T, int G) { return (long long)q * T / G; }
}  // namespace

__global__ void __launch_bounds__(DTHREADS, 1)
    k_gdots2_ws(const float4* __restrict__ basis, long long basis_rhs_stride, long long vec_stride, int J,
                const float4* __restrict__ u, long long u_rhs_stride, const float4* __restrict__ z,
                long long z_rhs_stride, long long nunits, int nrhs, int nslot, double2* __restrict__ partial,
                const int* __restrict__ active, int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[DS];
    __shared__ __align__(8) uint64_t empty[DS];
    __shared__ float scratch[2][TW][32];
    __shared__ double sx[TW][3];
    __shared__ int abort_flag;
    double* acc = reinterpret_cast<double*>(smem + DS * kDStage);  // [2J + 2][2]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x, q = blockIdx.x;
    const int S = 2 * J + 2;
    const long long cpr = (nunits + CU - 1) / CU;  // chunks per right-hand side
    const long long T = cpr * nrhs;
    const long long lo = range_lo(q, T, G), hi = range_lo(q + 1, T, G);
    const int ngroups = (J + TG - 1) / TG;
    volatile int* abort = &abort_flag;
    if (tid == 0) {
        for (int k = 0; k < DS; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], TW);
        }
        abort_flag = 0;
        mbar_fence_init();
    }
    __syncthreads();

    if (warp == TW) {  // ---- producer warp: one lane issues every stage
        if (lane != 0 || ngroups == 0) return;
        int n = 0;  // stages issued
        bool ok = true;
        for (long long it = lo; it < hi && ok; ++it) {
            const long long r = it / cpr, c = it - r * cpr;
            if (active != nullptr && active[r] == 0) continue;
            const long long u0 = c * CU;
            const int len = (int)min((long long)CU, nunits - u0);
            const float4* Vr = basis + r * basis_rhs_stride + u0;
            for (int g = 0; g < ngroups && ok; ++g) {
                const int nv = min(TG, J - g * TG);
                for (int t = 0; t < DNT; ++t) {
                    const int s = n % DS;
                    if (n >= DS) {  // the consumers' release of this stage's previous use
                        if (!mbar_wait_or_abort(&empty[s], (uint32_t)((n / DS - 1) & 1), abort)) {
                            ok = false;
                            break;
                        }
                        fence_proxy_async_smem();
                    }
                    const int units = min(DU, len - t * DU);
                    if (units <= 0) {  // tile beyond a short chunk: complete the phase without bytes
                        mbar_expect_tx(&full[s], 0);
                    } else {
                        const uint32_t bytes = (uint32_t)units * 16u;
                        unsigned char* dst = smem + (size_t)s * kDStage;
                        mbar_expect_tx(&full[s], bytes * nv);
                        for (int v = 0; v < nv; ++v)
                            bulk_load(dst + (size_t)v * DU * 16, Vr + (long long)(g * TG + v) * vec_stride + t * DU,
                                      bytes, &full[s]);
                    }
                    ++n;
                }
            }
        }
        // the block's shared memory must outlive every copy: wait until the
        // consumers have released the last stages, or, if they gave up, until
        // the copies still in flight have landed (bounded)
        for (int k = max(0, n - DS); k < n && ok; ++k)
            ok = mbar_wait_or_abort(&empty[k % DS], (uint32_t)((k / DS) & 1), abort);
        if (!ok) {
            atomicExch(err, OVS_ETIMEOUT_CODE);
            abort_flag = 1;
            for (int k = max(0, n - DS); k < n; ++k) mbar_wait_bounded(&full[k % DS], (uint32_t)((k / DS) & 1));
        }
        return;
    }

    // ---- consumer warps
    // zero this block's share of the unused slots: the block owning the first
    // chunk of r clears r's slots past the last block that works on r
    for (long long r = 0; r < nrhs; ++r) {
        if (owner_of(r * cpr, T, G) != q) continue;
        const int used = owner_of((r + 1) * cpr - 1, T, G) - q + 1;
        double* base = reinterpret_cast<double*>(partial + ((size_t)r * nslot) * S);
        for (long long i = (long long)used * 2 * S + tid; i < (long long)nslot * 2 * S; i += TB) base[i] = 0.0;
    }
    int n = 0;   // stages consumed
    int gg = 0;  // groups completed, over all chunks (selects the scratch buffer)
    long long seg_r = -1;
    bool bad = false;
    double ea = 0.0, ebr = 0.0, ebi = 0.0;  // u^H u, u^H z of the segment (per thread)

    auto flush = [&](long long r) {
        ea = wsum_d(ea);
        ebr = wsum_d(ebr);
        ebi = wsum_d(ebi);
        if (lane == 0) {
            sx[warp][0] = ea;
            sx[warp][1] = ebr;
            sx[warp][2] = ebi;
        }
        ea = ebr = ebi = 0.0;
        consumers_sync();
        if (tid == 0) {
            double a = 0.0, br = 0.0, bi = 0.0;
            for (int w = 0; w < TW; ++w) {
                a += sx[w][0];
                br += sx[w][1];
                bi += sx[w][2];
            }
            acc[(2 * J) * 2] = a;
            acc[(2 * J) * 2 + 1] = 0.0;
            acc[(2 * J + 1) * 2] = br;
            acc[(2 * J + 1) * 2 + 1] = bi;
        }
        consumers_sync();
        const int slot = q - owner_of(r * cpr, T, G);
        double* out = reinterpret_cast<double*>(partial + ((size_t)r * nslot + slot) * S);
        for (int i = tid; i < 2 * S; i += TB) out[i] = acc[i];
        consumers_sync();
    };

    for (long long it = lo; it < hi; ++it) {
        const long long r = it / cpr, c = it - r * cpr;
        if (active != nullptr && active[r] == 0) continue;
        if (r != seg_r) {
            if (seg_r >= 0) flush(seg_r);
            for (int i = tid; i < 2 * S; i += TB) acc[i] = 0.0;
            seg_r = r;
        }
        const long long u0 = c * CU;
        const int len = (int)min((long long)CU, nunits - u0);
        float4 ur[DNT * DE], zr[DNT * DE];
        const float4* up = u + r * u_rhs_stride + u0;
        const float4* zp = z + r * z_rhs_stride + u0;
#pragma unroll
        for (int k = 0; k < DNT * DE; ++k) {
            const int p = k * TB + tid;  // tile k / DE, unit (k % DE) * TB + tid of it
            ur[k] = p < len ? up[p] : make_float4(0.f, 0.f, 0.f, 0.f);
            zr[k] = p < len ? zp[p] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < DNT * DE; ++k) {
            cf uc[2], zc[2];
            Unit<float>::split(ur[k], uc);
            Unit<float>::split(zr[k], zc);
            cf aa = {0.f, 0.f}, bz = {0.f, 0.f};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                cfmac(aa, uc[h], uc[h]);
                cfmac(bz, uc[h], zc[h]);
            }
            ea += aa.re;
            ebr += bz.re;
            ebi += bz.im;
        }
        for (int g = 0; g < ngroups; ++g) {
            float v[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) v[k] = 0.f;
            const int nv = min(TG, J - g * TG);
#pragma unroll
            for (int t = 0; t < DNT; ++t) {
                const int s = n % DS;
                const bool got = bad || mbar_wait_or_abort(&full[s], (uint32_t)((n / DS) & 1), abort);
                if (!__all_sync(0xffffffffu, got)) {  // keep `bad` uniform over the warp
                    if (lane == 0) {
                        atomicExch(err, OVS_ETIMEOUT_CODE);
                        abort_flag = 1;
                    }
                    bad = true;
                }
                if (!bad) {
                    const float4* st4 = reinterpret_cast<const float4*>(smem + (size_t)s * kDStage);
#pragma unroll
                    for (int e = 0; e < DE; ++e) {
                        const int k = t * DE + e;
                        if (k * TB + tid < len) {
                            cf uc[2], zc[2];
                            Unit<float>::split(ur[k], uc);
                            Unit<float>::split(zr[k], zc);
#pragma unroll
                            for (int gi = 0; gi < TG; ++gi) {
                                if (gi < nv) {
                                    cf vc[2];
                                    Unit<float>::split(st4[gi * DU + e * TB + tid], vc);
#pragma unroll
                                    for (int h = 0; h < 2; ++h) {
                                        cf a = {v[2 * gi], v[2 * gi + 1]};
                                        cfmac(a, vc[h], uc[h]);
                                        v[2 * gi] = a.re;
                                        v[2 * gi + 1] = a.im;
                                        cf bz = {v[2 * (TG + gi)], v[2 * (TG + gi) + 1]};
                                        cfmac(bz, vc[h], zc[h]);
                                        v[2 * (TG + gi)] = bz.re;
                                        v[2 * (TG + gi) + 1] = bz.im;
                                    }
                                }
                            }
                        }
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&empty[s]);  // this warp is done with the stage
                }
                ++n;
            }
            // group complete: warp partials of the 8 vectors, lane l holding
            // item l/2 = which * 8 + gi, component l % 2
            tstep32<32, 16>(v, (lane & 16) != 0);
            tstep32<16, 8>(v, (lane & 8) != 0);
            tstep32<8, 4>(v, (lane & 4) != 0);
            tstep32<4, 2>(v, (lane & 2) != 0);
            tstep32<2, 1>(v, (lane & 1) != 0);
            scratch[gg & 1][warp][lane] = v[0];
            // all consumers leave together; the producer waits for the copies
            if (consumers_sync_or(bad)) return;
            if (warp == 0) {
                double sum = 0.0;
#pragma unroll
                for (int w = 0; w < TW; ++w) sum += (double)scratch[gg & 1][w][lane];
                const int item = lane >> 1, comp = lane & 1;
                const int which = item / TG, gi = item - which * TG;
                if (gi < nv) acc[(which * J + g * TG + gi) * 2 + comp] += sum;
            }
            // this buffer is next written at the end of the group after the
            // next one, behind a barrier that warp 0 reaches only now
            ++gg;
        }
    }
    if (seg_r >= 0) flush(seg_r);
}

// Update sweep of the delayed-reorthogonalisation Arnoldi step, complex64:
//   v_J = (u - sum_i V_i s_i) / beta -> basis slot J,
//   u   <- (z - sum_i V_i t_i) / beta - v_J d
// with s, t from red[r] (s at 0, t at J), 1/beta = inv_beta[r], d = dcoef[r].
// Persistent and warp-specialised like k_gdots2_ws: the work items are the
// tiles of TU = 512 units of every right-hand side, flattened as (r, tile)
// and split into one contiguous range per block; a tile takes one stage per
// group of 8 basis vectors. A consumer thread keeps the two sums of its 2
// units in registers across the groups of a tile and loads its u and z for
// the tile's epilogue before the first group, so that load is hidden behind
// the basis stream. The FP32 copies of s and t are reloaded into shared
// memory when the block moves on to the next right-hand side.
__global__ void __launch_bounds__(DTHREADS, 1)
    k_arnoldi_update_ws(float4* __restrict__ basis, long long basis_rhs_stride, long long vec_stride, int J,
                        const double2* __restrict__ red, long long red_stride, const double* __restrict__ inv_beta,
                        const double2* __restrict__ dcoef, float4* __restrict__ u, long long u_rhs_stride,
                        const float4* __restrict__ z, long long z_rhs_stride, long long nunits, int nrhs,
                        const int* __restrict__ active, int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[TNS];
    __shared__ __align__(8) uint64_t empty[TNS];
    __shared__ int abort_flag;
    cf* sc = reinterpret_cast<cf*>(smem + TNS * kStageBytes);  // s at [0, J), t at [J, 2J)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x, q = blockIdx.x;
    const long long tpr = (nunits + TU - 1) / TU;  // tiles per right-hand side
    const long long T = tpr * nrhs;
    const long long lo = range_lo(q, T, G), hi = range_lo(q + 1, T, G);
    const int ngroups = (J + TG - 1) / TG;
    volatile int* abort = &abort_flag;
    if (tid == 0) {
        for (int k = 0; k < TNS; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], TW);
        }
        abort_flag = 0;
        mbar_fence_init();
    }
    __syncthreads();

    if (warp == TW) {  // ---- producer warp: one lane issues every stage
        if (lane != 0 || ngroups == 0) return;
        int n = 0;  // stages issued
        bool ok = true;
        for (long long it = lo; it < hi && ok; ++it) {
            const long long r = it / tpr, base = (it - r * tpr) * TU;
            if (active != nullptr && active[r] == 0) continue;
            const uint32_t bytes = (uint32_t)min((long long)TU, nunits - base) * 16u;
            const float4* Vr = basis + r * basis_rhs_stride + base;
            for (int g = 0; g < ngroups; ++g) {
                const int s = n % TNS;
                if (n >= TNS) {  // the consumers' release of this stage's previous use
                    if (!mbar_wait_or_abort(&empty[s], (uint32_t)((n / TNS - 1) & 1), abort)) {
                        ok = false;
                        break;
                    }
                    fence_proxy_async_smem();
                }
                const int nv = min(TG, J - g * TG);
                unsigned char* dst = smem + (size_t)s * kStageBytes;
                mbar_expect_tx(&full[s], bytes * nv);
                for (int v = 0; v < nv; ++v)
                    bulk_load(dst + (size_t)v * TU * 16, Vr + (long long)(g * TG + v) * vec_stride, bytes, &full[s]);
                ++n;
            }
        }
        for (int k = max(0, n - TNS); k < n && ok; ++k)
            ok = mbar_wait_or_abort(&empty[k % TNS], (uint32_t)((k / TNS) & 1), abort);
        if (!ok) {
            atomicExch(err, OVS_ETIMEOUT_CODE);
            abort_flag = 1;
            for (int k = max(0, n - TNS); k < n; ++k) mbar_wait_bounded(&full[k % TNS], (uint32_t)((k / TNS) & 1));
        }
        return;
    }

    // ---- consumer warps
    int n = 0;  // stages consumed
    long long seg_r = -1;
    bool bad = false;
    float ib = 0.f;
    cf d = {0.f, 0.f};
    for (long long it = lo; it < hi; ++it) {
        const long long r = it / tpr, base = (it - r * tpr) * TU;
        if (active != nullptr && active[r] == 0) continue;
        if (r != seg_r) {  // coefficients of the next right-hand side
            if (consumers_sync_or(bad)) return;  // everyone is done with the old ones
            for (int i = tid; i < 2 * J; i += TB) {
                const double2 c = red[r * red_stride + i];
                sc[i] = {float(c.x), float(c.y)};
            }
            if (consumers_sync_or(bad)) return;
            ib = float(inv_beta[r]);
            const double2 dd = dcoef[r];
            d = {float(dd.x), float(dd.y)};
            seg_r = r;
        }
        float4* ur = u + r * u_rhs_stride;
        const float4* zr = z + r * z_rhs_stride;
        float4 up[TE], zp[TE];
#pragma unroll
        for (int e = 0; e < TE; ++e) {
            const long long p = base + tid + (long long)TB * e;
            up[e] = p < nunits ? ur[p] : make_float4(0.f, 0.f, 0.f, 0.f);
            zp[e] = p < nunits ? __ldg(zr + p) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        cf a[TE][2], bb[TE][2];
#pragma unroll
        for (int e = 0; e < TE; ++e) a[e][0] = a[e][1] = bb[e][0] = bb[e][1] = {0.f, 0.f};
        for (int g = 0; g < ngroups; ++g) {
            const int s = n % TNS;
            const bool got = bad || mbar_wait_or_abort(&full[s], (uint32_t)((n / TNS) & 1), abort);
            if (!__all_sync(0xffffffffu, got)) {  // keep `bad` uniform over the warp
                if (lane == 0) {
                    atomicExch(err, OVS_ETIMEOUT_CODE);
                    abort_flag = 1;
                }
                bad = true;
            }
            if (!bad) {
                const float4* st4 = reinterpret_cast<const float4*>(smem + (size_t)s * kStageBytes);
                const int nv = min(TG, J - g * TG);
#pragma unroll
                for (int gi = 0; gi < TG; ++gi) {
                    if (gi < nv) {
                        const cf si = sc[g * TG + gi], ti = sc[J + g * TG + gi];
#pragma unroll
                        for (int e = 0; e < TE; ++e) {
                            cf vc[2];
                            Unit<float>::split(st4[gi * TU + tid + TB * e], vc);
#pragma unroll
                            for (int c = 0; c < 2; ++c) {
                                cfma(a[e][c], vc[c], si);
                                cfma(bb[e][c], vc[c], ti);
                            }
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);  // this warp is done with the stage
            }
            ++n;
        }
        if (bad) continue;
        float4* vout = basis + r * basis_rhs_stride + (long long)J * vec_stride;
#pragma unroll
        for (int e = 0; e < TE; ++e) {
            const long long p = base + tid + (long long)TB * e;
            if (p >= nunits) continue;
            cf uc[2], zc[2], vo[2], un[2];
            Unit<float>::split(up[e], uc);
            Unit<float>::split(zp[e], zc);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                vo[c] = (uc[c] - a[e][c]) * ib;
                un[c] = (zc[c] - bb[e][c]) * ib - cmul(vo[c], d);
            }
            vout[p] = Unit<float>::join(vo);
            ur[p] = Unit<float>::join(un);
        }
    }
}

// Recombination y += alpha * sum_{i < J_r} V_i c_i (Eqs. yproj3, fAxLRArn)
// of a complex64 basis into a complex128 vector, J_r = min(J, Jdev[r]) (the
// Krylov depth of right-hand side r). Persistent and warp-specialised like
// k_arnoldi_update_ws: tiles of TU = 512 units of every right-hand side, one
// stage per group of 8 basis vectors. A consumer thread sums each group in
// FP32 (8 terms per entry) and adds the partial to its FP64 accumulators, so
// the FP64 work is two additions per complex entry and group. y (complex128
// internal layout: complex64 unit u <-> complex128 entries 2u, 2u+1) is read
// and written once per tile; its load is issued before the first group.
__global__ void __launch_bounds__(DTHREADS, 1)
    k_recombine_ws(const float4* __restrict__ basis, long long basis_rhs_stride, long long vec_stride, int J,
                   const int* __restrict__ Jdev, const double2* __restrict__ coef, long long coef_stride,
                   double alpha, double2* __restrict__ y, long long y_rhs_stride, long long nunits, int nrhs,
                   const int* __restrict__ active, int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[TNS];
    __shared__ __align__(8) uint64_t empty[TNS];
    __shared__ int abort_flag;
    cf* sc = reinterpret_cast<cf*>(smem + TNS * kStageBytes);  // alpha * c, FP32, [0, J)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x, q = blockIdx.x;
    const long long tpr = (nunits + TU - 1) / TU;
    const long long T = tpr * nrhs;
    const long long lo = range_lo(q, T, G), hi = range_lo(q + 1, T, G);
    volatile int* abort = &abort_flag;
    auto depth = [&](long long r) { return Jdev != nullptr ? min(J, Jdev[r]) : J; };
    if (tid == 0) {
        for (int k = 0; k < TNS; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], TW);
        }
        abort_flag = 0;
        mbar_fence_init();
    }
    __syncthreads();

    if (warp == TW) {  // ---- producer warp: one lane issues every stage
        if (lane != 0) return;
        int n = 0;
        bool ok = true;
        for (long long it = lo; it < hi && ok; ++it) {
            const long long r = it / tpr, base = (it - r * tpr) * TU;
            if (active != nullptr && active[r] == 0) continue;
            const int Jr = depth(r);
            const int ngroups = (Jr + TG - 1) / TG;
            const uint32_t bytes = (uint32_t)min((long long)TU, nunits - base) * 16u;
            const float4* Vr = basis + r * basis_rhs_stride + base;
            for (int g = 0; g < ngroups; ++g) {
                const int s = n % TNS;
                if (n >= TNS) {
                    if (!mbar_wait_or_abort(&empty[s], (uint32_t)((n / TNS - 1) & 1), abort)) {
                        ok = false;
                        break;
                    }
                    fence_proxy_async_smem();
                }
                const int nv = min(TG, Jr - g * TG);
                unsigned char* dst = smem + (size_t)s * kStageBytes;
                mbar_expect_tx(&full[s], bytes * nv);
                for (int v = 0; v < nv; ++v)
                    bulk_load(dst + (size_t)v * TU * 16, Vr + (long long)(g * TG + v) * vec_stride, bytes, &full[s]);
                ++n;
            }
        }
        for (int k = max(0, n - TNS); k < n && ok; ++k)
            ok = mbar_wait_or_abort(&empty[k % TNS], (uint32_t)((k / TNS) & 1), abort);
        if (!ok) {
            atomicExch(err, OVS_ETIMEOUT_CODE);
            abort_flag = 1;
            for (int k = max(0, n - TNS); k < n; ++k) mbar_wait_bounded(&full[k % TNS], (uint32_t)((k / TNS) & 1));
        }
        return;
    }

    // ---- consumer warps
    int n = 0;
    long long seg_r = -1;
    int Jr = 0;
    bool bad = false;
    for (long long it = lo; it < hi; ++it) {
        const long long r = it / tpr, base = (it - r * tpr) * TU;
        if (active != nullptr && active[r] == 0) continue;
        if (r != seg_r) {  // coefficients of the next right-hand side
            if (consumers_sync_or(bad)) return;
            Jr = depth(r);
            for (int i = tid; i < Jr; i += TB) {
                const double2 c = coef[r * coef_stride + i];
                sc[i] = {float(alpha * c.x), float(alpha * c.y)};
            }
            if (consumers_sync_or(bad)) return;
            seg_r = r;
        }
        const int ngroups = (Jr + TG - 1) / TG;
        double2* yr = y + r * y_rhs_stride;
        double2 yo[TE][2];
#pragma unroll
        for (int e = 0; e < TE; ++e) {
            const long long p = base + tid + (long long)TB * e;
            yo[e][0] = p < nunits ? yr[2 * p] : make_double2(0.0, 0.0);
            yo[e][1] = p < nunits ? yr[2 * p + 1] : make_double2(0.0, 0.0);
        }
        for (int g = 0; g < ngroups; ++g) {
            const int s = n % TNS;
            const bool got = bad || mbar_wait_or_abort(&full[s], (uint32_t)((n / TNS) & 1), abort);
            if (!__all_sync(0xffffffffu, got)) {
                if (lane == 0) {
                    atomicExch(err, OVS_ETIMEOUT_CODE);
                    abort_flag = 1;
                }
                bad = true;
            }
            if (!bad) {
                const float4* st4 = reinterpret_cast<const float4*>(smem + (size_t)s * kStageBytes);
                const int nv = min(TG, Jr - g * TG);
                cf a[TE][2];
#pragma unroll
                for (int e = 0; e < TE; ++e) a[e][0] = a[e][1] = {0.f, 0.f};
#pragma unroll
                for (int gi = 0; gi < TG; ++gi) {
                    if (gi < nv) {
                        const cf ci = sc[g * TG + gi];
#pragma unroll
                        for (int e = 0; e < TE; ++e) {
                            cf vc[2];
                            Unit<float>::split(st4[gi * TU + tid + TB * e], vc);
#pragma unroll
                            for (int c = 0; c < 2; ++c) cfma(a[e][c], vc[c], ci);
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
#pragma unroll
                for (int e = 0; e < TE; ++e)
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        yo[e][c].x += double(a[e][c].re);
                        yo[e][c].y += double(a[e][c].im);
                    }
            }
            ++n;
        }
        if (bad) continue;
#pragma unroll
        for (int e = 0; e < TE; ++e) {
            const long long p = base + tid + (long long)TB * e;
            if (p >= nunits) continue;
            yr[2 * p] = yo[e][0];
            yr[2 * p + 1] = yo[e][1];
        }
    }
}

bool tma_update_fits(int J) { return TNS * kStageBytes + (size_t)(2 * J + 1) * sizeof(cf) <= 220 * 1024; }

static size_t gdots_chunk_smem(int J) { return DS * kDStage + (size_t)(2 * J + 2) * 16; }

bool gdots_chunk_fits(int J) { return gdots_chunk_smem(J) <= 222 * 1024; }

static int gdots_chunk_grid(long long nunits, int nrhs, int num_sms) {
    const long long T = (nunits + CU - 1) / CU * nrhs;
    return (int)std::max<long long>(1, std::min<long long>(num_sms, T));
}

int gdots_chunk_slots(long long nunits, int nrhs, int num_sms) {
    const long long cpr = (nunits + CU - 1) / CU, T = cpr * nrhs;
    const int G = gdots_chunk_grid(nunits, nrhs, num_sms);
    int n = 1;
    for (long long r = 0; r < nrhs; ++r)
        n = std::max(n, owner_of((r + 1) * cpr - 1, T, G) - owner_of(r * cpr, T, G) + 1);
    return n;
}

cudaError_t launch_gdots2_chunk(const void* basis, long long basis_rhs_stride, long long vec_stride, int J,
                                const void* u, long long u_rhs_stride, const void* z, long long z_rhs_stride,
                                long long nunits, int nrhs, int num_sms, int nslot, void* partial, const int* active,
                                int* err, cudaStream_t st) {
    const size_t smem = gdots_chunk_smem(J);
    const cudaError_t e = ensure_dyn_smem((const void*)k_gdots2_ws, smem);
    if (e != cudaSuccess) return e;
    if (nslot != gdots_chunk_slots(nunits, nrhs, num_sms)) return cudaErrorInvalidValue;
    const int G = gdots_chunk_grid(nunits, nrhs, num_sms);
    k_gdots2_ws<<<G, DTHREADS, smem, st>>>((const float4*)basis, basis_rhs_stride, vec_stride, J, (const float4*)u,
                                           u_rhs_stride, (const float4*)z, z_rhs_stride, nunits, nrhs, nslot,
                                           (double2*)partial, active, err);
    return cudaGetLastError();
}

cudaError_t launch_arnoldi_update_tma(void* basis, long long basis_rhs_stride, long long vec_stride, int J,
                                      const void* red, long long red_stride, const double* inv_beta,
                                      const void* dcoef, void* u, long long u_rhs_stride, const void* z,
                                      long long z_rhs_stride, long long nunits, int nrhs, int num_sms,
                                      const int* active, int* err, cudaStream_t st) {
    const size_t smem = TNS * kStageBytes + (size_t)(2 * J + 1) * sizeof(cf);
    const cudaError_t e = ensure_dyn_smem((const void*)k_arnoldi_update_ws, smem);
    if (e != cudaSuccess) return e;
    const long long T = (nunits + TU - 1) / TU * nrhs;
    const int G = (int)std::max<long long>(1, std::min<long long>(num_sms, T));
    k_arnoldi_update_ws<<<G, DTHREADS, smem, st>>>((float4*)basis, basis_rhs_stride, vec_stride, J,
                                                   (const double2*)red, red_stride, inv_beta, (const double2*)dcoef,
                                                   (float4*)u, u_rhs_stride, (const float4*)z, z_rhs_stride, nunits,
                                                   nrhs, active, err);
    return cudaGetLastError();
}

bool recombine_tma_fits(int J) { return TNS * kStageBytes + (size_t)std::max(J, 1) * sizeof(cf) <= 220 * 1024; }

cudaError_t launch_recombine_tma(const void* basis, long long basis_rhs_stride, long long vec_stride, int J,
                                 const int* Jdev, const void* coef, long long coef_stride, double alpha, void* y,
                                 long long y_rhs_stride, long long nunits, int nrhs, int num_sms, const int* active,
                                 int* err, cudaStream_t st) {
    const size_t smem = TNS * kStageBytes + (size_t)std::max(J, 1) * sizeof(cf);
    const cudaError_t e = ensure_dyn_smem((const void*)k_recombine_ws, smem);
    if (e != cudaSuccess) return e;
    const long long T = (nunits + TU - 1) / TU * nrhs;
    const int G = (int)std::max<long long>(1, std::min<long long>(num_sms, T));
    k_recombine_ws<<<G, DTHREADS, smem, st>>>((const float4*)basis, basis_rhs_stride, vec_stride, J, Jdev,
                                              (const double2*)coef, coef_stride, alpha, (double2*)y, y_rhs_stride,
                                              nunits, nrhs, active, err);
    return cudaGetLastError();
}

// Self-check of the bounded waits: one thread waits on an mbarrier on which
// nothing ever arrives; after kWaitNs it records OVS_ETIMEOUT in the error
// word and returns, as the sweeps do when a copy never lands.
static __device__ int g_wait_check_err;

__global__ void k_wait_timeout_check() {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        g_wait_check_err = 0;
        mbar_init(&bar, 1);
        mbar_fence_init();
        if (!mbar_wait_bounded(&bar, 0)) g_wait_check_err = OVS_ETIMEOUT_CODE;
    }
}

cudaError_t check_wait_timeout(cudaStream_t st, int* code) {
    k_wait_timeout_check<<<1, 32, 0, st>>>();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(code, g_wait_check_err, sizeof(int));
    return e;
}

}  // namespace ovs
