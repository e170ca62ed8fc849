// TMA-pipelined update sweep of the complex64 Arnoldi basis (K2).
//
// The update sweep of an Arnoldi step (see blas.cu) streams the whole basis
// of every right-hand side. Here the basis tiles reach shared memory through
// 1D bulk asynchronous copies (cp.async.bulk, completion counted in bytes on
// an mbarrier): a stage holds 8 basis vectors x 512 16-byte units (64 KB),
// and 3 stages are in flight per block, so ~128 KB of loads per SM stay
// outstanding without occupying registers. Thread 0 issues the copies; all
// 256 threads consume a stage from shared memory and release it with a
// block barrier (which also agrees on the wait), after which its buffer is
// refilled (after a proxy fence, since generic loads read it before the
// asynchronous copy overwrites it). The two sums of each thread's units stay
// in registers across the stages of a tile.
//
// Every wait on a stage is bounded: if a copy does not complete the block
// records OVS_ETIMEOUT in *err, waits (bounded) for the copies it still has
// in flight, and returns.
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
constexpr long long kWaitLimit = 1LL << 24;  // try_wait polls before giving up
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
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (long long n = 0; n < kWaitLimit; ++n)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Stage sequence of one block: for each tile of its row chunk, the groups
// of TG basis vectors.
template <int U, int NS>
struct Seq {
    const float4* V;  // basis of this right-hand side
    long long vec_stride, u0, u1;
    int J, ngroups;
    __device__ void issue(int idx, unsigned char* stages, uint64_t* full) const {
        const int s = idx % NS;
        const int t = idx / ngroups, g = idx - t * ngroups;
        const long long base = u0 + (long long)t * U;
        const int units = (int)min((long long)U, u1 - base);
        const int nv = min(TG, J - g * TG);
        const uint32_t bytes = (uint32_t)units * 16u;
        unsigned char* dst = stages + (size_t)s * TG * U * 16;
        mbar_expect_tx(&full[s], bytes * nv);
        for (int v = 0; v < nv; ++v)
            bulk_load(dst + (size_t)v * U * 16, V + (long long)(g * TG + v) * vec_stride + base, bytes, &full[s]);
    }
};

// Abort path (all threads): record the timeout and wait (bounded) for the
// copies still in flight, so that no copy lands after the block has left.
template <int NS>
__device__ void drain(int idx, int total, uint64_t* full, int* err) {
    if (threadIdx.x == 0) {
        atomicExch(err, OVS_ETIMEOUT_CODE);
        for (int q = idx; q < min(idx + NS, total); ++q) mbar_wait_bounded(&full[q % NS], (uint32_t)((q / NS) & 1));
    }
    __syncthreads();
}

}  // namespace

// Update sweep of the delayed-reorthogonalisation Arnoldi step, complex64:
//   v_J = (u - sum_i V_i s_i) / beta -> basis slot J,
//   u   <- (z - sum_i V_i t_i) / beta - v_J d
// with s, t from red[r] (s at 0, t at J), 1/beta = inv_beta[r], d = dcoef[r].
// The basis streams through the same staged pipeline; the two sums of each
// thread's units stay in registers across the groups of a tile.
__global__ void __launch_bounds__(TB, 1)
    k_arnoldi_update_tma(float4* __restrict__ basis, long long basis_rhs_stride, long long vec_stride, int J,
                         const double2* __restrict__ red, long long red_stride, const double* __restrict__ inv_beta,
                         const double2* __restrict__ dcoef, float4* __restrict__ u, long long u_rhs_stride,
                         const float4* __restrict__ z, long long z_rhs_stride, long long nunits, long long chunk,
                         const int* __restrict__ active, int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[TNS];
    unsigned char* stages = smem;
    cf* sc = reinterpret_cast<cf*>(smem + TNS * kStageBytes);  // s at [0, J), t at [J, 2J)
    const int r = blockIdx.y, b = blockIdx.x;
    if (active != nullptr && active[r] == 0) return;
    const int tid = threadIdx.x;
    for (int i = tid; i < 2 * J; i += TB) {
        const double2 c = red[r * red_stride + i];
        sc[i] = {float(c.x), float(c.y)};
    }
    Seq<TU, TNS> q;
    q.V = basis + r * basis_rhs_stride;
    q.vec_stride = vec_stride;
    q.u0 = (long long)b * chunk;
    q.u1 = min(q.u0 + chunk, nunits);
    q.J = J;
    q.ngroups = (J + TG - 1) / TG;
    const int ntiles = (int)((q.u1 - q.u0 + TU - 1) / TU);
    const int total = ntiles * q.ngroups;
    if (tid == 0) {
        for (int s = 0; s < TNS; ++s) mbar_init(&full[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0)
        for (int idx = 0; idx < min(TNS, total); ++idx) q.issue(idx, stages, full);
    const float ib = float(inv_beta[r]);
    const double2 dd = dcoef[r];
    const cf d = {float(dd.x), float(dd.y)};
    float4* vout = basis + r * basis_rhs_stride + (long long)J * vec_stride;
    float4* ur = u + r * u_rhs_stride;
    const float4* zr = z + r * z_rhs_stride;
    cf a[TE][2], bb[TE][2];
    for (int t = 0; t < ntiles; ++t) {
        const long long base = q.u0 + (long long)t * TU;
#pragma unroll
        for (int e = 0; e < TE; ++e) a[e][0] = a[e][1] = bb[e][0] = bb[e][1] = {0.f, 0.f};
        for (int g = 0; g < q.ngroups; ++g) {
            const int idx = t * q.ngroups + g, s = idx % TNS;
            const bool got = mbar_wait_bounded(&full[s], (uint32_t)((idx / TNS) & 1));
            const float4* st4 = reinterpret_cast<const float4*>(stages + (size_t)s * kStageBytes);
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
            if (!__syncthreads_and(got)) {  // wait agreement + release of stage s
                drain<TNS>(idx, total, full, err);
                return;
            }
            if (tid == 0 && idx + TNS < total) {
                fence_proxy_async_smem();
                q.issue(idx + TNS, stages, full);
            }
        }
#pragma unroll
        for (int e = 0; e < TE; ++e) {
            const long long p = base + tid + (long long)TB * e;
            if (p >= q.u1) continue;
            cf uc[2], zc[2], vo[2], un[2];
            Unit<float>::split(ur[p], uc);
            Unit<float>::split(__ldg(zr + p), zc);
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

bool tma_update_fits(int J) { return TNS * kStageBytes + (size_t)(2 * J + 1) * sizeof(cf) <= 220 * 1024; }

cudaError_t launch_arnoldi_update_tma(void* basis, long long basis_rhs_stride, long long vec_stride, int J,
                                      const void* red, long long red_stride, const double* inv_beta,
                                      const void* dcoef, void* u, long long u_rhs_stride, const void* z,
                                      long long z_rhs_stride, long long nunits, const BlasPlan& plan, int nrhs,
                                      const int* active, int* err, cudaStream_t st) {
    static size_t set = 0;
    const size_t smem = TNS * kStageBytes + (size_t)(2 * J + 1) * sizeof(cf);
    if (smem > set) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_arnoldi_update_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        set = smem;
    }
    dim3 grid(plan.nblk, nrhs);
    k_arnoldi_update_tma<<<grid, TB, smem, st>>>((float4*)basis, basis_rhs_stride, vec_stride, J,
                                                 (const double2*)red, red_stride, inv_beta, (const double2*)dcoef,
                                                 (float4*)u, u_rhs_stride, (const float4*)z, z_rhs_stride, nunits,
                                                 plan.chunk, active, err);
    return cudaGetLastError();
}

}  // namespace ovs
