// ovs_matvec_noalloc: ovs_matvec without any device allocation.
//
// Some callers cannot let a library allocate device memory: programs whose
// device memory is already handed out by another allocator (a framework's
// caching allocator that reserved the whole pool, so a cudaMalloc would
// fail or steal from it), and loops that must not pay the implicit
// device-wide synchronisation of cudaMalloc/cudaFree. For them this entry
// point keeps its two work fields (the input and output of the stencil in
// the library's internal layout) in one fixed array compiled into the
// library, so the call allocates nothing; only the handle's links, created
// earlier, are used besides the caller's x and y.
//
// Every GPU that loads the library holds the array (2 x 8 MiB) until the
// process exits. All calls share it: calls that overlap on the GPU (on
// different streams, or from different threads) race on its contents and
// must be serialised by the caller. No entry needs to start at zero: each
// entry a call reads was written earlier in the same call.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/ovsign.h"
#include "common.cuh"
#include "handle.h"
#include "kernels.h"

namespace ovs {

constexpr size_t kNoAllocFieldBytes = (size_t)8 << 20;  // per work field

// Two work fields back to back; 256-byte alignment keeps every 16-byte
// vector access of the stencil and layout kernels aligned.
static __device__ __align__(256) unsigned char g_noalloc_scratch[2 * kNoAllocFieldBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the array on the current device, looked up once per
// device (with that device current) and cached for the life of the process.
// A cudaDeviceReset destroys the context that holds the array: the cached
// address is then stale, so a caller that resets a device must not call
// this entry point on it afterwards.
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (g_scratch_ptr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}
}  // namespace

}  // namespace ovs

using namespace ovs;

extern "C" int ovs_matvec_noalloc(ovs_gauge_t g, int32_t op, const void* x, void* y, int32_t nrhs, int32_t prec,
                                  void* stream) {
    if (!g || !x || !y) return lib_fail(OVS_EINVAL, "ovs_matvec_noalloc: NULL argument");
    if (nrhs < 0) return lib_fail(OVS_EINVAL, "ovs_matvec_noalloc: nrhs < 0");
    if (nrhs == 0) return OVS_OK;
    if (op != OVS_OP_DW && op != OVS_OP_HW && op != OVS_OP_HW2)
        return lib_fail(OVS_EINVAL, "ovs_matvec_noalloc: bad op");
    if (prec != OVS_F64 && prec != OVS_MIXED) return lib_fail(OVS_EINVAL, "ovs_matvec_noalloc: bad prec");
    if (prec == OVS_MIXED && g->links32 == nullptr)
        return lib_fail(OVS_ESTATE, "ovs_matvec_noalloc: handle was created without OVS_MIXED");
    if (!g->mu_set) return lib_fail(OVS_ESTATE, "ovs_matvec_noalloc: call ovs_set_mu first");
    const int tp = prec == OVS_MIXED ? PREC_F32 : PREC_F64;
    const size_t fb = (size_t)g->N * (tp == PREC_F64 ? 16 : 8);
    if (fb * (size_t)nrhs > kNoAllocFieldBytes)
        return lib_fail(OVS_EINVAL,
                        "ovs_matvec_noalloc: nrhs * N exceeds the fixed work array (8 MiB per field: "
                        "nrhs * N <= 524288 for OVS_F64, <= 1048576 for OVS_MIXED); use ovs_matvec");
    // host buffers would need staging memory: only device (or managed)
    // pointers, on the current device, which must be the handle's (its links
    // and the array used below live there)
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        return lib_fail(OVS_ECUDA, "ovs_matvec_noalloc: no current device");
    }
    if (cur != g->device) return lib_fail(OVS_EINVAL, "ovs_matvec_noalloc: the current device is not the handle's");
    for (const void* p : {x, (const void*)y}) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess ||
            (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return lib_fail(OVS_EINVAL, "ovs_matvec_noalloc: x and y must be device pointers");
        }
        if (a.type == cudaMemoryTypeDevice && a.device != cur)
            return lib_fail(OVS_EINVAL, "ovs_matvec_noalloc: x and y must be on the current device");
    }
    void* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return lib_fail(OVS_ECUDA, cudaGetErrorString(e));
    char* f0 = static_cast<char*>(base);
    char* f1 = f0 + kNoAllocFieldBytes;
    cudaStream_t st = (cudaStream_t)stream;
    const long long N = g->N;
    const void* L = tp == PREC_F64 ? g->links64 : g->links32;
    // the stencil shape already chosen for (precision, nrhs) on this handle,
    // if any (no tuning here: it would time launches on the caller's stream)
    StencilShape sh{};
    const auto tuned = g->tuned.find(std::make_pair(tp, (int)nrhs));
    if (tuned != g->tuned.end()) sh = tuned->second.best;
    e = launch_to_internal(tp, x, N, f0, fb, (int)g->V, nrhs, st);
    if (e == cudaSuccess) {
        if (op == OVS_OP_HW2) {
            e = launch_wilson(tp, true, L, f0, fb, f1, fb, g->geom, nrhs, g->kappa, g->mu, nullptr, st, sh);
            if (e == cudaSuccess)
                e = launch_wilson(tp, true, L, f1, fb, f0, fb, g->geom, nrhs, g->kappa, g->mu, nullptr, st, sh);
            if (e == cudaSuccess) e = launch_to_canonical(tp, f0, fb, y, N, (int)g->V, nrhs, st);
        } else {
            e = launch_wilson(tp, op == OVS_OP_HW, L, f0, fb, f1, fb, g->geom, nrhs, g->kappa, g->mu, nullptr, st, sh);
            if (e == cudaSuccess) e = launch_to_canonical(tp, f1, fb, y, N, (int)g->V, nrhs, st);
        }
    }
    if (e != cudaSuccess) return lib_fail(OVS_ECUDA, cudaGetErrorString(e));
    return OVS_OK;
}
