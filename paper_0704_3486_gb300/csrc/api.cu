// C ABI (include/ovsign.h): handles, operator set-up, deflation basis and
// the sign application
//
//   y = R sgn(Lambda) L^+ x + beta V_k sgn(H_k) e_1,  x_ominus = x - R L^+ x
//
// (Sec. 5.3, Eqs. xdec, fARLx, LRArnoldi, fAxLRArn; Sec. 4, Eq. yproj3),
// enqueued on the caller's stream as a sequence of kernels:
// K7 layout -> K5 projection -> norm -> k x (K1 matvec, K2 CGS2 sweeps)
// -> K3 Newton sign of H_k -> K4 recombination -> K7 layout.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ovsign.h"
#include "common.cuh"
#include "kernels.h"
#include "handle.h"

namespace ovs {
void generate_links(long long V, uint64_t seed, double eps, double* links);
int eig_setup(struct ovs_gauge_s* g, int m, double tol, double* eig_out, bool schur);
}  // namespace ovs

using namespace ovs;

// --------------------------------------------------------------- errors
static thread_local std::string g_err = "no error";

// Record the message and return code. A failed runtime call (e.g. an
// allocation beyond the device) leaves a non-sticky "last error" that the
// next launch check would report again: it is cleared here, so the handle
// stays usable after a reported failure. Sticky errors are not affected.
static int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    if (code == OVS_ECUDA || code == OVS_ENOMEM) cudaGetLastError();
    return code;
}

#define CK(call)                                                                                      \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) {                                                                      \
            if (e_ == cudaErrorMemoryAllocation)                                                      \
                return fail(OVS_ENOMEM, "%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
            return fail(OVS_ECUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
        }                                                                                             \
    } while (0)

#define TRY(call)                 \
    do {                          \
        int s_ = (call);          \
        if (s_ < 0) return s_;    \
    } while (0)

// --------------------------------------------------------------- handle
template <typename T> static cudaError_t dalloc(T** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return cudaSuccess;
    return cudaMalloc((void**)p, bytes);
}
template <typename T> static void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

// helpers exposed to other translation units of the library
namespace ovs {
int lib_fail(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace ovs

// ------------------------------------------------------------- tracing
static const int kEventPool = 16384;

static void prof_flush(ovs_gauge_s* g) {
    if (g->pending.empty()) return;
    cudaEventSynchronize(g->events[g->pending.back().ev + 1]);
    for (const auto& p : g->pending) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, g->events[p.ev], g->events[p.ev + 1]) == cudaSuccess) g->prof_ms[p.cls] += t;
    }
    cudaGetLastError();
    g->pending.clear();
}

static void prof_begin(ovs_gauge_s* g, int cls, cudaStream_t st) {
    ++g->prof_launches[cls];
    if (!g->timing || g->capturing) return;
    if (g->events.empty()) {
        g->events.resize(kEventPool);
        for (auto& e : g->events) cudaEventCreate(&e);
    }
    if ((int)(2 * g->pending.size() + 2) > kEventPool) prof_flush(g);
    const int ev = (int)(2 * g->pending.size());
    g->pending.push_back({cls, ev});
    cudaEventRecord(g->events[ev], st);
}

static void prof_end(ovs_gauge_s* g, int cls, double bytes, cudaStream_t st) {
    g->prof_bytes[cls] += bytes;
    if (!g->timing || g->capturing) return;
    cudaEventRecord(g->events[g->pending.back().ev + 1], st);
}

// Launch `call` as a kernel of tracing class `cls` moving `bytes` algorithmic bytes.
#define KL(cls, bytes, call)              \
    do {                                  \
        prof_begin(g, (cls), st);         \
        CK(call);                         \
        prof_end(g, (cls), (bytes), st);  \
    } while (0)

static double sz_of(int tprec) { return tprec == PREC_F64 ? 16.0 : 8.0; }
// K1: links read once, each right-hand side read and written once
static double bytes_wilson(long long V, int tp, int nrhs) { return (double)V * sz_of(tp) * (36.0 + 24.0 * nrhs); }
// K2 dot sweep: J basis vectors (shared or per rhs) and w
static double bytes_dots(long long N, int tp, int J, int nrhs, bool shared) {
    return (double)N * sz_of(tp) * ((shared ? J : (double)J * nrhs) + nrhs);
}
// update sweep: J basis vectors, optional input, output
static double bytes_update(long long N, int tpv, int tpo, int J, int nrhs, bool shared, bool has_in) {
    return (double)N * (sz_of(tpv) * (shared ? J : (double)J * nrhs) + sz_of(tpo) * nrhs * (has_in ? 2.0 : 1.0));
}
static double bytes_layout(long long N, int tp, int nrhs) { return (double)N * nrhs * (16.0 + sz_of(tp)); }

// Largest Krylov dimension: the inner-product sweep keeps 8 warps x (2k+2)
// complex128 accumulators in shared memory (<= 200 KB).
static const int kMaxK = 790;

static size_t field_bytes(long long N, int tprec) { return (size_t)N * (tprec == PREC_F64 ? 16 : 8); }
static long long field_units(long long N, int tprec) { return tprec == PREC_F64 ? N : N / 2; }
static int tprec_of(int prec) { return prec == OVS_MIXED ? PREC_F32 : PREC_F64; }
static const void* links_for(const ovs_gauge_s* g, int tprec) { return tprec == PREC_F64 ? g->links64 : g->links32; }

// Stencil autotuner (see ovs_stencil_tuning): every candidate shape timed
// on st, one warm-up and up to 3 timed launches each, the fastest kept.
StencilShape ovs::stencil_shape(ovs_gauge_s* g, int tp, int nrhs, const void* in, size_t in_stride, void* out,
                                size_t out_stride, cudaStream_t st) {
    const auto key = std::make_pair(tp, nrhs);
    const auto it = g->tuned.find(key);
    if (it != g->tuned.end()) return it->second.best;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (g->capturing || cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return StencilShape{};
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return StencilShape{};
    }
    const void* L = links_for(g, tp);
    ovs_gauge_s::Tuned t;
    t.best = StencilShape{};
    float best = -1.0f;
    for (int i = 0; i < kNumStencilShapes; ++i) {
        const StencilShape sh = kStencilShapes[i];
        t.ms[i] = -1.0f;
        if (tp == PREC_F64 && sh.rt != 1) continue;
        auto run = [&]() {
            return launch_wilson(tp, true, L, in, in_stride, out, out_stride, g->geom, nrhs, g->kappa, g->mu, nullptr,
                                 st, sh);
        };
        // warm-up (timed: a launch over 1 ms is timed once more, else 3 times)
        float ms = -1.0f;
        cudaError_t e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = run();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        const int reps = (e == cudaSuccess && ms > 1.0f) ? 1 : 3;
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int rep = 0; rep < reps && e == cudaSuccess; ++rep) e = run();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        t.ms[i] = ms / reps;
        if (best < 0.0f || t.ms[i] < best) {
            best = t.ms[i];
            t.best = sh;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g->tuned[key] = t;
    return t.best;
}

static void free_vec(VecWork& w) {
    dfree(w.xint);
    dfree(w.wvec);
    dfree(w.yacc);
    dfree(w.sx);
    dfree(w.sy);
    w.nrhs = 0;
    w.prec = -1;
}

static void free_kry(KryWork& k) {
    dfree(k.basis);
    dfree(k.H);
    dfree(k.htmp);
    dfree(k.dcoef);
    dfree(k.err);
    dfree(k.ccheck[0]);
    dfree(k.ccheck[1]);
    dfree(k.est);
    dfree(k.due);
    dfree(k.cstate);
    dfree(k.partial);
    dfree(k.norm_part);
    dfree(k.beta);
    dfree(k.inv_beta);
    dfree(k.hnorm2);
    dfree(k.active);
    dfree(k.k_used);
    dfree(k.iters);
    dfree(k.status);
    dfree(k.coeff);
    dfree(k.newton);
    dfree(k.cdef);
    dfree(k.cdef2);
    dfree(k.X);
    dfree(k.sylv);
    dfree(k.cS);
    k.nrhs = k.kmax = k.jcap = k.nblk = k.mdef = 0;
    k.prec = -1;
}

static void drop_graphs(ovs_gauge_s* g) {
    for (auto& e : g->graphs) cudaGraphDestroy(e.graph);
    g->graphs.clear();
    ++g->gen;
}

// Combined graphs of the batched form: one per set of instances (handle
// uid and generation), right-hand-side counts and options; every instance's
// recorded application is a child graph, so one launch runs them all.
namespace {
struct BatchEntry {
    std::vector<unsigned long long> uids;
    std::vector<unsigned> gens;
    std::vector<int> nrhs;
    int kmax, prec, every, flags;
    double tol;
    cudaGraphExec_t exec;
};
std::mutex g_batch_mu;
std::vector<BatchEntry> g_batches;
std::atomic<unsigned long long> g_next_uid{1};

// Drop the combined graphs that contain handle uid (all of them if uid = 0
// is never used: uids start at 1).
void drop_batches_of(unsigned long long uid) {
    std::lock_guard<std::mutex> lock(g_batch_mu);
    for (size_t i = 0; i < g_batches.size();) {
        const auto& u = g_batches[i].uids;
        if (std::find(u.begin(), u.end(), uid) != u.end()) {
            cudaGraphExecDestroy(g_batches[i].exec);
            g_batches.erase(g_batches.begin() + i);
        } else {
            ++i;
        }
    }
}
}  // namespace

void ovs::free_deflation(ovs_gauge_s* g) {
    drop_graphs(g);
    dfree(g->R64);
    dfree(g->L64);
    dfree(g->R32);
    dfree(g->L32);
    dfree(g->sgn);
    dfree(g->schurT);
    dfree(g->schurFT);
    g->m = 0;
    g->scheme = DEFL_NONE;
    g->lambda.clear();
}

static int ensure_vec(ovs_gauge_s* g, int nrhs, int tprec) {
    VecWork& w = g->vw;
    if (w.nrhs >= nrhs && w.prec == tprec) return OVS_OK;
    const int n = std::max(nrhs, w.prec == tprec ? w.nrhs : 0);
    drop_graphs(g);
    free_vec(w);
    const size_t fb = field_bytes(g->N, tprec), f64 = field_bytes(g->N, PREC_F64);
    CK(dalloc(&w.xint, fb * n));
    CK(dalloc(&w.wvec, fb * n));
    CK(dalloc(&w.yacc, f64 * n));
    CK(dalloc(&w.sx, f64 * n));
    CK(dalloc(&w.sy, f64 * n));
    w.nrhs = n;
    w.prec = tprec;
    return OVS_OK;
}

static int ensure_kry(ovs_gauge_s* g, int nrhs, int kmax, int tprec) {
    KryWork& k = g->kw;
    const int jneed = std::max(gdots_stride(2, kmax), gdots_stride(1, std::max(kmax, g->m)));
    const BlasPlan plan = blas_plan(field_units(g->N, tprec), nrhs, g->num_sms);
    const BlasPlan plan1 = blas_plan(field_units(g->N, tprec), 1, g->num_sms);
    const int nblk_need =
        std::max(std::max(plan.nblk, plan1.nblk),
                 tprec == PREC_F32 ? gdots_chunk_slots(field_units(g->N, tprec), nrhs, g->num_sms) : 0);
    const bool schur = g->scheme == DEFL_SCHUR;
    if (k.prec == tprec && k.nrhs >= nrhs && k.kmax >= kmax && k.jcap >= jneed && k.nblk >= nblk_need &&
        k.mdef >= g->m && (!schur || k.X != nullptr))
        return OVS_OK;
    const bool same = (k.prec == tprec);
    const int n = std::max(nrhs, same ? k.nrhs : 0);
    const int km = std::max(kmax, same ? k.kmax : 0);
    const int jc = std::max(gdots_stride(2, km), jneed);
    const int nb = std::max(nblk_need, blas_plan(field_units(g->N, tprec), 1, g->num_sms).nblk);
    drop_graphs(g);
    free_kry(k);
    const size_t fb = field_bytes(g->N, tprec);
    CK(dalloc(&k.basis, fb * (size_t)(km + 1) * n));
    CK(dalloc(&k.H, sizeof(double2) * (size_t)(km + 1) * km * n));
    CK(dalloc(&k.htmp, sizeof(double2) * (size_t)jc * n));
    CK(dalloc(&k.dcoef, sizeof(double2) * (size_t)n));
    CK(dalloc(&k.err, sizeof(int)));
    CK(dalloc(&k.ccheck[0], sizeof(double2) * (size_t)km * n));
    CK(dalloc(&k.ccheck[1], sizeof(double2) * (size_t)km * n));
    CK(dalloc(&k.est, sizeof(double) * n));
    CK(dalloc(&k.due, sizeof(int) * n));
    CK(dalloc(&k.cstate, sizeof(CheckState) * n));
    CK(cudaMemset(k.err, 0, sizeof(int)));
    CK(dalloc(&k.partial, sizeof(double2) * (size_t)nb * jc * n));
    CK(dalloc(&k.norm_part, sizeof(double) * (size_t)nb * n));
    CK(dalloc(&k.beta, sizeof(double) * n));
    CK(dalloc(&k.inv_beta, sizeof(double) * n));
    CK(dalloc(&k.hnorm2, sizeof(double) * n));
    CK(dalloc(&k.active, sizeof(int) * n));
    CK(dalloc(&k.k_used, sizeof(int) * n));
    CK(dalloc(&k.iters, sizeof(int) * n));
    CK(dalloc(&k.status, sizeof(int) * n));
    CK(dalloc(&k.coeff, sizeof(double2) * (size_t)km * n));
    CK(dalloc(&k.newton, sizeof(double2) * 2 * (size_t)km * km * n));
    const int md = std::max(std::max(g->m, 1), same ? k.mdef : 0);
    CK(dalloc(&k.cdef, sizeof(double2) * (size_t)md * n));
    CK(dalloc(&k.cdef2, sizeof(double2) * (size_t)md * n));
    if (schur) {
        CK(dalloc(&k.X, sizeof(double2) * (size_t)md * km * n));
        CK(dalloc(&k.sylv, sizeof(double2) * (size_t)schur_scratch_per_rhs(md) * n));
        CK(dalloc(&k.cS, sizeof(double2) * (size_t)md * n));
    }
    k.mdef = md;
    k.nrhs = n;
    k.kmax = km;
    k.jcap = jc;
    k.nblk = nb;
    k.prec = tprec;
    return OVS_OK;
}

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static int check_dims(const int32_t dims[4]) {
    if (!dims) return fail(OVS_EINVAL, "dims is NULL");
    long long v = 1;
    for (int i = 0; i < 4; ++i) {
        if (dims[i] < 2) return fail(OVS_EINVAL, "lattice extent %d of direction %d is below 2", dims[i], i);
        v *= dims[i];
    }
    if (v * 12 > (1LL << 31) - 1) return fail(OVS_EINVAL, "lattice too large (12 V must fit in 31 bits)");
    return OVS_OK;
}

static int new_handle(const int32_t dims[4], const double* links_host, int32_t prec, ovs_gauge_t* out) {
    if (!out) return fail(OVS_EINVAL, "out is NULL");
    *out = nullptr;
    TRY(check_dims(dims));
    if (prec != OVS_F64 && prec != OVS_MIXED) return fail(OVS_EINVAL, "prec must be OVS_F64 or OVS_MIXED");
    ovs_gauge_s* g = new ovs_gauge_s();
    g->uid = g_next_uid.fetch_add(1);
    for (int i = 0; i < 4; ++i) g->dims[i] = dims[i];
    g->geom = make_geom(dims);
    g->V = g->geom.V;
    g->N = 12 * g->V;
    g->prec = prec;
    cudaGetDevice(&g->device);
    cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    void* tmp = nullptr;
    const size_t lb = (size_t)g->V * 72 * sizeof(double);
    cudaError_t e = cudaMalloc(&g->links64, (size_t)g->V * 36 * sizeof(double2));
    if (e == cudaSuccess && prec == OVS_MIXED) e = cudaMalloc(&g->links32, (size_t)g->V * 36 * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&tmp, lb);
    if (e == cudaSuccess) e = cudaMemcpy(tmp, links_host, lb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_links_to_internal(tmp, g->links64, g->links32, (int)g->V, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) {
        ovs_destroy(g);
        return fail(e == cudaErrorMemoryAllocation ? OVS_ENOMEM : OVS_ECUDA, "gauge upload: %s",
                    cudaGetErrorString(e));
    }
    *out = g;
    return OVS_OK;
}

// ----------------------------------------------------------------- ABI
extern "C" {

const char* ovs_last_error(void) { return g_err.c_str(); }

const char* ovs_version(void) { return "ovsign 0.1 (sm_103a)"; }

int ovs_create_gauge(const int32_t dims[4], uint64_t seed, double eps, int32_t prec, ovs_gauge_t* out) {
    TRY(check_dims(dims));
    if (!(eps >= 0.0) || !std::isfinite(eps)) return fail(OVS_EINVAL, "eps must be finite and >= 0");
    const long long V = (long long)dims[0] * dims[1] * dims[2] * dims[3];
    std::vector<double> links((size_t)V * 72);
    generate_links(V, seed, eps, links.data());
    return new_handle(dims, links.data(), prec, out);
}

int ovs_create_gauge_from_links(const int32_t dims[4], const double* links, int32_t prec, ovs_gauge_t* out) {
    if (!links) return fail(OVS_EINVAL, "links is NULL");
    return new_handle(dims, links, prec, out);
}

int ovs_get_links(ovs_gauge_t g, double* links_out) {
    if (!g || !links_out) return fail(OVS_EINVAL, "NULL argument");
    void* tmp = nullptr;
    const size_t lb = (size_t)g->V * 72 * sizeof(double);
    CK(cudaMalloc(&tmp, lb));
    cudaError_t e = launch_links_to_canonical(g->links64, tmp, (int)g->V, 0);
    if (e == cudaSuccess) e = cudaMemcpy(links_out, tmp, lb, cudaMemcpyDeviceToHost);
    cudaFree(tmp);
    CK(e);
    return OVS_OK;
}

int ovs_set_mu(ovs_gauge_t g, double mu, double m_w) {
    if (!g) return fail(OVS_EINVAL, "NULL handle");
    if (!std::isfinite(mu) || !std::isfinite(m_w) || 8.0 + 2.0 * m_w == 0.0)
        return fail(OVS_EINVAL, "mu and m_w must be finite and 8 + 2 m_w != 0");
    g->mu = mu;
    g->m_w = m_w;
    g->kappa = 1.0 / (8.0 + 2.0 * m_w);
    g->mu_set = true;
    free_deflation(g);  // also drops recorded applications (kappa, mu are kernel arguments)
    return OVS_OK;
}

int ovs_matvec(ovs_gauge_t g, int32_t op, const void* x, void* y, int32_t nrhs, int32_t prec, void* stream) {
    if (!g || !x || !y) return fail(OVS_EINVAL, "NULL argument");
    if (nrhs < 0) return fail(OVS_EINVAL, "nrhs < 0");
    if (nrhs == 0) return OVS_OK;
    if (op != OVS_OP_DW && op != OVS_OP_HW && op != OVS_OP_HW2) return fail(OVS_EINVAL, "bad op");
    if (prec != OVS_F64 && prec != OVS_MIXED) return fail(OVS_EINVAL, "bad prec");
    if (prec == OVS_MIXED && g->prec != OVS_MIXED) return fail(OVS_ESTATE, "handle was created without OVS_MIXED");
    if (!g->mu_set) return fail(OVS_ESTATE, "call ovs_set_mu first");
    cudaStream_t st = (cudaStream_t)stream;
    const int tp = tprec_of(prec);
    TRY(ensure_vec(g, nrhs, tp));
    const long long N = g->N;
    const size_t f64 = field_bytes(N, PREC_F64), fb = field_bytes(N, tp);
    const bool xdev = is_device_ptr(x), ydev = is_device_ptr(y);
    const void* xd = x;
    if (!xdev) {
        CK(cudaMemcpyAsync(g->vw.sx, x, f64 * nrhs, cudaMemcpyHostToDevice, st));
        xd = g->vw.sx;
    }
    void* yd = ydev ? y : g->vw.sy;
    VecWork& w = g->vw;
    const double bl = bytes_layout(N, tp, nrhs), bw = bytes_wilson(g->V, tp, nrhs);
    KL(OVS_PROF_LAYOUT, bl, launch_to_internal(tp, xd, N, w.xint, fb, (int)g->V, nrhs, st));
    const void* L = links_for(g, tp);
    const StencilShape sh = stencil_shape(g, tp, nrhs, w.xint, fb, w.wvec, fb, st);
    if (op == OVS_OP_HW2) {
        KL(OVS_PROF_MATVEC, bw,
           launch_wilson(tp, true, L, w.xint, fb, w.wvec, fb, g->geom, nrhs, g->kappa, g->mu, nullptr, st, sh));
        KL(OVS_PROF_MATVEC, bw,
           launch_wilson(tp, true, L, w.wvec, fb, w.xint, fb, g->geom, nrhs, g->kappa, g->mu, nullptr, st, sh));
        KL(OVS_PROF_LAYOUT, bl, launch_to_canonical(tp, w.xint, fb, yd, N, (int)g->V, nrhs, st));
    } else {
        KL(OVS_PROF_MATVEC, bw,
           launch_wilson(tp, op == OVS_OP_HW, L, w.xint, fb, w.wvec, fb, g->geom, nrhs, g->kappa, g->mu, nullptr,
                         st, sh));
        KL(OVS_PROF_LAYOUT, bl, launch_to_canonical(tp, w.wvec, fb, yd, N, (int)g->V, nrhs, st));
    }
    if (!ydev) {
        CK(cudaMemcpyAsync(y, yd, f64 * nrhs, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    return OVS_OK;
}

// ------------------------------------------------------------ deflation
static void host_inverse(std::vector<std::complex<double>>& a, int n, bool& ok) {
    // Gauss-Jordan with partial pivoting, row-major, in place
    std::vector<int> perm(n);
    ok = true;
    for (int p = 0; p < n; ++p) {
        int piv = p;
        double best = std::abs(a[(size_t)p * n + p]);
        for (int i = p + 1; i < n; ++i)
            if (std::abs(a[(size_t)i * n + p]) > best) { best = std::abs(a[(size_t)i * n + p]); piv = i; }
        if (!(best > 0.0)) { ok = false; return; }
        perm[p] = piv;
        if (piv != p)
            for (int j = 0; j < n; ++j) std::swap(a[(size_t)p * n + j], a[(size_t)piv * n + j]);
        const std::complex<double> inv = 1.0 / a[(size_t)p * n + p];
        for (int j = 0; j < n; ++j) a[(size_t)p * n + j] *= inv;
        a[(size_t)p * n + p] = inv;
        for (int i = 0; i < n; ++i) {
            if (i == p) continue;
            const std::complex<double> f = a[(size_t)i * n + p];
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j)
                if (j != p) a[(size_t)i * n + j] -= f * a[(size_t)p * n + j];
            a[(size_t)i * n + p] = -f * inv;
        }
    }
    for (int p = n - 1; p >= 0; --p)
        if (perm[p] != p)
            for (int i = 0; i < n; ++i) std::swap(a[(size_t)i * n + p], a[(size_t)i * n + perm[p]]);
}

}  // extern "C"

namespace ovs {
// Install R (right vectors) and L (left vectors), both device canonical
// complex128 [m][N]; biorthonormalise L; keep FP32 copies for OVS_MIXED.
int install_deflation(ovs_gauge_s* g, int m, const void* Rc, const void* Lc, const double* lambda) {
    cudaStream_t st = 0;
    free_deflation(g);
    if (m == 0) return OVS_OK;
    double lmax = 0.0;
    for (int i = 0; i < m; ++i) lmax = std::max(lmax, std::hypot(lambda[2 * i], lambda[2 * i + 1]));
    std::vector<double> sg(m);
    for (int i = 0; i < m; ++i) {
        if (!(std::fabs(lambda[2 * i]) > 1e-12 * lmax))
            return fail(OVS_ESIGN, "deflated eigenvalue %d has Re lambda = %g: sign undefined", i, lambda[2 * i]);
        sg[i] = lambda[2 * i] > 0 ? 1.0 : -1.0;
    }
    const long long N = g->N;
    const int V = (int)g->V;
    const size_t f64 = field_bytes(N, PREC_F64);
    CK(dalloc(&g->R64, f64 * m));
    CK(dalloc(&g->L64, f64 * m));
    CK(dalloc(&g->sgn, sizeof(double) * m));
    CK(cudaMemcpy(g->sgn, sg.data(), sizeof(double) * m, cudaMemcpyHostToDevice));
    void* Ltmp = nullptr;
    CK(dalloc(&Ltmp, f64 * m));
    KL(OVS_PROF_LAYOUT, 0.0, launch_to_internal(PREC_F64, Rc, N, g->R64, f64, V, m, 0));
    KL(OVS_PROF_LAYOUT, 0.0, launch_to_internal(PREC_F64, Lc, N, Ltmp, f64, V, m, 0));
    // G[j][i] = L_j^+ R_i  (right-hand side i = R_i, basis = L shared)
    const BlasPlan plan = blas_plan(N, m, g->num_sms);
    void* part = nullptr;
    void* G = nullptr;
    const int S = gdots_stride(1, m);
    CK(dalloc(&part, sizeof(double2) * (size_t)plan.nblk * S * m));
    CK(dalloc(&G, sizeof(double2) * (size_t)m * m));
    KL(OVS_PROF_DOTS, 0.0,
       launch_gdots(PREC_F64, 1, Ltmp, 0, N, m, g->R64, N, nullptr, 0, false, N, plan, m, part, nullptr, 0));
    KL(OVS_PROF_SMALL, 0.0, launch_reduce(part, plan.nblk, S, m, m, G, m, false, nullptr, 0));
    std::vector<std::complex<double>> gh((size_t)m * m), a((size_t)m * m);
    CK(cudaMemcpy(gh.data(), G, sizeof(double2) * (size_t)m * m, cudaMemcpyDeviceToHost));
    // gh[i*m + j] = L_j^+ R_i = G_ji with G = L^+ R. Row-major a = G.
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) a[(size_t)j * m + i] = gh[(size_t)i * m + j];
    bool ok = true;
    host_inverse(a, m, ok);
    if (!ok) {
        cudaFree(part); cudaFree(G); cudaFree(Ltmp);
        return fail(OVS_EINVAL, "L^+ R is singular: left and right vectors do not span dual spaces");
    }
    // Lbi = L G^{-+}: Lbi_i = sum_j L_j (G^{-+})_{j i} = sum_j L_j conj(Ginv_{i j})
    std::vector<std::complex<double>> cf((size_t)m * m);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) cf[(size_t)i * m + j] = std::conj(a[(size_t)i * m + j]);
    CK(cudaMemcpy(G, cf.data(), sizeof(double2) * (size_t)m * m, cudaMemcpyHostToDevice));
    KL(OVS_PROF_UPDATE, 0.0, launch_update(PREC_F64, PREC_F64, Ltmp, 0, N, m, nullptr, G, m, 1.0, nullptr, 0, g->L64, N, N, plan, m,
                     nullptr, nullptr, 0));
    CK(cudaDeviceSynchronize());
    cudaFree(part);
    cudaFree(G);
    if (g->prec == OVS_MIXED) {
        const size_t f32 = field_bytes(N, PREC_F32);
        CK(dalloc(&g->R32, f32 * m));
        CK(dalloc(&g->L32, f32 * m));
        KL(OVS_PROF_LAYOUT, 0.0, launch_to_internal(PREC_F32, Rc, N, g->R32, f32, V, m, 0));
        KL(OVS_PROF_LAYOUT, 0.0, launch_to_canonical(PREC_F64, g->L64, f64, Ltmp, N, V, m, 0));
        KL(OVS_PROF_LAYOUT, 0.0, launch_to_internal(PREC_F32, Ltmp, N, g->L32, f32, V, m, 0));
        CK(cudaDeviceSynchronize());
    }
    cudaFree(Ltmp);
    g->m = m;
    g->scheme = DEFL_LR;
    g->lambda.assign(lambda, lambda + 2 * m);
    return OVS_OK;
}
}  // namespace ovs

extern "C" {

int ovs_deflate_load(ovs_gauge_t g, int32_t m, const double* R, const double* L, const double* lambda) {
    if (!g) return fail(OVS_EINVAL, "NULL handle");
    if (!g->mu_set) return fail(OVS_ESTATE, "call ovs_set_mu first");
    if (m < 0 || (long long)m > g->N) return fail(OVS_EINVAL, "m out of range");
    if (m > 0 && (!R || !L || !lambda)) return fail(OVS_EINVAL, "NULL R, L or lambda");
    if (m == 0) {
        free_deflation(g);
        return OVS_OK;
    }
    const size_t f64 = field_bytes(g->N, PREC_F64);
    void *Rd = nullptr, *Ld = nullptr;
    CK(dalloc(&Rd, f64 * m));
    cudaError_t e = dalloc(&Ld, f64 * m);
    if (e == cudaSuccess) e = cudaMemcpy(Rd, R, f64 * m, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(Ld, L, f64 * m, cudaMemcpyHostToDevice);
    int rc = OVS_OK;
    if (e != cudaSuccess) rc = fail(OVS_ECUDA, "deflate_load upload: %s", cudaGetErrorString(e));
    if (rc == OVS_OK) rc = install_deflation(g, m, Rd, Ld, lambda);
    cudaFree(Rd);
    cudaFree(Ld);
    return rc;
}

int ovs_deflate_load_schur(ovs_gauge_t g, int32_t m, const double* R) {
    if (!g) return fail(OVS_EINVAL, "NULL handle");
    if (!g->mu_set) return fail(OVS_ESTATE, "call ovs_set_mu first");
    if (m < 0 || (long long)m > g->N) return fail(OVS_EINVAL, "m out of range");
    if (m > 0 && !R) return fail(OVS_EINVAL, "NULL R");
    if (m == 0) {
        free_deflation(g);
        return OVS_OK;
    }
    const size_t f64 = field_bytes(g->N, PREC_F64);
    void* Rd = nullptr;
    CK(dalloc(&Rd, f64 * m));
    const cudaError_t e = cudaMemcpy(Rd, R, f64 * m, cudaMemcpyHostToDevice);
    int rc = e == cudaSuccess ? install_schur(g, m, Rd) : fail(OVS_ECUDA, "deflate_load_schur upload: %s",
                                                              cudaGetErrorString(e));
    cudaFree(Rd);
    return rc;
}

int ovs_deflate_scheme(ovs_gauge_t g) {
    if (!g) return fail(OVS_EINVAL, "NULL handle");
    return g->scheme;
}

int ovs_deflate_get(ovs_gauge_t g, int32_t* m_out, double* R, double* L, double* lambda) {
    if (!g) return fail(OVS_EINVAL, "NULL handle");
    if (L && g->scheme == DEFL_SCHUR) return fail(OVS_ESTATE, "Schur deflation keeps no left vectors");
    if (m_out) *m_out = g->m;
    const int m = g->m;
    if (m == 0) return OVS_OK;
    if (lambda) std::memcpy(lambda, g->lambda.data(), sizeof(double) * 2 * m);
    const size_t f64 = field_bytes(g->N, PREC_F64);
    void* tmp = nullptr;
    if (R || L) CK(dalloc(&tmp, f64 * m));
    cudaStream_t st = 0;
    if (R) {
        KL(OVS_PROF_LAYOUT, 0.0, launch_to_canonical(PREC_F64, g->R64, f64, tmp, g->N, (int)g->V, m, 0));
        CK(cudaMemcpy(R, tmp, f64 * m, cudaMemcpyDeviceToHost));
    }
    if (L) {
        KL(OVS_PROF_LAYOUT, 0.0, launch_to_canonical(PREC_F64, g->L64, f64, tmp, g->N, (int)g->V, m, 0));
        CK(cudaMemcpy(L, tmp, f64 * m, cudaMemcpyDeviceToHost));
    }
    if (tmp) cudaFree(tmp);
    return OVS_OK;
}

static uint64_t fnv1a(const void* p, size_t n, uint64_t h) {
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ULL;
    }
    return h;
}

struct DeflHeader {
    char magic[8];
    int32_t dims[4];
    double mu, m_w;
    int64_t m, N;
    uint64_t checksum;
};

int ovs_deflate_save(ovs_gauge_t g, const char* path) {
    if (!g || !path) return fail(OVS_EINVAL, "NULL argument");
    if (g->m == 0) return fail(OVS_ESTATE, "no deflation basis installed");
    if (g->scheme != DEFL_LR) return fail(OVS_ESTATE, "only an LR deflation basis can be saved");
    const int m = g->m;
    const size_t f64 = field_bytes(g->N, PREC_F64);
    std::vector<double> R((size_t)m * g->N * 2), L((size_t)m * g->N * 2), lam(2 * m);
    TRY(ovs_deflate_get(g, nullptr, R.data(), L.data(), lam.data()));
    DeflHeader h;
    std::memcpy(h.magic, "OVSDEFL1", 8);
    for (int i = 0; i < 4; ++i) h.dims[i] = g->dims[i];
    h.mu = g->mu;
    h.m_w = g->m_w;
    h.m = m;
    h.N = g->N;
    uint64_t c = 1469598103934665603ULL;
    c = fnv1a(lam.data(), lam.size() * sizeof(double), c);
    c = fnv1a(R.data(), f64 * m, c);
    c = fnv1a(L.data(), f64 * m, c);
    h.checksum = c;
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(OVS_EIO, "cannot open %s for writing", path);
    bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1;
    ok = ok && std::fwrite(lam.data(), sizeof(double), lam.size(), f) == lam.size();
    ok = ok && std::fwrite(R.data(), 1, f64 * m, f) == f64 * m;
    ok = ok && std::fwrite(L.data(), 1, f64 * m, f) == f64 * m;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(OVS_EIO, "write to %s failed", path);
    return OVS_OK;
}

int ovs_deflate_restore(ovs_gauge_t g, const char* path) {
    if (!g || !path) return fail(OVS_EINVAL, "NULL argument");
    if (!g->mu_set) return fail(OVS_ESTATE, "call ovs_set_mu first");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(OVS_EIO, "cannot open %s", path);
    DeflHeader h;
    if (std::fread(&h, sizeof(h), 1, f) != 1 || std::memcmp(h.magic, "OVSDEFL1", 8) != 0) {
        std::fclose(f);
        return fail(OVS_EIO, "%s is not a deflation file", path);
    }
    bool same = h.N == g->N && h.mu == g->mu && h.m_w == g->m_w && h.m > 0 && h.m <= g->N;
    for (int i = 0; i < 4; ++i) same = same && h.dims[i] == g->dims[i];
    if (!same) {
        std::fclose(f);
        return fail(OVS_ESTATE, "%s was saved for another lattice, mu or m_w", path);
    }
    const int m = (int)h.m;
    const size_t f64 = field_bytes(g->N, PREC_F64);
    std::vector<double> R((size_t)m * g->N * 2), L((size_t)m * g->N * 2), lam(2 * m);
    bool ok = std::fread(lam.data(), sizeof(double), lam.size(), f) == lam.size();
    ok = ok && std::fread(R.data(), 1, f64 * m, f) == f64 * m;
    ok = ok && std::fread(L.data(), 1, f64 * m, f) == f64 * m;
    std::fclose(f);
    if (!ok) return fail(OVS_EIO, "%s is truncated", path);
    uint64_t c = 1469598103934665603ULL;
    c = fnv1a(lam.data(), lam.size() * sizeof(double), c);
    c = fnv1a(R.data(), f64 * m, c);
    c = fnv1a(L.data(), f64 * m, c);
    if (c != h.checksum) return fail(OVS_EIO, "%s: checksum mismatch", path);
    return ovs_deflate_load(g, m, R.data(), L.data(), lam.data());
}

int ovs_deflate_stats(ovs_gauge_t g, int32_t* iters, int64_t* matvecs, double* max_resid) {
    if (!g) return fail(OVS_EINVAL, "NULL handle");
    if (iters) {
        iters[0] = g->setup_iters[0];
        iters[1] = g->setup_iters[1];
    }
    if (matvecs) *matvecs = g->setup_matvecs;
    if (max_resid) *max_resid = g->setup_resid;
    return OVS_OK;
}

int ovs_set_setup_budget(ovs_gauge_t g, double max_seconds) {
    if (!g) return fail(OVS_EINVAL, "NULL handle");
    if (!(max_seconds >= 0.0)) return fail(OVS_EINVAL, "max_seconds must be >= 0");
    g->setup_budget_s = max_seconds;
    return OVS_OK;
}

int ovs_deflate_setup(ovs_gauge_t g, int32_t m, double tol, double* eig_out) {
    if (!g) return fail(OVS_EINVAL, "NULL handle");
    if (!g->mu_set) return fail(OVS_ESTATE, "call ovs_set_mu first");
    if (m <= 0 || (long long)m * 4 > g->N) return fail(OVS_EINVAL, "m must be in [1, N/4]");
    if (!(tol > 0.0)) return fail(OVS_EINVAL, "tol must be > 0");
    return eig_setup(g, m, tol, eig_out, false);
}

int ovs_deflate_setup_schur(ovs_gauge_t g, int32_t m, double tol, double* eig_out) {
    if (!g) return fail(OVS_EINVAL, "NULL handle");
    if (!g->mu_set) return fail(OVS_ESTATE, "call ovs_set_mu first");
    if (m <= 0 || (long long)m * 4 > g->N) return fail(OVS_EINVAL, "m must be in [1, N/4]");
    if (!(tol > 0.0)) return fail(OVS_EINVAL, "tol must be > 0");
    return eig_setup(g, m, tol, eig_out, true);
}

// ---------------------------------------------------------- sign apply
}  // extern "C"

// Argument checks shared by the single and batched forms.
static int check_apply(ovs_gauge_s* g, int nrhs, const ovs_apply_opts* opts) {
    if (!g || !opts) return fail(OVS_EINVAL, "NULL argument");
    if (nrhs <= 0) return fail(OVS_EINVAL, "nrhs must be >= 1");
    if (nrhs > 65535) return fail(OVS_EINVAL, "nrhs must be <= 65535");
    if (!g->mu_set) return fail(OVS_ESTATE, "call ovs_set_mu first");
    const int k = opts->k_max;
    if (k < 1 || k > kMaxK) return fail(OVS_EINVAL, "k_max must be in [1, %d]", kMaxK);
    if ((long long)k + 1 > g->N) return fail(OVS_EINVAL, "k_max must be < N");
    if (opts->prec != OVS_F64 && opts->prec != OVS_MIXED) return fail(OVS_EINVAL, "bad prec");
    if (opts->prec == OVS_MIXED && g->prec != OVS_MIXED) return fail(OVS_ESTATE, "handle was created without OVS_MIXED");
    const int every = opts->check_every;
    if (every < 0 || (every % 2) != 0) return fail(OVS_EINVAL, "check_every must be 0 or a positive even number");
    if (every > 0 && !(opts->tol > 0.0)) return fail(OVS_EINVAL, "check_every > 0 needs tol > 0");
    if ((opts->flags & ~(OVS_APPLY_HARMONIC | OVS_APPLY_SKIP_AHEAD)) != 0)
        return fail(OVS_EINVAL, "unknown bits in opts->flags");
    const bool harmonic = (opts->flags & OVS_APPLY_HARMONIC) != 0;
    if (harmonic && every > 0) return fail(OVS_EINVAL, "OVS_APPLY_HARMONIC needs check_every = 0");
    if ((opts->flags & OVS_APPLY_SKIP_AHEAD) != 0 && every == 0)
        return fail(OVS_EINVAL, "OVS_APPLY_SKIP_AHEAD needs check_every > 0");
    if (g->scheme == DEFL_SCHUR && (every > 0 || harmonic))
        return fail(OVS_EINVAL, "Schur deflation supports fixed-k applications without OVS_APPLY_HARMONIC");
    if (g->scheme == DEFL_SCHUR && !schur_coeff_fits(k)) return fail(OVS_EINVAL, "k_max too large for Schur deflation");
    return OVS_OK;
}

// Enqueue the whole application on st, from the device canonical input xd
// to the device canonical output yd. Buffers must already be sized
// (ensure_vec / ensure_kry); no allocation happens here, and no host
// synchronisation except the stencil autotuner's one-time timing of a new
// (precision, nrhs) pair, which is skipped during stream capture (the
// batched form tunes before it records), so the sequence can be recorded as
// a CUDA graph.
static int sign_apply_core(ovs_gauge_s* g, const void* xd, void* yd, int nrhs, const ovs_apply_opts* opts,
                           cudaStream_t st, bool overlap = false) {
    const int k = opts->k_max;
    const int every = opts->check_every;
    const int tp = tprec_of(opts->prec);
    VecWork& w = g->vw;
    KryWork& kw = g->kw;
    const long long N = g->N;
    const int V = (int)g->V;
    const size_t fb = field_bytes(N, tp), f64 = field_bytes(N, PREC_F64);
    const long long units = field_units(N, tp);
    const long long kmax = kw.kmax;
    const long long basis_rhs_units = (kmax + 1) * units;
    const int ldh = (int)(kmax + 1);
    const long long h_rhs = (long long)(kmax + 1) * kmax;
    const BlasPlan plan = blas_plan(units, nrhs, g->num_sms);
    const BlasPlan plan64 = blas_plan(N, nrhs, g->num_sms);
    const int dslots = tp == PREC_F32 ? gdots_chunk_slots(units, nrhs, g->num_sms) : 0;
    char* basis = (char*)kw.basis;

    // input, canonical complex128 -> internal precision
    KL(OVS_PROF_LAYOUT, bytes_layout(N, tp, nrhs), launch_to_internal(tp, xd, N, w.xint, fb, V, nrhs, st));
    CK(cudaMemsetAsync(kw.H, 0, sizeof(double2) * h_rhs * nrhs, st));

    // K5: LR projection (Sec. 5.3 step iii) and the exact deflated part, or
    // the Schur projection (Sec. 5.2 step iii)
    const int m = g->m;
    const bool schur = m > 0 && g->scheme == DEFL_SCHUR;
    const void* Sb = tp == PREC_F64 ? g->R64 : g->R32;  // Schur vectors (schur)
    const int S1 = gdots_stride(1, std::max(m, 1));
    const long long x_rhs = (long long)kw.mdef * kmax;  // Schur: X = S^H H_w V_k per right-hand side
    // v_r -= S coef_r (the Schur vectors shared by all right-hand sides)
    auto schur_out = [&](const void* coef, long long coef_stride, void* v) -> int {
        if (tp == PREC_F32 && m <= 1536)
            KL(OVS_PROF_PROJ, bytes_update(N, tp, tp, m, nrhs, true, true),
               launch_shared_combine(PREC_F32, Sb, units, m, coef, coef_stride, -1.0, v, N, v, N, units, nrhs, st));
        else
            KL(OVS_PROF_PROJ, bytes_update(N, tp, tp, m, nrhs, true, true),
               launch_update(tp, tp, Sb, 0, units, m, nullptr, coef, coef_stride, -1.0, v, N, v, N, units, plan, nrhs,
                             nullptr, nullptr, st));
        return OVS_OK;
    };
    // partial sums of S^H v_r over pblk blocks (reduced by the caller): in the
    // mixed form the shared-basis kernel that reads S once for all
    // right-hand sides, else the register sweep
    const int sdb = (tp == PREC_F32 && m > 0) ? shared_dots_blocks(m, nrhs, units, g->num_sms, kw.nblk) : 0;
    const int pblk = sdb > 0 ? sdb : plan.nblk;
    auto shared_dots = [&](const void* basis, const void* v, const int* act) -> int {
        if (sdb > 0)
            KL(OVS_PROF_PROJ, bytes_dots(N, tp, m, nrhs, true),
               launch_shared_dots(basis, units, m, v, units, nrhs, units, sdb, kw.partial, S1, act, st));
        else
            KL(OVS_PROF_PROJ, bytes_dots(N, tp, m, nrhs, true),
               launch_gdots(tp, 1, basis, 0, units, m, v, units, nullptr, 0, false, units, plan, nrhs, kw.partial, act,
                            st));
        return OVS_OK;
    };
    auto schur_dots = [&](const void* v) -> int { return shared_dots(Sb, v, kw.active); };
    if (schur) {
        // c = S^H x, x_perp = x - S c, classical Gram-Schmidt applied twice
        CK(cudaMemsetAsync(kw.active, 0xff, sizeof(int) * nrhs, st));
        TRY(schur_dots(w.xint));
        KL(OVS_PROF_SMALL, 16.0 * pblk * S1 * nrhs,
           launch_reduce(kw.partial, pblk, S1, m, nrhs, kw.cdef, m, false, nullptr, st));
        TRY(schur_out(kw.cdef, m, w.xint));
        TRY(schur_dots(w.xint));
        KL(OVS_PROF_SMALL, 16.0 * pblk * S1 * nrhs,
           launch_reduce(kw.partial, pblk, S1, m, nrhs, kw.cdef2, m, false, nullptr, st));
        TRY(schur_out(kw.cdef2, m, w.xint));
        KL(OVS_PROF_SMALL, 16.0 * pblk * S1 * nrhs,
           launch_reduce(kw.partial, pblk, S1, m, nrhs, kw.cdef, m, true, nullptr, st));
        CK(cudaMemsetAsync(w.yacc, 0, f64 * nrhs, st));
    } else if (m > 0) {
        const void* Lb = tp == PREC_F64 ? g->L64 : g->L32;
        const void* Rb = tp == PREC_F64 ? g->R64 : g->R32;
        TRY(shared_dots(Lb, w.xint, nullptr));
        KL(OVS_PROF_SMALL, 16.0 * pblk * S1 * nrhs,
           launch_reduce(kw.partial, pblk, S1, m, nrhs, kw.cdef, m, false, nullptr, st));
        KL(OVS_PROF_SMALL, 32.0 * m * nrhs, launch_sign_scale(kw.cdef, g->sgn, m, nrhs, kw.cdef2, st));
        if (tp == PREC_F32 && m <= 1536)
            KL(OVS_PROF_PROJ, bytes_update(N, tp, tp, m, nrhs, true, true),
               launch_shared_combine(PREC_F32, Rb, units, m, kw.cdef, m, -1.0, w.xint, N, w.xint, N, units, nrhs, st));
        else
            KL(OVS_PROF_PROJ, bytes_update(N, tp, tp, m, nrhs, true, true),
               launch_update(tp, tp, Rb, 0, units, m, nullptr, kw.cdef, m, -1.0, w.xint, N, w.xint, N, units, plan,
                             nrhs, nullptr, nullptr, st));
        // y = R sgn(Lambda) c into the complex128 accumulator: from the FP64
        // copy of R in the FP64 form; from the complex64 copy (FP32 products,
        // FP64 sums over 16 terms) in the mixed form, whose FP64 units would
        // otherwise bound it (4 DFMA per complex entry and vector)
        if (tp == PREC_F64)
            KL(OVS_PROF_PROJ, bytes_update(N, PREC_F64, PREC_F64, m, nrhs, true, false),
               launch_update(PREC_F64, PREC_F64, g->R64, 0, N, m, nullptr, kw.cdef2, m, 1.0, nullptr, 0, w.yacc, N, N,
                             plan64, nrhs, nullptr, nullptr, st));
        else if (m <= 1536)
            KL(OVS_PROF_PROJ, bytes_update(N, PREC_F32, PREC_F64, m, nrhs, true, false),
               launch_shared_combine(PREC_F64, g->R32, units, m, kw.cdef2, m, 1.0, nullptr, 0, w.yacc, N, units, nrhs,
                                     st));
        else
            KL(OVS_PROF_PROJ, bytes_update(N, PREC_F32, PREC_F64, m, nrhs, true, false),
               launch_update(PREC_F32, PREC_F64, g->R32, 0, units, m, nullptr, kw.cdef2, m, 1.0, nullptr, 0, w.yacc,
                             N, units, plan, nrhs, nullptr, nullptr, st));
    } else {
        CK(cudaMemsetAsync(w.yacc, 0, f64 * nrhs, st));
    }
    CK(cudaMemsetAsync(kw.active, 0xff, sizeof(int) * nrhs, st));  // every rhs starts active (-1 != 0)
    CK(cudaMemsetAsync(kw.est, 0, sizeof(double) * nrhs, st));
    CheckState* cstate = static_cast<CheckState*>(kw.cstate);
    const bool skip = (opts->flags & OVS_APPLY_SKIP_AHEAD) != 0;
    const int check_cap = every > 0 ? every * ((k - 1) / every) : 0;
    if (every > 0) {  // ccheck[0]: the coefficients of the last check (none yet: zero)
        CK(cudaMemsetAsync(kw.ccheck[0], 0, sizeof(double2) * kmax * nrhs, st));
        KL(OVS_PROF_SMALL, 32.0 * nrhs, launch_check_init(cstate, every, nrhs, st));
    }

    // Arnoldi (Sec. 4, Eq. Arnoldi; Sec. 5.3 Eq. LRArnoldi) with classical
    // Gram-Schmidt applied twice, the second pass of step j-1 done in the
    // same sweep as the first pass of step j. u (in xint) is the first-pass
    // residual, x_ominus at the start; z = A u (in wvec).
    const double bw = bytes_wilson(g->V, tp, nrhs);
    const StencilShape sh = stencil_shape(g, tp, nrhs, w.xint, fb, w.wvec, fb, st);
    for (int j = 0; j < k; ++j) {
        const int S = gdots_stride(2, j);
        KL(OVS_PROF_MATVEC, bw,
           launch_wilson(tp, true, links_for(g, tp), w.xint, fb, w.wvec, fb, g->geom, nrhs, g->kappa, g->mu,
                         kw.active, st, sh));
        if (schur) {
            // modified Arnoldi (Eq. modArnoldi): z <- z - S (S^H z), twice;
            // xz = S^H z (both passes) lands in column j of X
            char* Xj = (char*)kw.X + sizeof(double2) * (size_t)j * m;
            TRY(schur_dots(w.wvec));
            KL(OVS_PROF_SMALL, 16.0 * pblk * S1 * nrhs,
               launch_reduce(kw.partial, pblk, S1, m, nrhs, Xj, x_rhs, false, kw.active, st));
            TRY(schur_out(Xj, x_rhs, w.wvec));
            TRY(schur_dots(w.wvec));
            KL(OVS_PROF_SMALL, 16.0 * pblk * S1 * nrhs,
               launch_reduce(kw.partial, pblk, S1, m, nrhs, kw.cdef2, m, false, kw.active, st));
            TRY(schur_out(kw.cdef2, m, w.wvec));
            KL(OVS_PROF_SMALL, 16.0 * pblk * S1 * nrhs,
               launch_reduce(kw.partial, pblk, S1, m, nrhs, Xj, x_rhs, true, kw.active, st));
        }
        const bool tma = (tp == PREC_F32) && tma_update_fits(j);
        const bool chunked = (tp == PREC_F32) && gdots_chunk_fits(j);
        const int dblk = chunked ? dslots : plan.nblk;
        if (chunked)
            KL(OVS_PROF_DOTS, (double)N * sz_of(tp) * nrhs * (j + 2.0),
               launch_gdots2_chunk(basis, basis_rhs_units, units, j, w.xint, units, w.wvec, units, units, nrhs,
                                   g->num_sms, dslots, kw.partial, kw.active, kw.err, st));
        else
            KL(OVS_PROF_DOTS, (double)N * sz_of(tp) * nrhs * (j + 2.0),
               launch_gdots(tp, 2, basis, basis_rhs_units, units, j, w.xint, units, w.wvec, units, true, units, plan,
                            nrhs, kw.partial, kw.active, st));
        KL(OVS_PROF_SMALL, 16.0 * dblk * S * nrhs,
           launch_reduce(kw.partial, dblk, S, S, nrhs, kw.htmp, kw.jcap, false, kw.active, st));
        KL(OVS_PROF_SMALL, 16.0 * 3.0 * j * nrhs,
           launch_arnoldi_step(kw.htmp, kw.jcap, j, kw.H, h_rhs, ldh, kw.beta, kw.inv_beta, kw.dcoef, kw.hnorm2,
                               kw.active, kw.k_used, nrhs, st));
        if (schur)  // X[:, j] = (xz - X[:, <j] s) / beta_j
            KL(OVS_PROF_SMALL, 16.0 * ((double)m * j + 2.0 * m) * nrhs,
               launch_schur_xcol(kw.X, x_rhs, m, j, kw.htmp, kw.jcap, kw.inv_beta, kw.active, nrhs, st));
        KL(OVS_PROF_SMALL, 16.0 * ((double)j * j / 2 + 2.0 * j) * nrhs,
           launch_arnoldi_column(kw.htmp, kw.jcap, j, kw.H, h_rhs, ldh, kw.inv_beta, kw.dcoef, kw.active, nrhs, st));
        // A7 (batched form): at the checks (every `every` steps, or on the
        // skip-ahead schedule) the sign of the complete H_j of each active
        // right-hand side that is due; stop it once successive coefficient
        // vectors agree to tol (V orthonormal, so this is the change of its
        // Krylov part).
        if (every > 0 && j > 0 && j % every == 0) {
            KL(OVS_PROF_SMALL, 12.0 * nrhs, launch_check_due(kw.active, cstate, j, kw.due, nrhs, st));
            KL(OVS_PROF_NEWTON, 16.0 * (double)j * j * nrhs,
               launch_newton(kw.H, h_rhs, ldh, kw.k_used, kw.beta, kw.ccheck[1], kmax, kw.newton, (int)kmax, nrhs,
                             kw.iters, kw.status, st, kw.due, j));
            KL(OVS_PROF_SMALL, 48.0 * j * nrhs,
               launch_conv_check(kw.ccheck[1], kw.ccheck[0], kmax, j, opts->tol, kw.active, kw.k_used, kw.est,
                                 kw.due, cstate, every, check_cap, skip, nrhs, st));
        }
        if (tma)
            KL(OVS_PROF_UPDATE, (double)N * sz_of(tp) * nrhs * (j + 4.0),
               launch_arnoldi_update_tma(basis, basis_rhs_units, units, j, kw.htmp, kw.jcap, kw.inv_beta, kw.dcoef,
                                         w.xint, units, w.wvec, units, units, nrhs, g->num_sms, kw.active, kw.err, st));
        else
            KL(OVS_PROF_UPDATE, (double)N * sz_of(tp) * nrhs * (j + 4.0),
               launch_arnoldi_update(tp, basis, basis_rhs_units, units, j, kw.htmp, kw.jcap, kw.inv_beta, kw.dcoef,
                                     w.xint, units, w.wvec, units, units, plan, nrhs, kw.active, st));
    }
    if (tp == PREC_F32 && gdots_chunk_fits(k)) {  // second Gram-Schmidt pass of the last column
        // the two-vector TMA sweep with z = u: s (and a copy as t), u^H u at 2k
        const int S = gdots_stride(2, k);
        KL(OVS_PROF_DOTS, (double)N * sz_of(tp) * nrhs * (k + 1.0),
           launch_gdots2_chunk(basis, basis_rhs_units, units, k, w.xint, units, w.xint, units, units, nrhs,
                               g->num_sms, dslots, kw.partial, kw.active, kw.err, st));
        KL(OVS_PROF_SMALL, 16.0 * dslots * S * nrhs,
           launch_reduce(kw.partial, dslots, S, S, nrhs, kw.htmp, kw.jcap, false, kw.active, st));
        KL(OVS_PROF_SMALL, 16.0 * 2.0 * k * nrhs,
           launch_arnoldi_final(kw.htmp, kw.jcap, k, 2 * k, kw.H, h_rhs, ldh, kw.active, nrhs, st));
    } else {
        const int S = gdots_stride(1, k);
        KL(OVS_PROF_DOTS, (double)N * sz_of(tp) * nrhs * (k + 1.0),
           launch_gdots(tp, 1, basis, basis_rhs_units, units, k, w.xint, units, nullptr, 0, true, units, plan, nrhs,
                        kw.partial, kw.active, st));
        KL(OVS_PROF_SMALL, 16.0 * plan.nblk * S * nrhs,
           launch_reduce(kw.partial, plan.nblk, S, S, nrhs, kw.htmp, kw.jcap, false, kw.active, st));
        KL(OVS_PROF_SMALL, 16.0 * 2.0 * k * nrhs,
           launch_arnoldi_final(kw.htmp, kw.jcap, k, k, kw.H, h_rhs, ldh, kw.active, nrhs, st));
    }
    // harmonic variant (Sec. 4): H_k -> H_k + |h_(k+1,k)|^2 H_k^-H e_k e_k^T
    if (opts->flags & OVS_APPLY_HARMONIC)
        KL(OVS_PROF_SMALL, 16.0 * (double)k * (k + 1) * nrhs,
           launch_harmonic(kw.H, h_rhs, ldh, kw.k_used, kw.newton, (int)kmax, nrhs, st));
    // K3: beta sgn(H_k) e_1 (Sec. 5.3 step v; Sec. 5.2 step v for H_k); a
    // right-hand side stopped by a convergence check has it already
    if (every > 0)
        KL(OVS_PROF_SMALL, 32.0 * k * nrhs,
           launch_check_final(cstate, kw.ccheck[0], kw.coeff, kmax, kw.k_used, kw.due, nrhs, st));
    KL(OVS_PROF_NEWTON, 16.0 * (double)k * k * nrhs,
       launch_newton(kw.H, h_rhs, ldh, kw.k_used, kw.beta, kw.coeff, kmax, kw.newton, (int)kmax, nrhs, kw.iters,
                     kw.status, st, every > 0 ? kw.due : nullptr, 0, k));  // k_used[r] <= k
    if (schur) {
        // Schur coefficients sgn(T) c + beta Y e_1 (App. A), then y = S cS
        KL(OVS_PROF_SMALL, 16.0 * ((double)m * k * 4 + (double)k * k) * nrhs,
           launch_schur_coeff(g->schurT, g->schurFT, m, kw.X, x_rhs, kw.H, h_rhs, ldh, kw.newton, 2 * kmax * kmax,
                              kw.k_used, kw.status, kw.beta, kw.cdef, m, kw.sylv, kw.cS, m, nrhs, k, st));
        if (tp == PREC_F64)
            KL(OVS_PROF_PROJ, bytes_update(N, PREC_F64, PREC_F64, m, nrhs, true, false),
               launch_update(PREC_F64, PREC_F64, g->R64, 0, N, m, nullptr, kw.cS, m, 1.0, nullptr, 0, w.yacc, N, N,
                             plan64, nrhs, nullptr, nullptr, st));
        else if (m <= 1536)
            KL(OVS_PROF_PROJ, bytes_update(N, PREC_F32, PREC_F64, m, nrhs, true, false),
               launch_shared_combine(PREC_F64, g->R32, units, m, kw.cS, m, 1.0, nullptr, 0, w.yacc, N, units, nrhs,
                                     st));
        else
            KL(OVS_PROF_PROJ, bytes_update(N, PREC_F32, PREC_F64, m, nrhs, true, false),
               launch_update(PREC_F32, PREC_F64, g->R32, 0, units, m, nullptr, kw.cS, m, 1.0, nullptr, 0, w.yacc,
                             N, units, plan, nrhs, nullptr, nullptr, st));
    }
    // K4: y += V_k c (Sec. 5.3 step vi)
    if (tp == PREC_F32 && recombine_tma_fits(k))
        KL(OVS_PROF_PROJ, bytes_update(N, tp, PREC_F64, k, nrhs, false, true),
           launch_recombine_tma(basis, basis_rhs_units, units, k, kw.k_used, kw.coeff, kmax, 1.0, w.yacc, N, units,
                                nrhs, g->num_sms, nullptr, kw.err, st));
    else
        KL(OVS_PROF_PROJ, bytes_update(N, tp, PREC_F64, k, nrhs, false, true),
           launch_update(tp, PREC_F64, basis, basis_rhs_units, units, k, kw.k_used, kw.coeff, kmax, 1.0, w.yacc, N,
                         w.yacc, N, units, plan, nrhs, nullptr, nullptr, st));
    if (overlap)  // D_ov(mu) x = x + gamma5 sgn(H_w) x (Sec. 2, Eq. Dov), fused into the layout pass
        KL(OVS_PROF_LAYOUT, bytes_layout(N, PREC_F64, nrhs) + 16.0 * N * nrhs,
           launch_to_canonical_overlap(w.yacc, f64, xd, N, yd, N, V, nrhs, st));
    else
        KL(OVS_PROF_LAYOUT, bytes_layout(N, PREC_F64, nrhs),
           launch_to_canonical(PREC_F64, w.yacc, f64, yd, N, V, nrhs, st));
    return OVS_OK;
}

static void remember_apply(ovs_gauge_s* g, int nrhs, const ovs_apply_opts* opts, cudaStream_t st) {
    g->last_nrhs = nrhs;
    g->last_stream = st;
    g->last_every = opts->check_every;
    g->last_tol = opts->tol;
    g->last_kmax = opts->k_max;
}

extern "C" {

}  // extern "C"

// ovs_sign_apply (overlap = false) and ovs_overlap_apply (overlap = true)
static int apply_entry(ovs_gauge_t g, const void* x, void* y, int32_t nrhs, const ovs_apply_opts* opts,
                       ovs_apply_info* info, void* stream, bool overlap) {
    if (!x || !y) return fail(OVS_EINVAL, "NULL argument");
    TRY(check_apply(g, nrhs, opts));
    cudaStream_t st = (cudaStream_t)stream;
    const int tp = tprec_of(opts->prec);
    TRY(ensure_vec(g, nrhs, tp));
    TRY(ensure_kry(g, nrhs, opts->k_max, tp));
    const size_t f64 = field_bytes(g->N, PREC_F64);
    const bool xdev = is_device_ptr(x), ydev = is_device_ptr(y);
    const void* xd = x;
    if (!xdev) {
        CK(cudaMemcpyAsync(g->vw.sx, x, f64 * nrhs, cudaMemcpyHostToDevice, st));
        xd = g->vw.sx;
    }
    void* yd = ydev ? y : g->vw.sy;
    TRY(sign_apply_core(g, xd, yd, nrhs, opts, st, overlap));
    if (!ydev) CK(cudaMemcpyAsync(y, yd, f64 * nrhs, cudaMemcpyDeviceToHost, st));
    remember_apply(g, nrhs, opts, st);
    if (info) return ovs_get_info(g, info, nrhs);
    if (!ydev) CK(cudaStreamSynchronize(st));
    return OVS_OK;
}

extern "C" {

int ovs_sign_apply(ovs_gauge_t g, const void* x, void* y, int32_t nrhs, const ovs_apply_opts* opts,
                   ovs_apply_info* info, void* stream) {
    return apply_entry(g, x, y, nrhs, opts, info, stream, false);
}

int ovs_overlap_apply(ovs_gauge_t g, const void* x, void* y, int32_t nrhs, const ovs_apply_opts* opts,
                      ovs_apply_info* info, void* stream) {
    return apply_entry(g, x, y, nrhs, opts, info, stream, true);
}

int ovs_overlap_solve(ovs_gauge_t g, const void* b, void* x, int32_t nrhs, const ovs_apply_opts* inner,
                      const ovs_solve_opts* outer, ovs_solve_info* info, void* stream) {
    if (!b || !x || !outer) return fail(OVS_EINVAL, "NULL argument");
    TRY(check_apply(g, nrhs, inner));
    const int restart = outer->restart;
    if (restart < 1 || restart > 256) return fail(OVS_EINVAL, "restart must be in [1, 256]");
    if (outer->max_cycles < 1) return fail(OVS_EINVAL, "max_cycles must be >= 1");
    if (!(outer->tol > 0.0)) return fail(OVS_EINVAL, "tol must be > 0");
    cudaStream_t st = (cudaStream_t)stream;
    const int tp = tprec_of(inner->prec);
    TRY(ensure_vec(g, nrhs, tp));
    TRY(ensure_kry(g, nrhs, inner->k_max, tp));
    const long long N = g->N;
    const size_t f64 = field_bytes(N, PREC_F64);
    const int jc = gdots_stride(1, restart + 1);
    const BlasPlan plan = blas_plan(N, nrhs, g->num_sms);
    const int nb = norm_blocks();
    // work space of the outer iteration, owned by this call
    struct Bufs {
        std::vector<void*> p;
        ~Bufs() {
            for (void* q : p)
                if (q) cudaFree(q);
        }
        void* get(size_t bytes) {  // nullptr (recorded) when the allocation fails
            void* q = nullptr;
            if (cudaMalloc(&q, bytes) != cudaSuccess) {
                cudaGetLastError();
                q = nullptr;
            }
            p.push_back(q);
            return q;
        }
    } bufs;
    void* W = bufs.get(f64 * (size_t)(restart + 1) * nrhs);
    void* z = bufs.get(f64 * nrhs);
    void* r = bufs.get(f64 * nrhs);
    const bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
    void* bd = bdev ? const_cast<void*>(b) : bufs.get(f64 * nrhs);
    void* xd = xdev ? x : bufs.get(f64 * nrhs);
    void* red1 = bufs.get(sizeof(double2) * (size_t)jc * nrhs);
    void* red2 = bufs.get(sizeof(double2) * (size_t)jc * nrhs);
    void* part = bufs.get(sizeof(double2) * (size_t)plan.nblk * jc * nrhs);
    double* npart = (double*)bufs.get(sizeof(double) * (size_t)nb * nrhs);
    void* R = bufs.get(sizeof(double2) * (size_t)restart * restart * nrhs);
    void* rot = bufs.get(sizeof(double2) * 2 * (size_t)restart * nrhs);
    void* gv = bufs.get(sizeof(double2) * (size_t)(restart + 1) * nrhs);
    void* yv = bufs.get(sizeof(double2) * (size_t)restart * nrhs);
    double* sc = (double*)bufs.get(sizeof(double) * 5 * (size_t)nrhs);  // beta, 1/beta, est, 1/h, |r|
    for (void* q : bufs.p)
        if (!q) return fail(OVS_ENOMEM, "overlap_solve: device memory for the outer basis");
    double *beta = sc, *inv_beta = sc + nrhs, *est = sc + 2 * nrhs, *inv_hn = sc + 3 * nrhs, *rn = sc + 4 * nrhs;
    if (!bdev) CK(cudaMemcpyAsync(bd, b, f64 * nrhs, cudaMemcpyHostToDevice, st));
    std::vector<double> bnorm(nrhs), h_est(nrhs), h_ih(nrhs), h_rn(nrhs);
    CK(launch_norms(bd, N, N, nrhs, npart, rn, nullptr, st));
    CK(cudaMemcpyAsync(bnorm.data(), rn, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
    CK(cudaMemsetAsync(xd, 0, f64 * nrhs, st));
    CK(cudaMemcpyAsync(r, bd, f64 * nrhs, cudaMemcpyDeviceToDevice, st));
    CK(cudaStreamSynchronize(st));
    int iters = 0, cycles = 0;
    bool converged = false;
    for (int cyc = 1; cyc <= outer->max_cycles && !converged; ++cyc) {
        // w_0 = r / ||r||, g = ||r|| e_1
        CK(launch_norms(r, N, N, nrhs, npart, beta, inv_beta, st));
        CK(launch_scale(r, N, W, N, inv_beta, N, nrhs, st));
        CK(launch_gmres_start(beta, gv, restart, nrhs, st));
        int jj = 0;
        for (int j = 0; j < restart; ++j) {
            char* Wj = (char*)W + f64 * (size_t)j * nrhs;
            TRY(sign_apply_core(g, Wj, z, nrhs, inner, st, true));  // z = D_ov w_j
            ++iters;
            for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice
                void* red = pass ? red2 : red1;
                CK(launch_gdots(PREC_F64, 1, W, N, (long long)nrhs * N, j + 1, z, N, nullptr, 0, false, N, plan, nrhs,
                                part, nullptr, st));
                CK(launch_reduce(part, plan.nblk, gdots_stride(1, j + 1), j + 1, nrhs, red, jc, false, nullptr, st));
                CK(launch_update(PREC_F64, PREC_F64, W, N, (long long)nrhs * N, j + 1, nullptr, red, jc, -1.0, z, N, z,
                                 N, N, plan, nrhs, nullptr, nullptr, st));
            }
            CK(launch_norm_partials(z, N, N, nrhs, npart, st));
            CK(launch_gmres_col(red1, red2, jc, npart, j, restart, R, rot, gv, est, inv_hn, nrhs, st));
            jj = j + 1;
            if (j + 1 < restart) CK(launch_scale(z, N, (char*)W + f64 * (size_t)(j + 1) * nrhs, N, inv_hn, N, nrhs, st));
            CK(cudaMemcpyAsync(h_est.data(), est, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(h_ih.data(), inv_hn, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            bool all = true, breakdown = false;
            for (int q = 0; q < nrhs; ++q) {
                all = all && !(h_est[q] > outer->tol * bnorm[q]);
                breakdown = breakdown || h_ih[q] == 0.0;
            }
            if (all || breakdown) break;
        }
        // x += W y with y = R^-1 g; true residual r = b - D_ov x
        CK(launch_gmres_backsub(R, gv, jj, restart, yv, nrhs, st));
        CK(launch_update(PREC_F64, PREC_F64, W, N, (long long)nrhs * N, jj, nullptr, yv, restart, 1.0, xd, N, xd, N, N,
                         plan, nrhs, nullptr, nullptr, st));
        TRY(sign_apply_core(g, xd, z, nrhs, inner, st, true));
        CK(launch_sub(bd, z, r, N, nrhs, st));
        CK(launch_norms(r, N, N, nrhs, npart, rn, nullptr, st));
        CK(cudaMemcpyAsync(h_rn.data(), rn, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        cycles = cyc;
        converged = true;
        for (int q = 0; q < nrhs; ++q) converged = converged && !(h_rn[q] > outer->tol * bnorm[q]);
    }
    if (!xdev) CK(cudaMemcpyAsync(x, xd, f64 * nrhs, cudaMemcpyDeviceToHost, st));
    remember_apply(g, nrhs, inner, st);
    // reports of the last inner application: timeouts and sign failures
    std::vector<ovs_apply_info> ii(nrhs);
    const int inner_rc = ovs_get_info(g, ii.data(), nrhs);
    if (inner_rc < 0) return inner_rc;
    int worst = OVS_OK;
    for (int q = 0; q < nrhs; ++q) {
        const double rel = bnorm[q] > 0.0 ? h_rn[q] / bnorm[q] : 0.0;
        const bool ok = !(h_rn[q] > outer->tol * bnorm[q]);
        int stq = ok ? OVS_OK : OVS_NOT_CONVERGED;
        if (ii[q].status == OVS_ESIGN) stq = OVS_ESIGN;
        if (stq == OVS_ESIGN) worst = OVS_ESIGN;
        else if (stq == OVS_NOT_CONVERGED && worst == OVS_OK) worst = OVS_NOT_CONVERGED;
        if (info) {
            info[q].iters = iters;
            info[q].cycles = cycles;
            info[q].status = stq;
            info[q].reserved = 0;
            info[q].rel_resid = rel;
        }
    }
    return worst;
}

int ovs_get_krylov(ovs_gauge_t g, int32_t rhs, int32_t* k_out, double* V, double* H) {
    if (!g || !k_out) return fail(OVS_EINVAL, "NULL argument");
    if (rhs < 0 || rhs >= g->last_nrhs) return fail(OVS_EINVAL, "rhs outside the last application");
    KryWork& kw = g->kw;
    CK(cudaStreamSynchronize(g->last_stream));
    int k = 0;
    CK(cudaMemcpy(&k, kw.k_used + rhs, sizeof(int), cudaMemcpyDeviceToHost));
    *k_out = k;
    if (k <= 0) return OVS_OK;
    const long long N = g->N;
    const int tp = kw.prec;
    const size_t fb = field_bytes(N, tp), f64 = field_bytes(N, PREC_F64);
    if (V) {
        void* tmp = nullptr;
        CK(dalloc(&tmp, f64 * k));
        const char* b = (const char*)kw.basis + fb * (size_t)(kw.kmax + 1) * rhs;
        cudaError_t e = launch_to_canonical(tp, b, fb, tmp, N, (int)g->V, k, 0);
        if (e == cudaSuccess) e = cudaMemcpy(V, tmp, f64 * k, cudaMemcpyDeviceToHost);
        cudaFree(tmp);
        CK(e);
    }
    if (H) {
        const int ldh = kw.kmax + 1;
        const double2* Hr = (const double2*)kw.H + (size_t)(kw.kmax + 1) * kw.kmax * rhs;
        CK(cudaMemcpy2D(H, sizeof(double2) * (k + 1), Hr, sizeof(double2) * ldh, sizeof(double2) * (k + 1), k,
                        cudaMemcpyDeviceToHost));
    }
    return OVS_OK;
}

}  // extern "C"

// Recorded application of a handle for (nrhs, opts): sign_apply_core from
// the staging buffers sx to sy, captured once on the handle's stream.
static int get_graph(ovs_gauge_s* g, int nrhs, const ovs_apply_opts* opts, ovs_gauge_s::GraphEntry** out) {
    for (auto& e : g->graphs)
        if (e.gen == g->gen && e.nrhs == nrhs && e.kmax == opts->k_max && e.prec == opts->prec &&
            e.every == opts->check_every && e.flags == opts->flags && e.tol == opts->tol) {
            *out = &e;
            return OVS_OK;
        }
    ovs_gauge_s::GraphEntry e;
    e.nrhs = nrhs;
    e.kmax = opts->k_max;
    e.prec = opts->prec;
    e.every = opts->check_every;
    e.flags = opts->flags;
    e.tol = opts->tol;
    e.gen = g->gen;
    long long l0[OVS_PROF_NCLASS];
    double b0[OVS_PROF_NCLASS];
    for (int c = 0; c < OVS_PROF_NCLASS; ++c) {
        l0[c] = g->prof_launches[c];
        b0[c] = g->prof_bytes[c];
    }
    CK(cudaStreamBeginCapture(g->istream, cudaStreamCaptureModeThreadLocal));
    g->capturing = true;
    const int rc = sign_apply_core(g, g->vw.sx, g->vw.sy, nrhs, opts, g->istream);
    g->capturing = false;
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(g->istream, &graph);
    for (int c = 0; c < OVS_PROF_NCLASS; ++c) {  // counted at replay time instead
        e.launches[c] = g->prof_launches[c] - l0[c];
        e.bytes[c] = g->prof_bytes[c] - b0[c];
        g->prof_launches[c] = l0[c];
        g->prof_bytes[c] = b0[c];
    }
    if (rc < 0) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    CK(ec);
    e.graph = graph;
    g->graphs.push_back(e);
    *out = &g->graphs.back();
    return OVS_OK;
}

extern "C" {

int ovs_sign_apply_batched(int32_t n, const ovs_gauge_t* gs, const void* const* x, void* const* y,
                           const int32_t* nrhs, const ovs_apply_opts* opts, ovs_apply_info* info, void* stream) {
    if (n <= 0 || !gs || !x || !y || !nrhs || !opts) return fail(OVS_EINVAL, "NULL argument or n <= 0");
    for (int i = 0; i < n; ++i) {
        if (!x[i] || !y[i]) return fail(OVS_EINVAL, "x[%d] or y[%d] is NULL", i, i);
        for (int j = 0; j < i; ++j)
            if (gs[j] == gs[i]) return fail(OVS_EINVAL, "handle %d appears twice (its buffers are not shared)", i);
        TRY(check_apply(gs[i], nrhs[i], opts));
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int tp = tprec_of(opts->prec);
    std::vector<ovs_gauge_s::GraphEntry*> ges(n);
    for (int i = 0; i < n; ++i) {
        ovs_gauge_s* g = gs[i];
        TRY(ensure_vec(g, nrhs[i], tp));
        TRY(ensure_kry(g, nrhs[i], opts->k_max, tp));
        // choose the stencil shape now: the recorded application cannot time it
        stencil_shape(g, tp, nrhs[i], g->vw.xint, field_bytes(g->N, tp), g->vw.wvec, field_bytes(g->N, tp), st);
        if (!g->istream) CK(cudaStreamCreateWithFlags(&g->istream, cudaStreamNonBlocking));
        TRY(get_graph(g, nrhs[i], opts, &ges[i]));
    }
    // the combined graph of these instances (built once, then replayed)
    cudaGraphExec_t exec = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_batch_mu);
        for (auto it = g_batches.begin(); it != g_batches.end() && !exec; ++it) {
            if ((int)it->uids.size() != n || it->kmax != opts->k_max || it->prec != opts->prec ||
                it->every != opts->check_every || it->flags != opts->flags || it->tol != opts->tol)
                continue;
            bool same = true;
            for (int i = 0; i < n && same; ++i)
                same = it->uids[i] == gs[i]->uid && it->gens[i] == gs[i]->gen && it->nrhs[i] == nrhs[i];
            if (same) exec = it->exec;
        }
        if (!exec) {
            // entries of these handles at older generations can never match again
            for (size_t q = 0; q < g_batches.size();) {
                bool stale = false;
                for (int i = 0; i < n && !stale; ++i)
                    for (size_t u = 0; u < g_batches[q].uids.size(); ++u)
                        stale = stale || (g_batches[q].uids[u] == gs[i]->uid && g_batches[q].gens[u] != gs[i]->gen);
                if (stale) {
                    cudaGraphExecDestroy(g_batches[q].exec);
                    g_batches.erase(g_batches.begin() + q);
                } else {
                    ++q;
                }
            }
            cudaGraph_t parent = nullptr;
            CK(cudaGraphCreate(&parent, 0));
            cudaError_t e = cudaSuccess;
            for (int i = 0; i < n && e == cudaSuccess; ++i) {
                cudaGraphNode_t node;
                e = cudaGraphAddChildGraphNode(&node, parent, nullptr, 0, ges[i]->graph);
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, parent, 0);
            cudaGraphDestroy(parent);
            CK(e);
            BatchEntry be;
            be.kmax = opts->k_max;
            be.prec = opts->prec;
            be.every = opts->check_every;
            be.flags = opts->flags;
            be.tol = opts->tol;
            be.exec = exec;
            for (int i = 0; i < n; ++i) {
                be.uids.push_back(gs[i]->uid);
                be.gens.push_back(gs[i]->gen);
                be.nrhs.push_back(nrhs[i]);
            }
            g_batches.push_back(be);
        }
    }
    // inputs into the instances' staging buffers, one launch for all
    // instances, outputs back; all on the caller's stream
    bool any_host = false;
    for (int i = 0; i < n; ++i) {
        ovs_gauge_s* g = gs[i];
        const size_t bytes = field_bytes(g->N, PREC_F64) * nrhs[i];
        const bool xdev = is_device_ptr(x[i]);
        CK(cudaMemcpyAsync(g->vw.sx, x[i], bytes, xdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    }
    CK(cudaGraphLaunch(exec, st));
    for (int i = 0; i < n; ++i) {
        ovs_gauge_s* g = gs[i];
        const size_t bytes = field_bytes(g->N, PREC_F64) * nrhs[i];
        const bool ydev = is_device_ptr(y[i]);
        any_host = any_host || !ydev;
        CK(cudaMemcpyAsync(y[i], g->vw.sy, bytes, ydev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
        for (int c = 0; c < OVS_PROF_NCLASS; ++c) {
            g->prof_launches[c] += ges[i]->launches[c];
            g->prof_bytes[c] += ges[i]->bytes[c];
        }
        remember_apply(g, nrhs[i], opts, st);
    }
    if (info) {
        int worst = OVS_OK, off = 0;
        for (int i = 0; i < n; ++i) {
            const int s = ovs_get_info(gs[i], info + off, nrhs[i]);
            if (s < 0) return s;
            if (s == OVS_ESIGN || worst == OVS_ESIGN) worst = OVS_ESIGN;
            else if (s == OVS_NOT_CONVERGED) worst = OVS_NOT_CONVERGED;
            off += nrhs[i];
        }
        return worst;
    }
    if (any_host) CK(cudaStreamSynchronize(st));
    return OVS_OK;
}

int ovs_get_info(ovs_gauge_t g, ovs_apply_info* info, int32_t nrhs) {
    if (!g || !info) return fail(OVS_EINVAL, "NULL argument");
    if (nrhs <= 0 || nrhs > g->last_nrhs) return fail(OVS_EINVAL, "nrhs exceeds the last application");
    CK(cudaStreamSynchronize(g->last_stream));
    std::vector<int> ku(nrhs), it(nrhs), stt(nrhs);
    std::vector<double> beta(nrhs), est(nrhs);
    CK(cudaMemcpy(est.data(), g->kw.est, sizeof(double) * nrhs, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(ku.data(), g->kw.k_used, sizeof(int) * nrhs, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(it.data(), g->kw.iters, sizeof(int) * nrhs, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(stt.data(), g->kw.status, sizeof(int) * nrhs, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(beta.data(), g->kw.beta, sizeof(double) * nrhs, cudaMemcpyDeviceToHost));
    int derr = 0;
    CK(cudaMemcpy(&derr, g->kw.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (derr != 0) {
        CK(cudaMemset(g->kw.err, 0, sizeof(int)));
        return fail(OVS_ETIMEOUT, "a bounded device wait gave up during the last sign application");
    }
    int worst = OVS_OK, bad_rhs = -1;
    for (int r = 0; r < nrhs; ++r) {
        if (!std::isfinite(beta[r])) {  // the (deflated) source had a NaN or an infinity
            stt[r] = OVS_EINVAL;
            if (bad_rhs < 0) bad_rhs = r;
        }
        info[r].k_used = ku[r];
        info[r].newton_iters = it[r];
        info[r].status = stt[r];
        info[r].reserved = 0;
        info[r].beta = beta[r];
        info[r].est_err = est[r];
        if (g->last_every > 0 && stt[r] == OVS_OK && !(est[r] < g->last_tol) && ku[r] >= g->last_kmax) {
            stt[r] = OVS_NOT_CONVERGED;  // the estimate never reached tol within k_max
            info[r].status = stt[r];
        }
        if (stt[r] == OVS_ESIGN) worst = OVS_ESIGN;
        else if (stt[r] == OVS_NOT_CONVERGED && worst == OVS_OK) worst = OVS_NOT_CONVERGED;
    }
    if (bad_rhs >= 0) {
        char msg[128];
        snprintf(msg, sizeof(msg), "right-hand side %d: the source is not finite (NaN or infinity)", bad_rhs);
        return fail(OVS_EINVAL, msg);
    }
    return worst;
}

int ovs_check_wait_timeout(void* stream) {
    int code = 0;
    const cudaError_t e = check_wait_timeout((cudaStream_t)stream, &code);
    if (e != cudaSuccess) return fail(OVS_ECUDA, cudaGetErrorString(e));
    if (code != OVS_ETIMEOUT) return fail(OVS_ECUDA, "the bounded wait of the self-check did not report a timeout");
    return OVS_ETIMEOUT;
}

int ovs_stencil_tuning(ovs_gauge_t g, int32_t prec, int32_t nrhs, int32_t* shape, float* ms) {
    if (!g || !shape) return fail(OVS_EINVAL, "NULL argument");
    if (prec != OVS_F64 && prec != OVS_MIXED) return fail(OVS_EINVAL, "bad prec");
    if (nrhs < 1) return fail(OVS_EINVAL, "nrhs < 1");
    const auto it = g->tuned.find(std::make_pair(tprec_of(prec), (int)nrhs));
    if (it == g->tuned.end()) return fail(OVS_ESTATE, "no stencil shape chosen yet for this (prec, nrhs)");
    shape[0] = it->second.best.rt;
    shape[1] = it->second.best.sites;
    shape[2] = it->second.best.rb;
    if (ms)
        for (int i = 0; i < kNumStencilShapes; ++i) ms[i] = it->second.ms[i];
    return OVS_OK;
}

int ovs_set_stencil_shape(ovs_gauge_t g, int32_t prec, int32_t nrhs, int32_t rt, int32_t sites, int32_t rb) {
    if (!g) return fail(OVS_EINVAL, "NULL handle");
    if (prec != OVS_F64 && prec != OVS_MIXED) return fail(OVS_EINVAL, "bad prec");
    if (nrhs < 1) return fail(OVS_EINVAL, "nrhs < 1");
    const auto key = std::make_pair(tprec_of(prec), (int)nrhs);
    if (rt == 0) {
        drop_graphs(g);
        g->tuned.erase(key);
        return OVS_OK;
    }
    for (int i = 0; i < kNumStencilShapes; ++i) {
        const StencilShape& c = kStencilShapes[i];
        if (c.rt == rt && c.sites == sites && c.rb == rb) {
            drop_graphs(g);
            ovs_gauge_s::Tuned t;
            t.best = c;
            for (int q = 0; q < kNumStencilShapes; ++q) t.ms[q] = 0.0f;
            g->tuned[key] = t;
            return OVS_OK;
        }
    }
    return fail(OVS_EINVAL, "not one of the stencil shapes (see ovs_stencil_tuning)");
}

int ovs_profile_enable(ovs_gauge_t g, int32_t timing) {
    if (!g) return fail(OVS_EINVAL, "NULL handle");
    prof_flush(g);
    for (int c = 0; c < OVS_PROF_NCLASS; ++c) {
        g->prof_ms[c] = 0.0;
        g->prof_bytes[c] = 0.0;
        g->prof_launches[c] = 0;
    }
    g->timing = timing != 0;
    return OVS_OK;
}

int ovs_profile_read(ovs_gauge_t g, double* ms, int64_t* launches, double* bytes) {
    if (!g) return fail(OVS_EINVAL, "NULL handle");
    prof_flush(g);
    for (int c = 0; c < OVS_PROF_NCLASS; ++c) {
        if (ms) ms[c] = g->prof_ms[c];
        if (launches) launches[c] = g->prof_launches[c];
        if (bytes) bytes[c] = g->prof_bytes[c];
    }
    return OVS_OK;
}

void ovs_destroy(ovs_gauge_t g) {
    if (!g) return;
    prof_flush(g);
    drop_batches_of(g->uid);
    drop_graphs(g);
    if (g->ev_join) cudaEventDestroy(g->ev_join);
    if (g->istream) cudaStreamDestroy(g->istream);
    for (auto& e : g->events) cudaEventDestroy(e);
    free_deflation(g);
    free_vec(g->vw);
    free_kry(g->kw);
    dfree(g->links64);
    dfree(g->links32);
    delete g;
}

}  // extern "C"
