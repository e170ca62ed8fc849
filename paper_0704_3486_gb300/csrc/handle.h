// Private definition of the library handle (shared by api.cu and eig.cu).
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <utility>
#include <vector>

#include "../../include/ovsign.h"
#include "common.cuh"
#include "kernels.h"

struct VecWork {  // per-right-hand-side vectors
    int nrhs = 0, prec = -1;
    void* xint = nullptr;  // [nrhs][N] precision prec (x, then x_ominus)
    void* wvec = nullptr;  // [nrhs][N] precision prec (Arnoldi w)
    void* yacc = nullptr;  // [nrhs][N] complex128 internal (y accumulator)
    void* sx = nullptr;    // [nrhs][N] complex128 canonical staging (host x)
    void* sy = nullptr;    // [nrhs][N] complex128 canonical staging (host y)
};

struct KryWork {  // Krylov basis and small matrices
    int nrhs = 0, kmax = 0, prec = -1, jcap = 0, nblk = 0;
    void* basis = nullptr;       // [nrhs][kmax+1][N] precision prec
    void* H = nullptr;           // [nrhs][(kmax+1) x kmax] complex128, column-major
    void* htmp = nullptr;        // [nrhs][jcap] complex128: reduced inner products of a sweep
    void* dcoef = nullptr;       // [nrhs] complex128
    int* err = nullptr;          // device error word (OVS_ETIMEOUT from bounded waits)
    void* ccheck[2] = {nullptr, nullptr};  // [nrhs][kmax] coefficient vectors of successive checks
    double* est = nullptr;                 // [nrhs] last convergence estimate
    int* due = nullptr;                    // [nrhs] checked at this step (A7)
    void* cstate = nullptr;                // [nrhs] CheckState: the check schedule (A7)
    void* partial = nullptr;     // [nrhs][nblk][jcap] complex128
    double* norm_part = nullptr; // [nrhs][nblk]
    double* beta = nullptr;
    double* inv_beta = nullptr;
    double* hnorm2 = nullptr;
    int* active = nullptr;
    int* k_used = nullptr;
    int* iters = nullptr;
    int* status = nullptr;
    void* coeff = nullptr;  // [nrhs][kmax] complex128
    void* newton = nullptr; // [nrhs][2 kmax^2] complex128
    void* cdef = nullptr;   // [nrhs][m] complex128 deflation coefficients
    void* cdef2 = nullptr;  // [nrhs][m] complex128 sgn-scaled (Schur: second-pass scratch)
    int mdef = 0;           // m the deflation buffers below were sized for
    void* X = nullptr;      // Schur: [nrhs][m x kmax] complex128, X = S^H H_w V_k (column-major)
    void* sylv = nullptr;   // Schur: [nrhs][2 m 800] complex128 Sylvester scratch (C, Y)
    void* cS = nullptr;     // Schur: [nrhs][m] complex128 coefficients of S in y
};

// deflation scheme installed on a handle
enum { DEFL_NONE = 0, DEFL_LR = 1, DEFL_SCHUR = 2 };

struct ovs_gauge_s {
    int dims[4];
    ovs::Geom geom;
    long long V = 0, N = 0;
    int prec = OVS_F64;
    int device = 0, num_sms = 148;
    bool mu_set = false;
    double mu = 0.0, m_w = 0.0, kappa = 0.0;
    void* links64 = nullptr;  // [4][9][V] double2
    void* links32 = nullptr;  // [4][9][V] float2 (OVS_MIXED)
    // deflation basis (internal layout). LR: R (right eigenvectors) and L
    // (left, biorthonormalised). Schur: R holds the Schur vectors S_m, L is
    // absent, schurT / schurFT are T_m and sgn(T_m) (column-major m x m).
    int m = 0;
    int scheme = DEFL_NONE;
    void* schurT = nullptr;
    void* schurFT = nullptr;
    void* R64 = nullptr;  // [m][N] double2 planes
    void* L64 = nullptr;  // biorthonormalised
    void* R32 = nullptr;  // [m][N/2] float4 planes
    void* L32 = nullptr;
    double* sgn = nullptr;  // device [m]
    std::vector<double> lambda;  // host 2m
    VecWork vw;
    KryWork kw;
    int last_nrhs = 0;
    cudaStream_t last_stream = nullptr;
    int last_every = 0, last_kmax = 0;
    double last_tol = 0.0;
    // tracing (ovs_profile_*)
    struct Pending {
        int cls, ev;
    };
    bool timing = false;
    double prof_ms[OVS_PROF_NCLASS] = {};
    double prof_bytes[OVS_PROF_NCLASS] = {};
    long long prof_launches[OVS_PROF_NCLASS] = {};
    std::vector<cudaEvent_t> events;
    std::vector<Pending> pending;
    cudaStream_t prof_stream = nullptr;
    // batched form: recorded applications (CUDA graphs) and a private stream
    struct GraphEntry {
        int nrhs, kmax, prec, every, flags;
        double tol;
        unsigned gen;
        cudaGraph_t graph;  // the recorded application (a child of the batched form's graphs)
        long long launches[OVS_PROF_NCLASS];
        double bytes[OVS_PROF_NCLASS];
    };
    std::vector<GraphEntry> graphs;
    unsigned gen = 1;  // bumped whenever buffers, mu or the deflation basis change
    unsigned long long uid = 0;  // unique over the process (keys of the combined batched graphs)
    bool capturing = false;
    cudaStream_t istream = nullptr;
    cudaEvent_t ev_join = nullptr;
    // stencil launch shapes chosen per (internal precision, nrhs)
    struct Tuned {
        ovs::StencilShape best;
        float ms[ovs::kNumStencilShapes];
    };
    std::map<std::pair<int, int>, Tuned> tuned;
    // statistics of the last ovs_deflate_setup
    int setup_iters[2] = {0, 0};
    long long setup_matvecs = 0;
    double setup_resid = 0.0;
    double setup_budget_s = 0.0;
};


namespace ovs {
int lib_fail(int code, const char* msg);
// Install R (right) and L (left) vectors given as device canonical
// complex128 [m][N]; L is biorthonormalised against R.
int install_deflation(ovs_gauge_s* g, int m, const void* Rc, const void* Lc, const double* lambda);
// Install Schur deflation from m right vectors (device canonical complex128
// [m][N]): S_m, T_m = S_m^H H_w S_m and sgn(T_m) (schur.cu).
int install_schur(ovs_gauge_s* g, int m, const void* Rc);
// Drop the deflation basis (and the recorded applications that used it).
void free_deflation(ovs_gauge_s* g);
// Stencil shape for (tp, nrhs) on this handle: the cached choice, else (not
// capturing) the fastest candidate timed on st with in -> out as operands.
StencilShape stencil_shape(ovs_gauge_s* g, int tp, int nrhs, const void* in, size_t in_stride, void* out,
                           size_t out_stride, cudaStream_t st);
}  // namespace ovs
