/*
 * ovsign.h -- C ABI of a GB300 (sm_103a) library that computes
 *
 *     y = sgn(H_w(mu)) x,      H_w(mu) = gamma5 D_w(mu),
 *
 * for the Wilson-Dirac operator at quark chemical potential mu, by the
 * deflated Arnoldi method of Bloch, Frommer, Lang and Wettig (2007):
 * LR deflation of critical eigenvectors (Sec. 5.3, Eq. fAxLRArn), an
 * Arnoldi basis of the deflated Krylov space (Sec. 4, Eq. Arnoldi) and the
 * sign of the small Hessenberg matrix by Roberts' Newton iteration
 * (Sec. 5.2, Eq. Roberts). Also: Schur deflation with the Sylvester solver
 * of App. A (Sec. 5.2), the harmonic (see-saw-free) variant of Sec. 4, and
 * the overlap operator D_ov(mu) = 1 + gamma5 sgn(H_w(mu)) (Sec. 2, Eq. Dov)
 * with its nested inversion.
 *
 * Conventions used throughout
 * ---------------------------
 *  - dims = {Lx, Ly, Lz, Lt}; V = Lx Ly Lz Lt sites; N = 12 V unknowns.
 *    Site s = ((t*Lz + z)*Ly + y)*Lx + x. Direction nu = 0,1,2,3 is x,y,z,t.
 *    Every extent must be >= 2. Boundaries: periodic in space, antiperiodic
 *    in time.
 *  - Vectors are complex128, interleaved (re, im), entry
 *    (s*4 + spin)*3 + colour; nrhs vectors are stored one after another
 *    ([nrhs][N]). Spin basis: chiral, gamma5 = diag(1, 1, -1, -1).
 *  - Links are complex128 [V][4][3][3] (row, column); U_nu(s) joins s to
 *    s + nu-hat.
 *  - D_w(mu) x(s) = x(s) - kappa sum_nu [ (1 - gamma_nu) e^{+mu d_nu3}
 *    U_nu(s) x(s+nu) + (1 + gamma_nu) e^{-mu d_nu3} U_nu(s-nu)^+ x(s-nu) ],
 *    kappa = 1/(8 + 2 m_w)  (Sec. 2, Eq. Dw, with the projectors in the
 *    order (1 - gamma) forward, which is gamma5-conjugate to the printed
 *    order and has the same spectrum).
 *  - Pointers to vectors may be device or host memory; the library asks the
 *    CUDA runtime which. Host buffers are staged through device memory with
 *    copies on the given stream. All device work is enqueued on `stream`
 *    (a cudaStream_t; NULL means the legacy default stream).
 *  - Every entry point returns an ovs_status; no C++ exception crosses
 *    the ABI. On error ovs_last_error() returns a message (thread local).
 *  - A handle is not thread safe: use one handle per host thread. The
 *    library owns the device memory behind a handle (links, deflation
 *    basis, Krylov workspaces, grown on demand with cudaMalloc) until
 *    ovs_destroy.
 */
#ifndef OVSIGN_H
#define OVSIGN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ovs_gauge_s* ovs_gauge_t;

typedef enum {
    OVS_OK = 0,
    OVS_NOT_CONVERGED = 1, /* result usable but flagged (see ovs_apply_info) */
    OVS_EINVAL = -1,       /* bad argument */
    OVS_ENOMEM = -2,       /* device or host allocation failed */
    OVS_ECUDA = -3,        /* CUDA runtime or library error */
    OVS_ESTATE = -4,       /* mu not set, or deflation required but absent */
    OVS_EEIG = -5,         /* eigensolver did not converge */
    OVS_ESIGN = -6,        /* sign undefined: eigenvalue on the imaginary axis */
    OVS_ETIMEOUT = -7,     /* a bounded device wait gave up */
    OVS_EIO = -8           /* file read/write failed or bad file */
} ovs_status;

/* Arithmetic of the path. OVS_F64: links, vectors and Krylov basis in
 * complex128. OVS_MIXED: links, matvec and Krylov basis in complex64 with
 * FP64 accumulation of Gram-Schmidt inner products, FP64 Hessenberg
 * entries, FP64 deflation coefficients and FP64 Newton sign; input and
 * output vectors stay complex128. */
enum { OVS_F64 = 0, OVS_MIXED = 1 };

/* Operators for ovs_matvec. */
enum { OVS_OP_DW = 0, OVS_OP_HW = 1, OVS_OP_HW2 = 2 };

/* Create a handle on the current CUDA device with a seeded SU(3) field:
 * per link l = 4 s + nu, eighteen normals from Philox4x32-10 (counter
 * (l mod 2^32, l div 2^32, j, 0), j = 0..8, key = seed) by Box-Muller,
 * A = normals as a complex 3x3, X = traceless Hermitian part of A,
 * U = exp(i eps X) (Taylor series with scaling and squaring), reunitarised
 * to SU(3). This is the synthetic stand-in for the paper's gauge ensembles
 * (Sec. 6). prec: OVS_F64 or OVS_MIXED (which precisions the handle keeps
 * on the device; OVS_MIXED keeps both). Errors: EINVAL (dims < 2, eps < 0,
 * bad prec), ENOMEM, ECUDA. */
int ovs_create_gauge(const int32_t dims[4], uint64_t seed, double eps, int32_t prec,
                     ovs_gauge_t* out);

/* Create a handle from caller links (host, complex128 [V][4][3][3]). The
 * library copies them; the caller keeps ownership of `links`. The links
 * need not be unitary. Errors: as ovs_create_gauge. */
int ovs_create_gauge_from_links(const int32_t dims[4], const double* links, int32_t prec,
                                ovs_gauge_t* out);

/* Copy the handle's complex128 links back to host `links_out`
 * ([V][4][3][3], 72 V doubles). Synchronises the device. */
int ovs_get_links(ovs_gauge_t g, double* links_out);

/* Set mu and the Wilson mass m_w (kappa = 1/(8 + 2 m_w), Sec. 2). The paper
 * takes m_w in (-2, 0); any m_w with 8 + 2 m_w != 0 is accepted. Clears any
 * deflation basis (it belongs to the old operator). Host only. */
int ovs_set_mu(ovs_gauge_t g, double mu, double m_w);

/* y = op x for nrhs vectors, op = OVS_OP_DW (D_w(mu)), OVS_OP_HW (H_w(mu)),
 * OVS_OP_HW2 (H_w(mu)^2, used to find the critical eigenvalues, Sec. 6).
 * prec selects the arithmetic (OVS_F64 or OVS_MIXED); x and y are
 * complex128 either way. x and y must not overlap. Errors: EINVAL, ESTATE
 * (mu not set), ECUDA. */
int ovs_matvec(ovs_gauge_t g, int32_t op, const void* x, void* y, int32_t nrhs, int32_t prec,
               void* stream);

/* ovs_matvec without any device allocation, for callers that cannot let a
 * library allocate: programs whose device memory is already handed out by
 * another allocator (so a cudaMalloc would fail or take memory it owns), and
 * loops that must not pay the device-wide synchronisation of cudaMalloc and
 * cudaFree. The paper has no counterpart: this is a service of the library.
 * The two work fields live in one fixed array compiled into the library,
 * 8 MiB per field, which every GPU that loads the library holds until the
 * process exits: nrhs * N <= 524288 (OVS_F64) or <= 1048576 (OVS_MIXED),
 * larger requests fail with OVS_EINVAL. x and y must be device pointers
 * (complex128, canonical layout, [nrhs][N]); host pointers fail with
 * OVS_EINVAL. The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture. The address is kept for the life of the
 * process: after a cudaDeviceReset of that device this entry point must not
 * be called again. All calls share the array: calls that overlap on the GPU
 * race on it and must be serialised by the caller. The current device must
 * be the handle's, and x and y on it (else OVS_EINVAL). The stencil uses the
 * launch shape the handle has chosen for (prec, nrhs), if any, without
 * tuning. Same results as ovs_matvec; errors as ovs_matvec plus the size
 * limit. */
int ovs_matvec_noalloc(ovs_gauge_t g, int32_t op, const void* x, void* y, int32_t nrhs, int32_t prec,
                       void* stream);

/* Compute the m critical eigenpairs of H_w(mu) on the GPU for LR deflation
 * (Sec. 5.3 step i, Sec. 6): eigenvalues of smallest |lambda| found through
 * H_w(mu)^2 (the paper's choice), right vectors R with H R = R Lambda, left
 * vectors as right eigenvectors of H_w(mu)^+ = H_w(-mu) (gamma5-
 * hermiticity), biorthonormalised so that L^+ R = I. The m kept are those
 * of smallest |Re lambda| among the converged right pairs that have a
 * converged left partner (eigenvalue conj(lambda) within relative distance
 * 1e-6); the left iteration starts from the right one's final block and
 * runs until m such pairs exist. tol: relative residual
 * ||H r - lambda r|| / ||H|| asked of each pair (e.g. 1e-10). eig_out, if
 * not NULL, receives the m eigenvalues as 2m doubles (re, im), sorted by
 * |Re lambda|. Synchronises the device. Errors: EINVAL, ESTATE, EEIG (fewer
 * than m matched pairs reached tol within the iteration budget; the nearest
 * pairs are installed instead and eig_out filled), ENOMEM, ECUDA. */
int ovs_deflate_setup(ovs_gauge_t g, int32_t m, double tol, double* eig_out);

/* Statistics of the last ovs_deflate_setup on this handle: iterations of
 * the right (iters[0]) and left (iters[1]) subspace iterations, the total
 * number of single-vector H_w applications, and the largest relative
 * residual ||H r - lambda r|| / ||H|| of the installed right pairs (any
 * pointer may be NULL). */
int ovs_deflate_stats(ovs_gauge_t g, int32_t* iters, int64_t* matvecs, double* max_resid);

/* Work limit of ovs_deflate_setup on this handle: wall-clock seconds for
 * the whole set-up (0 = no limit; default 0). When the limit is reached the
 * current Ritz pairs are installed and ovs_deflate_setup returns OVS_EEIG. */
int ovs_set_setup_budget(ovs_gauge_t g, double max_seconds);

/* Install a deflation basis given by the caller (host complex128 arrays
 * R and L of [m][N], lambda of 2m doubles). L is biorthonormalised against
 * R (L <- L (L^+ R)^-+). m = 0 removes deflation. Errors: EINVAL, ESTATE
 * (mu not set), ESIGN (some Re lambda == 0), ENOMEM, ECUDA. */
int ovs_deflate_load(ovs_gauge_t g, int32_t m, const double* R, const double* L,
                     const double* lambda);

/* Copy the installed basis to host buffers (any may be NULL):
 * R, L: [m][N] complex128 (L biorthonormalised), lambda: 2m doubles.
 * m_out receives m. Synchronises the device. */
int ovs_deflate_get(ovs_gauge_t g, int32_t* m_out, double* R, double* L, double* lambda);

/* Schur deflation (Sec. 5.2). Install it from m right eigenvectors of
 * H_w(mu) given by the caller (host complex128 [m][N], in the order their
 * Schur vectors are to take): S_m = orthonormal basis of their span with
 * the leading columns spanning the leading vectors (Cholesky QR, twice),
 * T_m = S_m^H H_w S_m with its strictly lower part (the eigenvectors'
 * residual) dropped, and sgn(T_m) by Roberts' iteration on the device
 * (Sec. 5.2 steps i-ii). Replaces any installed basis; m = 0 removes
 * deflation. ovs_deflate_get then returns S_m as R and diag(T_m) as lambda.
 * Errors: EINVAL (dependent vectors), ESTATE (mu not set), ESIGN (an
 * eigenvalue on the imaginary axis), ENOMEM, ECUDA. */
int ovs_deflate_load_schur(ovs_gauge_t g, int32_t m, const double* R);

/* ovs_deflate_setup for Schur deflation: the right eigenvectors only (the
 * paper's reason for the scheme: about half the set-up of LR deflation,
 * Sec. 5.4), the m of smallest |Re lambda| among the converged pairs, then
 * installed as by ovs_deflate_load_schur. ovs_set_setup_budget's limit
 * applies to the one iteration. Errors as ovs_deflate_setup. */
int ovs_deflate_setup_schur(ovs_gauge_t g, int32_t m, double tol, double* eig_out);

/* Scheme of the installed basis: 0 none, 1 LR (Sec. 5.3), 2 Schur
 * (Sec. 5.2); EINVAL for a NULL handle. */
int ovs_deflate_scheme(ovs_gauge_t g);

/* Save / restore an LR deflation basis to a binary file (header with dims,
 * mu, m_w, m and a checksum, then lambda, R, L in complex128). Restore
 * checks that dims, mu and m_w match the handle. Errors: EIO, ESTATE (also:
 * a Schur basis, which is rebuilt from its right vectors instead). */
int ovs_deflate_save(ovs_gauge_t g, const char* path);
int ovs_deflate_restore(ovs_gauge_t g, const char* path);

/* Options of a sign application. */
typedef struct {
    int32_t k_max;       /* Krylov dimension, 1..790 (Sec. 4 suggests even
                            values) */
    int32_t check_every; /* 0: run exactly k_max steps (stop only at breakdown);
                            >0 (even): every check_every steps compute
                            c_j = beta sgn(H_j) e_1 and stop a right-hand
                            side once ||c_j - c_{j-check_every}|| / ||c_j||
                            (zero-padded) is below tol; V is orthonormal,
                            so this is the change of its Krylov part */
    int32_t prec;        /* OVS_F64 or OVS_MIXED */
    int32_t flags;       /* 0, OVS_APPLY_HARMONIC or OVS_APPLY_SKIP_AHEAD
                            (other bits: EINVAL) */
    double tol;          /* tolerance for check_every > 0 */
} ovs_apply_opts;

/* opts->flags: the harmonic variant of Sec. 4, which removes the even/odd
 * see-saw of the error in k: sgn(H_k) is replaced by sgn(H^_k) with
 * H^_k = H_k + |h_(k+1,k)|^2 H_k^-H e_k e_k^T (its eigenvalues are the
 * harmonic Ritz values of H_w on the Krylov space); y = ... + beta V_k
 * sgn(H^_k) e_1. Needs check_every = 0 and no Schur deflation. */
#define OVS_APPLY_HARMONIC 1

/* opts->flags: skip-ahead schedule of the convergence checks (needs
 * check_every > 0; not a method of the paper, which fixes k). The checks
 * stay on multiples of check_every, up to J = check_every floor((k_max-1) /
 * check_every). A check whose previous check lies check_every steps back
 * gives a one-interval estimate. After two of them, e0 at j0 and e1 < e0 at
 * j1, the estimate is extrapolated geometrically: it reaches tol after
 * n = log(tol/e1) / (log(e1/e0)/(j1-j0)) more steps, and the checks (and
 * their sign computations) are skipped up to P = check_every floor((j1 + n)
 * / check_every) - check_every (at most J - check_every). The check at P
 * only stores its coefficients, unless its estimate (over the longer
 * interval) is already below tol; the check at P + check_every gives the
 * next one-interval estimate. Every stop still needs an estimate below tol;
 * est_err is the last estimate formed. */
#define OVS_APPLY_SKIP_AHEAD 2

/* Per right-hand-side report. */
typedef struct {
    int32_t k_used;       /* Krylov dimension used (< k_max after breakdown) */
    int32_t newton_iters; /* Roberts iterations on H_k */
    int32_t status;       /* OVS_OK, OVS_NOT_CONVERGED, OVS_ESIGN, or OVS_EINVAL
                             when the source of this right-hand side is not
                             finite (the call then returns OVS_EINVAL) */
    int32_t reserved;
    double beta;          /* ||x_ominus||, the norm of the deflated source */
    double est_err;       /* last error estimate (check_every > 0), else 0 */
} ovs_apply_info;

/* y = sgn(H_w(mu)) x for nrhs vectors (Sec. 5.3, Eq. fAxLRArn):
 *   c = L^+ x, x_ominus = x - R c, y = R sgn(Re Lambda) c
 *     + beta V_k sgn(H_k) e_1 with the Arnoldi basis V_k of
 *   K_k(H_w, x_ominus), beta = ||x_ominus||; without a deflation basis the
 *   first three terms vanish (Sec. 4, Eq. yproj3). With Schur deflation
 *   (Sec. 5.2, Eq. formula): c = S^H x, x_perp = x - S c, V_k from the
 *   modified Arnoldi recurrence that also orthogonalises against S
 *   (Eq. modArnoldi), X = S^H H_w V_k, Y from T Y - Y H_k = sgn(T) X
 *   - X sgn(H_k) by the row recurrences of App. A, and y = S (sgn(T) c
 *   + beta Y e_1) + beta V_k sgn(H_k) e_1 (check_every must be 0).
 * Each right-hand side has its own Krylov basis; all are advanced together.
 * x: input [nrhs][N], y: output [nrhs][N] (complex128, host or device, must
 * not overlap). If info is not NULL the call waits for the stream and fills
 * nrhs reports; if NULL the call returns once the work is enqueued and
 * ovs_get_info() reads the reports later. Returns the worst per-RHS status
 * when info is given. Errors: EINVAL (also: a right-hand side whose source
 * is not finite, reported when the reports are read), ESTATE (mu not set),
 * ENOMEM (the handle stays usable), ECUDA, ETIMEOUT (a bounded device wait
 * gave up; reported when the reports are read). */
int ovs_sign_apply(ovs_gauge_t g, const void* x, void* y, int32_t nrhs, const ovs_apply_opts* opts,
                   ovs_apply_info* info, void* stream);

/* y = D_ov(mu) x = x + gamma5 sgn(H_w(mu)) x for nrhs vectors (Sec. 2,
 * Eq. Dov): ovs_sign_apply with the last step fused into the output layout
 * pass. Arguments, reports and errors as ovs_sign_apply. */
int ovs_overlap_apply(ovs_gauge_t g, const void* x, void* y, int32_t nrhs, const ovs_apply_opts* opts,
                      ovs_apply_info* info, void* stream);

/* Options and per-right-hand-side report of the nested inversion. */
typedef struct {
    int32_t restart;    /* outer Krylov dimension per cycle, 1..256 */
    int32_t max_cycles; /* restarts allowed, >= 1 */
    double tol;         /* stop once ||b - D_ov x|| <= tol ||b|| */
} ovs_solve_opts;

typedef struct {
    int32_t iters;      /* D_ov applications inside the cycles (all rhs advance together) */
    int32_t cycles;     /* cycles run */
    int32_t status;     /* OVS_OK, OVS_NOT_CONVERGED or OVS_ESIGN */
    int32_t reserved;
    double rel_resid;   /* ||b - D_ov x|| / ||b||, recomputed at the end of the last cycle */
} ovs_solve_info;

/* Solve D_ov(mu) x = b for nrhs right-hand sides by nested iteration: an
 * outer restarted GMRES (zero initial guess, classical Gram-Schmidt applied
 * twice, the least-squares problem updated by Givens rotations on the
 * device) whose every iteration applies D_ov through the deflated Arnoldi
 * method with `inner` and the installed deflation basis, which is set up
 * once and reused by every application (the use of the method the paper
 * names, Secs. 6 and 7; the outer method is not given there). All
 * right-hand sides advance together; a cycle ends when every one has a
 * least-squares residual below tol ||b|| (or the outer Krylov space became
 * invariant), and the true residual b - D_ov x is recomputed at the end of
 * each cycle. The host reads the residual estimates once per outer
 * iteration. b, x: [nrhs][N] complex128, host or device. The outer basis
 * ((restart + 1) nrhs N complex128) is allocated for the call and freed.
 * info (if not NULL): nrhs reports. Returns OVS_OK when all converged,
 * OVS_NOT_CONVERGED if some did not within max_cycles, or an error as
 * ovs_sign_apply. */
int ovs_overlap_solve(ovs_gauge_t g, const void* b, void* x, int32_t nrhs, const ovs_apply_opts* inner,
                      const ovs_solve_opts* outer, ovs_solve_info* info, void* stream);

/* Diagnosis and test hook (no counterpart in the paper): the Krylov basis
 * and Hessenberg matrix of right-hand side `rhs` of the last application
 * on this handle. *k_out = k_used; V (if not NULL): host complex128
 * [k][N] canonical, v_1..v_k (converted from the basis precision); H (if
 * not NULL): host complex128 column-major (k+1) x k, Hbar_k with
 * h_(k+1,k) in its last row (after OVS_APPLY_HARMONIC its last column is
 * the harmonic one). Synchronises the device. Errors: EINVAL. */
int ovs_get_krylov(ovs_gauge_t g, int32_t rhs, int32_t* k_out, double* V, double* H);

/* Batched form: n instances, each a handle with its own gauge field, mu and
 * deflation basis, and nrhs[i] right-hand sides x[i] -> y[i] (layout and
 * host/device rules of ovs_sign_apply; the n handles must be distinct).
 * Each instance's whole application (A1-A7 of ovs_sign_apply, from an
 * internal copy of x to an internal y) is recorded once per (nrhs, opts) as
 * a CUDA graph; the recorded applications of the n instances are the child
 * graphs of one combined graph, built once per set of instances, nrhs and
 * opts, so one graph launch on `stream` runs all instances concurrently
 * (lattices of different sizes, uneven Krylov depths). set_mu, deflation
 * changes and buffer growth drop the recorded graphs, ovs_destroy the
 * combined ones that contain the handle. With opts->check_every > 0 every
 * right-hand side stops at its own Krylov dimension. info, if not NULL,
 * receives sum(nrhs) reports in instance order; the call then waits for
 * `stream`. Returns the worst status as ovs_sign_apply. */
int ovs_sign_apply_batched(int32_t n, const ovs_gauge_t* g, const void* const* x, void* const* y,
                           const int32_t* nrhs, const ovs_apply_opts* opts, ovs_apply_info* info, void* stream);

/* Reports of the last ovs_sign_apply on this handle (waits for its stream). */
int ovs_get_info(ovs_gauge_t g, ovs_apply_info* info, int32_t nrhs);

/* Launch shape of the stencil (K1). A shape is (rt, sites, rb): rt
 * right-hand sides per thread (1 or 2: the thread loads each link once for
 * them) and a thread block of `sites` sites times `rb` right-hand-side
 * tiles (the warps of a block share the links of their sites through L1),
 * at most 256 threads. The 18 candidates are, in this order:
 *   (1,32,1) (1,32,2) (1,32,4) (1,32,8) (1,64,1) (1,64,2) (1,64,4)
 *   (1,128,1) (1,128,2) (2,32,1) (2,32,2) (2,32,4) (2,32,8) (2,64,1)
 *   (2,64,2) (2,64,4) (2,128,1) (2,128,2).
 * The first stencil launch of a handle for a (prec, nrhs) pair, made outside
 * stream capture, times the candidates on the caller's stream with CUDA
 * events (one warm-up and up to three timed launches each, on that call's
 * operands; this synchronises the stream once) and keeps the fastest for
 * the handle. OVS_F64 times only the rt = 1 shapes (the FP64 stencil is
 * bound by the FP64 units whatever the shape). ovs_sign_apply_batched tunes
 * before it records its graphs. A launch inside a capture that finds no
 * choice uses (1, 128, 1) without storing it. Every shape gives
 * bit-identical results. The paper has no counterpart: this is a service
 * of the library. */

/* The shape chosen for (prec, nrhs) in shape[0..2] = (rt, sites, rb) and, if
 * ms is not NULL, the mean time in ms of each of the 18 candidates in the
 * order above (negative: not timed or not launchable; 0 for all: the shape
 * was pinned by ovs_set_stencil_shape). OVS_ESTATE if no shape has been
 * chosen for the pair yet; EINVAL on bad arguments. */
int ovs_stencil_tuning(ovs_gauge_t g, int32_t prec, int32_t nrhs, int32_t* shape, float* ms);

/* Pin the shape (rt, sites, rb) used for (prec, nrhs) instead of timing the
 * candidates; rt = 0 forgets the choice, so the next launch tunes again.
 * The handle's recorded batched applications are dropped. EINVAL if the
 * shape is not one of the 18 candidates. */
int ovs_set_stencil_shape(ovs_gauge_t g, int32_t prec, int32_t nrhs, int32_t rt, int32_t sites, int32_t rb);

/* Tracing. Every kernel a handle launches is counted per class, together
 * with its algorithmic bytes (the bytes the operation must move at least:
 * each operand read once, each result written once). With timing on, every
 * launch is also bracketed by two CUDA events on its stream, so per-class
 * device times can be read back; this costs two event records per launch
 * and no host synchronisation except when the event pool (8192 launches)
 * fills up. */
enum {
    OVS_PROF_MATVEC = 0, /* K1: H_w / D_w stencil */
    OVS_PROF_DOTS = 1,   /* K2: Gram-Schmidt inner products of the Arnoldi steps */
    OVS_PROF_UPDATE = 2, /* K2: basis updates of the Arnoldi steps */
    OVS_PROF_SMALL = 3,  /* reductions, Hessenberg column, norms, scaling */
    OVS_PROF_NEWTON = 4, /* K3: Roberts iteration on H_k */
    OVS_PROF_LAYOUT = 5, /* K7: canonical <-> internal layout */
    OVS_PROF_PROJ = 6,   /* K4/K5: deflation projection (L^+ x, x - R c, R sgn c), recombination V_k c */
    OVS_PROF_NCLASS = 7
};

/* Reset the counters; timing != 0 turns event timing on, 0 turns it off. */
int ovs_profile_enable(ovs_gauge_t g, int32_t timing);

/* Totals since the last ovs_profile_enable (any pointer may be NULL):
 * ms[c] device milliseconds (0 without timing), launches[c], bytes[c]
 * algorithmic bytes, for c < OVS_PROF_NCLASS. Waits for timed launches. */
int ovs_profile_read(ovs_gauge_t g, double* ms, int64_t* launches, double* bytes);

/* Self-check of the timeout path of the bounded device waits (the paper has
 * no counterpart). Every wait of the library's kernels on a flag or an
 * mbarrier is bounded: when it gives up, the kernel records OVS_ETIMEOUT in
 * an error word, lets its copies in flight land, and returns, and the call
 * reports OVS_ETIMEOUT. This launches one block whose wait can never
 * complete (nothing arrives on its mbarrier) and waits for it on `stream`
 * (about a second). Returns OVS_ETIMEOUT when the bound works, OVS_ECUDA
 * otherwise. The context stays usable. */
int ovs_check_wait_timeout(void* stream);

/* Thread-local message of the last error (never NULL). */
const char* ovs_last_error(void);

/* Library version string. */
const char* ovs_version(void);

/* Release the handle and all device memory it owns. NULL is ignored. */
void ovs_destroy(ovs_gauge_t g);

#ifdef __cplusplus
}
#endif

#endif /* OVSIGN_H */
