"""Python binding of libovsign (include/ovsign.h): sgn(H_w(mu)) x on GB300.

Argument marshalling only: every step of the computation runs in the CUDA
library. Vectors are torch tensors of dtype complex128 with shape
[nrhs, N] (N = 12 V, entry (site*4 + spin)*3 + colour), on the GPU or on
the host (the library stages host buffers itself). Functions mirror the C
entry points without the ``ovs_`` prefix and raise ``OvsError`` on a
negative status.

There is no CPU fallback: ``load()`` raises if the shared library is
missing, and the library needs a CUDA device to do any work.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libovsign.so")

F64 = 0
MIXED = 1
OP_DW, OP_HW, OP_HW2 = 0, 1, 2
STATUS = {
    0: "OVS_OK", 1: "OVS_NOT_CONVERGED", -1: "OVS_EINVAL", -2: "OVS_ENOMEM", -3: "OVS_ECUDA",
    -4: "OVS_ESTATE", -5: "OVS_EEIG", -6: "OVS_ESIGN", -7: "OVS_ETIMEOUT", -8: "OVS_EIO",
}
EXPORTS = [
    "ovs_create_gauge", "ovs_create_gauge_from_links", "ovs_get_links", "ovs_set_mu", "ovs_matvec",
    "ovs_matvec_noalloc",
    "ovs_deflate_setup", "ovs_deflate_stats", "ovs_set_setup_budget", "ovs_deflate_load", "ovs_deflate_get", "ovs_deflate_save", "ovs_deflate_restore",
    "ovs_deflate_load_schur", "ovs_deflate_setup_schur", "ovs_deflate_scheme",
    "ovs_sign_apply", "ovs_sign_apply_batched", "ovs_get_info", "ovs_stencil_tuning", "ovs_set_stencil_shape",
    "ovs_overlap_apply", "ovs_overlap_solve", "ovs_get_krylov",
    "ovs_profile_enable", "ovs_profile_read", "ovs_check_wait_timeout", "ovs_last_error", "ovs_version",
    "ovs_destroy",
]
PROF_CLASSES = ["matvec", "dots", "update", "small", "newton", "layout", "proj"]
APPLY_HARMONIC = 1
APPLY_SKIP_AHEAD = 2
SCHEME = {0: "none", 1: "lr", 2: "schur"}


class OvsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class ApplyOpts(ctypes.Structure):
    _fields_ = [("k_max", ctypes.c_int32), ("check_every", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("tol", ctypes.c_double)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int32), ("max_cycles", ctypes.c_int32), ("tol", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("cycles", ctypes.c_int32), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("rel_resid", ctypes.c_double)]

    def as_dict(self):
        return {"iters": self.iters, "cycles": self.cycles, "status": self.status, "rel_resid": self.rel_resid}


class ApplyInfo(ctypes.Structure):
    _fields_ = [("k_used", ctypes.c_int32), ("newton_iters", ctypes.c_int32), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("beta", ctypes.c_double), ("est_err", ctypes.c_double)]

    def as_dict(self):
        return {"k_used": self.k_used, "newton_iters": self.newton_iters, "status": self.status,
                "beta": self.beta, "est_err": self.est_err}


_lib = None


def load(path=None):
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise OSError(f"{path} not found: build it with paper_0704_3486_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i32, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    p_i32 = ctypes.POINTER(ctypes.c_int32)
    p_dbl = ctypes.POINTER(ctypes.c_double)
    sig = {
        "ovs_create_gauge": ([p_i32, ctypes.c_uint64, dbl, i32, ctypes.POINTER(vp)], i32),
        "ovs_create_gauge_from_links": ([p_i32, vp, i32, ctypes.POINTER(vp)], i32),
        "ovs_get_links": ([vp, vp], i32),
        "ovs_set_mu": ([vp, dbl, dbl], i32),
        "ovs_matvec": ([vp, i32, vp, vp, i32, i32, vp], i32),
        "ovs_matvec_noalloc": ([vp, i32, vp, vp, i32, i32, vp], i32),
        "ovs_deflate_setup": ([vp, i32, dbl, vp], i32),
        "ovs_deflate_stats": ([vp, vp, vp, vp], i32),
        "ovs_set_setup_budget": ([vp, dbl], i32),
        "ovs_deflate_load": ([vp, i32, vp, vp, vp], i32),
        "ovs_deflate_get": ([vp, p_i32, vp, vp, vp], i32),
        "ovs_deflate_save": ([vp, ctypes.c_char_p], i32),
        "ovs_deflate_restore": ([vp, ctypes.c_char_p], i32),
        "ovs_deflate_load_schur": ([vp, i32, vp], i32),
        "ovs_deflate_setup_schur": ([vp, i32, dbl, vp], i32),
        "ovs_deflate_scheme": ([vp], i32),
        "ovs_overlap_apply": ([vp, vp, vp, i32, ctypes.POINTER(ApplyOpts), ctypes.POINTER(ApplyInfo), vp], i32),
        "ovs_overlap_solve": ([vp, vp, vp, i32, ctypes.POINTER(ApplyOpts), ctypes.POINTER(SolveOpts),
                               ctypes.POINTER(SolveInfo), vp], i32),
        "ovs_get_krylov": ([vp, i32, p_i32, vp, vp], i32),
        "ovs_sign_apply": ([vp, vp, vp, i32, ctypes.POINTER(ApplyOpts), ctypes.POINTER(ApplyInfo), vp], i32),
        "ovs_sign_apply_batched": ([i32, vp, vp, vp, vp, ctypes.POINTER(ApplyOpts), ctypes.POINTER(ApplyInfo), vp],
                                   i32),
        "ovs_get_info": ([vp, ctypes.POINTER(ApplyInfo), i32], i32),
        "ovs_stencil_tuning": ([vp, i32, i32, p_i32, vp], i32),
        "ovs_set_stencil_shape": ([vp, i32, i32, i32, i32, i32], i32),
        "ovs_profile_enable": ([vp, i32], i32),
        "ovs_check_wait_timeout": ([vp], i32),
        "ovs_profile_read": ([vp, vp, vp, vp], i32),
        "ovs_last_error": ([], ctypes.c_char_p),
        "ovs_version": ([], ctypes.c_char_p),
        "ovs_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    del p_dbl
    _lib = lib
    return lib


def _check(status):
    if status < 0:
        raise OvsError(status, _lib.ovs_last_error().decode())
    return status


def _dims(dims):
    return (ctypes.c_int32 * 4)(*[int(d) for d in dims])


def _ptr(t):
    """Data pointer of a contiguous complex128 tensor or numpy array."""
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(t.data_ptr())
    if not t.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C contiguous")
    return ctypes.c_void_p(t.ctypes.data)


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:  # pragma: no cover
            pass
        return ctypes.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


class Gauge:
    """Owns an ``ovs_gauge_t`` handle (released by ``destroy`` or GC)."""

    def __init__(self, handle, dims):
        self.handle = handle
        self.dims = tuple(int(d) for d in dims)
        self.V = self.dims[0] * self.dims[1] * self.dims[2] * self.dims[3]
        self.N = 12 * self.V

    def destroy(self):
        if self.handle:
            load().ovs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def create_gauge(dims, seed, eps, prec=MIXED):
    lib = load()
    h = ctypes.c_void_p()
    _check(lib.ovs_create_gauge(_dims(dims), ctypes.c_uint64(int(seed)), float(eps), int(prec), ctypes.byref(h)))
    return Gauge(h, dims)


def create_gauge_from_links(dims, links, prec=MIXED):
    """links: complex128 array [V][4][3][3] (numpy or CPU tensor)."""
    import numpy as np
    lib = load()
    arr = np.ascontiguousarray(np.asarray(links, dtype=np.complex128))
    h = ctypes.c_void_p()
    _check(lib.ovs_create_gauge_from_links(_dims(dims), _ptr(arr), int(prec), ctypes.byref(h)))
    return Gauge(h, dims)


def get_links(g):
    import numpy as np
    out = np.empty((g.V, 4, 3, 3), dtype=np.complex128)
    _check(load().ovs_get_links(g.handle, _ptr(out)))
    return out


def set_mu(g, mu, m_w):
    _check(load().ovs_set_mu(g.handle, float(mu), float(m_w)))


def matvec(g, op, x, y, nrhs=None, prec=F64, stream=None):
    nrhs = x.shape[0] if nrhs is None else nrhs
    _check(load().ovs_matvec(g.handle, int(op), _ptr(x), _ptr(y), int(nrhs), int(prec), _stream(stream)))


def matvec_noalloc(g, op, x, y, nrhs=None, prec=F64, stream=None):
    """matvec for callers that cannot have the library allocate device
    memory (their pool belongs to another allocator, or cudaMalloc's
    synchronisation is not allowed in their loop). Uses a fixed 2 x 8 MiB
    work array inside the library: nrhs*N <= 524288 (F64) / 1048576 (MIXED);
    x, y must be device tensors. Calls that overlap on the GPU race."""
    nrhs = x.shape[0] if nrhs is None else nrhs
    _check(load().ovs_matvec_noalloc(g.handle, int(op), _ptr(x), _ptr(y), int(nrhs), int(prec),
                                     _stream(stream)))


def deflate_setup(g, m, tol=1e-10, allow_unconverged=False, scheme="lr"):
    """Returns (eigenvalues, status). scheme "lr" (left and right vectors,
    Sec. 5.3) or "schur" (right vectors only, Sec. 5.2). With
    allow_unconverged, OVS_EEIG (basis installed but not at tol) is returned
    as a status instead of raised."""
    import numpy as np
    eig = np.empty(2 * m, dtype=np.float64)
    fn = load().ovs_deflate_setup_schur if scheme == "schur" else load().ovs_deflate_setup
    status = fn(g.handle, int(m), float(tol), _ptr(eig))
    if not (allow_unconverged and status == -5):
        _check(status)
    return eig[0::2] + 1j * eig[1::2], status


def deflate_load_schur(g, R):
    """Schur deflation from right eigenvectors R: complex128 [m][N] (host)."""
    import numpy as np
    R = np.ascontiguousarray(np.asarray(R, dtype=np.complex128))
    m = R.shape[0]
    _check(load().ovs_deflate_load_schur(g.handle, int(m), _ptr(R) if m else None))


def deflate_scheme(g):
    return SCHEME[_check(load().ovs_deflate_scheme(g.handle))]


def deflate_stats(g):
    """{'iterations': (right, left), 'matvecs': n} of the last deflate_setup."""
    import numpy as np
    it = np.zeros(2, dtype=np.int32)
    mv = np.zeros(1, dtype=np.int64)
    rs = np.zeros(1, dtype=np.float64)
    _check(load().ovs_deflate_stats(g.handle, _ptr(it), _ptr(mv), _ptr(rs)))
    return {"iterations": (int(it[0]), int(it[1])), "matvecs": int(mv[0]), "max_resid": float(rs[0])}


def set_setup_budget(g, max_seconds):
    _check(load().ovs_set_setup_budget(g.handle, float(max_seconds)))


def deflate_load(g, R, L, lam):
    """R, L: complex128 [m][N] (host); lam: m complex eigenvalues."""
    import numpy as np
    R = np.ascontiguousarray(np.asarray(R, dtype=np.complex128))
    L = np.ascontiguousarray(np.asarray(L, dtype=np.complex128))
    lam = np.asarray(lam, dtype=np.complex128)
    lam2 = np.ascontiguousarray(np.stack([lam.real, lam.imag], axis=-1).reshape(-1))
    m = lam.shape[0]
    if m == 0:
        _check(load().ovs_deflate_load(g.handle, 0, None, None, None))
        return
    _check(load().ovs_deflate_load(g.handle, int(m), _ptr(R), _ptr(L), _ptr(lam2)))


def deflate_get(g):
    """(R, L, lambda); for Schur deflation R holds S_m and L is None."""
    import numpy as np
    m = ctypes.c_int32()
    lib = load()
    _check(lib.ovs_deflate_get(g.handle, ctypes.byref(m), None, None, None))
    m = m.value
    schur = lib.ovs_deflate_scheme(g.handle) == 2
    R = np.empty((m, g.N), dtype=np.complex128)
    L = None if schur else np.empty((m, g.N), dtype=np.complex128)
    lam = np.empty(2 * m, dtype=np.float64)
    if m:
        _check(lib.ovs_deflate_get(g.handle, None, _ptr(R), None if schur else _ptr(L), _ptr(lam)))
    return R, L, lam[0::2] + 1j * lam[1::2]


def deflate_save(g, path):
    _check(load().ovs_deflate_save(g.handle, os.fsencode(path)))


def deflate_restore(g, path):
    _check(load().ovs_deflate_restore(g.handle, os.fsencode(path)))


def _flags(harmonic=False, skip_ahead=False):
    return (APPLY_HARMONIC if harmonic else 0) | (APPLY_SKIP_AHEAD if skip_ahead else 0)


def _apply(fn, g, x, y, k_max, prec, nrhs, check_every, tol, stream, want_info, harmonic, skip_ahead=False):
    nrhs = x.shape[0] if nrhs is None else nrhs
    opts = ApplyOpts(int(k_max), int(check_every), int(prec), _flags(harmonic, skip_ahead), float(tol))
    if want_info:
        info = (ApplyInfo * nrhs)()
        st = _check(fn(g.handle, _ptr(x), _ptr(y), int(nrhs), ctypes.byref(opts), info, _stream(stream)))
        return st, [i.as_dict() for i in info]
    return _check(fn(g.handle, _ptr(x), _ptr(y), int(nrhs), ctypes.byref(opts), None, _stream(stream)))


def sign_apply(g, x, y, k_max, prec=MIXED, nrhs=None, check_every=0, tol=0.0, stream=None, want_info=True,
               harmonic=False, skip_ahead=False):
    """y = sgn(H_w(mu)) x. Returns (status, [info dicts]) if want_info, else status.
    skip_ahead: the skip-ahead schedule of the convergence checks."""
    return _apply(load().ovs_sign_apply, g, x, y, k_max, prec, nrhs, check_every, tol, stream, want_info, harmonic,
                  skip_ahead)


def overlap_apply(g, x, y, k_max, prec=MIXED, nrhs=None, check_every=0, tol=0.0, stream=None, want_info=True,
                  harmonic=False):
    """y = D_ov(mu) x = x + gamma5 sgn(H_w(mu)) x (Sec. 2, Eq. Dov)."""
    return _apply(load().ovs_overlap_apply, g, x, y, k_max, prec, nrhs, check_every, tol, stream, want_info,
                  harmonic)


def overlap_solve(g, b, x, k_max, restart, tol, max_cycles=50, prec=MIXED, nrhs=None, harmonic=False, stream=None):
    """Solve D_ov(mu) x = b by restarted GMRES around the sign application.
    Returns (status, [info dicts: iters, cycles, status, rel_resid])."""
    nrhs = b.shape[0] if nrhs is None else nrhs
    inner = ApplyOpts(int(k_max), 0, int(prec), APPLY_HARMONIC if harmonic else 0, 0.0)
    outer = SolveOpts(int(restart), int(max_cycles), float(tol))
    info = (SolveInfo * nrhs)()
    st = _check(load().ovs_overlap_solve(g.handle, _ptr(b), _ptr(x), int(nrhs), ctypes.byref(inner),
                                         ctypes.byref(outer), info, _stream(stream)))
    return st, [i.as_dict() for i in info]


def get_krylov(g, rhs):
    """(V [k][N] complex128, Hbar [(k+1) x k] complex128) of right-hand side
    rhs of the last application (a test and diagnosis hook)."""
    import numpy as np
    lib = load()
    k = ctypes.c_int32()
    _check(lib.ovs_get_krylov(g.handle, int(rhs), ctypes.byref(k), None, None))
    k = k.value
    V = np.empty((k, g.N), dtype=np.complex128)
    H = np.empty((k, k + 1), dtype=np.complex128)  # column-major (k+1) x k
    if k:
        _check(lib.ovs_get_krylov(g.handle, int(rhs), ctypes.byref(ctypes.c_int32()), _ptr(V), _ptr(H)))
    return V, H.T.copy()


def sign_apply_batched(gauges, xs, ys, k_max, prec=MIXED, check_every=0, tol=0.0, stream=None, want_info=True,
                       skip_ahead=False):
    """Batched form over several handles: y_i = sgn(H_w(mu_i)) x_i for each
    instance i (xs[i], ys[i] of shape [nrhs_i, N_i])."""
    n = len(gauges)
    handles = (ctypes.c_void_p * n)(*[g.handle.value if hasattr(g.handle, "value") else g.handle for g in gauges])
    xp = (ctypes.c_void_p * n)(*[_ptr(x).value for x in xs])
    yp = (ctypes.c_void_p * n)(*[_ptr(y).value for y in ys])
    nr = (ctypes.c_int32 * n)(*[int(x.shape[0]) for x in xs])
    opts = ApplyOpts(int(k_max), int(check_every), int(prec), _flags(skip_ahead=skip_ahead), float(tol))
    lib = load()
    if want_info:
        total = sum(int(x.shape[0]) for x in xs)
        info = (ApplyInfo * total)()
        st = _check(lib.ovs_sign_apply_batched(n, handles, xp, yp, nr, ctypes.byref(opts), info, _stream(stream)))
        return st, [i.as_dict() for i in info]
    return _check(lib.ovs_sign_apply_batched(n, handles, xp, yp, nr, ctypes.byref(opts), None, _stream(stream)))


def get_info(g, nrhs):
    info = (ApplyInfo * nrhs)()
    st = _check(load().ovs_get_info(g.handle, info, int(nrhs)))
    return st, [i.as_dict() for i in info]


STENCIL_SHAPES = [(1, 32, 1), (1, 32, 2), (1, 32, 4), (1, 32, 8), (1, 64, 1), (1, 64, 2), (1, 64, 4), (1, 128, 1),
                  (1, 128, 2), (2, 32, 1), (2, 32, 2), (2, 32, 4), (2, 32, 8), (2, 64, 1), (2, 64, 2), (2, 64, 4),
                  (2, 128, 1), (2, 128, 2)]


def stencil_tuning(g, prec, nrhs):
    """The stencil shape chosen for (prec, nrhs): {'shape': (rt, sites, rb),
    'ms': {shape: mean ms of that candidate (negative: not timed)}}; None if
    no shape has been chosen yet."""
    import numpy as np
    shape = (ctypes.c_int32 * 3)()
    ms = np.zeros(len(STENCIL_SHAPES), dtype=np.float32)
    st = load().ovs_stencil_tuning(g.handle, int(prec), int(nrhs), shape, _ptr(ms))
    if st == -4:  # OVS_ESTATE: not chosen yet
        return None
    _check(st)
    return {"shape": tuple(shape), "ms": {sh: float(v) for sh, v in zip(STENCIL_SHAPES, ms)}}


def set_stencil_shape(g, prec, nrhs, shape):
    """Pin the stencil shape (rt, sites, rb) for (prec, nrhs); None forgets it."""
    rt, sites, rb = shape if shape is not None else (0, 0, 0)
    _check(load().ovs_set_stencil_shape(g.handle, int(prec), int(nrhs), int(rt), int(sites), int(rb)))


def profile_enable(g, timing=True):
    _check(load().ovs_profile_enable(g.handle, 1 if timing else 0))


def profile_read(g):
    """Per kernel class: {'matvec': {'ms':..., 'launches':..., 'bytes':...}, ...}."""
    import numpy as np
    n = len(PROF_CLASSES)
    ms = np.zeros(n, dtype=np.float64)
    launches = np.zeros(n, dtype=np.int64)
    nbytes = np.zeros(n, dtype=np.float64)
    _check(load().ovs_profile_read(g.handle, _ptr(ms), _ptr(launches), _ptr(nbytes)))
    return {c: {"ms": float(ms[i]), "launches": int(launches[i]), "bytes": float(nbytes[i])}
            for i, c in enumerate(PROF_CLASSES)}


def check_wait_timeout(stream=None):
    """Run the bounded-wait self-check; returns the status (OVS_ETIMEOUT = -7
    when the timeout path works)."""
    return load().ovs_check_wait_timeout(_stream(stream))


def version():
    return load().ovs_version().decode()
