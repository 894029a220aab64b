"""ctypes binding of libcfie.so (include/cfie.h), argument marshalling only.

Every function of the C ABI is exposed under the same name; device buffers are
passed as torch tensors (complex128, contiguous, on the context's device) or as
raw integer addresses.  Loading fails loudly when the library has not been
built: there is no CPU fallback.

A thin object layer (Context, Geometry, Operator) wraps the handles for tests
and the benchmark.
"""
import ctypes
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcfie.so")

CFIE_OK, CFIE_EINVAL, CFIE_ENOMEM, CFIE_ECUDA, CFIE_ENOCONV, CFIE_ETIMEOUT, CFIE_EBUSY = range(7)
STATUS_NAMES = ["CFIE_OK", "CFIE_EINVAL", "CFIE_ENOMEM", "CFIE_ECUDA", "CFIE_ENOCONV",
                "CFIE_ETIMEOUT", "CFIE_EBUSY"]
CFIE_SOUND_SOFT, CFIE_SOUND_HARD = 0, 1
CFIE_FP64, CFIE_FP32_REFINED, CFIE_TENSOR_REFINED = 0, 1, 2
CFIE_MATRIX_FREE, CFIE_STORED = 0, 1
CFIE_CURVE_CIRCLE, CFIE_CURVE_ELLIPSE, CFIE_CURVE_STAR, CFIE_CURVE_KITE = 0, 1, 2, 3
CURVE = {"circle": CFIE_CURVE_CIRCLE, "ellipse": CFIE_CURVE_ELLIPSE, "star": CFIE_CURVE_STAR,
         "kite": CFIE_CURVE_KITE}
(CFIE_K_MATVEC_FP64, CFIE_K_MATVEC_FP32, CFIE_K_MATVEC_TENSOR, CFIE_K_ARNOLDI,
 CFIE_K_SPECTRAL, CFIE_K_COUNT) = range(6)
KERNEL_CLASS_NAMES = ["matvec_fp64", "matvec_fp32", "matvec_tensor", "arnoldi", "spectral"]

BC = {"soft": CFIE_SOUND_SOFT, "hard": CFIE_SOUND_HARD}
PRECISION = {"fp64": CFIE_FP64, "fp32": CFIE_FP32_REFINED, "tensor": CFIE_TENSOR_REFINED}
LAYOUT = {"matrix_free": CFIE_MATRIX_FREE, "stored": CFIE_STORED}


class cfie_request(ctypes.Structure):
    _fields_ = [("bc", ctypes.c_int), ("precision", ctypes.c_int), ("K", ctypes.c_int),
                ("a", ctypes.POINTER(ctypes.c_double)), ("b", ctypes.POINTER(ctypes.c_double)),
                ("n", ctypes.c_int), ("omega", ctypes.c_double), ("eta", ctypes.c_double),
                ("nrhs", ctypes.c_int), ("theta", ctypes.POINTER(ctypes.c_double)),
                ("rtol", ctypes.c_double), ("restart", ctypes.c_int), ("maxit", ctypes.c_int)]


class cfie_result(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int), ("started", ctypes.c_int), ("status", ctypes.c_int),
                ("iters_max", ctypes.c_int), ("relres_max", ctypes.c_double),
                ("queued_s", ctypes.c_double), ("service_s", ctypes.c_double),
                ("latency_s", ctypes.c_double)]


class cfie_server_counters(ctypes.Structure):
    _fields_ = [(k, ctypes.c_longlong) for k in
                ("completed", "solves", "queued", "running", "peak_running", "budget_bytes",
                 "in_use_bytes", "peak_in_use_bytes")]


class cfie_solve_stats(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("refinements", ctypes.c_int),
                ("inner_matvecs", ctypes.c_int), ("fp64_matvecs", ctypes.c_int),
                ("arnoldi_steps", ctypes.c_int), ("matvec_variant", ctypes.c_int),
                ("basis_fp32", ctypes.c_int), ("residual_variant", ctypes.c_int),
                ("arnoldi_elems", ctypes.c_longlong)]


class cfie_peaks(ctypes.Structure):
    _fields_ = [("sms", ctypes.c_int), ("fp32_fma_per_s", ctypes.c_double),
                ("mufu_per_s", ctypes.c_double), ("fp64_fma_per_s", ctypes.c_double)]


class CfieError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {message}")
        self.status = status


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)
_LLP = ctypes.POINTER(ctypes.c_longlong)

# name -> (restype, argtypes), in the order of include/cfie.h
SIGNATURES = {
    "cfie_ctx_create": (_I, [_I, _P, ctypes.POINTER(_P)]),
    "cfie_ctx_destroy": (None, [_P]),
    "cfie_last_error": (ctypes.c_char_p, [_P]),
    "cfie_geometry_circle": (_I, [_P, _D, ctypes.POINTER(_P)]),
    "cfie_geometry_ellipse": (_I, [_P, _D, _D, ctypes.POINTER(_P)]),
    "cfie_geometry_fourier_star": (_I, [_P, _I, _DP, _DP, ctypes.POINTER(_P)]),
    "cfie_geometry_kite": (_I, [_P, ctypes.POINTER(_P)]),
    "cfie_geometry_samples": (_I, [_P, _I, _DP, _DP, _DP, ctypes.POINTER(_P)]),
    "cfie_geom_destroy": (None, [_P]),
    "cfie_arclength_samples": (_I, [_I, _DP, _I, _I, _DP, _DP, _DP, _DP]),
    "cfie_dirprec_plan": (_I, [_I, _DP, _I, _I, _I, _D, _I, _I, _IP, _IP, _IP, _IP]),
    "cfie_dirprec_w_pattern": (_I, [_I, _IP, _IP, _I, _IP, _IP, _IP, _IP]),
    "cfie_dirprec_level": (_I, [_I, _I, _I, _D, _D, _D, _DP, _DP, _DP, _DP]),
    "cfie_dirprec_threshold": (_I, [_I, _DP, _I, _DP]),
    "cfie_dirprec_create": (_I, [_P, _I, _DP, _I, _I, _I, _I, _I, ctypes.POINTER(_P)]),
    "cfie_dirprec_apply": (_I, [_P, _P, _P, _I]),
    "cfie_dirprec_coefficients": (_I, [_P, _IP, _DP]),
    "cfie_op_set_preconditioner": (_I, [_P, _P]),
    "cfie_dirprec_destroy": (None, [_P]),
    "cfie_discretise": (_I, [_P, _I, _D, _D, _I, _I, _I, ctypes.POINTER(_P)]),
    "cfie_discretise_many": (_I, [_I, ctypes.POINTER(_P), _IP, _DP, _DP, _I, _I, _I,
                                  ctypes.POINTER(_P)]),
    "cfie_op_destroy": (None, [_P]),
    "cfie_op_n": (_I, [_P]),
    "cfie_rhs_plane_waves": (_I, [_P, _I, _DP, _P]),
    "cfie_apply": (_I, [_P, _P, _P, _I]),
    "cfie_apply_fp64": (_I, [_P, _P, _P, _I]),
    "cfie_apply_fp64_static": (_I, [_P, _P, _P, _I]),
    "cfie_apply_residual": (_I, [_P, _P, _P, _I]),
    "cfie_op_set_variant": (_I, [_P, _I]),
    "cfie_gmres_solve": (_I, [_P, _P, _P, _I, _D, _I, _I, _IP, _DP]),
    "cfie_op_set_inner_basis": (_I, [_P, _I]),
    "cfie_op_set_block_gmres": (_I, [_P, _I]),
    "cfie_op_set_residual_variant": (_I, [_P, _I]),
    "cfie_field_eval": (_I, [_P, _P, _I, _I, _P, _P]),
    "cfie_op_last_stats": (_I, [_P, ctypes.POINTER(cfie_solve_stats)]),
    "cfie_ctx_set_profiling": (_I, [_P, _I]),
    "cfie_ctx_kernel_times": (_I, [_P, _DP, _LLP]),
    "cfie_launch_count": (ctypes.c_longlong, []),
    "cfie_measure_peaks": (_I, [_P, ctypes.POINTER(cfie_peaks)]),
    "cfie_batch_create": (_I, [_P, _I, ctypes.POINTER(_P), _IP, ctypes.POINTER(_P)]),
    "cfie_batch_length": (ctypes.c_longlong, [_P]),
    "cfie_batch_apply": (_I, [_P, _P, _P]),
    "cfie_batch_gmres_solve": (_I, [_P, _P, _P, _D, _I, _I, _IP, _DP]),
    "cfie_batch_last_stats": (_I, [_P, ctypes.POINTER(cfie_solve_stats)]),
    "cfie_batch_set_inner_basis": (_I, [_P, _I]),
    "cfie_batch_tuning": (_I, [_P, _IP, ctypes.POINTER(ctypes.c_float)]),
    "cfie_batch_set_dealing": (_I, [_P, _I]),
    "cfie_batch_destroy": (None, [_P]),
    "cfie_server_create": (_I, [_I, ctypes.c_size_t, _I, ctypes.POINTER(_P)]),
    "cfie_server_submit": (_I, [_P, ctypes.POINTER(cfie_request), ctypes.POINTER(ctypes.c_longlong)]),
    "cfie_server_poll": (_I, [_P, ctypes.c_longlong, ctypes.POINTER(cfie_result), _P]),
    "cfie_server_wait_all": (_I, [_P, _D]),
    "cfie_server_release": (_I, [_P, ctypes.c_longlong]),
    "cfie_server_stats": (_I, [_P, ctypes.POINTER(cfie_server_counters)]),
    "cfie_server_last_error": (ctypes.c_char_p, [_P]),
    "cfie_server_request_error": (_I, [_P, ctypes.c_longlong, ctypes.c_char_p, ctypes.c_size_t]),
    "cfie_server_destroy": (None, [_P]),
    "cfie_server_set_batching": (_I, [_P, _I]),
    "cfie_server_set_block_gmres": (_I, [_P, _I, _I]),
}

_lib = None


def load():
    """Load libcfie.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_1408_1578_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _addr(buf):
    if buf is None:
        return None
    if isinstance(buf, int):
        return buf
    import torch
    if not isinstance(buf, torch.Tensor):
        raise TypeError("device buffers are torch tensors or integer addresses")
    if buf.dtype != torch.complex128 or not buf.is_cuda or not buf.is_contiguous():
        raise ValueError("device buffers must be contiguous complex128 CUDA tensors")
    return buf.data_ptr()


def _dptr(a):
    return a.ctypes.data_as(_DP)


# ---------------------------------------------------------------------------
# raw entry points under their C names
# ---------------------------------------------------------------------------
def __getattr__(name):
    if name in SIGNATURES:
        return getattr(load(), name)
    raise AttributeError(name)


def _curve_params(kind, params):
    if kind == "circle":
        p = [params.get("radius", 1.0)]
    elif kind == "ellipse":
        p = [params["a"], params["b"]]
    elif kind == "star":
        p = list(np.asarray(params["a"], dtype=np.float64)) + \
            list(np.asarray(params["b"], dtype=np.float64))
    elif kind == "kite":
        p = []
    else:
        raise ValueError(kind)
    return np.ascontiguousarray(p, dtype=np.float64)


def dirprec_plan(kind, q, p, omega, m_leaf=2, **params):
    """cfie_dirprec_plan: (first, level, kpair) of the directional
    preconditioner's segments for the named curve (host; no GPU needed);
    kpair has shape (m, m, 2)."""
    par = _curve_params(kind, params)
    pp = _dptr(par) if par.size else None
    m = ctypes.c_int()
    lib = load()
    args = (CURVE[kind], pp, int(par.size), int(q), int(p), float(omega), int(m_leaf))
    st = lib.cfie_dirprec_plan(*args, 0, ctypes.byref(m), None, None, None)
    if st != CFIE_OK:
        raise CfieError(st, "cfie_dirprec_plan: invalid curve or sizes")
    k = m.value
    first = np.zeros(k, dtype=np.int32)
    level = np.zeros(k, dtype=np.int32)
    kpair = np.zeros((k, k, 2), dtype=np.int32)
    st = lib.cfie_dirprec_plan(*args, k, ctypes.byref(m), first.ctypes.data_as(_IP),
                               level.ctypes.data_as(_IP), kpair.ctypes.data_as(_IP))
    if st != CFIE_OK:
        raise CfieError(st, "cfie_dirprec_plan")
    return first, level, kpair


def dirprec_w_pattern(level, kpair):
    """cfie_dirprec_w_pattern: (koff, row, col) of W~ = E + antidiag(T) from a
    plan's levels and wave-number pairs (host; no GPU needed)."""
    level = np.ascontiguousarray(level, dtype=np.int32)
    kpair = np.ascontiguousarray(kpair, dtype=np.int32)
    m = int(level.size)
    koff = np.zeros(m + 1, dtype=np.int32)
    nnz = ctypes.c_int()
    lib = load()
    args = (m, level.ctypes.data_as(_IP), kpair.ctypes.data_as(_IP))
    st = lib.cfie_dirprec_w_pattern(*args, 0, koff.ctypes.data_as(_IP), ctypes.byref(nnz), None, None)
    if st != CFIE_OK:
        raise CfieError(st, "cfie_dirprec_w_pattern")
    row = np.zeros(nnz.value, dtype=np.int32)
    col = np.zeros(nnz.value, dtype=np.int32)
    st = lib.cfie_dirprec_w_pattern(*args, nnz.value, koff.ctypes.data_as(_IP), ctypes.byref(nnz),
                                    row.ctypes.data_as(_IP), col.ctypes.data_as(_IP))
    if st != CFIE_OK:
        raise CfieError(st, "cfie_dirprec_w_pattern")
    return koff, row, col


def dirprec_level(n, p, level, omega, eta, L):
    """cfie_dirprec_level: (B, B^-1, U, T) of one level as complex arrays (host;
    no GPU needed)."""
    c, K = (1 << level) * p, (1 << (level + 1)) + 1
    out = [np.empty((c, c), np.complex128), np.empty((c, c), np.complex128),
           np.empty((c, K), np.complex128), np.empty((K, K), np.complex128)]
    st = load().cfie_dirprec_level(int(n), int(p), int(level), float(omega), float(eta), float(L),
                                   *[a.view(np.float64).ctypes.data_as(_DP) for a in out])
    if st != CFIE_OK:
        raise CfieError(st, "cfie_dirprec_level: invalid sizes or a singular block")
    return tuple(out)


def dirprec_threshold(T, keep):
    """cfie_dirprec_threshold: T~, the `keep` entries of T largest in modulus
    (host; no GPU needed)."""
    T = np.ascontiguousarray(T, dtype=np.complex128)
    out = np.empty_like(T)
    st = load().cfie_dirprec_threshold(int(T.shape[0]), T.view(np.float64).ctypes.data_as(_DP),
                                       int(keep), out.view(np.float64).ctypes.data_as(_DP))
    if st != CFIE_OK:
        raise CfieError(st, "cfie_dirprec_threshold: invalid size")
    return out


def arclength_samples(kind, n, **params):
    """cfie_arclength_samples: (z, dz, ddz, L) of the named curve at n points
    equispaced in arclength, each an (n, 2) array (host; no GPU needed).
    params as for Context.geometry: circle radius, ellipse a and b, star a and b."""
    par = _curve_params(kind, params)
    out = [np.empty((int(n), 2)) for _ in range(3)]
    L = ctypes.c_double()
    st = load().cfie_arclength_samples(CURVE[kind], _dptr(par) if par.size else None, int(par.size),
                                       int(n), *[_dptr(a) for a in out], ctypes.byref(L))
    if st != CFIE_OK:
        raise CfieError(st, "cfie_arclength_samples: invalid curve parameters or n")
    return out[0], out[1], out[2], L.value


# ---------------------------------------------------------------------------
# object layer
# ---------------------------------------------------------------------------
class Context:
    def __init__(self, device=0, stream=None):
        lib = load()
        h = _P()
        handle = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
        st = lib.cfie_ctx_create(device, handle, ctypes.byref(h))
        if st != CFIE_OK:
            raise CfieError(st, "cfie_ctx_create failed")
        self.h = h
        self.lib = lib
        self.device = device
        self._children = weakref.WeakSet()   # geometries / operators to destroy first

    def check(self, st, what):
        if st != CFIE_OK:
            raise CfieError(st, f"{what}: {self.lib.cfie_last_error(self.h).decode()}")

    def last_error(self):
        return self.lib.cfie_last_error(self.h).decode()

    def set_profiling(self, on):
        self.check(self.lib.cfie_ctx_set_profiling(self.h, 1 if on else 0), "cfie_ctx_set_profiling")

    def kernel_times(self):
        ms = np.zeros(CFIE_K_COUNT)
        ln = np.zeros(CFIE_K_COUNT, dtype=np.int64)
        self.check(self.lib.cfie_ctx_kernel_times(self.h, _dptr(ms), ln.ctypes.data_as(_LLP)),
                   "cfie_ctx_kernel_times")
        return {KERNEL_CLASS_NAMES[k]: (float(ms[k]), int(ln[k])) for k in range(CFIE_K_COUNT)}

    def measure_peaks(self):
        """Issue rates of the FP32 FMA, MUFU and FP64 FMA pipes (per second)."""
        p = cfie_peaks()
        self.check(self.lib.cfie_measure_peaks(self.h, ctypes.byref(p)), "cfie_measure_peaks")
        return {k: getattr(p, k) for k, _ in p._fields_}

    def close(self):
        """Destroy the context; batches, operators and geometries made from it
        are destroyed first (the C ABI needs the context alive for them)."""
        if self.h:
            kids = list(self._children)
            for child in [c for c in kids if isinstance(c, Batch)] + \
                    [c for c in kids if not isinstance(c, Batch)]:
                child.close()
            self.lib.cfie_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # geometry constructors
    def _geom(self, fn, *args):
        g = _P()
        self.check(fn(self.h, *args, ctypes.byref(g)), fn.__name__)
        geom = Geometry(self, g)
        self._children.add(geom)
        return geom

    def circle(self, radius=1.0):
        return self._geom(self.lib.cfie_geometry_circle, float(radius))

    def ellipse(self, a, b):
        return self._geom(self.lib.cfie_geometry_ellipse, float(a), float(b))

    def fourier_star(self, a, b):
        a = np.ascontiguousarray(a, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        return self._geom(self.lib.cfie_geometry_fourier_star, int(a.size), _dptr(a), _dptr(b))

    def kite(self):
        return self._geom(self.lib.cfie_geometry_kite)

    def samples(self, z, dz, ddz):
        z = np.ascontiguousarray(z, dtype=np.float64)
        dz = np.ascontiguousarray(dz, dtype=np.float64)
        ddz = np.ascontiguousarray(ddz, dtype=np.float64)
        return self._geom(self.lib.cfie_geometry_samples, int(z.shape[0]), _dptr(z), _dptr(dz),
                          _dptr(ddz))

    def discretise_many(self, geoms, n, omega, eta=None, bc="soft", precision="fp64",
                        layout="matrix_free"):
        """cfie_discretise for many geometries of this context at once (their
        set-up overlapping on the GPU); returns the operators in order."""
        count = len(geoms)
        hs = (_P * count)(*[g.h for g in geoms])
        nn = np.ascontiguousarray(n, dtype=np.int32)
        om = np.ascontiguousarray(omega, dtype=np.float64)
        et = np.ascontiguousarray(om if eta is None else eta, dtype=np.float64)
        out = (_P * count)()
        self.check(self.lib.cfie_discretise_many(count, hs, nn.ctypes.data_as(_IP), _dptr(om),
                                                 _dptr(et), BC[bc], PRECISION[precision],
                                                 LAYOUT[layout], out), "cfie_discretise_many")
        ops = [Operator(self, _P(out[k]), int(nn[k])) for k in range(count)]
        for op in ops:
            self._children.add(op)
        return ops

    def geometry(self, kind, **params):
        if kind == "circle":
            return self.circle(params.get("radius", 1.0))
        if kind == "ellipse":
            return self.ellipse(params["a"], params["b"])
        if kind == "star":
            return self.fourier_star(params["a"], params["b"])
        if kind == "kite":
            return self.kite()
        raise ValueError(kind)


class Batch:
    """Operators solved in lockstep (cfie_batch_*).  Vectors are the operators'
    (nrhs_k, n_k) blocks concatenated; `split` / `join` convert."""

    def __init__(self, ctx, ops, nrhs):
        self.ctx = ctx
        self.ops = list(ops)
        self.nrhs = [int(k) for k in nrhs]
        arr = (_P * len(self.ops))(*[op.h for op in self.ops])
        nr = np.ascontiguousarray(self.nrhs, dtype=np.int32)
        h = _P()
        ctx.check(ctx.lib.cfie_batch_create(ctx.h, len(self.ops), arr, nr.ctypes.data_as(_IP),
                                            ctypes.byref(h)), "cfie_batch_create")
        self.h = h
        self.length = int(ctx.lib.cfie_batch_length(h))
        self.offsets = np.cumsum([0] + [op.n * k for op, k in zip(self.ops, self.nrhs)])[:-1]
        ctx._children.add(self)

    def apply(self, x, y):
        self.ctx.check(self.ctx.lib.cfie_batch_apply(self.h, _addr(x), _addr(y)), "cfie_batch_apply")

    def gmres_solve(self, f, x, rtol=1e-6, restart=80, maxit=1000, allow_noconv=False):
        P = int(sum(self.nrhs))
        its = np.zeros(P, dtype=np.int32)
        rel = np.zeros(P)
        st = self.ctx.lib.cfie_batch_gmres_solve(self.h, _addr(f), _addr(x), float(rtol), int(restart),
                                                 int(maxit), its.ctypes.data_as(_IP), _dptr(rel))
        if not (st == CFIE_OK or (allow_noconv and st == CFIE_ENOCONV)):
            self.ctx.check(st, "cfie_batch_gmres_solve")
        return its, rel, st

    def last_stats(self):
        s = cfie_solve_stats()
        self.ctx.check(self.ctx.lib.cfie_batch_last_stats(self.h, ctypes.byref(s)),
                       "cfie_batch_last_stats")
        return {k: getattr(s, k) for k, _ in s._fields_}

    def set_dealing(self, dealing):
        """Force the contraction's work dealing (0 round-robin, 1 greedy, 2 stream-K)."""
        self.ctx.check(self.ctx.lib.cfie_batch_set_dealing(self.h, int(dealing)),
                       "cfie_batch_set_dealing")

    def tuning(self):
        """(dealing, [ms of each candidate]) of the batch's contraction autotuner."""
        d = ctypes.c_int()
        ms = (ctypes.c_float * 3)()
        self.ctx.check(self.ctx.lib.cfie_batch_tuning(self.h, ctypes.byref(d), ms), "cfie_batch_tuning")
        return d.value, [float(v) for v in ms]

    def set_inner_basis(self, fp32):
        self.ctx.check(self.ctx.lib.cfie_batch_set_inner_basis(self.h, 1 if fp32 else 0),
                       "cfie_batch_set_inner_basis")

    def block(self, vec, k):
        """View of operator k's (nrhs_k, n_k) block of a flat batch vector."""
        o = int(self.offsets[k])
        return vec[o:o + self.ops[k].n * self.nrhs[k]].view(self.nrhs[k], self.ops[k].n)

    def close(self):
        if self.h:
            self.ctx.lib.cfie_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Request server (cfie_server_*): continuous batching of independent solves."""

    def __init__(self, device=0, hbm_budget_bytes=64 << 30, slots=4, batch=1, block_min_rhs=0,
                 block_min_n=0):
        lib = load()
        h = _P()
        st = lib.cfie_server_create(device, int(hbm_budget_bytes), int(slots), ctypes.byref(h))
        if st != CFIE_OK:
            raise CfieError(st, "cfie_server_create failed")
        self.lib = lib
        self.h = h
        self.shapes = {}
        if batch != 1:
            self.set_batching(batch)
        if block_min_rhs:
            self.set_block_gmres(block_min_rhs, block_min_n)

    def set_block_gmres(self, min_rhs, min_n=0):
        """Requests with at least min_rhs directions and min_n nodes run alone
        with block GMRES (min_rhs 0: off)."""
        st = self.lib.cfie_server_set_block_gmres(self.h, int(min_rhs), int(min_n))
        if st != CFIE_OK:
            raise CfieError(st, "min_rhs must be in [0, 1024], min_n >= 0")

    def set_batching(self, max_requests):
        """Requests a free slot takes at once and solves as one lockstep batch."""
        st = self.lib.cfie_server_set_batching(self.h, int(max_requests))
        if st != CFIE_OK:
            raise CfieError(st, "max_requests must be in [1, 256]")

    def submit(self, a, b, n, omega, nrhs=1, theta=None, bc="soft", precision="fp32", eta=None,
               rtol=1e-8, restart=80, maxit=4000):
        a = np.ascontiguousarray(a, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        theta = np.ascontiguousarray(
            2 * np.pi * np.arange(nrhs) / nrhs if theta is None else theta, dtype=np.float64)
        req = cfie_request(BC[bc], PRECISION[precision], int(a.size), _dptr(a), _dptr(b), int(n),
                           float(omega), float(omega if eta is None else eta), int(theta.size),
                           _dptr(theta), float(rtol), int(restart), int(maxit))
        t = ctypes.c_longlong()
        st = self.lib.cfie_server_submit(self.h, ctypes.byref(req), ctypes.byref(t))
        if st != CFIE_OK:
            raise CfieError(st, self.lib.cfie_server_last_error(self.h).decode())
        self.shapes[t.value] = (int(theta.size), int(n))
        return t.value

    def poll(self, ticket, want_x=False):
        r = cfie_result()
        x = None
        ptr = None
        if want_x:
            x = np.zeros(self.shapes[ticket], dtype=np.complex128)
            ptr = x.ctypes.data
        st = self.lib.cfie_server_poll(self.h, ticket, ctypes.byref(r), ptr)
        if st != CFIE_OK:
            raise CfieError(st, self.lib.cfie_server_last_error(self.h).decode())
        out = {k: getattr(r, k) for k, _ in r._fields_}
        if want_x and r.done:
            out["x"] = x
        if r.done and r.status != CFIE_OK:
            buf = ctypes.create_string_buffer(512)
            self.lib.cfie_server_request_error(self.h, ticket, buf, 512)
            out["error"] = buf.value.decode(errors="replace")
        return out

    def wait_all(self, timeout_s=600.0):
        return self.lib.cfie_server_wait_all(self.h, float(timeout_s)) == CFIE_OK

    def release(self, ticket):
        self.lib.cfie_server_release(self.h, ticket)

    def stats(self):
        c = cfie_server_counters()
        self.lib.cfie_server_stats(self.h, ctypes.byref(c))
        return {k: getattr(c, k) for k, _ in c._fields_}

    def close(self):
        if self.h:
            self.lib.cfie_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Geometry:
    def __init__(self, ctx, h):
        self.ctx = ctx
        self.h = h

    def discretise(self, n, omega, eta=None, bc="soft", precision="fp64", layout="matrix_free"):
        op = _P()
        eta = omega if eta is None else eta
        self.ctx.check(self.ctx.lib.cfie_discretise(self.h, int(n), float(omega), float(eta), BC[bc],
                                                    PRECISION[precision], LAYOUT[layout],
                                                    ctypes.byref(op)), "cfie_discretise")
        oper = Operator(self.ctx, op, n)
        self.ctx._children.add(oper)
        return oper

    def close(self):
        if self.h:
            self.ctx.lib.cfie_geom_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Operator:
    def __init__(self, ctx, h, n):
        self.ctx = ctx
        self.h = h
        self.n = n

    def rhs_plane_waves(self, theta, f):
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        self.ctx.check(self.ctx.lib.cfie_rhs_plane_waves(self.h, int(theta.size), _dptr(theta), _addr(f)),
                       "cfie_rhs_plane_waves")

    def apply(self, x, y, nrhs=None):
        nrhs = x.numel() // self.n if nrhs is None else nrhs
        self.ctx.check(self.ctx.lib.cfie_apply(self.h, _addr(x), _addr(y), int(nrhs)), "cfie_apply")

    def set_variant(self, variant):
        """0 = autotuned, 1 = FP32-pipe sums, 2 = tensor-core sums."""
        self.ctx.check(self.ctx.lib.cfie_op_set_variant(self.h, int(variant)), "cfie_op_set_variant")

    def field_eval(self, q, pts, u):
        """u (nrhs, npts) = scattered field of the densities q (nrhs, n) at the
        points pts (npts,), given as complex128 x + i y (the (x, y) double pairs
        of the C ABI); all complex128 device tensors."""
        nrhs = q.numel() // self.n
        npts = pts.numel()
        self.ctx.check(self.ctx.lib.cfie_field_eval(self.h, _addr(q), int(nrhs), int(npts),
                                                    _addr(pts), _addr(u)), "cfie_field_eval")

    def set_residual_variant(self, variant):
        """0 automatic, 1 double-float Dot2 on the CUDA cores, 2 sliced on the tensor cores."""
        self.ctx.check(self.ctx.lib.cfie_op_set_residual_variant(self.h, int(variant)),
                       "cfie_op_set_residual_variant")

    def set_inner_basis(self, fp32):
        """Refined precisions: inner Krylov basis in FP32 (True, default) or FP64."""
        self.ctx.check(self.ctx.lib.cfie_op_set_inner_basis(self.h, 1 if fp32 else 0),
                       "cfie_op_set_inner_basis")

    def set_block_gmres(self, on):
        """gmres_solve as one block GMRES over all right-hand sides (True) or
        one GMRES per right-hand side (False, default)."""
        self.ctx.check(self.ctx.lib.cfie_op_set_block_gmres(self.h, 1 if on else 0),
                       "cfie_op_set_block_gmres")

    def apply_residual(self, x, y, nrhs=None):
        nrhs = x.numel() // self.n if nrhs is None else nrhs
        self.ctx.check(self.ctx.lib.cfie_apply_residual(self.h, _addr(x), _addr(y), int(nrhs)),
                       "cfie_apply_residual")

    def apply_fp64(self, x, y, nrhs=None):
        nrhs = x.numel() // self.n if nrhs is None else nrhs
        self.ctx.check(self.ctx.lib.cfie_apply_fp64(self.h, _addr(x), _addr(y), int(nrhs)),
                       "cfie_apply_fp64")

    def gmres_solve(self, f, x, rtol=1e-6, restart=80, maxit=1000, nrhs=None, allow_noconv=False):
        nrhs = f.numel() // self.n if nrhs is None else nrhs
        its = np.zeros(nrhs, dtype=np.int32)
        rel = np.zeros(nrhs)
        st = self.ctx.lib.cfie_gmres_solve(self.h, _addr(f), _addr(x), int(nrhs), float(rtol),
                                           int(restart), int(maxit), its.ctypes.data_as(_IP),
                                           _dptr(rel))
        if not (st == CFIE_OK or (allow_noconv and st == CFIE_ENOCONV)):
            self.ctx.check(st, "cfie_gmres_solve")
        return its, rel, st

    def last_stats(self):
        s = cfie_solve_stats()
        self.ctx.check(self.ctx.lib.cfie_op_last_stats(self.h, ctypes.byref(s)), "cfie_op_last_stats")
        return {k: getattr(s, k) for k, _ in s._fields_}

    def dirprec(self, kind, q, p, m_leaf=2, t_keep=4, **params):
        """cfie_dirprec_create: the directional preconditioner of Section 2 for
        this operator, whose nodes must be the named curve's n = 4^q p
        arclength samples (arclength_samples + Context.samples)."""
        par = _curve_params(kind, params)
        h = _P()
        self.ctx.check(self.ctx.lib.cfie_dirprec_create(self.h, CURVE[kind],
                                                        _dptr(par) if par.size else None,
                                                        int(par.size), int(q), int(p), int(m_leaf),
                                                        int(t_keep), ctypes.byref(h)),
                       "cfie_dirprec_create")
        prec = Preconditioner(self.ctx, h, self.n)
        self.ctx._children.add(prec)
        return prec

    def set_preconditioner(self, prec):
        """Right preconditioner of gmres_solve (None detaches)."""
        self.ctx.check(self.ctx.lib.cfie_op_set_preconditioner(self.h, prec.h if prec else None),
                       "cfie_op_set_preconditioner")
        if getattr(self, "_prec", None) is not None:
            self._prec._users.discard(self)
        self._prec = prec
        if prec is not None:
            prec._users.add(self)

    def close(self):
        if self.h:
            if getattr(self, "_prec", None) is not None:
                self._prec._users.discard(self)
                self._prec = None
            self.ctx.lib.cfie_op_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Preconditioner:
    """A cfie_dirprec handle: apply(x, y) computes y = P x (eq. eapp)."""

    def __init__(self, ctx, h, n):
        self.ctx = ctx
        self.h = h
        self.n = n
        self._users = weakref.WeakSet()   # operators that use it as their preconditioner

    def apply(self, x, y, nrhs=None):
        nrhs = x.numel() // self.n if nrhs is None else nrhs
        self.ctx.check(self.ctx.lib.cfie_dirprec_apply(self.h, _addr(x), _addr(y), int(nrhs)),
                       "cfie_dirprec_apply")

    def coefficients(self):
        """The m x m block coefficients e_ij (complex128, zero diagonal)."""
        m = ctypes.c_int()
        self.ctx.check(self.ctx.lib.cfie_dirprec_coefficients(self.h, ctypes.byref(m), None),
                       "cfie_dirprec_coefficients")
        e = np.zeros((m.value, m.value), dtype=np.complex128)
        self.ctx.check(self.ctx.lib.cfie_dirprec_coefficients(
            self.h, ctypes.byref(m), e.ctypes.data_as(_DP)), "cfie_dirprec_coefficients")
        return e

    def close(self):
        if self.h:
            for op in list(self._users):
                if op.h:
                    op.set_preconditioner(None)
            self.ctx.lib.cfie_dirprec_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
