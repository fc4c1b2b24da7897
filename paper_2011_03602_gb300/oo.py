"""ctypes binding of liboo (include/oo.h), same names as the C entry points.

Argument marshalling only: every step of the computation runs inside the
library.  Host arrays are numpy arrays; device arrays are anything with a
``data_ptr()`` (torch CUDA tensors) or a raw integer address.  A non-zero
status raises OOError carrying the status and the library's error text.
If liboo.so has not been built the first call raises; there is no fallback.
"""
import ctypes
import math
import os

import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liboo.so")

OO_OK, OO_EINVAL, OO_ENOMEM, OO_ECUDA, OO_ETIMEOUT = 0, -1, -2, -3, -4
OO_ETOLERANCE, OO_EBUSY, OO_ENOTFOUND, OO_ESTATE, OO_EUSER = -5, -6, -7, -8, -9
OO_BLOCK_GEMM, OO_BLOCK_FFT = 1, 2
OO_LANG_C, OO_LANG_PYTHON, OO_LANG_JAVA = 0, 1, 2

_c = ctypes
_u64, _i32, _dbl, _vp = _c.c_uint64, _c.c_int32, _c.c_double, _c.c_void_p


class OOError(RuntimeError):
    def __init__(self, status, text):
        super().__init__("%s (%d): %s" % (oo_status_str(status), status, text))
        self.status = status


class oo_var(_c.Structure):
    _fields_ = [("name", _c.c_char_p), ("bytes", _u64)]


class oo_nest(_c.Structure):
    _fields_ = [("name", _c.c_char_p), ("level", _i32), ("parallelisable", _i32),
                ("reads", _u64), ("writes", _u64), ("partial", _u64)]


class oo_xfer(_c.Structure):
    _fields_ = [("point", _i32), ("var", _i32), ("dir", _i32), ("pad", _i32), ("bytes", _u64)]


class oo_jacobi(_c.Structure):
    _fields_ = [("I", _i32), ("J", _i32), ("K", _i32), ("iters", _i32),
                ("omega", _c.c_float), ("timing", _i32)]


class oo_req(_c.Structure):
    _fields_ = [("kind", _i32), ("prec", _i32), ("m", _c.c_int64), ("n", _c.c_int64), ("k", _c.c_int64),
                ("in0", _vp), ("in1", _vp), ("out", _vp), ("dir", _i32), ("pad", _i32)]


class oo_serve_req(_c.Structure):
    _fields_ = [("kind", _i32), ("prec", _i32), ("m", _c.c_int64), ("n", _c.c_int64), ("k", _c.c_int64),
                ("dir", _i32), ("iters", _i32), ("omega", _c.c_float), ("client", _i32),
                ("in0", _vp), ("in1", _vp), ("out", _vp), ("res", _vp)]


class oo_fb_site(_c.Structure):
    _fields_ = [("callee", _c.c_char_p), ("lang", _i32), ("calls", _i32),
                ("m", _c.c_int64), ("n", _c.c_int64), ("k", _c.c_int64)]


class oo_serve_stats_t(_c.Structure):
    _fields_ = [(n, _u64) for n in ("submitted", "completed", "rejected_busy", "failed", "queued", "running",
                                    "device_free_bytes", "device_budget_bytes")] + [("stage_ms", _dbl * 5)]


class oo_run_stats(_c.Structure):
    _fields_ = [("wall_ms", _dbl), ("nest_ms", _dbl * 6), ("xfer_ms", _dbl),
                ("h2d_bytes", _u64), ("d2h_bytes", _u64), ("n_xfers", _i32),
                ("n_launches", _i32)]

    def as_dict(self):
        return {"wall_ms": self.wall_ms, "nest_ms": list(self.nest_ms), "xfer_ms": self.xfer_ms,
                "h2d_bytes": self.h2d_bytes, "d2h_bytes": self.d2h_bytes,
                "n_xfers": self.n_xfers, "n_launches": self.n_launches}


# generic loop programs: nest body and result check callbacks
OO_NEST_FN = _c.CFUNCTYPE(_c.c_int, _vp, _c.c_int, _c.c_int, _c.c_int64, _c.POINTER(_vp), _vp)
OO_CHECK_FN = _c.CFUNCTYPE(_c.c_int, _vp, _c.POINTER(_vp))

_lib = None


def lib():
    """Load liboo.so once; raise if it is missing (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise OSError("liboo.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    L = _c.CDLL(LIB_PATH)
    P = _c.POINTER
    sig = {
        "oo_create": (_c.c_int, [_c.c_int, _vp, P(_vp)]),
        "oo_destroy": (None, [_vp]),
        "oo_status_str": (_c.c_char_p, [_c.c_int]),
        "oo_last_error": (_c.c_char_p, [_vp]),
        "oo_sync": (_c.c_int, [_vp]),
        "oo_inject_wait_timeout": (_c.c_int, [_vp, _c.c_int]),
        "oo_tune_stencil": (_c.c_int, [_vp, _c.c_int, _c.c_int, _c.c_int, P(_c.c_int), _vp]),
        "oo_load_nests": (_c.c_int, [_vp, P(oo_nest), _c.c_int, P(oo_var), _c.c_int, _u64, P(_c.c_int)]),
        "oo_load_jacobi_nests": (_c.c_int, [_vp, _c.c_int, _c.c_int, _c.c_int, _c.c_int, P(_c.c_int)]),
        "oo_transfer_plan": (_c.c_int, [_vp, _u64, _c.c_int, _c.c_int, P(oo_xfer), _c.c_int,
                                        P(_c.c_int), P(_u64), P(_u64)]),
        "oo_run_pattern": (_c.c_int, [_vp, _u64, _c.c_int, P(oo_jacobi), _vp, _vp, P(oo_run_stats)]),
        "oo_run_pattern_dev": (_c.c_int, [_vp, _u64, _c.c_int, P(oo_jacobi), _vp, _vp, P(oo_run_stats)]),
        "oo_stencil_dev": (_c.c_int, [_vp, _c.c_int, _c.c_int, _c.c_int, _c.c_int, P(_vp), _vp,
                                      _c.c_float, _vp, _vp]),
        "oo_stencil_noalloc_dev": (_c.c_int, [_vp, _c.c_int, _c.c_int, _c.c_int, _c.c_int, P(_vp), _vp,
                                              _c.c_float, _vp, _vp]),
        "oo_stencil_check": (_c.c_int, [_vp]),
        "oo_stencil_noalloc_check": (_c.c_int, [_vp]),
        "oo_set_option": (_c.c_int, [_vp, _c.c_int, _c.c_int]),
        "oo_get_option": (_c.c_int, [_vp, _c.c_int, P(_c.c_int)]),
        "oo_jacobi_pitch": (_c.c_int, [_c.c_int]),
        "oo_ga_search": (_c.c_int, [_vp, P(oo_jacobi), _c.c_int, _c.c_int, _c.c_int, _dbl, _dbl, _u64,
                                    _dbl, P(_u64), P(_dbl), _vp, _vp]),
        "oo_ga_search_resume": (_c.c_int, [_vp, P(oo_jacobi), _c.c_int, _c.c_int, _c.c_int, _dbl, _dbl, _u64,
                                           _dbl, _vp, P(_u64), P(_dbl), _vp, _vp]),
        "oo_ga_table": (_c.c_int, [_c.c_int, _c.c_int, _c.c_int, _dbl, _dbl, _u64, _vp, _vp,
                                   P(_u64), P(_dbl)]),
        "oo_lookup_block": (_c.c_int, [_c.c_char_p, _c.c_int, P(_c.c_int)]),
        "oo_fft_c128": (_c.c_int, [_vp, _c.c_int64, _c.c_int, _vp, _vp]),
        "oo_gemm_f64": (_c.c_int, [_vp, _c.c_int, _c.c_int, _c.c_int, _c.c_int, _vp, _c.c_int, _vp, _c.c_int,
                                   _vp, _c.c_int]),
        "oo_gemm_f64_dev": (_c.c_int, [_vp, _c.c_int, _c.c_int, _c.c_int, _c.c_int, _vp, _c.c_int, _vp,
                                       _c.c_int, _vp, _c.c_int]),
        "oo_gemm_check": (_c.c_int, [_vp, _c.c_int, _c.c_int, _c.c_int]),
        "oo_fb_search": (_c.c_int, [_vp, _vp, _c.c_int, _c.c_int, _dbl, _u64, _vp, _vp, P(_c.c_uint32), P(_dbl)]),
        "oo_fb_best": (_c.c_int, [_c.c_int, _vp, P(_c.c_uint32), P(_dbl)]),
        "oo_offload_search": (_c.c_int, [_vp, _vp, _c.c_int, _c.c_int, _dbl, _u64, P(oo_jacobi), _c.c_int,
                                         _c.c_int, _c.c_int, _dbl, _dbl, _u64, _dbl, P(_c.c_uint32), P(_u64),
                                         P(_dbl), P(_dbl)]),
        "oo_run_program": (_c.c_int, [_vp, _u64, _c.c_int, _c.c_int, OO_NEST_FN, _vp, _vp, _vp, P(oo_run_stats)]),
        "oo_ga_program": (_c.c_int, [_vp, _c.c_int, _c.c_int, OO_NEST_FN, OO_CHECK_FN, _vp, _vp, _vp, _c.c_int,
                                     _c.c_int, _dbl, _dbl, _u64, P(_u64), P(_dbl), _vp, _vp]),
        "oo_gemm_plan": (_c.c_int, [_c.c_int, _c.c_int, P(_c.c_int), P(_c.c_int), P(_c.c_int), P(_c.c_int)]),
        "oo_gemm_scheme": (_c.c_int, [_c.c_int, P(_c.c_int), P(_c.c_int)]),
        "oo_tune_gemm_tiles": (_c.c_int, [_vp, _vp, _vp]),
        "oo_get_gemm_tiles": (_c.c_int, [_vp, _vp]),
        "oo_set_gemm_tiles": (_c.c_int, [_vp, _vp]),
        "oo_batch_create": (_c.c_int, [_vp, P(oo_req), _c.c_int, P(_vp)]),
        "oo_batch_run": (_c.c_int, [_vp, _c.c_int]),
        "oo_batch_check": (_c.c_int, [_vp]),
        "oo_batch_info": (_c.c_int, [_vp, P(_dbl), P(_dbl), P(_c.c_int), P(_c.c_int)]),
        "oo_batch_destroy": (None, [_vp]),
        "oo_serve_start": (_c.c_int, [_vp, _c.c_int, _u64, _c.c_int]),
        "oo_serve_start_resident": (_c.c_int, [_vp, _u64, _c.c_int, _c.c_int]),
        "oo_submit": (_c.c_int, [_vp, P(oo_serve_req), P(_u64)]),
        "oo_wait": (_c.c_int, [_vp, _u64, _c.c_int, P(_dbl)]),
        "oo_serve_stats": (_c.c_int, [_vp, P(oo_serve_stats_t)]),
        "oo_serve_stop": (_c.c_int, [_vp]),
        "oo_router_create": (_c.c_int, [_vp, _c.c_int, P(_vp)]),
        "oo_router_submit": (_c.c_int, [_vp, P(oo_serve_req), P(_c.c_int), P(_u64)]),
        "oo_router_wait": (_c.c_int, [_vp, _c.c_int, _u64, _c.c_int, P(_dbl)]),
        "oo_router_destroy": (None, [_vp]),
        "oo_route_pick": (_c.c_int, [_vp, _vp, _c.c_int, _u64, P(_c.c_int)]),
        "oo_route_batch": (_c.c_int, [_vp, _vp, _c.c_int, _vp, _c.c_int, _vp]),
        "oo_serve_footprint": (_c.c_int, [P(oo_serve_req), P(_u64)]),
        "oo_fft_c128_dev": (_c.c_int, [_vp, _c.c_int64, _c.c_int, _c.c_int, _vp, _vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(ctx, st):
    if st != OO_OK:
        txt = lib().oo_last_error(ctx)
        raise OOError(st, (txt or b"").decode(errors="replace"))


def _host_ptr(a, dtype, n=None):
    if a is None:
        return None
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous:
        raise TypeError("expected a C-contiguous numpy %s array" % np.dtype(dtype).name)
    if n is not None and a.size != n:
        raise ValueError("expected %d elements, got %d" % (n, a.size))
    return a.ctypes.data_as(_vp)


def _dev_ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return _vp(t)
    if hasattr(t, "is_cuda") and not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if hasattr(t, "is_contiguous") and not t.is_contiguous():
        raise TypeError("expected a contiguous tensor")
    return _vp(t.data_ptr())


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return _vp(stream)
    return _vp(stream.cuda_stream)


# ------------------------------------------------------------------ context
def oo_status_str(status):
    return lib().oo_status_str(status).decode()


def oo_create(device=0, stream=None):
    """Returns an opaque context handle (c_void_p)."""
    h = _vp()
    st = lib().oo_create(device, _stream_handle(stream), _c.byref(h))
    if st != OO_OK:
        raise OOError(st, (lib().oo_last_error(None) or b"").decode(errors="replace"))
    return h


def oo_destroy(ctx):
    lib().oo_destroy(ctx)
    k = _ctx_key(ctx)
    with _in_flight_lock:  # a service still running stopped with the context
        for key in [key for key in _in_flight if key[0] == k]:
            del _in_flight[key]


def oo_last_error(ctx):
    return (lib().oo_last_error(ctx) or b"").decode(errors="replace")


def oo_sync(ctx):
    _check(ctx, lib().oo_sync(ctx))


OO_STENCIL_VARIANTS = 5


def oo_tune_stencil(ctx, I, J, K):
    """Time every stencil tile variant for the grid; the fastest is kept for
    it.  Returns (variant, ms per variant)."""
    v = _c.c_int()
    ms = np.empty(OO_STENCIL_VARIANTS, np.float64)
    _check(ctx, lib().oo_tune_stencil(ctx, I, J, K, _c.byref(v), ms.ctypes.data_as(_vp)))
    return v.value, ms


OO_INJECT_NONE, OO_INJECT_STENCIL_LOAD, OO_INJECT_FUSED_BARRIER, OO_INJECT_SERVE_STALL = 0, 1, 2, 3
OO_OPT_JACOBI_FUSED, OO_OPT_STENCIL_VARIANT, OO_OPT_GEMM_PAIR = 1, 2, 3


def oo_set_option(ctx, option, value):
    """Set a per-context option (OO_OPT_JACOBI_FUSED, OO_OPT_STENCIL_VARIANT, OO_OPT_GEMM_PAIR)."""
    _check(ctx, lib().oo_set_option(ctx, option, value))


def oo_get_option(ctx, option):
    v = _c.c_int()
    _check(ctx, lib().oo_get_option(ctx, option, _c.byref(v)))
    return v.value


def oo_inject_wait_timeout(ctx, what):
    """Arm a one-shot bounded-wait failure (tests of the timeout paths)."""
    _check(ctx, lib().oo_inject_wait_timeout(ctx, what))


# -------------------------------------------------------------- nest table
def oo_load_nests(ctx, nests, var_bytes, outputs, var_names=None):
    """nests: sequence of dicts(name, level, parallelisable, reads, writes, partial)."""
    n = len(nests)
    arr = (oo_nest * n)()
    keep = []
    for i, d in enumerate(nests):
        nm = d.get("name", "n%d" % i).encode()
        keep.append(nm)
        arr[i] = oo_nest(nm, d["level"], d["parallelisable"], d["reads"], d["writes"], d["partial"])
    v = (oo_var * len(var_bytes))()
    for i, b in enumerate(var_bytes):
        nm = (var_names[i] if var_names else "v%d" % i).encode()
        keep.append(nm)
        v[i] = oo_var(nm, b)
    gl = _c.c_int()
    _check(ctx, lib().oo_load_nests(ctx, arr, n, v, len(var_bytes), outputs, _c.byref(gl)))
    return gl.value


def oo_load_jacobi_nests(ctx, I, J, K, iters):
    gl = _c.c_int()
    _check(ctx, lib().oo_load_jacobi_nests(ctx, I, J, K, iters, _c.byref(gl)))
    return gl.value


def oo_transfer_plan(ctx, gene, hoist, iters):
    """-> (list of (point, var, dir, bytes), h2d_bytes, d2h_bytes)."""
    n = _c.c_int()
    h2d, d2h = _u64(), _u64()
    _check(ctx, lib().oo_transfer_plan(ctx, gene, hoist, iters, None, 0, _c.byref(n), None, None))
    buf = (oo_xfer * max(n.value, 1))()
    _check(ctx, lib().oo_transfer_plan(ctx, gene, hoist, iters, buf, n.value, _c.byref(n),
                                       _c.byref(h2d), _c.byref(d2h)))
    return [(x.point, x.var, x.dir, x.bytes) for x in buf[:n.value]], h2d.value, d2h.value


# ------------------------------------------------------------------ Jacobi
def jacobi(I, J, K, iters, omega=0.8, timing=False):
    return oo_jacobi(I, J, K, iters, omega, 1 if timing else 0)


def oo_jacobi_pitch(K):
    return lib().oo_jacobi_pitch(K)


def oo_run_pattern(ctx, gene, hoist, prob, p_out=None, res_out=None):
    """Host outputs (numpy float32 [I*J*K] / float64 [iters]); returns stats dict."""
    st = oo_run_stats()
    n = prob.I * prob.J * prob.K
    _check(ctx, lib().oo_run_pattern(ctx, gene, hoist, _c.byref(prob), _host_ptr(p_out, np.float32, n),
                                     _host_ptr(res_out, np.float64, prob.iters), _c.byref(st)))
    return st.as_dict()


def oo_run_pattern_dev(ctx, gene, hoist, prob, p_dev=None, res_dev=None):
    """Device outputs (torch tensors or raw addresses); returns stats dict."""
    st = oo_run_stats()
    _check(ctx, lib().oo_run_pattern_dev(ctx, gene, hoist, _c.byref(prob), _dev_ptr(p_dev),
                                         _dev_ptr(res_dev), _c.byref(st)))
    return st.as_dict()


def oo_stencil_dev(ctx, I, J, K, pitch, coef, p, omega, wrk2, res_dev):
    """coef: 12 device arrays (a0 a1 a2 a3 b0 b1 b2 c0 c1 c2 bnd wrk1)."""
    if len(coef) != 12:
        raise ValueError("need 12 coefficient arrays")
    ptrs = (_vp * 12)(*[_dev_ptr(c).value for c in coef])
    _check(ctx, lib().oo_stencil_dev(ctx, I, J, K, pitch, ptrs, _dev_ptr(p), _c.c_float(omega),
                                     _dev_ptr(wrk2), _dev_ptr(res_dev)))


def oo_stencil_noalloc_dev(ctx, I, J, K, pitch, coef, p, omega, wrk2, res_dev):
    """oo_stencil_dev without any device allocation (static scratch); see oo.h."""
    if len(coef) != 12:
        raise ValueError("need 12 coefficient arrays")
    ptrs = (_vp * 12)(*[_dev_ptr(c).value for c in coef])
    _check(ctx, lib().oo_stencil_noalloc_dev(ctx, I, J, K, pitch, ptrs, _dev_ptr(p), _c.c_float(omega),
                                             _dev_ptr(wrk2), _dev_ptr(res_dev)))


def oo_stencil_check(ctx):
    """Synchronise; raise OOError(OO_ETIMEOUT) if an oo_stencil_dev sweep's bounded wait ran out."""
    _check(ctx, lib().oo_stencil_check(ctx))


def oo_stencil_noalloc_check(ctx):
    """Synchronise; raise OOError(OO_ETIMEOUT) if an oo_stencil_noalloc_dev sweep's bounded wait ran out."""
    _check(ctx, lib().oo_stencil_noalloc_check(ctx))


# ---------------------------------------------------------------------- GA
def oo_ga_table(L, pop, gens, pc, pm, seed, times):
    times = np.ascontiguousarray(times, np.float64)
    if times.size != (1 << L):
        raise ValueError("need 2^L times")
    hist = np.empty(gens * pop, np.uint64)
    bg, bt = _u64(), _dbl()
    _check(None, lib().oo_ga_table(L, pop, gens, pc, pm, seed, times.ctypes.data_as(_vp),
                                   hist.ctypes.data_as(_vp), _c.byref(bg), _c.byref(bt)))
    return hist.reshape(gens, pop), bg.value, bt.value


def oo_ga_search(ctx, prob, hoist, pop, gens, pc, pm, seed, eval_timeout_ms=0.0, known_ms=None):
    """known_ms (64 floats, NaN = not measured yet): resume from a saved
    gene_ms table (oo_ga_search_resume)."""
    hist = np.empty(gens * pop, np.uint64)
    gene_ms = np.empty(64, np.float64)
    bg, bt = _u64(), _dbl()
    if known_ms is None:
        st = lib().oo_ga_search(ctx, _c.byref(prob), hoist, pop, gens, pc, pm, seed, eval_timeout_ms,
                                _c.byref(bg), _c.byref(bt), hist.ctypes.data_as(_vp), gene_ms.ctypes.data_as(_vp))
    else:
        known = np.ascontiguousarray(known_ms, dtype=np.float64)
        if known.shape != (64,):
            raise ValueError("known_ms must have 64 entries")
        st = lib().oo_ga_search_resume(ctx, _c.byref(prob), hoist, pop, gens, pc, pm, seed, eval_timeout_ms,
                                       known.ctypes.data_as(_vp), _c.byref(bg), _c.byref(bt),
                                       hist.ctypes.data_as(_vp), gene_ms.ctypes.data_as(_vp))
    _check(ctx, st)
    return {"best_gene": bg.value, "best_ms": bt.value, "history": hist.reshape(gens, pop),
            "gene_ms": gene_ms}


# ------------------------------------------------- generic loop programs
def _addr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise TypeError("host buffers must be C-contiguous")
        return x.ctypes.data
    return _dev_ptr(x).value


def _ptr_array(bufs):
    arr = (_vp * len(bufs))()
    for i, b in enumerate(bufs):
        arr[i] = _addr(b)
    return arr


def _nest_callback(body):
    """body(nest, on_gpu, iteration, stream_handle) -> None; exceptions abort the run."""
    def cb(user, nest, on_gpu, it, vars_, stream):
        try:
            body(nest, bool(on_gpu), it, stream)
            return 0
        except Exception:  # reported to the library as a failed nest
            import traceback
            traceback.print_exc()
            return 1
    return OO_NEST_FN(cb)


def oo_run_program(ctx, gene, hoist, iters, body, host_vars, dev_vars):
    """Run the loaded table's program; body(nest, on_gpu, iteration, stream)
    executes a nest on the caller's own host / device buffers (the same
    objects passed here, in table order).  Returns the stats dict."""
    cb = _nest_callback(body)
    st = oo_run_stats()
    _check(ctx, lib().oo_run_program(ctx, gene, hoist, iters, cb, None, _ptr_array(host_vars),
                                     _ptr_array(dev_vars), _c.byref(st)))
    return st.as_dict()


def oo_ga_program(ctx, gene_len, hoist, iters, body, host_vars, dev_vars, pop, gens, pc, pm, seed, check=None):
    """GA over the loaded program's genes (gene_len as oo_load_nests returned
    it); check() -> bool accepts or rejects the result left in the host buffers."""
    cb = _nest_callback(body)
    ck = OO_CHECK_FN(lambda user, hv: 0 if check is None or check() else 1)
    hist = np.empty(gens * pop, np.uint64)
    bg, bt = _u64(), _dbl()
    gm = np.empty(1 << gene_len, np.float64)
    _check(ctx, lib().oo_ga_program(ctx, hoist, iters, cb, ck, None, _ptr_array(host_vars), _ptr_array(dev_vars),
                                    pop, gens, pc, pm, seed, _c.byref(bg), _c.byref(bt),
                                    hist.ctypes.data_as(_vp), gm.ctypes.data_as(_vp)))
    return {"best_gene": bg.value, "best_ms": bt.value, "history": hist.reshape(gens, pop), "gene_ms": gm}


# ------------------------------------------- function-block trial order
def fb_sites(sites):
    """[(callee, lang, calls, m, n, k), ...] -> ctypes array of oo_fb_site
    (the callee byte strings are kept alive on the array)."""
    arr = (oo_fb_site * len(sites))()
    keep = []
    for i, (callee, lang, calls, m, n, k) in enumerate(sites):
        b = callee.encode() if isinstance(callee, str) else callee
        keep.append(b)
        arr[i] = oo_fb_site(b, lang, calls, m, n, k)
    arr._keep = keep
    return arr


def oo_fb_search(ctx, sites, prec=None, tol=1e-10, seed=1):
    """Sec. 4.2.1 trial over every combination of the known sites."""
    prec = OO_PREC_FP64EQ if prec is None else prec
    arr = fb_sites(sites)
    n = len(sites)
    ids = np.zeros(n, np.int32)
    ms = np.empty(1 << n, np.float64)
    bm, bt = _c.c_uint32(), _dbl()
    _check(ctx, lib().oo_fb_search(ctx, arr, n, prec, tol, seed, ids.ctypes.data_as(_vp), ms.ctypes.data_as(_vp),
                                   _c.byref(bm), _c.byref(bt)))
    return {"block_ids": ids, "mask_ms": ms, "best_mask": bm.value, "best_ms": bt.value}


def oo_fb_best(mask_ms):
    ms = np.ascontiguousarray(mask_ms, np.float64)
    n = ms.size.bit_length() - 1
    if ms.size != (1 << n):
        raise ValueError("need 2^n times")
    bm, bt = _c.c_uint32(), _dbl()
    _check(None, lib().oo_fb_best(n, ms.ctypes.data_as(_vp), _c.byref(bm), _c.byref(bt)))
    return bm.value, bt.value


def oo_offload_search(ctx, sites, prob, hoist, pop, gens, pc, pm, ga_seed, eval_timeout_ms=0.0, prec=None,
                      tol=1e-10, seed=1):
    """Sec. 4.2: function blocks first, then the loop GA."""
    prec = OO_PREC_FP64EQ if prec is None else prec
    arr = fb_sites(sites) if sites else None
    bm, bg, fms, lms = _c.c_uint32(), _u64(), _dbl(), _dbl()
    _check(ctx, lib().oo_offload_search(ctx, arr, len(sites), prec, tol, seed, _c.byref(prob), hoist, pop, gens,
                                        pc, pm, ga_seed, eval_timeout_ms, _c.byref(bm), _c.byref(bg),
                                        _c.byref(fms), _c.byref(lms)))
    return {"best_mask": bm.value, "best_gene": bg.value, "fb_ms": fms.value, "loop_ms": lms.value}


# --------------------------------------------------------- function blocks
def oo_fft_c128(ctx, x, direction=-1, out=None):
    """Host complex128 array -> its FFT (new array unless out is given)."""
    x = np.ascontiguousarray(x, np.complex128)
    if out is None:
        out = np.empty_like(x)
    _check(ctx, lib().oo_fft_c128(ctx, x.size, direction, x.ctypes.data_as(_vp), _host_ptr(out, np.complex128)))
    return out


OO_PREC_SPLIT3_BF16 = 0
OO_PREC_SPLIT3_TF32 = 1
OO_PREC_FP64EQ = 2


def oo_gemm_f64(ctx, A, B, prec=OO_PREC_SPLIT3_BF16, out=None):
    """Host float64 A (m x k) @ B (k x n) -> C (m x n) float64."""
    A = np.ascontiguousarray(A, np.float64)
    B = np.ascontiguousarray(B, np.float64)
    m, k = A.shape
    k2, n = B.shape
    if k != k2:
        raise ValueError("inner dimensions differ")
    C = np.empty((m, n), np.float64) if out is None else out
    _check(ctx, lib().oo_gemm_f64(ctx, prec, m, n, k, A.ctypes.data_as(_vp), k, B.ctypes.data_as(_vp), n,
                                  _host_ptr(C, np.float64, m * n), n))
    return C


def oo_gemm_f64_dev(ctx, m, n, k, dA, lda, dB, ldb, dC, ldc, prec=OO_PREC_SPLIT3_BF16):
    _check(ctx, lib().oo_gemm_f64_dev(ctx, prec, m, n, k, _dev_ptr(dA), lda, _dev_ptr(dB), ldb,
                                      _dev_ptr(dC), ldc))


def oo_gemm_check(ctx, m, n, k):
    _check(ctx, lib().oo_gemm_check(ctx, m, n, k))


def oo_gemm_plan(prec, k):
    """(BF16 products, digit bits beta, level bound L, exact K-block) of a
    product with inner dimension k in precision pattern prec."""
    v = [_c.c_int() for _ in range(4)]
    _check(None, lib().oo_gemm_plan(prec, k, *[_c.byref(x) for x in v]))
    return tuple(x.value for x in v)


OO_EQ_PAIRS, OO_EQ_LEVELS = 0, 1
OO_TILE_NBUCKETS, OO_TILE_KBUCKETS = 6, 5


def oo_gemm_scheme(k):
    """(scheme, most products summed in one FP32 accumulator) of an
    FP64-equivalent product with inner dimension k."""
    s, per = _c.c_int(), _c.c_int()
    _check(None, lib().oo_gemm_scheme(k, _c.byref(s), _c.byref(per)))
    return s.value, per.value


def oo_tune_gemm_tiles(ctx):
    """Autotune the FP64-equivalent tile widths; returns (widths table
    OO_TILE_NBUCKETS x OO_TILE_KBUCKETS, mean ms per bucket and width 32/64/128)."""
    w = np.zeros(OO_TILE_NBUCKETS * OO_TILE_KBUCKETS, np.int32)
    ms = np.zeros(OO_TILE_NBUCKETS * OO_TILE_KBUCKETS * 3, np.float64)
    _check(ctx, lib().oo_tune_gemm_tiles(ctx, w.ctypes.data_as(_vp), ms.ctypes.data_as(_vp)))
    return w.reshape(OO_TILE_NBUCKETS, OO_TILE_KBUCKETS), ms.reshape(OO_TILE_NBUCKETS, OO_TILE_KBUCKETS, 3)


def oo_get_gemm_tiles(ctx):
    w = np.zeros(OO_TILE_NBUCKETS * OO_TILE_KBUCKETS, np.int32)
    _check(ctx, lib().oo_get_gemm_tiles(ctx, w.ctypes.data_as(_vp)))
    return w.reshape(OO_TILE_NBUCKETS, OO_TILE_KBUCKETS)


def oo_set_gemm_tiles(ctx, widths):
    w = np.ascontiguousarray(widths, np.int32).reshape(-1)
    if w.size != OO_TILE_NBUCKETS * OO_TILE_KBUCKETS:
        raise ValueError("need %d widths" % (OO_TILE_NBUCKETS * OO_TILE_KBUCKETS))
    _check(ctx, lib().oo_set_gemm_tiles(ctx, w.ctypes.data_as(_vp)))


def oo_fft_c128_dev(ctx, n, batch, direction, din, dout):
    """Device buffers of batch * n complex128 (torch tensors or addresses)."""
    _check(ctx, lib().oo_fft_c128_dev(ctx, n, batch, direction, _dev_ptr(din), _dev_ptr(dout)))


# ------------------------------------------------------ batched function blocks
def oo_batch_create(ctx, reqs):
    """reqs: dicts kind ('gemm' | 'fft'), sizes and device buffers:
    gemm: m, n, k, A, B, C (contiguous row-major); fft: n, x, X, dir."""
    arr = (oo_req * len(reqs))()
    for i, r in enumerate(reqs):
        if r["kind"] == "gemm":
            arr[i] = oo_req(OO_BLOCK_GEMM, r.get("prec", 0), r["m"], r["n"], r["k"], _dev_ptr(r["A"]),
                            _dev_ptr(r["B"]), _dev_ptr(r["C"]), 0, 0)
        else:
            arr[i] = oo_req(OO_BLOCK_FFT, 0, 0, r["n"], 0, _dev_ptr(r["x"]), None, _dev_ptr(r["X"]),
                            r.get("dir", -1), 0)
    h = _vp()
    _check(ctx, lib().oo_batch_create(ctx, arr, len(reqs), _c.byref(h)))
    return h


def oo_batch_run(ctx, b, mode):
    """mode 0 grouped, 1 grouped in a CUDA graph, 2 one call per request."""
    _check(ctx, lib().oo_batch_run(b, mode))


def oo_batch_check(ctx, b):
    _check(ctx, lib().oo_batch_check(b))


def oo_batch_info(b):
    fl, pts, ng, nf = _dbl(), _dbl(), _c.c_int(), _c.c_int()
    lib().oo_batch_info(b, _c.byref(fl), _c.byref(pts), _c.byref(ng), _c.byref(nf))
    return {"gemm_flops": fl.value, "fft_points": pts.value, "n_gemm": ng.value, "n_fft": nf.value}


def oo_batch_destroy(b):
    lib().oo_batch_destroy(b)


# ------------------------------------------------------------------- serving
OO_BLOCK_JACOBI = 3


def oo_serve_start(ctx, slots=8, hbm_budget_bytes=8 << 30, queue_cap=4096):
    _check(ctx, lib().oo_serve_start(ctx, slots, hbm_budget_bytes, queue_cap))


def serve_request(kind, **kw):
    """Build an oo_serve_req from numpy host arrays: gemm(A, B, C, prec),
    fft(x, X, dir), jacobi(I, J, K, iters, p, res, omega).  GEMMs default to
    the FP64-equivalent pattern.  The request holds its arrays, and oo_submit
    holds them from submission until oo_wait returns for the ticket (the
    library reads and writes them in between)."""
    r = oo_serve_req()
    r._arrays = tuple(v for v in kw.values() if isinstance(v, np.ndarray))
    r.client = kw.get("client", OO_LANG_PYTHON)
    if kind == "gemm":
        A, B, C = kw["A"], kw["B"], kw["C"]
        r.kind, r.prec, (r.m, r.k), r.n = OO_BLOCK_GEMM, kw.get("prec", OO_PREC_FP64EQ), A.shape, B.shape[1]
        r.in0, r.in1, r.out = _host_ptr(A, np.float64), _host_ptr(B, np.float64), _host_ptr(C, np.float64)
    elif kind == "fft":
        x, X = kw["x"], kw["X"]
        r.kind, r.n, r.dir = OO_BLOCK_FFT, x.size, kw.get("dir", -1)
        r.in0, r.out = _host_ptr(x, np.complex128), _host_ptr(X, np.complex128)
    else:
        r.kind, r.m, r.n, r.k = OO_BLOCK_JACOBI, kw["I"], kw["J"], kw["K"]
        r.iters, r.omega = kw["iters"], kw.get("omega", 0.8)
        r.out = _host_ptr(kw["p"], np.float32, kw["I"] * kw["J"] * kw["K"])
        res = kw.get("res")
        if res is not None and res.size < kw["iters"]:
            raise ValueError("res needs at least iters elements")
        r.res = None if res is None else _host_ptr(res, np.float64)
    return r


def oo_serve_start_resident(ctx, hbm_budget_bytes, queue_cap=1024, tensor_ctas=0):
    """Serve with the request loop resident on the device (persistent
    workers fed through rings; no kernel launch per request)."""
    _check(ctx, lib().oo_serve_start_resident(ctx, hbm_budget_bytes, queue_cap, tensor_ctas))


# arrays of submitted requests, by (context, ticket), until oo_wait returns
_in_flight = {}
_in_flight_lock = threading.Lock()


def _ctx_key(ctx):
    return ctx.value if hasattr(ctx, "value") else ctx


def _hold(ctx, req, ticket):
    with _in_flight_lock:
        _in_flight[(_ctx_key(ctx), ticket)] = getattr(req, "_arrays", ())


def oo_submit(ctx, req):
    """-> ticket; raises OOError (status OO_EBUSY when back-pressured)."""
    t = _u64()
    _check(ctx, lib().oo_submit(ctx, _c.byref(req), _c.byref(t)))
    _hold(ctx, req, t.value)
    return t.value


def oo_submit_status(ctx, req):
    """-> (status, ticket) without raising (for load generators)."""
    t = _u64()
    st = lib().oo_submit(ctx, _c.byref(req), _c.byref(t))
    if st == 0:
        _hold(ctx, req, t.value)
    return st, t.value


def oo_wait(ctx, ticket, timeout_ms=60000):
    """-> latency in ms; raises OOError (OO_ETIMEOUT if not done in time,
    and the ticket and its arrays stay held)."""
    lat = _dbl()
    st = lib().oo_wait(ctx, ticket, timeout_ms, _c.byref(lat))
    if st != OO_ETIMEOUT:
        with _in_flight_lock:
            _in_flight.pop((_ctx_key(ctx), ticket), None)
    _check(ctx, st)
    return lat.value


def oo_serve_stats(ctx):
    st = oo_serve_stats_t()
    _check(ctx, lib().oo_serve_stats(ctx, _c.byref(st)))
    out = {n: getattr(st, n) for n, _ in oo_serve_stats_t._fields_[:-1]}
    out["stage_ms"] = dict(zip(("queued", "input", "staging", "device", "output"), list(st.stage_ms)))
    return out


def oo_serve_stop(ctx):
    _check(ctx, lib().oo_serve_stop(ctx))
    k = _ctx_key(ctx)
    with _in_flight_lock:  # tickets not waited for are discarded with the service
        for key in [key for key in _in_flight if key[0] == k]:
            del _in_flight[key]


def oo_route_pick(free_bytes, queued, need):
    """The replica a request of `need` bytes goes to (host-only)."""
    f = np.ascontiguousarray(free_bytes, dtype=np.uint64)
    q = np.ascontiguousarray(queued, dtype=np.uint64)
    if f.size != q.size or f.size < 1:
        raise ValueError("one free-bytes and one queued figure per replica")
    r = _c.c_int()
    _check(None, lib().oo_route_pick(f.ctypes.data_as(_vp), q.ctypes.data_as(_vp), f.size, int(need), _c.byref(r)))
    return r.value


def oo_route_batch(free_bytes, queued, needs):
    """Owners of requests routed in order (host-only; see oo.h)."""
    f = np.ascontiguousarray(free_bytes, dtype=np.uint64)
    q = np.ascontiguousarray(queued, dtype=np.uint64)
    nd = np.ascontiguousarray(needs, dtype=np.uint64)
    if f.size != q.size or f.size < 1:
        raise ValueError("one free-bytes and one queued figure per replica")
    out = np.empty(nd.size, dtype=np.int32)
    _check(None, lib().oo_route_batch(f.ctypes.data_as(_vp), q.ctypes.data_as(_vp), f.size,
                                      nd.ctypes.data_as(_vp), nd.size, out.ctypes.data_as(_vp)))
    return out


def oo_serve_footprint(req):
    b = _u64()
    _check(None, lib().oo_serve_footprint(_c.byref(req), _c.byref(b)))
    return b.value


class Router:
    """Serving replicas (oo_router_*): requests routed over serving contexts
    by free device memory.  submit -> (replica, ticket); wait(replica,
    ticket) -> latency ms.  The request's arrays are held until waited."""

    def __init__(self, ctxs):
        self.ctxs = list(ctxs)
        arr = (_vp * len(self.ctxs))(*[_ctx_key(c) for c in self.ctxs])
        h = _vp()
        _check(None, lib().oo_router_create(arr, len(self.ctxs), _c.byref(h)))
        self.h = h

    def submit(self, req):
        r, t = _c.c_int(), _u64()
        st = lib().oo_router_submit(self.h, _c.byref(req), _c.byref(r), _c.byref(t))
        if st != OO_OK:
            raise OOError(st, "router: " + oo_status_str(st))
        _hold(self.ctxs[r.value], req, t.value)
        return r.value, t.value

    def wait(self, replica, ticket, timeout_ms=60000):
        lat = _dbl()
        st = lib().oo_router_wait(self.h, replica, ticket, timeout_ms, _c.byref(lat))
        if st != OO_ETIMEOUT:
            with _in_flight_lock:
                _in_flight.pop((_ctx_key(self.ctxs[replica]), ticket), None)
        _check(self.ctxs[replica], st)
        return lat.value

    def close(self):
        if self.h:
            lib().oo_router_destroy(self.h)
            self.h = None


def oo_lookup_block(callee, lang):
    b = _c.c_int()
    _check(None, lib().oo_lookup_block(callee.encode(), lang, _c.byref(b)))
    return b.value


__all__ = [n for n in dir() if n.startswith("oo_") or n in ("OOError", "jacobi", "lib")]
del math
