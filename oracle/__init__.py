"""Python access to the plain FP64 C oracle.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
CPU-baseline leg of bench.py, never by the library.  See oracle.h for what
each routine computes and which passage of the paper it follows.
"""
import ctypes
import numpy as np

from .build import build as _build

_lib = None

ORC_NCOEF = 12


class Xfer(ctypes.Structure):
    _fields_ = [("point", ctypes.c_int32), ("var", ctypes.c_int32),
                ("dir", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("bytes", ctypes.c_uint64)]


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build())
        d, i, u64, vp = ctypes.c_double, ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p
        _lib.oracle_jacobi_setup.argtypes = [i, i, i, vp, vp]
        _lib.oracle_stencil.argtypes = [i, i, i, vp, vp, d, vp, vp]
        _lib.oracle_jacobi_run.argtypes = [i, i, i, i, ctypes.c_float, i, vp, vp, vp, vp]
        _lib.oracle_jacobi_run.restype = i
        _lib.oracle_plan.argtypes = [i, vp, vp, vp, vp, vp, i, vp, u64, u64, i, i, vp, i, vp, vp]
        _lib.oracle_plan.restype = i
        _lib.oracle_splitmix64.argtypes = [ctypes.POINTER(u64)]
        _lib.oracle_splitmix64.restype = u64
        _lib.oracle_rng_seed.argtypes = [vp, u64]
        _lib.oracle_rng_next.argtypes = [vp]
        _lib.oracle_rng_next.restype = u64
        _lib.oracle_ga.argtypes = [i, i, i, d, d, u64, vp, vp, vp, vp]
        _lib.oracle_ga.restype = i
        _lib.oracle_gemm.argtypes = [i, i, i, vp, i, vp, i, vp, i, i, i]
        _lib.oracle_dft.argtypes = [ctypes.c_int64, i, vp, vp]
        _lib.oracle_fft.argtypes = [ctypes.c_int64, i, vp, vp]
        _lib.oracle_fft.restype = i
        _lib.oracle_fb_best.argtypes = [i, vp, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(d)]
        _lib.oracle_fb_best.restype = i
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------------ Jacobi
def jacobi_setup(I, J, K):
    """(coef[12, I, J, K] float32, p[I, J, K] float32) as the setup nests make them."""
    coef = np.empty((ORC_NCOEF, I, J, K), np.float32)
    p = np.empty((I, J, K), np.float32)
    lib().oracle_jacobi_setup(I, J, K, _p(coef), _p(p))
    return coef, p


def stencil(coef, p, omega):
    """One N2 sweep in FP64 on float inputs -> (wrk2 float64 [I,J,K], res float)."""
    coef = np.ascontiguousarray(coef, np.float32)
    p = np.ascontiguousarray(p, np.float64)
    I, J, K = p.shape
    wrk2 = np.empty_like(p)
    res = ctypes.c_double()
    lib().oracle_stencil(I, J, K, _p(coef), _p(p), float(omega), _p(wrk2), ctypes.byref(res))
    return wrk2, res.value


def jacobi_run(I, J, K, iters, omega=0.8, mode=1, coef=None, p0=None, want_p=True):
    """Whole program. mode 1 = float stores (oracle-s32), 0 = FP64 storage."""
    res = np.empty(iters, np.float64)
    pout = np.empty((I, J, K), np.float64) if want_p else None
    c = None if coef is None else np.ascontiguousarray(coef, np.float32)
    q = None if p0 is None else np.ascontiguousarray(p0, np.float32)
    rc = lib().oracle_jacobi_run(I, J, K, iters, ctypes.c_float(omega), mode,
                                 None if c is None else _p(c), None if q is None else _p(q),
                                 _p(res), None if pout is None else _p(pout))
    if rc != 0:
        raise ValueError("oracle_jacobi_run: bad arguments")
    return res, pout


# ----------------------------------------------------------- transfer plan
def plan(nests, var_bytes, outputs, gene, hoist, iters):
    """nests: list of dicts(level, parallelisable, reads, writes, partial) with
    bit masks.  Returns (list of (point, var, dir, bytes), h2d, d2h)."""
    n = len(nests)
    level = np.array([x["level"] for x in nests], np.int32)
    par = np.array([x["parallelisable"] for x in nests], np.int32)
    rd = np.array([x["reads"] for x in nests], np.uint64)
    wr = np.array([x["writes"] for x in nests], np.uint64)
    pa = np.array([x["partial"] for x in nests], np.uint64)
    vb = np.array(var_bytes, np.uint64)
    h2d, d2h = ctypes.c_uint64(), ctypes.c_uint64()
    cnt = lib().oracle_plan(n, _p(level), _p(par), _p(rd), _p(wr), _p(pa), len(vb), _p(vb),
                            outputs, gene, hoist, iters, None, 0, None, None)
    if cnt < 0:
        raise ValueError("oracle_plan: bad arguments")
    buf = (Xfer * max(cnt, 1))()
    lib().oracle_plan(n, _p(level), _p(par), _p(rd), _p(wr), _p(pa), len(vb), _p(vb),
                      outputs, gene, hoist, iters, ctypes.cast(buf, ctypes.c_void_p), cnt,
                      ctypes.byref(h2d), ctypes.byref(d2h))
    return [(x.point, x.var, x.dir, x.bytes) for x in buf[:cnt]], h2d.value, d2h.value


# ---------------------------------------------------------------------- GA
def splitmix64(state):
    s = ctypes.c_uint64(state)
    out = lib().oracle_splitmix64(ctypes.byref(s))
    return out, s.value


def rng_stream(seed, n):
    st = (ctypes.c_uint64 * 4)()
    lib().oracle_rng_seed(ctypes.cast(st, ctypes.c_void_p), seed)
    return [lib().oracle_rng_next(ctypes.cast(st, ctypes.c_void_p)) for _ in range(n)]


def rng_from_state(state, n):
    st = (ctypes.c_uint64 * 4)(*state)
    return [lib().oracle_rng_next(ctypes.cast(st, ctypes.c_void_p)) for _ in range(n)]


def ga(L, pop, gens, pc, pm, seed, times):
    times = np.ascontiguousarray(times, np.float64)
    assert times.shape == (1 << L,)
    hist = np.empty((gens, pop), np.uint64)
    bg, bt = ctypes.c_uint64(), ctypes.c_double()
    rc = lib().oracle_ga(L, pop, gens, pc, pm, seed, _p(times), _p(hist),
                         ctypes.byref(bg), ctypes.byref(bt))
    if rc != 0:
        raise ValueError("oracle_ga: bad arguments")
    return hist, bg.value, bt.value


# -------------------------------------------------------------------- GEMM
def gemm(A, B, rows=None):
    A = np.ascontiguousarray(A, np.float64)
    B = np.ascontiguousarray(B, np.float64)
    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    r0, r1 = (0, m) if rows is None else rows
    C = np.zeros((m, n), np.float64)
    lib().oracle_gemm(m, n, k, _p(A), k, _p(B), n, _p(C), n, r0, r1)
    return C


# --------------------------------------------------------------------- FFT
def dft(x, direction=-1):
    x = np.ascontiguousarray(x, np.complex128)
    out = np.empty_like(x)
    lib().oracle_dft(x.size, direction, _p(x), _p(out))
    return out


def fft(x, direction=-1):
    x = np.ascontiguousarray(x, np.complex128)
    out = np.empty_like(x)
    if lib().oracle_fft(x.size, direction, _p(x), _p(out)) != 0:
        raise ValueError("oracle_fft: length must be a power of two")
    return out


# ------------------------------------------------- function-block decision
def fb_best(times):
    t = np.ascontiguousarray(times, np.float64)
    n = t.size.bit_length() - 1
    bm, bt = ctypes.c_uint32(), ctypes.c_double()
    if t.size != (1 << n) or lib().oracle_fb_best(n, _p(t), ctypes.byref(bm), ctypes.byref(bt)) != 0:
        raise ValueError("oracle_fb_best: bad arguments")
    return bm.value, bt.value
