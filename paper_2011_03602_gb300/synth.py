"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle calls.

This module holds no arithmetic of the offload method itself: only the
random streams that feed it.  Every generator is a pure function of its seed.

Stream: splitmix64 (Steele, Lea & Flood, 2014): state_t = seed + t * 0x9e3779b97f4a7c15
(mod 2^64), then the mix; a uniform is (x >> 11) * 2^-53 in [0, 1).
GEMM entries: 2u - 1 (uniform on [-1, 1)).
Complex normal: Box-Muller, |z|^2 = -ln(1 - u1), arg z = 2 pi u2, so the real
and imaginary parts are each N(0, 1/2) and E|z|^2 = 1.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_stream(seed: int, n: int) -> np.ndarray:
    """The first n splitmix64 outputs for `seed` (uint64 array)."""
    with np.errstate(over="ignore"):
        t = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + t * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, n: int) -> np.ndarray:
    """n float64 uniforms in [0, 1)."""
    return (splitmix64_stream(seed, n) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def gemm_matrix(seed: int, rows: int, cols: int) -> np.ndarray:
    """Row-major float64 matrix with entries uniform on [-1, 1)."""
    return (2.0 * uniform(seed, rows * cols) - 1.0).reshape(rows, cols)


def complex_normal(seed: int, n: int) -> np.ndarray:
    """n complex128 values, real and imaginary parts independent N(0, 1/2)."""
    u = uniform(seed, 2 * n)
    r = np.sqrt(-np.log1p(-u[0::2]))
    th = 2.0 * np.pi * u[1::2]
    return r * np.cos(th) + 1j * (r * np.sin(th))


def field(seed: int, shape, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """float32 array of the given shape, uniform on [lo, hi)."""
    n = int(np.prod(shape))
    return (lo + (hi - lo) * uniform(seed, n)).astype(np.float32).reshape(shape)


def log_uniform_int(seed: int, n: int, lo: int, hi: int) -> np.ndarray:
    """n integers log-uniform on [lo, hi]."""
    u = uniform(seed, n)
    v = np.exp(np.log(lo) + u * (np.log(hi + 1) - np.log(lo)))
    return np.clip(np.floor(v).astype(np.int64), lo, hi)
