"""The C-ABI library loads, exports every entry point include/*.h declares,
and its host-only logic matches the oracle (no GPU calls here)."""
import glob
import os
import re

import numpy as np
import pytest

from paper_2011_03602_gb300 import build as pkg_build
from paper_2011_03602_gb300 import oo

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg_build.build()


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(oo_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported():
    names = declared_symbols()
    assert "oo_run_pattern" in names and "oo_create" in names
    L = oo.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings():
    assert oo.oo_status_str(0) == "ok"
    assert oo.oo_status_str(oo.OO_ETIMEOUT) == "timed out"


def test_lookup_block_by_language():
    assert oo.oo_lookup_block("cblas_dgemm", oo.OO_LANG_C) == oo.OO_BLOCK_GEMM
    assert oo.oo_lookup_block("numpy.fft.fft", oo.OO_LANG_PYTHON) == oo.OO_BLOCK_FFT
    assert oo.oo_lookup_block("org.jtransforms.fft.DoubleFFT_1D.complexForward",
                              oo.OO_LANG_JAVA) == oo.OO_BLOCK_FFT
    with pytest.raises(oo.OOError) as e:
        oo.oo_lookup_block("cblas_dgemm", oo.OO_LANG_JAVA)
    assert e.value.status == oo.OO_ENOTFOUND


def test_lookup_accepts_spelling_variants():
    assert oo.oo_lookup_block("np.dot", oo.OO_LANG_PYTHON) == oo.OO_BLOCK_GEMM
    assert oo.oo_lookup_block("np.fft.fft", oo.OO_LANG_PYTHON) == oo.OO_BLOCK_FFT
    assert oo.oo_lookup_block("sp.fft.fft", oo.OO_LANG_PYTHON) == oo.OO_BLOCK_FFT
    assert oo.oo_lookup_block("la.blas.dgemm", oo.OO_LANG_PYTHON) == oo.OO_BLOCK_GEMM
    assert oo.oo_lookup_block("DGEMM", oo.OO_LANG_C) == oo.OO_BLOCK_GEMM
    assert oo.oo_lookup_block("DoubleFFT_1D.complexForward", oo.OO_LANG_JAVA) == oo.OO_BLOCK_FFT
    assert oo.oo_lookup_block("CommonOps_DDRM.mult", oo.OO_LANG_JAVA) == oo.OO_BLOCK_GEMM
    for name, lang in (("np.linalg.svd", oo.OO_LANG_PYTHON), ("FFT_1D.complexForward", oo.OO_LANG_JAVA),
                       ("multiply", oo.OO_LANG_JAVA), ("dgemm", oo.OO_LANG_PYTHON)):
        with pytest.raises(oo.OOError) as e:
            oo.oo_lookup_block(name, lang)
        assert e.value.status == oo.OO_ENOTFOUND


def test_host_only_context_rejects_gpu_work():
    ctx = oo.oo_create(-1)
    try:
        assert oo.oo_load_jacobi_nests(ctx, 5, 5, 5, 2) == 6
        with pytest.raises(oo.OOError) as e:
            oo.oo_run_pattern(ctx, 63, 1, oo.jacobi(5, 5, 5, 2))
        assert e.value.status == oo.OO_ESTATE
    finally:
        oo.oo_destroy(ctx)


def test_bad_tables_are_rejected():
    ctx = oo.oo_create(-1)
    try:
        with pytest.raises(oo.OOError) as e:
            oo.oo_load_nests(ctx, [dict(level=2, parallelisable=1, reads=0, writes=1, partial=0)],
                             [8], 1)
        assert e.value.status == oo.OO_EINVAL
        with pytest.raises(oo.OOError):
            oo.oo_load_nests(ctx, [dict(level=0, parallelisable=1, reads=0, writes=1, partial=2)],
                             [8, 8], 1)
        with pytest.raises(oo.OOError) as e:
            oo.oo_transfer_plan(ctx, 1, 1, 1)   # no table loaded yet
        assert e.value.status == oo.OO_ESTATE
    finally:
        oo.oo_destroy(ctx)


def test_missing_gpu_fails_loudly_or_creates():
    # on a machine without a GPU the context cannot be created on device 0
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(oo.OOError) as e:
        oo.oo_create(0)
    assert e.value.status in (oo.OO_ECUDA, oo.OO_EINVAL)


def test_gemm_plan_follows_the_exactness_rule():
    """FP64-equivalent split: K-block kb, digit width beta and the number of
    products one FP32 accumulator sums keep every accumulator exact,
    per_acc * kb * (2^beta - 1)^2 < 2^24, and the level bound L is the
    smallest with 4 (L + 2) 2^(-beta (L - 1)) <= 2^-42."""
    assert oo.oo_gemm_plan(oo.OO_PREC_SPLIT3_BF16, 4096) == (3, 0, 0, 0)
    for k in (1, 63, 64, 65, 128, 129, 200, 256, 257, 512, 513, 1000, 1024, 1025, 4096, 10000):
        prods, beta, L, kb = oo.oo_gemm_plan(oo.OO_PREC_FP64EQ, k)
        scheme, per_acc = oo.oo_gemm_scheme(k)
        assert kb % 64 == 0 and kb <= 1024
        assert per_acc == (1 if scheme == oo.OO_EQ_PAIRS else L - 1)
        assert per_acc * kb * (2 ** beta - 1) ** 2 < 2 ** 24 and beta <= 8
        assert 4 * (L + 2) * 2.0 ** (-beta * (L - 1)) <= 2.0 ** -42
        assert 4 * (L + 1) * 2.0 ** (-beta * (L - 2)) > 2.0 ** -42
        assert prods == L * (L - 1) // 2
    # levels with 7-bit digits up to k = 128, 6-bit up to 512, pairs beyond
    assert oo.oo_gemm_scheme(128) == (oo.OO_EQ_LEVELS, 7)
    assert oo.oo_gemm_plan(oo.OO_PREC_FP64EQ, 100) == (28, 7, 8, 128)
    assert oo.oo_gemm_scheme(512) == (oo.OO_EQ_LEVELS, 8)
    assert oo.oo_gemm_plan(oo.OO_PREC_FP64EQ, 256) == (36, 6, 9, 256)
    assert oo.oo_gemm_scheme(513) == (oo.OO_EQ_PAIRS, 1)
    assert oo.oo_gemm_plan(oo.OO_PREC_FP64EQ, 4096) == (28, 7, 8, 1024)
    assert oo.oo_gemm_plan(oo.OO_PREC_SPLIT3_TF32, 64) == (3, 0, 0, 0)
    with pytest.raises(oo.OOError):
        oo.oo_gemm_plan(3, 64)


def test_gemm_tile_table_host_only():
    """The tile-width table of a context: built-in widths are 32, 64 or 128;
    set / get round trip; other widths refused."""
    ctx = oo.oo_create(-1)
    try:
        w = oo.oo_get_gemm_tiles(ctx)
        assert w.shape == (oo.OO_TILE_NBUCKETS, oo.OO_TILE_KBUCKETS)
        assert set(np.unique(w)) <= {32, 64, 128}
        new = np.full_like(w, 64)
        new[0, :] = 32
        oo.oo_set_gemm_tiles(ctx, new)
        assert np.array_equal(oo.oo_get_gemm_tiles(ctx), new)
        bad = new.copy()
        bad[2, 3] = 96
        with pytest.raises(oo.OOError) as e:
            oo.oo_set_gemm_tiles(ctx, bad)
        assert e.value.status == oo.OO_EINVAL
        assert np.array_equal(oo.oo_get_gemm_tiles(ctx), new)
    finally:
        oo.oo_destroy(ctx)


def test_generic_program_needs_a_device_and_a_table():
    ctx = oo.oo_create(-1)
    try:
        body = lambda nest, on_gpu, it, stream: None  # noqa: E731
        with pytest.raises(oo.OOError) as e:
            oo.oo_run_program(ctx, 0, 1, 1, body, [None], [None])
        assert e.value.status == oo.OO_ESTATE
    finally:
        oo.oo_destroy(ctx)
    assert oo.oo_status_str(oo.OO_EUSER) == "nest function failed"


def test_host_only_context_rejects_tuning_and_bad_injections():
    """A host-only context (device -1) refuses the stencil tuner with
    OO_ESTATE instead of touching CUDA; injection arguments are checked on
    any context."""
    ctx = oo.oo_create(-1)
    try:
        with pytest.raises(oo.OOError) as e:
            oo.oo_tune_stencil(ctx, 9, 9, 9)
        assert e.value.status == oo.OO_ESTATE
        with pytest.raises(oo.OOError) as e:
            oo.oo_inject_wait_timeout(ctx, 9)
        assert e.value.status == oo.OO_EINVAL
        oo.oo_inject_wait_timeout(ctx, oo.OO_INJECT_NONE)
    finally:
        oo.oo_destroy(ctx)


def test_context_options_host_only():
    """Per-context options replace process-wide switches: set, read back,
    bad options and values refused; the library reads no environment."""
    ctx = oo.oo_create(-1)
    try:
        assert oo.oo_get_option(ctx, oo.OO_OPT_JACOBI_FUSED) == -1
        assert oo.oo_get_option(ctx, oo.OO_OPT_STENCIL_VARIANT) == -1
        oo.oo_set_option(ctx, oo.OO_OPT_JACOBI_FUSED, 0)
        oo.oo_set_option(ctx, oo.OO_OPT_STENCIL_VARIANT, oo.OO_STENCIL_VARIANTS - 1)
        assert oo.oo_get_option(ctx, oo.OO_OPT_JACOBI_FUSED) == 0
        assert oo.oo_get_option(ctx, oo.OO_OPT_STENCIL_VARIANT) == oo.OO_STENCIL_VARIANTS - 1
        assert oo.oo_get_option(ctx, oo.OO_OPT_GEMM_PAIR) == 1
        for v in (0, 160, 192, 224, 256, 1):
            oo.oo_set_option(ctx, oo.OO_OPT_GEMM_PAIR, v)
            assert oo.oo_get_option(ctx, oo.OO_OPT_GEMM_PAIR) == v
        for opt, val in ((oo.OO_OPT_JACOBI_FUSED, 2), (oo.OO_OPT_STENCIL_VARIANT, oo.OO_STENCIL_VARIANTS),
                         (oo.OO_OPT_STENCIL_VARIANT, -2), (oo.OO_OPT_GEMM_PAIR, 2), (oo.OO_OPT_GEMM_PAIR, -1),
                         (oo.OO_OPT_GEMM_PAIR, 128), (oo.OO_OPT_GEMM_PAIR, 200),
                         (99, 0)):
            with pytest.raises(oo.OOError) as e:
                oo.oo_set_option(ctx, opt, val)
            assert e.value.status == oo.OO_EINVAL
    finally:
        oo.oo_destroy(ctx)
    csrc = os.path.join(ROOT, "paper_2011_03602_gb300", "csrc")
    for f in os.listdir(csrc):
        assert "getenv" not in open(os.path.join(csrc, f), errors="replace").read(), f


def test_serve_requests_hold_their_arrays_until_waited():
    """The Python binding keeps a request's arrays alive from oo_submit until
    oo_wait returns: the library reads inputs and writes outputs in between
    (the device-resident loop copies them when the request is admitted and
    when it completes), so arrays the caller dropped must not be freed."""
    from paper_2011_03602_gb300 import oo
    A, B, C = np.ones((4, 3)), np.ones((3, 5)), np.empty((4, 5))
    r = oo.serve_request("gemm", A=A, B=B, C=C)
    assert all(any(x is y for y in r._arrays) for x in (A, B, C))
    p, res = np.empty(27, np.float32), np.empty(2)
    r = oo.serve_request("jacobi", I=3, J=3, K=3, iters=2, p=p, res=res)
    assert all(any(x is y for y in r._arrays) for x in (p, res))
    oo._hold(7, r, 11)
    assert oo._in_flight[(7, 11)] == r._arrays
    with oo._in_flight_lock:
        del oo._in_flight[(7, 11)]


def test_resident_loop_launches_its_workers_only_at_start():
    """The device-resident serving loop launches no kernel per request: the
    only launch sites in its source are the two workers', inside
    oo_serve_start_resident, and the scheduler, admission, I/O and wait
    code issue copies, events and stream queries only."""
    src = open(os.path.join(os.path.dirname(oo.__file__), "csrc", "serve_resident.cu")).read()
    start = src.index("oo_status oo_serve_start_resident(")
    end = src.index("\n}\n", start)
    launches = [m.start() for m in re.finditer(r"<<<", src)]
    tiles = [m.start() for m in re.finditer(r"\blaunch_resident_tiles\(", src)]
    assert len(launches) == 1 and start < launches[0] < end
    calls = [t for t in tiles if not src[max(0, t - 5):t].startswith("void ")]
    assert len(calls) == 1 and start < calls[0] < end
    assert "cudaLaunch" not in src and "cudaGraphLaunch" not in src
