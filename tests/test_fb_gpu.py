"""Function-block trial (Sec. 4.2.1) and the whole trial order (Sec. 4.2)
measured on the GPU: known call sites of the three front-end languages are
candidates, unknown ones are not; every combination is timed; the result
gate makes a too-coarse precision pattern infinitely slow; the decision on
the measured table is the oracle's."""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def oo_mod():
    from paper_2011_03602_gb300 import build as pkg_build
    from paper_2011_03602_gb300 import oo
    pkg_build.build()
    return oo


@pytest.fixture(scope="module")
def ctx(oo_mod):
    c = oo_mod.oo_create(0)
    yield c
    oo_mod.oo_destroy(c)


def sites(oo):
    return [("cblas_dgemm", oo.OO_LANG_C, 2, 384, 320, 700),
            ("my_solver_step", oo.OO_LANG_C, 3, 64, 64, 64),        # not in the table
            ("numpy.fft.fft", oo.OO_LANG_PYTHON, 4, 0, 1 << 16, 0),
            ("org.jtransforms.fft.DoubleFFT_1D.complexForward", oo.OO_LANG_JAVA, 1, 0, 1 << 12, 0)]


def test_every_combination_measured(oo_mod, ctx):
    r = oo_mod.oo_fb_search(ctx, sites(oo_mod), prec=oo_mod.OO_PREC_FP64EQ, tol=1e-10, seed=5)
    assert list(r["block_ids"]) == [oo_mod.OO_BLOCK_GEMM, 0, oo_mod.OO_BLOCK_FFT, oo_mod.OO_BLOCK_FFT]
    ms = r["mask_ms"]
    for mask in range(16):
        if mask & 0b0010:
            assert math.isinf(ms[mask])       # unknown site cannot be offloaded
        else:
            assert 0.0 < ms[mask] < 60000.0   # measured, results within tol
    assert (r["best_mask"], r["best_ms"]) == oracle.fb_best(ms)
    assert not (r["best_mask"] & 0b0010)


def test_gate_rejects_coarse_precision(oo_mod, ctx):
    """split-BF16 GEMM (~1e-5) fails a 1e-10 check: every mask offloading the
    GEMM site is infinitely slow; FP64-equivalent passes it."""
    s = [("cblas_dgemm", oo_mod.OO_LANG_C, 1, 256, 256, 512),
         ("fftw_execute", oo_mod.OO_LANG_C, 1, 0, 1 << 14, 0)]
    r = oo_mod.oo_fb_search(ctx, s, prec=oo_mod.OO_PREC_SPLIT3_BF16, tol=1e-10, seed=9)
    ms = r["mask_ms"]
    assert math.isinf(ms[0b01]) and math.isinf(ms[0b11])
    assert np.isfinite(ms[0b00]) and np.isfinite(ms[0b10])
    assert not (r["best_mask"] & 1)
    r2 = oo_mod.oo_fb_search(ctx, s, prec=oo_mod.OO_PREC_SPLIT3_BF16, tol=1e-3, seed=9)
    assert np.all(np.isfinite(r2["mask_ms"]))
    r3 = oo_mod.oo_fb_search(ctx, s, prec=oo_mod.OO_PREC_FP64EQ, tol=1e-10, seed=9)
    assert np.all(np.isfinite(r3["mask_ms"]))


def test_trial_order_end_to_end(oo_mod, ctx):
    """Blocks first, then the loop GA on the Jacobi program's nests."""
    prob = oo_mod.jacobi(17, 19, 33, 5)
    r = oo_mod.oo_offload_search(ctx, sites(oo_mod)[:1], prob, 1, 6, 3, 0.9, 0.05, 7)
    assert r["best_mask"] in (0, 1) and math.isfinite(r["fb_ms"])
    assert 0 <= r["best_gene"] < 64 and math.isfinite(r["loop_ms"])
