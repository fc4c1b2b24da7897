"""The split-BF16 matrix product (Sec. 3.2.2 function block) on CTA pairs
(cta_group::2: 256 x W tiles, W = 160 .. 256 columns, each CTA of a pair
holding 128 rows of A and half of the tile's columns of B) against the
single-CTA kernel (128 x 128 tiles) and the FP64 Dot2 oracle.

Both kernels form the same three BF16 products per K step, in the same K
order, into one FP32 accumulator, and share the epilogue, so their outputs
must agree bit for bit; shapes cover one element, partial slabs in m (the
second CTA of a pair holding no valid row), partial column halves in n,
ragged k, every tile width and more units than resident clusters."""
import numpy as np
import pytest

import oracle
from paper_2011_03602_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPLIT3_TOL = 1e-4


@pytest.fixture(scope="module")
def oo_mod():
    from paper_2011_03602_gb300 import build as pkg_build
    from paper_2011_03602_gb300 import oo
    pkg_build.build()
    return oo


@pytest.fixture(scope="module")
def ctxs(oo_mod):
    pair, single = oo_mod.oo_create(0), oo_mod.oo_create(0)
    oo_mod.oo_set_option(single, oo_mod.OO_OPT_GEMM_PAIR, 0)
    assert oo_mod.oo_get_option(pair, oo_mod.OO_OPT_GEMM_PAIR) == 1
    yield pair, single
    oo_mod.oo_destroy(pair)
    oo_mod.oo_destroy(single)


def err_metric(C, ref, A, B):
    return np.max(np.abs(C - ref) / np.maximum(np.abs(A) @ np.abs(B), 1e-300))


def test_small_first(oo_mod, ctxs):
    """One 256 x 128 unit (one cluster), then one element."""
    pair, single = ctxs
    for m, n, k in ((256, 128, 64), (1, 1, 1)):
        A = synth.gemm_matrix(11, m, k)
        B = synth.gemm_matrix(12, k, n)
        Cp = oo_mod.oo_gemm_f64(pair, A, B)
        Cs = oo_mod.oo_gemm_f64(single, A, B)
        np.testing.assert_array_equal(Cp, Cs)
        assert err_metric(Cp, oracle.gemm(A, B), A, B) <= SPLIT3_TOL


@pytest.mark.parametrize("m,n,k", [(128, 128, 64), (129, 65, 70), (300, 200, 1000), (513, 257, 129),
                                   (77, 513, 129), (1024, 1024, 1024), (2048, 384, 512), (640, 1000, 3)])
def test_pair_equals_single_and_oracle(oo_mod, ctxs, m, n, k):
    pair, single = ctxs
    A = synth.gemm_matrix(100 + m, m, k)
    B = synth.gemm_matrix(200 + n, k, n)
    Cp = oo_mod.oo_gemm_f64(pair, A, B)
    Cs = oo_mod.oo_gemm_f64(single, A, B)
    np.testing.assert_array_equal(Cp, Cs)
    assert err_metric(Cp, oracle.gemm(A, B), A, B) <= SPLIT3_TOL


@pytest.mark.parametrize("width", [160, 192, 224, 256])
def test_every_tile_width(oo_mod, ctxs, width):
    pair, single = ctxs
    oo_mod.oo_set_option(pair, oo_mod.OO_OPT_GEMM_PAIR, width)
    try:
        for m, n, k in ((300, 200, 1000), (513, 700, 129), (1024, 1024, 256), (256, width, 64)):
            A = synth.gemm_matrix(300 + m, m, k)
            B = synth.gemm_matrix(400 + n, k, n)
            Cp = oo_mod.oo_gemm_f64(pair, A, B)
            Cs = oo_mod.oo_gemm_f64(single, A, B)
            np.testing.assert_array_equal(Cp, Cs)
    finally:
        oo_mod.oo_set_option(pair, oo_mod.OO_OPT_GEMM_PAIR, 1)


def test_full_size_pair_equals_single(oo_mod, ctxs):
    """n = m = k = 4096 (512 units over the resident clusters, several per
    cluster): every element equal; sampled rows against the oracle."""
    pair, single = ctxs
    n = 4096
    A = synth.gemm_matrix(7, n, n)
    B = synth.gemm_matrix(8, n, n)
    Cp = oo_mod.oo_gemm_f64(pair, A, B)
    Cs = oo_mod.oo_gemm_f64(single, A, B)
    np.testing.assert_array_equal(Cp, Cs)
    rows = [0, 255, 256, 1234, 4095]
    ref = oracle.gemm(A[rows], B)
    assert err_metric(Cp[rows], ref, A[rows], B) <= SPLIT3_TOL


def test_nonfinite_rows_and_columns(oo_mod, ctxs):
    """A NaN / infinity in A's row i or B's column j gives NaN in row i /
    column j and leaves the rest finite, in both kernels alike."""
    pair, single = ctxs
    m, n, k = 300, 200, 96
    A = synth.gemm_matrix(21, m, k)
    B = synth.gemm_matrix(22, k, n)
    A[257, 5] = np.inf
    B[7, 131] = np.nan
    Cp = oo_mod.oo_gemm_f64(pair, A, B)
    Cs = oo_mod.oo_gemm_f64(single, A, B)
    np.testing.assert_array_equal(np.isnan(Cp), np.isnan(Cs))
    assert np.isnan(Cp[257]).all() and np.isnan(Cp[:, 131]).all()
    mask = np.ones_like(Cp, dtype=bool)
    mask[257] = False
    mask[:, 131] = False
    assert np.isfinite(Cp[mask]).all()
    np.testing.assert_array_equal(Cp[mask], Cs[mask])


# ----------------------------------------------- FP64-equivalent pattern
FP64EQ_TOL = 1e-12


@pytest.mark.parametrize("m,n,k", [(256, 128, 600), (300, 200, 1000), (513, 257, 1500), (77, 640, 2048),
                                   (1024, 1024, 4096)])
def test_fp64eq_pair_equals_single_and_oracle(oo_mod, ctxs, m, n, k):
    """Inner dimensions above 512 take the pair scheme (two-product units on
    N = 256 MMAs, one-product units on N = 128): CTA pairs and single CTAs
    give the same bits, within the FP64-equivalent tolerance of the oracle."""
    pair, single = ctxs
    A = synth.gemm_matrix(500 + m, m, k)
    B = synth.gemm_matrix(600 + n, k, n)
    Cp = oo_mod.oo_gemm_f64(pair, A, B, prec=oo_mod.OO_PREC_FP64EQ)
    Cs = oo_mod.oo_gemm_f64(single, A, B, prec=oo_mod.OO_PREC_FP64EQ)
    np.testing.assert_array_equal(Cp, Cs)
    rows = sorted({0, m // 2, m - 1})
    ref = oracle.gemm(A[rows], B)
    assert err_metric(Cp[rows], ref, A[rows], B) <= FP64EQ_TOL


def test_fp64eq_full_size_pair_equals_single(oo_mod, ctxs):
    pair, single = ctxs
    n = 4096
    A = synth.gemm_matrix(9, n, n)
    B = synth.gemm_matrix(10, n, n)
    Cp = oo_mod.oo_gemm_f64(pair, A, B, prec=oo_mod.OO_PREC_FP64EQ)
    Cs = oo_mod.oo_gemm_f64(single, A, B, prec=oo_mod.OO_PREC_FP64EQ)
    np.testing.assert_array_equal(Cp, Cs)
