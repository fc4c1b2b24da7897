"""GPU parity of the FP64-equivalent matrix product (precision pattern
OO_PREC_FP64EQ: Ozaki-type BF16 digit slices, exact FP32 K-block sums,
float-float term sum) against the FP64 Dot2 oracle.

Gate: max_ij |C - C*|_ij / (|A| |B|)_ij <= 1e-12 (the FP64-equivalent
tolerance for the matrix-product block; the mode's own bound is ~2.3e-13
for rows / columns of comparable magnitude).  Shapes cover the three
regimes of the split: k <= 256 (8-bit digits, 21 products), 256 < k <= 1024
(7-bit digits, 28 products, one K-block) and k > 1024 (several exact
K-blocks), with ragged m, n and k tails."""
import numpy as np
import pytest

import oracle
from paper_2011_03602_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64EQ_TOL = 1e-12


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


def err_metric(C, ref, A, B):
    return np.max(np.abs(C - ref) / np.maximum(np.abs(A) @ np.abs(B), 1e-300))


def gemm(oo_mod, ctx, A, B):
    return oo_mod.oo_gemm_f64(ctx, A, B, prec=oo_mod.OO_PREC_FP64EQ)


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (5, 7, 3), (128, 256, 64), (130, 300, 70), (129, 257, 1100)])
def test_small_integers_exact(oo_mod, ctx, m, n, k):
    rng = np.random.default_rng(m + 3 * n + k)
    A = rng.integers(-100, 101, (m, k)).astype(np.float64)
    B = rng.integers(-100, 101, (k, n)).astype(np.float64)
    assert np.array_equal(gemm(oo_mod, ctx, A, B), A @ B)


@pytest.mark.parametrize("m,n,k", [(256, 256, 256), (77, 513, 129), (300, 200, 1000), (129, 131, 1024),
                                   (130, 260, 1100), (200, 72, 2100), (1024, 1024, 1024)])
def test_uniform_against_oracle(oo_mod, ctx, m, n, k):
    A = synth.gemm_matrix(31 + m, m, k)
    B = synth.gemm_matrix(32 + n, k, n)
    C = gemm(oo_mod, ctx, A, B)
    e = err_metric(C, oracle.gemm(A, B), A, B)
    assert e <= FP64EQ_TOL, e


def test_row_and_column_scales(oo_mod, ctx):
    """Per-row / per-column powers of two are exact: extreme ranges keep the bound."""
    m, n, k = 200, 300, 700
    A = synth.gemm_matrix(3, m, k) * np.logspace(-150, 150, m)[:, None]
    B = synth.gemm_matrix(4, k, n) * np.logspace(120, -120, n)[None, :]
    C = gemm(oo_mod, ctx, A, B)
    assert err_metric(C, oracle.gemm(A, B), A, B) <= FP64EQ_TOL


def test_zero_and_subnormal_rows(oo_mod, ctx):
    m, n, k = 40, 50, 300
    A = synth.gemm_matrix(7, m, k)
    B = synth.gemm_matrix(8, k, n)
    A[3] = 0.0
    B[:, 5] = 0.0
    A[7] = A[7] * 1e-310  # every entry subnormal
    C = gemm(oo_mod, ctx, A, B)
    ref = oracle.gemm(A, B)
    assert np.all(C[3] == 0.0) and np.all(C[:, 5] == 0.0)
    mask = np.ones_like(C, bool)
    mask[3] = False
    mask[:, 5] = False
    e = np.abs(C - ref)[mask] / np.maximum((np.abs(A) @ np.abs(B))[mask], 1e-320)
    # the subnormal row's products are themselves subnormal (absolute spacing 2^-1074)
    assert np.max(e) <= 1e-11


def test_graded_rows_within_general_bound(oo_mod, ctx):
    """Entries of one row spanning many binades: the error stays within the
    general bound 4 (L+2) 2^(-beta (L-1)) k max|a_i.| max|b_.j|."""
    m, n, k = 64, 96, 1500
    rng = np.random.default_rng(5)
    A = synth.gemm_matrix(9, m, k) * 2.0 ** rng.integers(-40, 1, (m, k))
    B = synth.gemm_matrix(10, k, n) * 2.0 ** rng.integers(-40, 1, (k, n))
    C = gemm(oo_mod, ctx, A, B)
    ref = oracle.gemm(A, B)
    prods, beta, L, kb = oo_mod.oo_gemm_plan(oo_mod.OO_PREC_FP64EQ, k)
    bound = 4 * (L + 2) * 2.0 ** (-beta * (L - 1)) * k
    scale = np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=0)[None, :]
    assert np.max(np.abs(C - ref) / scale) <= bound


def test_device_api_leading_dimensions_and_determinism(oo_mod, ctx):
    m, n, k = 150, 260, 1090
    A = synth.gemm_matrix(5, m, k)
    B = synth.gemm_matrix(6, k, n)
    lda, ldb, ldc = k + 3, n + 5, n + 7
    dA = torch.zeros(m * lda, dtype=torch.float64, device="cuda")
    dB = torch.zeros(k * ldb, dtype=torch.float64, device="cuda")
    dC = torch.full((m * ldc,), -1.0, dtype=torch.float64, device="cuda")
    dA.view(m, lda)[:, :k] = torch.from_numpy(A).cuda()
    dB.view(k, ldb)[:, :n] = torch.from_numpy(B).cuda()
    oo_mod.oo_gemm_f64_dev(ctx, m, n, k, dA, lda, dB, ldb, dC, ldc, prec=oo_mod.OO_PREC_FP64EQ)
    oo_mod.oo_gemm_check(ctx, m, n, k)
    Cf = dC.view(m, ldc).cpu().numpy()
    assert np.all(Cf[:, n:] == -1.0)
    assert err_metric(Cf[:, :n], oracle.gemm(A, B), A, B) <= FP64EQ_TOL
    host = gemm(oo_mod, ctx, A, B)
    assert np.array_equal(host, Cf[:, :n])


def test_full_size_sampled_rows(oo_mod, ctx):
    """n = 4096, the largest size in the workload: rows sampled against the oracle."""
    n = 4096
    A = synth.gemm_matrix(21, n, n)
    B = synth.gemm_matrix(22, n, n)
    C = gemm(oo_mod, ctx, A, B)
    rows = np.random.default_rng(0).choice(n, 6, replace=False)
    for r in rows:
        ref = oracle.gemm(A[r:r + 1], B)
        e = np.max(np.abs(C[r] - ref[0]) / (np.abs(A[r]) @ np.abs(B)))
        assert e <= FP64EQ_TOL, (r, e)


def test_long_inner_dimension(oo_mod, ctx):
    """k = 20000: twenty exact K-blocks summed in float-float."""
    m, n, k = 130, 70, 20000
    A = synth.gemm_matrix(51, m, k)
    B = synth.gemm_matrix(52, k, n)
    C = gemm(oo_mod, ctx, A, B)
    e = err_metric(C, oracle.gemm(A, B), A, B)
    assert e <= FP64EQ_TOL, e
