"""GPU parity of the split-BF16 tensor-core matrix product (Sec. 3.2.2
function block) against the FP64 Dot2 oracle.

Error metric per element: |C - C*| / (|A| |B|)_ij; the split into two BF16
terms keeps ~16 bits, so the bound is 1e-4 (reported, not an FP64 claim).
Small-integer inputs are exact in every partial product and FP32 sum, so
there the result must be bit-exact."""
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
def ctx(oo_mod):
    c = oo_mod.oo_create(0)
    yield c
    oo_mod.oo_destroy(c)


def ints(seed, shape, lo=-8, hi=9):
    return np.random.default_rng(seed).integers(lo, hi, shape).astype(np.float64)


def err_metric(C, ref, A, B):
    return np.max(np.abs(C - ref) / np.maximum(np.abs(A) @ np.abs(B), 1e-300))


@pytest.mark.parametrize("m,n,k", [(128, 256, 64), (1, 1, 1), (5, 7, 3), (130, 300, 70),
                                   (256, 512, 256), (129, 257, 65)])
def test_small_integers_exact(oo_mod, ctx, m, n, k):
    A, B = ints(m + k, (m, k)), ints(n + 7 * k, (k, n))
    C = oo_mod.oo_gemm_f64(ctx, A, B)
    assert np.array_equal(C, A @ B)


@pytest.mark.parametrize("m,n,k", [(256, 256, 256), (300, 200, 1000), (1024, 1024, 1024), (77, 513, 129)])
def test_uniform_against_oracle(oo_mod, ctx, m, n, k):
    A = synth.gemm_matrix(11 + m, m, k)
    B = synth.gemm_matrix(12 + n, k, n)
    C = oo_mod.oo_gemm_f64(ctx, A, B)
    ref = oracle.gemm(A, B)
    e = err_metric(C, ref, A, B)
    assert e <= SPLIT3_TOL, e


def test_row_and_column_scales(oo_mod, ctx):
    m, n, k = 200, 300, 150
    A = synth.gemm_matrix(3, m, k) * np.logspace(-150, 150, m)[:, None]
    B = synth.gemm_matrix(4, k, n) * np.logspace(120, -120, n)[None, :]
    C = oo_mod.oo_gemm_f64(ctx, A, B)
    ref = oracle.gemm(A, B)
    assert err_metric(C, ref, A, B) <= SPLIT3_TOL


def test_device_api_with_leading_dimensions(oo_mod, ctx):
    m, n, k = 150, 260, 90
    A = synth.gemm_matrix(5, m, k)
    B = synth.gemm_matrix(6, k, n)
    lda, ldb, ldc = k + 3, n + 5, n + 7
    dA = torch.zeros(m * lda, dtype=torch.float64, device="cuda")
    dB = torch.zeros(k * ldb, dtype=torch.float64, device="cuda")
    dC = torch.full((m * ldc,), -1.0, dtype=torch.float64, device="cuda")
    dA.view(m, lda)[:, :k] = torch.from_numpy(A).cuda()
    dB.view(k, ldb)[:, :n] = torch.from_numpy(B).cuda()
    oo_mod.oo_gemm_f64_dev(ctx, m, n, k, dA, lda, dB, ldb, dC, ldc)
    oo_mod.oo_gemm_check(ctx, m, n, k)
    Cf = dC.view(m, ldc).cpu().numpy()
    assert np.all(Cf[:, n:] == -1.0)
    assert err_metric(Cf[:, :n], oracle.gemm(A, B), A, B) <= SPLIT3_TOL
    host = oo_mod.oo_gemm_f64(ctx, A, B)
    assert np.array_equal(host, Cf[:, :n])


def test_full_size_sampled_rows(oo_mod, ctx):
    """n = 4096, the largest size in the workload: rows sampled against the oracle."""
    n = 4096
    A = synth.gemm_matrix(21, n, n)
    B = synth.gemm_matrix(22, n, n)
    C = oo_mod.oo_gemm_f64(ctx, A, B)
    rows = np.random.default_rng(0).choice(n, 8, replace=False)
    for r in rows:
        ref = oracle.gemm(A[r:r + 1], B)
        e = np.max(np.abs(C[r] - ref[0]) / (np.abs(A[r]) @ np.abs(B)))
        assert e <= SPLIT3_TOL, (r, e)


def test_bad_arguments(oo_mod, ctx):
    with pytest.raises(oo_mod.OOError):
        oo_mod.oo_gemm_f64(ctx, np.ones((3, 4)), np.ones((4, 5)), prec=7)


def test_long_inner_dimension(oo_mod, ctx):
    m, n, k = 130, 70, 20000
    A = synth.gemm_matrix(53, m, k)
    B = synth.gemm_matrix(54, k, n)
    C = oo_mod.oo_gemm_f64(ctx, A, B)
    assert err_metric(C, oracle.gemm(A, B), A, B) <= SPLIT3_TOL
