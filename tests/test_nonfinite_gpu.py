"""Non-finite inputs of the function blocks, against the oracle.

The library's rule, which is what the FP64 oracle gives:
  - GEMM (both precision patterns, single calls and batches): an entry of C
    whose row of A or column of B holds a NaN or an infinity is NaN (the
    compensated FP64 dot product meets an undefined product error there);
    every other entry is computed as usual, to the pattern's tolerance;
  - FFT: a transform of length n >= 2 with a NaN or an infinity among its
    inputs is NaN in every output component; n = 1 is the identity.  The
    DFT definition summed term by term (oracle.dft) is non-finite in every
    component there too: a NaN input makes every term's real and imaginary
    parts NaN, an infinite one gives +-Inf or NaN depending on whether the
    twiddle's component is exactly zero.  (The radix-2 oracle keeps some
    components finite: its last butterflies add the even half without a
    twiddle product.)"""
import numpy as np
import pytest

import oracle
from paper_2011_03602_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-4, 2: 1e-12}  # split-BF16 (reported bound), FP64-equivalent


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


def poisoned(m, n, k, seed):
    A = synth.gemm_matrix(seed, m, k)
    B = synth.gemm_matrix(seed + 1, k, n)
    A[min(3, m - 1), min(5, k - 1)] = np.nan
    A[m - 1, 0] = np.inf
    B[min(7, k - 1), n - 1] = -np.inf
    if n > 2 and k > 2:
        B[2, 2] = np.inf
    return A, B


def check_gemm(C, A, B, prec):
    ref = oracle.gemm(A, B)
    bad = ~np.isfinite(A).all(1)[:, None] | ~np.isfinite(B).all(0)[None, :]
    assert np.array_equal(np.isnan(ref), bad)          # the oracle's own pattern
    assert np.array_equal(np.isnan(C), bad)
    Af, Bf = np.where(np.isfinite(A), A, 0.0), np.where(np.isfinite(B), B, 0.0)
    scale = np.maximum(np.abs(Af) @ np.abs(Bf), 1e-300)
    e = np.max(np.abs(C - ref)[~bad] / scale[~bad]) if (~bad).any() else 0.0
    assert e <= TOL[prec], e


# even and odd leading dimensions take different split kernels
@pytest.mark.parametrize("m,n,k", [(130, 70, 300), (33, 17, 9), (256, 256, 512)])
@pytest.mark.parametrize("prec", [0, 2])
def test_gemm_nonfinite_rows_and_columns_are_nan(oo_mod, ctx, m, n, k, prec):
    A, B = poisoned(m, n, k, 40 + m)
    C = oo_mod.oo_gemm_f64(ctx, A, B, prec=prec)
    check_gemm(C, A, B, prec)
    # the same context then multiplies clean inputs as before
    A2, B2 = synth.gemm_matrix(7, m, k), synth.gemm_matrix(8, k, n)
    check_gemm(oo_mod.oo_gemm_f64(ctx, A2, B2, prec=prec), A2, B2, prec)


@pytest.mark.parametrize("logn", [0, 1, 3, 12, 13, 16])
@pytest.mark.parametrize("val", [np.nan, np.inf, -np.inf])
@pytest.mark.parametrize("direction", [-1, 1])
def test_fft_nonfinite_input(oo_mod, ctx, logn, val, direction):
    n = 1 << logn
    x = synth.complex_normal(60 + logn, n)
    x.view(np.float64)[(2 * (n // 3) + 1) % (2 * n)] = val
    got = oo_mod.oo_fft_c128(ctx, x, direction)
    if n == 1:
        assert np.array_equal(got, x, equal_nan=True)
        # the radix-2 oracle returns a length-1 input unchanged; the summed
        # definition would multiply it by the complex 1 + 0i
        assert np.array_equal(oracle.fft(x, direction), x, equal_nan=True)
    else:
        assert np.isnan(got.view(np.float64)).all()
        if n <= 4096:
            ref = oracle.dft(x, direction).view(np.float64)
            assert not np.isfinite(ref).any()
            if np.isnan(val):
                assert np.isnan(ref).all()
    # a clean transform on the same context is unaffected
    y = synth.complex_normal(61 + logn, n)
    g2, r2 = oo_mod.oo_fft_c128(ctx, y, direction), oracle.fft(y, direction)
    assert np.linalg.norm(g2 - r2) <= 1e-12 * max(np.linalg.norm(r2), 1e-300)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_batch_nonfinite(oo_mod, ctx, mode):
    """A batch mixing clean and poisoned GEMMs (both patterns) and FFTs."""
    reqs, host = [], []
    for i, (m, n, k, prec, bad) in enumerate([(40, 33, 70, 0, True), (40, 33, 70, 0, False),
                                              (129, 65, 300, 2, True), (17, 200, 31, 2, False),
                                              (64, 64, 64, 2, True)]):
        if bad:
            A, B = poisoned(m, n, k, 90 + i)
        else:
            A, B = synth.gemm_matrix(90 + i, m, k), synth.gemm_matrix(91 + i, k, n)
        reqs.append(dict(kind="gemm", prec=prec, m=m, n=n, k=k, A=torch.from_numpy(A).cuda(),
                         B=torch.from_numpy(B).cuda(), C=torch.empty((m, n), dtype=torch.float64, device="cuda")))
        host.append((A, B, prec))
    for i, (logn, val) in enumerate([(8, np.nan), (10, None), (13, np.inf), (16, -np.inf), (0, np.nan)]):
        x = synth.complex_normal(120 + i, 1 << logn)
        if val is not None:
            x.view(np.float64)[5 % (2 << logn)] = val
        reqs.append(dict(kind="fft", n=1 << logn, dir=-1, x=torch.from_numpy(x.view(np.float64).copy()).cuda(),
                         X=torch.empty(2 << logn, dtype=torch.float64, device="cuda")))
        host.append((x, None, None))
    torch.cuda.synchronize()
    b = oo_mod.oo_batch_create(ctx, reqs)
    try:
        oo_mod.oo_batch_run(ctx, b, mode)
        oo_mod.oo_batch_check(ctx, b)
    finally:
        oo_mod.oo_batch_destroy(b)
    for r, (a0, a1, prec) in zip(reqs, host):
        if r["kind"] == "gemm":
            check_gemm(r["C"].cpu().numpy(), a0, a1, prec)
        else:
            got = r["X"].cpu().numpy().view(np.complex128)
            if a0.size == 1:
                assert np.array_equal(got, a0, equal_nan=True)
            elif np.isfinite(a0.view(np.float64)).all():
                ref = oracle.fft(a0, -1)
                assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
            else:
                assert np.isnan(got.view(np.float64)).all()
