"""GPU parity of the FFT function block against the FP64 oracle FFT.

Gate: relative L2 error ||X - X*|| / ||X*|| <= 1e-12 (complex128 block)."""
import numpy as np
import pytest

import oracle
from paper_2011_03602_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


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


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("logn", [0, 1, 2, 3, 4, 5, 7, 10, 11, 12, 13, 14, 15, 17, 20, 22])
@pytest.mark.parametrize("direction", [-1, 1])
def test_fft_matches_oracle(oo_mod, ctx, logn, direction):
    n = 1 << logn
    x = synth.complex_normal(1000 + logn, n)
    got = oo_mod.oo_fft_c128(ctx, x, direction)
    ref = oracle.fft(x, direction)
    assert rel(got, ref) <= TOL, rel(got, ref)


def test_closed_forms(oo_mod, ctx):
    n = 1 << 14
    d = np.zeros(n, complex)
    d[0] = 1
    np.testing.assert_allclose(oo_mod.oo_fft_c128(ctx, d), np.ones(n), atol=1e-15)
    k = np.arange(n)
    m = 1234
    tone = np.exp(2j * np.pi * m * k / n)
    X = oo_mod.oo_fft_c128(ctx, tone)
    expect = np.zeros(n, complex)
    expect[m] = n
    assert np.max(np.abs(X - expect)) <= 1e-12 * n


@pytest.mark.parametrize("scale", [1e-200, 1e-30, 1e30, 1e200])
def test_any_finite_magnitude(oo_mod, ctx, scale):
    n = 1 << 13
    x = synth.complex_normal(7, n) * scale
    got = oo_mod.oo_fft_c128(ctx, x)
    ref = oracle.fft(x)
    # compare in units of the scale: squares of 1e+-200 values over/underflow
    assert np.all(np.isfinite(got))
    assert rel(got / scale, ref / scale) <= TOL


def test_round_trip_and_parseval(oo_mod, ctx):
    n = 1 << 18
    x = synth.complex_normal(3, n)
    X = oo_mod.oo_fft_c128(ctx, x, -1)
    assert np.sum(np.abs(X) ** 2) == pytest.approx(n * np.sum(np.abs(x) ** 2), rel=1e-12)
    back = oo_mod.oo_fft_c128(ctx, X, 1)
    assert rel(back, x) <= TOL


@pytest.mark.parametrize("logn,batch", [(3, 5), (10, 7), (12, 3), (14, 4), (16, 2)])
def test_batched_device_in_place(oo_mod, ctx, logn, batch):
    n = 1 << logn
    xs = [synth.complex_normal(50 + b, n) * (10.0 ** (b - 2)) for b in range(batch)]
    host = np.concatenate(xs)
    d = torch.from_numpy(host.view(np.float64).copy()).cuda()
    oo_mod.oo_fft_c128_dev(ctx, n, batch, -1, d, d)
    oo_mod.oo_sync(ctx)
    got = d.cpu().numpy().view(np.complex128)
    for b in range(batch):
        assert rel(got[b * n:(b + 1) * n], oracle.fft(xs[b])) <= TOL, b


def test_bad_lengths(oo_mod, ctx):
    with pytest.raises(oo_mod.OOError):
        oo_mod.oo_fft_c128(ctx, np.ones(12, complex))
    with pytest.raises(oo_mod.OOError):
        oo_mod.oo_fft_c128(ctx, np.ones(8, complex), 0)


@pytest.mark.parametrize("logn", [23, 24])
def test_maximum_lengths(oo_mod, ctx, logn):
    """The two largest lengths (four-step with 2^12-point passes at 2^24)."""
    n = 1 << logn
    x = synth.complex_normal(3000 + logn, n)
    got = oo_mod.oo_fft_c128(ctx, x, -1)
    ref = oracle.fft(x, -1)
    assert rel(got, ref) <= TOL, rel(got, ref)
