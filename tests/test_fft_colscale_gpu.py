"""Per-column scales of the FFT block.  Each column of a CTA -- a whole
transform, or one first-pass column of a four-step transform -- is split at
the power of two that brings its own largest component into [1/2, 1); the
second pass brings every column to its transform's scale.  These tests give
the columns magnitudes far apart (2^-600 .. 2^600) and check the result
against the FP64 oracle (relative L2 <= 1e-12) and that every path -- one
call per transform, a batched call, the grouped batch -- gives the same
bits."""
import numpy as np
import pytest

import oracle
from paper_2011_03602_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12
EXPS = [-600, -300, -45, -1, 0, 3, 40, 300, 600]


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
    """Relative L2 error, with both scaled by b's largest magnitude first (the
    squares of components near 2^600 overflow)."""
    s = np.max(np.abs(b))
    if s == 0:
        return float(np.linalg.norm(a))
    return np.linalg.norm((a - b) / s) / np.linalg.norm(b / s)


def four_step_cols(logn):
    """log2 of the first pass's column count (the number of columns N2)."""
    return logn - logn // 2


def column_scaled(seed, logn, shift=0):
    """Complex normal input whose four-step column n mod N2 is scaled by
    2^EXPS[(n mod N2 + shift) mod len]."""
    n = 1 << logn
    x = synth.complex_normal(seed, n)
    n2 = 1 << four_step_cols(logn)
    e = np.array([EXPS[(j + shift) % len(EXPS)] for j in range(n2)], dtype=float)
    return x * np.exp2(e)[np.arange(n) % n2]


@pytest.mark.parametrize("logn", [13, 14, 17, 20])
@pytest.mark.parametrize("direction", [-1, 1])
def test_columns_far_apart_against_oracle(oo_mod, ctx, logn, direction):
    x = column_scaled(70 + logn, logn)
    got = oo_mod.oo_fft_c128(ctx, x, direction)
    ref = oracle.fft(x, direction)
    assert rel(got, ref) <= TOL


def test_batched_call_equals_single_calls(oo_mod, ctx):
    """Whole transforms of very different magnitudes in one batched call
    (several per CTA) give what each gives alone; four-step ones likewise."""
    for logn, batch in ((6, 40), (10, 9), (12, 3), (14, 3)):
        n = 1 << logn
        xs = [synth.complex_normal(300 + 7 * b + logn, n) * 2.0 ** EXPS[b % len(EXPS)] for b in range(batch)]
        if logn > 12:
            xs = [column_scaled(400 + b, logn, shift=b) for b in range(batch)]
        alone = [oo_mod.oo_fft_c128(ctx, x, -1) for x in xs]
        din = torch.from_numpy(np.concatenate(xs).view(np.float64).copy()).cuda()
        dout = torch.full_like(din, np.nan)
        torch.cuda.synchronize()
        oo_mod.oo_fft_c128_dev(ctx, n, batch, -1, din, dout)
        oo_mod.oo_sync(ctx)  # the call ran on the context's stream
        got = dout.cpu().numpy().view(np.complex128).reshape(batch, n)
        for b in range(batch):
            np.testing.assert_array_equal(got[b], alone[b], err_msg="logn %d transform %d" % (logn, b))
            assert rel(got[b], oracle.fft(xs[b], -1)) <= TOL


def test_grouped_batch_equals_single_calls(oo_mod, ctx):
    oo = oo_mod
    reqs, alone = [], []
    for i, logn in enumerate((0, 3, 8, 11, 12, 13, 16)):
        n = 1 << logn
        x = column_scaled(500 + i, logn, shift=i) if logn > 12 else \
            synth.complex_normal(500 + i, n) * 2.0 ** EXPS[i % len(EXPS)]
        d = -1 if i % 2 == 0 else 1
        alone.append(oo.oo_fft_c128(ctx, x, d))
        reqs.append(dict(kind="fft", n=n, dir=d, x=torch.from_numpy(x.view(np.float64).copy()).cuda(),
                         X=torch.full((2 * n,), np.nan, dtype=torch.float64, device="cuda")))
    torch.cuda.synchronize()
    b = oo.oo_batch_create(ctx, reqs)
    try:
        for mode in (0, 1, 2):
            for r in reqs:
                r["X"].fill_(np.nan)
            torch.cuda.synchronize()
            oo.oo_batch_run(ctx, b, mode)
            oo.oo_batch_check(ctx, b)
            for i, r in enumerate(reqs):
                got = r["X"].cpu().numpy().view(np.complex128)
                np.testing.assert_array_equal(got, alone[i], err_msg="mode %d request %d" % (mode, i))
    finally:
        oo.oo_batch_destroy(b)
