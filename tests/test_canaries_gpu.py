"""Canaries around device outputs (the sanitizer stand-in for this pool: no
compute-sanitizer run): every device entry point writes exactly its output
elements and nothing next to them.  Outputs are views into larger buffers
filled with a sentinel; after the call the sentinel must be intact before
and after each output, and the outputs must equal the host entry points'."""
import numpy as np
import pytest

from paper_2011_03602_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GUARD = 1024  # elements of sentinel on each side
SENT = -12345.0


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


def guarded(count, dtype=torch.float64):
    buf = torch.full((count + 2 * GUARD,), SENT, dtype=dtype, device="cuda")
    return buf, buf[GUARD:GUARD + count]


def guards_intact(buf):
    h = buf.cpu().numpy()
    return np.all(h[:GUARD] == SENT) and np.all(h[-GUARD:] == SENT)


@pytest.mark.parametrize("n,batch", [(1, 3), (8, 5), (1024, 4), (4096, 2), (1 << 13, 2), (1 << 16, 1)])
def test_fft_dev_writes_only_its_output(oo_mod, ctx, n, batch):
    x = synth.complex_normal(30 + n, n * batch)
    din = torch.from_numpy(x.view(np.float64).copy()).cuda()
    buf, dout = guarded(2 * n * batch)
    torch.cuda.synchronize()
    oo_mod.oo_fft_c128_dev(ctx, n, batch, -1, din, dout)
    oo_mod.oo_sync(ctx)
    assert guards_intact(buf)
    y = dout.cpu().numpy().view(np.complex128).reshape(batch, n)
    for b in range(batch):
        assert np.array_equal(y[b], oo_mod.oo_fft_c128(ctx, x[b * n:(b + 1) * n], -1))


def test_batch_outputs_write_only_their_elements(oo_mod, ctx):
    """Uneven GEMMs and FFTs whose outputs sit back to back in one buffer with
    sentinel gaps between them."""
    rng = np.random.default_rng(4)
    reqs, spans, host = [], [], []
    total = GUARD
    specs = [("gemm", int(m), int(nn), int(k)) for m, nn, k in rng.integers(16, 200, (10, 3))] + \
            [("fft", 1 << int(e)) for e in rng.integers(8, 14, 6)]
    for sp in specs:
        size = sp[1] * sp[2] if sp[0] == "gemm" else 2 * sp[1]
        spans.append((total, size))
        total += size + GUARD
    buf = torch.full((total,), SENT, dtype=torch.float64, device="cuda")
    for i, sp in enumerate(specs):
        off, size = spans[i]
        if sp[0] == "gemm":
            _, m, nn, k = sp
            A, B = synth.gemm_matrix(100 + i, m, k), synth.gemm_matrix(200 + i, k, nn)
            host.append(("gemm", A, B))
            reqs.append({"kind": "gemm", "m": m, "n": nn, "k": k, "A": torch.from_numpy(A).cuda(),
                         "B": torch.from_numpy(B).cuda(), "C": buf[off:off + size], "prec": oo_mod.OO_PREC_FP64EQ})
        else:
            n = sp[1]
            x = synth.complex_normal(300 + i, n)
            host.append(("fft", x))
            reqs.append({"kind": "fft", "n": n, "x": torch.from_numpy(x.view(np.float64).copy()).cuda(),
                         "X": buf[off:off + size], "dir": -1})
    torch.cuda.synchronize()
    b = oo_mod.oo_batch_create(ctx, reqs)
    try:
        for mode in (0, 1, 2):
            buf[GUARD:].fill_(SENT)  # outputs and gaps back to the sentinel
            for i, sp in enumerate(specs):
                off, size = spans[i]
                buf[off:off + size].fill_(0.0)
            torch.cuda.synchronize()
            oo_mod.oo_batch_run(ctx, b, mode)
            oo_mod.oo_batch_check(ctx, b)
            oo_mod.oo_sync(ctx)
            h = buf.cpu().numpy()
            prev = 0
            for i, sp in enumerate(specs):
                off, size = spans[i]
                assert np.all(h[prev:off] == SENT), (mode, i)
                prev = off + size
                if sp[0] == "gemm":
                    _, A, B = host[i]
                    want = oo_mod.oo_gemm_f64(ctx, A, B, prec=oo_mod.OO_PREC_FP64EQ)
                    assert np.array_equal(h[off:off + size].reshape(want.shape), want), (mode, i)
                else:
                    want = oo_mod.oo_fft_c128(ctx, host[i][1], -1)
                    assert np.array_equal(h[off:off + size].view(np.complex128), want), (mode, i)
            assert np.all(h[prev:] == SENT)
    finally:
        oo_mod.oo_batch_destroy(b)


def test_pattern_dev_outputs_write_only_their_elements(oo_mod, ctx):
    I, J, K, it = 17, 13, 29, 7
    pbuf, p = guarded(I * J * K, torch.float32)
    rbuf, r = guarded(it)
    torch.cuda.synchronize()
    oo_mod.oo_run_pattern_dev(ctx, 63, 1, oo_mod.jacobi(I, J, K, it), p, r)
    oo_mod.oo_sync(ctx)
    assert guards_intact(pbuf) and guards_intact(rbuf)
    p_h, r_h = np.empty(I * J * K, np.float32), np.empty(it)
    oo_mod.oo_run_pattern(ctx, 63, 1, oo_mod.jacobi(I, J, K, it), p_h, r_h)
    assert np.array_equal(p.cpu().numpy(), p_h)
    assert np.array_equal(r.cpu().numpy(), r_h)
