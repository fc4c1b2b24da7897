"""Serving loop: requests from three client threads are admitted as slots and
device memory free up, overlap on the GPU, and every result is exactly the
one the same request gives alone (and within the oracle tolerance)."""
import threading

import numpy as np
import pytest

import oracle
from paper_2011_03602_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def oo_mod():
    from paper_2011_03602_gb300 import build as pkg_build
    from paper_2011_03602_gb300 import oo
    pkg_build.build()
    return oo


def make_mix(seed, count):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        u = rng.random()
        if u < 0.5:
            n = int(rng.integers(16, 300))
            A, B = synth.gemm_matrix(seed * 1000 + 2 * i, n, n + 3), synth.gemm_matrix(seed * 1000 + 2 * i + 1, n + 3, n)
            prec = 2 if i % 2 else 0  # both precision patterns (FP64-equivalent, split-BF16)
            out.append(("gemm", dict(A=A, B=B, C=np.empty((n, n)), prec=prec)))
        elif u < 0.8:
            n = 1 << int(rng.integers(0, 15))
            x = synth.complex_normal(seed * 1000 + i, n)
            out.append(("fft", dict(x=x, X=np.empty(n, complex), dir=int(rng.choice([-1, 1])))))
        else:
            I, J, K = (int(v) for v in rng.integers(3, 24, 3))
            iters = int(rng.integers(0, 12))
            out.append(("jacobi", dict(I=I, J=J, K=K, iters=iters, p=np.empty(I * J * K, np.float32),
                                       res=np.empty(max(iters, 1)))))
    return out


def alone(oo, ctx, kind, kw):
    if kind == "gemm":
        return oo.oo_gemm_f64(ctx, kw["A"], kw["B"], prec=kw["prec"])
    if kind == "fft":
        return oo.oo_fft_c128(ctx, kw["x"], kw["dir"])
    p = np.empty(kw["I"] * kw["J"] * kw["K"], np.float32)
    res = np.empty(kw["iters"])
    oo.oo_run_pattern(ctx, 63, 1, oo.jacobi(kw["I"], kw["J"], kw["K"], kw["iters"]), p, res)
    return p, res


def test_each_result_same_alone_and_in_the_mix(oo_mod):
    """Served Jacobi requests run the separate nest kernels; alone, a small
    grid would take the fused-iteration kernel, whose residual is summed in
    another order (p is the same either way).  So the bit-for-bit reference
    is the request alone with the separate kernels, and the fused result is
    checked against it to 1e-12."""
    oo = oo_mod
    mix = make_mix(3, 60)
    ctx = oo.oo_create(0)
    try:
        fused = {i: alone(oo, ctx, k, kw) for i, (k, kw) in enumerate(mix) if k == "jacobi"}
        oo.oo_set_option(ctx, oo.OO_OPT_JACOBI_FUSED, 0)
        ref = [alone(oo, ctx, k, kw) for k, kw in mix]
        oo.oo_set_option(ctx, oo.OO_OPT_JACOBI_FUSED, -1)
        for i, (pf, rf) in fused.items():
            assert np.array_equal(pf, ref[i][0])
            assert np.allclose(rf, ref[i][1], rtol=1e-12, atol=0)
        oo.oo_serve_start(ctx, slots=8, hbm_budget_bytes=1 << 30, queue_cap=256)
        lat = [None] * len(mix)

        def client(tag, idx):
            tickets = []
            for i in idx:
                k, kw = mix[i]
                r = oo.serve_request(k, client=tag, **kw)
                tickets.append((i, oo.oo_submit(ctx, r)))
            for i, t in tickets:
                lat[i] = oo.oo_wait(ctx, t, 60000)

        ths = [threading.Thread(target=client, args=(tag, list(range(tag, len(mix), 3)))) for tag in (0, 1, 2)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        st = oo.oo_serve_stats(ctx)
        oo.oo_serve_stop(ctx)
        assert st["completed"] == len(mix) and st["failed"] == 0
        assert all(v is not None and v >= 0 for v in lat)
        for (k, kw), r in zip(mix, ref):
            if k == "gemm":
                assert np.array_equal(kw["C"], r)
                ref_o = oracle.gemm(kw["A"], kw["B"])
                tol = 1e-12 if kw["prec"] == oo.OO_PREC_FP64EQ else 1e-4
                assert np.max(np.abs(kw["C"] - ref_o) / (np.abs(kw["A"]) @ np.abs(kw["B"]))) <= tol
            elif k == "fft":
                assert np.array_equal(kw["X"], r)
                ref_o = oracle.fft(kw["x"], kw["dir"])
                assert np.linalg.norm(kw["X"] - ref_o) <= 1e-12 * np.linalg.norm(ref_o)
            else:
                assert np.array_equal(kw["p"], r[0])
                assert np.array_equal(kw["res"][:kw["iters"]], r[1])
    finally:
        oo.oo_destroy(ctx)


def test_backpressure_and_budget(oo_mod):
    oo = oo_mod
    ctx = oo.oo_create(0)
    try:
        # a budget that fits only a couple of 129^3 Jacobi workspaces at a time
        oo.oo_serve_start(ctx, slots=4, hbm_budget_bytes=700 << 20, queue_cap=3)
        I = J = K = 129
        big = dict(I=I, J=J, K=K, iters=5, p=np.empty(I * J * K, np.float32), res=np.empty(5))
        accepted, busy = [], 0
        bufs = []
        for i in range(12):
            kw = dict(big, p=np.empty(I * J * K, np.float32), res=np.empty(5))
            bufs.append(kw)
            st, t = oo.oo_submit_status(ctx, oo.serve_request("jacobi", **kw))
            if st == oo.OO_EBUSY:
                busy += 1
            else:
                assert st == 0
                accepted.append((t, kw))
        assert busy > 0 and accepted
        ref_p, ref_r = alone(oo, oo.oo_create(0), "jacobi", big)
        for t, kw in accepted:
            oo.oo_wait(ctx, t, 60000)
            assert np.array_equal(kw["p"], ref_p) and np.array_equal(kw["res"], ref_r)
        # larger than the whole budget: rejected outright
        huge = dict(I=400, J=400, K=400, iters=1, p=np.empty(400 ** 3, np.float32), res=np.empty(1))
        st, _ = oo.oo_submit_status(ctx, oo.serve_request("jacobi", **huge))
        assert st == oo.OO_EINVAL
        s = oo.oo_serve_stats(ctx)
        assert s["rejected_busy"] == busy and s["device_free_bytes"] == s["device_budget_bytes"]
        oo.oo_serve_stop(ctx)
    finally:
        oo.oo_destroy(ctx)


def test_wait_timeout_keeps_ticket(oo_mod):
    oo = oo_mod
    ctx = oo.oo_create(0)
    try:
        oo.oo_serve_start(ctx, slots=2, hbm_budget_bytes=1 << 30, queue_cap=16)
        I, J, K, it = 97, 97, 193, 60
        kw = dict(I=I, J=J, K=K, iters=it, p=np.empty(I * J * K, np.float32), res=np.empty(it))
        t = oo.oo_submit(ctx, oo.serve_request("jacobi", **kw))
        with pytest.raises(oo.OOError) as e:
            oo.oo_wait(ctx, t, 0)
        assert e.value.status == oo.OO_ETIMEOUT
        assert oo.oo_wait(ctx, t, 60000) > 0
        with pytest.raises(oo.OOError):
            oo.oo_wait(ctx, t, 10)        # ticket consumed
        oo.oo_serve_stop(ctx)
        with pytest.raises(oo.OOError) as e:
            oo.oo_submit(ctx, oo.serve_request("jacobi", **kw))
        assert e.value.status == oo.OO_ESTATE
    finally:
        oo.oo_destroy(ctx)
