"""The device-resident serving loop (oo_serve_start_resident): persistent
worker kernels take every request's work from rings the host fills; no
kernel is launched per request.  Every result is exactly what the same
request gives alone on the same loop, matches the library's single calls
(GEMM, FFT: same bits; Jacobi: p bits, residuals to summation order) and the
oracle; admission is by free device memory; a bounded device wait that runs
out fails the requests in flight with OO_ETIMEOUT and leaves the context
usable."""
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
        if u < 0.45:
            n = int(rng.integers(16, 300))
            k = int(rng.choice([n + 3, 700]))  # level schemes (k <= 512) and the pair scheme
            A, B = synth.gemm_matrix(seed * 1000 + 2 * i, n, k), synth.gemm_matrix(seed * 1000 + 2 * i + 1, k, n)
            out.append(("gemm", dict(A=A, B=B, C=np.empty((n, n)), prec=2)))
        elif u < 0.8:
            n = 1 << int(rng.integers(0, 15))
            x = synth.complex_normal(seed * 1000 + i, n)
            out.append(("fft", dict(x=x, X=np.empty(n, complex), dir=int(rng.choice([-1, 1])))))
        else:
            I, J, K = (int(v) for v in rng.integers(3, 40, 3))
            iters = int(rng.integers(0, 12))
            out.append(("jacobi", dict(I=I, J=J, K=K, iters=iters, p=np.empty(I * J * K, np.float32),
                                       res=np.empty(max(iters, 1)))))
    return out


def fresh(kind, kw):
    """A copy of a request's buffers with fresh outputs."""
    kw = dict(kw)
    if kind == "gemm":
        kw["C"] = np.empty_like(kw["C"])
    elif kind == "fft":
        kw["X"] = np.empty_like(kw["X"])
    else:
        kw["p"] = np.empty_like(kw["p"])
        kw["res"] = np.empty_like(kw["res"])
    return kw


def outputs(kind, kw):
    if kind == "gemm":
        return (kw["C"],)
    if kind == "fft":
        return (kw["X"],)
    return (kw["p"], kw["res"][:kw["iters"]])


def test_each_result_same_alone_and_in_the_mix(oo_mod):
    oo = oo_mod
    mix = make_mix(7, 48)
    ctx = oo.oo_create(0)
    try:
        oo.oo_serve_start_resident(ctx, 2 << 30, 256)
        # alone: one request at a time through the loop
        alone = []
        for k, kw in mix:
            kw1 = fresh(k, kw)
            oo.oo_wait(ctx, oo.oo_submit(ctx, oo.serve_request(k, **kw1)), 60000)
            alone.append(outputs(k, kw1))
        # in the mix: three client threads submitting everything at once
        lat = [None] * len(mix)

        def client(tag, idx):
            tickets = [(i, oo.oo_submit(ctx, oo.serve_request(mix[i][0], client=tag, **mix[i][1]))) for i in idx]
            for i, t in tickets:
                lat[i] = oo.oo_wait(ctx, t, 60000)

        ths = [threading.Thread(target=client, args=(tag, list(range(tag, len(mix), 3)))) for tag in (0, 1, 2)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        st = oo.oo_serve_stats(ctx)
        oo.oo_serve_stop(ctx)
        assert st["completed"] == 2 * len(mix) and st["failed"] == 0
        assert all(v is not None and v >= 0 for v in lat)
        for (k, kw), a in zip(mix, alone):
            for x, y in zip(outputs(k, kw), a):
                assert np.array_equal(x, y), k
        # against the library's single calls and the oracle
        for k, kw in mix:
            if k == "gemm":
                assert np.array_equal(kw["C"], oo.oo_gemm_f64(ctx, kw["A"], kw["B"], prec=oo.OO_PREC_FP64EQ))
                ref = oracle.gemm(kw["A"], kw["B"])
                assert np.max(np.abs(kw["C"] - ref) / (np.abs(kw["A"]) @ np.abs(kw["B"]))) <= 1e-12
            elif k == "fft":
                assert np.array_equal(kw["X"], oo.oo_fft_c128(ctx, kw["x"], kw["dir"]))
                ref = oracle.fft(kw["x"], kw["dir"])
                assert np.linalg.norm(kw["X"] - ref) <= 1e-12 * max(np.linalg.norm(ref), 1e-300)
            else:
                I, J, K, it = kw["I"], kw["J"], kw["K"], kw["iters"]
                res_o, p_o = oracle.jacobi_run(I, J, K, it, mode=1)
                assert np.array_equal(kw["p"], p_o.reshape(-1).astype(np.float32))
                if it:
                    assert np.max(np.abs(kw["res"][:it] - res_o) / np.abs(res_o)) <= 1e-9
    finally:
        oo.oo_destroy(ctx)


def test_jacobi_residuals_match_tiled_kernels(oo_mod):
    """A 65 x 65 x 129 solve: p bit for bit what the per-iteration kernels
    give, residuals to their summation order."""
    oo = oo_mod
    I, J, K, it = 65, 65, 129, 20
    ctx = oo.oo_create(0)
    try:
        oo.oo_set_option(ctx, oo.OO_OPT_JACOBI_FUSED, 0)
        p_ref, r_ref = np.empty(I * J * K, np.float32), np.empty(it)
        oo.oo_run_pattern(ctx, 63, 1, oo.jacobi(I, J, K, it), p_ref, r_ref)
        oo.oo_serve_start_resident(ctx, 1 << 30, 16)
        kw = dict(I=I, J=J, K=K, iters=it, p=np.empty(I * J * K, np.float32), res=np.empty(it))
        oo.oo_wait(ctx, oo.oo_submit(ctx, oo.serve_request("jacobi", **kw)), 60000)
        oo.oo_serve_stop(ctx)
        assert np.array_equal(kw["p"], p_ref)
        assert np.max(np.abs(kw["res"] - r_ref) / r_ref) <= 1e-12
    finally:
        oo.oo_destroy(ctx)


def test_admission_by_free_memory_and_rejections(oo_mod):
    oo = oo_mod
    ctx = oo.oo_create(0)
    try:
        oo.oo_serve_start_resident(ctx, 256 << 20, 3)  # room for one 129^3 workspace at a time
        I = J = K = 129
        accepted, busy = [], 0
        for i in range(10):
            kw = dict(I=I, J=J, K=K, iters=3, p=np.empty(I * J * K, np.float32), res=np.empty(3))
            st, t = oo.oo_submit_status(ctx, oo.serve_request("jacobi", **kw))
            if st == oo.OO_EBUSY:
                busy += 1
            else:
                assert st == 0
                accepted.append((t, kw))
        assert busy > 0 and len(accepted) >= 1
        for t, kw in accepted:
            oo.oo_wait(ctx, t, 60000)
        for _, kw in accepted[1:]:
            assert np.array_equal(kw["p"], accepted[0][1]["p"])
            assert np.array_equal(kw["res"], accepted[0][1]["res"])
        A, B = synth.gemm_matrix(1, 8, 3000), synth.gemm_matrix(2, 3000, 8)
        bad = [oo.serve_request("gemm", A=A, B=B, C=np.empty((8, 8))),                     # k > 2048
               oo.serve_request("gemm", A=A[:, :64].copy(), B=B[:64].copy(), C=np.empty((8, 8)),
                                prec=oo.OO_PREC_SPLIT3_BF16),                              # not FP64EQ
               oo.serve_request("jacobi", I=400, J=400, K=400, iters=1,
                                p=np.empty(400 ** 3, np.float32), res=np.empty(1))]         # above the budget
        for r in bad:
            st, _ = oo.oo_submit_status(ctx, r)
            assert st == oo.OO_EINVAL
        s = oo.oo_serve_stats(ctx)
        assert s["rejected_busy"] == busy and s["device_free_bytes"] == s["device_budget_bytes"]
        # the context's other GPU calls wait until the loop stops
        with pytest.raises(oo.OOError) as e:
            oo.oo_fft_c128(ctx, synth.complex_normal(5, 64), -1)
        assert e.value.status == oo.OO_ESTATE
        oo.oo_serve_stop(ctx)
        oo.oo_fft_c128(ctx, synth.complex_normal(5, 64), -1)
    finally:
        oo.oo_destroy(ctx)


def test_stalled_wait_fails_requests_and_context_recovers(oo_mod):
    """Fault injection: the first admitted request's entry waits for a counter
    value that never comes; the workers' bounded waits (about a second) run
    out, the request fails with OO_ETIMEOUT, later submissions get
    OO_ESTATE, and after oo_serve_stop the context serves again."""
    oo = oo_mod
    ctx = oo.oo_create(0)
    try:
        x = synth.complex_normal(3, 1024)
        oo.oo_inject_wait_timeout(ctx, oo.OO_INJECT_SERVE_STALL)
        oo.oo_serve_start_resident(ctx, 512 << 20, 16)
        X = np.empty_like(x)
        t = oo.oo_submit(ctx, oo.serve_request("fft", x=x, X=X, dir=-1))
        with pytest.raises(oo.OOError) as e:
            oo.oo_wait(ctx, t, 30000)
        assert e.value.status == oo.OO_ETIMEOUT
        st, _ = oo.oo_submit_status(ctx, oo.serve_request("fft", x=x, X=X, dir=-1))
        assert st == oo.OO_ESTATE
        oo.oo_serve_stop(ctx)
        oo.oo_serve_start_resident(ctx, 512 << 20, 16)
        oo.oo_wait(ctx, oo.oo_submit(ctx, oo.serve_request("fft", x=x, X=X, dir=-1)), 30000)
        oo.oo_serve_stop(ctx)
        assert np.array_equal(X, oo.oo_fft_c128(ctx, x, -1))
    finally:
        oo.oo_destroy(ctx)


def test_largest_requests_same_bits_as_single_calls(oo_mod):
    """The largest requests the loop takes: FFTs of 2^20 and 2^22 points (the
    four-step passes as SIMT items), a GEMM at k = 2048 (the digit-slice
    region's row pitch) with n = 2048, and a 129 x 129 x 257 Jacobi solve,
    in flight together; each result is bit for bit the library's single
    call (Jacobi: p bits, residuals to summation order)."""
    oo = oo_mod
    ctx = oo.oo_create(0)
    try:
        xs = {e: synth.complex_normal(70 + e, 1 << e) for e in (20, 22)}
        A, B = synth.gemm_matrix(71, 2048, 2048), synth.gemm_matrix(72, 2048, 2048)
        A2, B2 = synth.gemm_matrix(73, 300, 2048), synth.gemm_matrix(74, 2048, 200)
        I, J, K, it = 129, 129, 257, 12
        want_fft = {(e, d): oo.oo_fft_c128(ctx, xs[e], d) for e in xs for d in (-1, 1)}
        want_gemm = oo.oo_gemm_f64(ctx, A, B, prec=oo.OO_PREC_FP64EQ)
        want_gemm2 = oo.oo_gemm_f64(ctx, A2, B2, prec=oo.OO_PREC_FP64EQ)
        oo.oo_set_option(ctx, oo.OO_OPT_JACOBI_FUSED, 0)
        p_ref, r_ref = np.empty(I * J * K, np.float32), np.empty(it)
        oo.oo_run_pattern(ctx, 63, 1, oo.jacobi(I, J, K, it), p_ref, r_ref)
        oo.oo_serve_start_resident(ctx, 8 << 30, 64)
        outs = {key: np.empty_like(xs[key[0]]) for key in want_fft}
        C, C2 = np.empty((2048, 2048)), np.empty((300, 200))
        p, r = np.empty(I * J * K, np.float32), np.empty(it)
        tickets = [oo.oo_submit(ctx, oo.serve_request("fft", x=xs[e], X=outs[(e, d)], dir=d)) for e, d in want_fft]
        tickets.append(oo.oo_submit(ctx, oo.serve_request("gemm", A=A, B=B, C=C)))
        tickets.append(oo.oo_submit(ctx, oo.serve_request("gemm", A=A2, B=B2, C=C2)))
        tickets.append(oo.oo_submit(ctx, oo.serve_request("jacobi", I=I, J=J, K=K, iters=it, p=p, res=r)))
        for t in tickets:
            oo.oo_wait(ctx, t, 120000)
        oo.oo_serve_stop(ctx)
        for key, want in want_fft.items():
            assert np.array_equal(outs[key], want), key
        assert np.array_equal(C, want_gemm) and np.array_equal(C2, want_gemm2)
        assert np.array_equal(p, p_ref)
        assert np.max(np.abs(r - r_ref) / r_ref) <= 1e-12
    finally:
        oo.oo_destroy(ctx)


def test_idle_loop_stays_alive_past_the_wait_bound(oo_mod):
    """Workers wait (bounded, about a second) for published entries; an idle
    loop publishes keep-alive entries, so after three idle seconds requests
    are still served and nothing has failed."""
    import time
    oo = oo_mod
    ctx = oo.oo_create(0)
    try:
        oo.oo_serve_start_resident(ctx, 512 << 20, 16)
        time.sleep(3.0)
        x = synth.complex_normal(9, 4096)
        X = np.empty_like(x)
        A, B, C = synth.gemm_matrix(10, 64, 96), synth.gemm_matrix(11, 96, 80), np.empty((64, 80))
        t1 = oo.oo_submit(ctx, oo.serve_request("fft", x=x, X=X, dir=1))
        t2 = oo.oo_submit(ctx, oo.serve_request("gemm", A=A, B=B, C=C))
        oo.oo_wait(ctx, t1, 30000)
        oo.oo_wait(ctx, t2, 30000)
        time.sleep(1.5)
        st = oo.oo_serve_stats(ctx)
        assert st["failed"] == 0 and st["completed"] == 2
        oo.oo_serve_stop(ctx)
        assert np.array_equal(X, oo.oo_fft_c128(ctx, x, 1))
        assert np.array_equal(C, oo.oo_gemm_f64(ctx, A, B, prec=oo.OO_PREC_FP64EQ))
    finally:
        oo.oo_destroy(ctx)
