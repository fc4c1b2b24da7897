"""Serving replicas in one process (oo_router_*): two host-scheduled serving
contexts on the same GPU with different device budgets; requests go to the
replica with the most free device memory and give what the library's
single calls give; a context that is not serving is passed over."""
import numpy as np
import pytest

from paper_2011_03602_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def oo_mod():
    from paper_2011_03602_gb300 import build as pkg_build
    from paper_2011_03602_gb300 import oo
    pkg_build.build()
    return oo


def test_router_routes_by_free_memory(oo_mod):
    oo = oo_mod
    small, big, idle = oo.oo_create(0), oo.oo_create(0), oo.oo_create(0)
    try:
        oo.oo_serve_start(small, slots=2, hbm_budget_bytes=256 << 20, queue_cap=64)
        oo.oo_serve_start(big, slots=2, hbm_budget_bytes=320 << 20, queue_cap=64)
        router = oo.Router([idle, small, big])  # `idle` is not serving
        x = synth.complex_normal(5, 1 << 16)
        X = np.empty_like(x)
        rep, t = router.submit(oo.serve_request("fft", x=x, X=X, dir=-1))
        assert rep == 2  # the most free bytes
        router.wait(rep, t)
        assert np.array_equal(X, oo.oo_fft_c128(big, x, -1))
        # Jacobi solves (each ~30 MB on the device) routed while none is
        # waited for: the router charges each to its replica, so once the big
        # replica's remaining budget falls below the small one's, the small
        # one takes the next
        I, J, K = 65, 65, 129
        need = oo.oo_serve_footprint(oo.serve_request("jacobi", I=I, J=J, K=K, iters=20,
                                                      p=np.empty(I * J * K, np.float32), res=np.empty(20)))
        handles, outs = [], []
        for i in range(8):
            p, r = np.empty(I * J * K, np.float32), np.empty(20)
            rep, t = router.submit(oo.serve_request("jacobi", I=I, J=J, K=K, iters=20, p=p, res=r))
            handles.append((rep, t))
            outs.append(p)
        reps = [h[0] for h in handles]
        for rep, t in handles:
            router.wait(rep, t)
        # 320 MB against 256 MB: the big replica first, the small one once
        # the big one's remaining budget falls below it
        assert need > 16 << 20 and reps[0] == 2 and set(reps) == {1, 2}
        for o in outs[1:]:
            assert np.array_equal(o, outs[0])
        A, B = synth.gemm_matrix(1, 200, 300), synth.gemm_matrix(2, 300, 150)
        C = np.empty((200, 150))
        rep, t = router.submit(oo.serve_request("gemm", A=A, B=B, C=C))
        router.wait(rep, t)
        assert np.array_equal(C, oo.oo_gemm_f64(small, A, B, prec=oo.OO_PREC_FP64EQ))
        router.close()
    finally:
        for c in (small, big, idle):
            oo.oo_destroy(c)


def test_router_falls_over_to_the_next_replica_on_back_pressure(oo_mod):
    """A replica whose queue is full answers OO_EBUSY; the router then takes
    the next best replica, and OO_EBUSY comes back only when every replica
    refuses."""
    oo = oo_mod
    tiny, spare = oo.oo_create(0), oo.oo_create(0)
    try:
        oo.oo_serve_start(tiny, slots=1, hbm_budget_bytes=1 << 30, queue_cap=1)   # most free memory, no queue
        oo.oo_serve_start(spare, slots=1, hbm_budget_bytes=512 << 20, queue_cap=64)
        router = oo.Router([tiny, spare])
        I, J, K = 65, 65, 129
        handles, reps = [], []
        for i in range(6):
            p, r = np.empty(I * J * K, np.float32), np.empty(30)
            rep, t = router.submit(oo.serve_request("jacobi", I=I, J=J, K=K, iters=30, p=p, res=r))
            handles.append((rep, t, p))
            reps.append(rep)
        assert reps[0] == 0 and 1 in reps  # the full queue sent later requests to the spare replica
        for rep, t, _ in handles:
            router.wait(rep, t)
        for _, _, p in handles[1:]:
            assert np.array_equal(p, handles[0][2])
        oo.oo_serve_stop(spare)
        busy = 0
        for i in range(4):  # only the tiny replica serves now: its one-deep queue refuses some
            try:
                p, r = np.empty(I * J * K, np.float32), np.empty(30)
                rep, t = router.submit(oo.serve_request("jacobi", I=I, J=J, K=K, iters=30, p=p, res=r))
                handles.append((rep, t, p))
            except oo.OOError as e:
                assert e.status == oo.OO_EBUSY
                busy += 1
        assert busy >= 1
        for rep, t, _ in handles[6:]:
            router.wait(rep, t)
        router.close()
    finally:
        for c in (tiny, spare):
            oo.oo_destroy(c)
