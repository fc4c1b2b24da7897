"""Failure detection without a GPU fault: every device wait is bounded and a
wait that runs out comes back to the host as OO_ETIMEOUT with the context
still usable; an allocation the device cannot satisfy is OO_ENOMEM; a GA
evaluation cut off by its time limit counts as infinitely slow (fitness 0).
The timeouts are made on purpose by a one-shot injection: the stencil
producer skips one copy, or the fused kernel's grid barrier awaits one block
more than it launched; each kernel's wait gives up after about a second."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def oo_mod():
    from paper_2011_03602_gb300 import build as pkg_build
    from paper_2011_03602_gb300 import oo
    pkg_build.build()
    return oo


def run(oo, ctx, shape, iters):
    I, J, K = shape
    p = np.empty(I * J * K, np.float32)
    res = np.empty(iters)
    oo.oo_run_pattern(ctx, 63, 1, oo.jacobi(I, J, K, iters), p, res)
    return p, res


@pytest.mark.parametrize("what,fused", [("STENCIL_LOAD", "0"), ("FUSED_BARRIER", "1")])
def test_wait_timeout_reported_and_context_usable(oo_mod, what, fused):
    oo = oo_mod
    shape, iters = (20, 21, 70), 3
    ctx = oo.oo_create(0)
    try:
        oo.oo_set_option(ctx, oo.OO_OPT_JACOBI_FUSED, int(fused))
        oo.oo_inject_wait_timeout(ctx, getattr(oo, "OO_INJECT_" + what))
        with pytest.raises(oo.OOError) as e:
            run(oo, ctx, shape, iters)
        assert e.value.status == oo.OO_ETIMEOUT
        # one-shot: the same call now succeeds and matches the oracle
        p, res = run(oo, ctx, shape, iters)
        ref_res, ref_p = oracle.jacobi_run(*shape, iters, mode=1)
        assert np.array_equal(p, ref_p.reshape(-1).astype(np.float32))
        assert np.max(np.abs(res - ref_res) / ref_res) <= 1e-9
    finally:
        oo.oo_destroy(ctx)


def test_single_sweep_timeout_reported(oo_mod):
    """oo_stencil_dev on caller arrays: an injected wait time-out is reported
    by oo_stencil_check (then cleared), and the next sweep is whole."""
    from paper_2011_03602_gb300 import synth
    import torch
    oo = oo_mod
    I, J, K = 12, 19, 140
    pitch = oo.oo_jacobi_pitch(K)
    ctx = oo.oo_create(0)
    try:
        coef = np.stack([synth.field(500 + a, (I, J, K), -1.0, 1.0) for a in range(12)])
        p = synth.field(520, (I, J, K), 0.0, 1.0)

        def pad(a):
            t = torch.zeros((I, J, pitch), dtype=torch.float32, device="cuda")
            t[:, :, :K] = torch.from_numpy(np.ascontiguousarray(a)).cuda()
            return t
        dcoef = [pad(coef[a]) for a in range(12)]
        dp = pad(p)
        w = torch.zeros((I, J, pitch), dtype=torch.float32, device="cuda")
        r = torch.zeros(1, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        oo.oo_inject_wait_timeout(ctx, oo.OO_INJECT_STENCIL_LOAD)
        oo.oo_stencil_dev(ctx, I, J, K, pitch, dcoef, dp, 0.8, w, r)
        with pytest.raises(oo.OOError) as e:
            oo.oo_stencil_check(ctx)
        assert e.value.status == oo.OO_ETIMEOUT
        oo.oo_stencil_dev(ctx, I, J, K, pitch, dcoef, dp, 0.8, w, r)
        oo.oo_stencil_check(ctx)
        _, r_or = oracle.stencil(coef, p.astype(np.float64), np.float32(0.8))
        assert abs(r.item() - r_or) <= 1e-5 * abs(r_or)
    finally:
        oo.oo_destroy(ctx)


def test_injection_arguments(oo_mod):
    oo = oo_mod
    ctx = oo.oo_create(0)
    try:
        with pytest.raises(oo.OOError) as e:
            oo.oo_inject_wait_timeout(ctx, 7)
        assert e.value.status == oo.OO_EINVAL
        oo.oo_inject_wait_timeout(ctx, oo.OO_INJECT_STENCIL_LOAD)
        oo.oo_inject_wait_timeout(ctx, oo.OO_INJECT_NONE)  # disarmed: the run succeeds
        run(oo, ctx, (9, 10, 131), 2)
    finally:
        oo.oo_destroy(ctx)


def test_device_allocation_failure(oo_mod):
    oo = oo_mod
    ctx = oo.oo_create(0)
    try:
        with pytest.raises(oo.OOError) as e:
            oo.oo_serve_start(ctx, slots=2, hbm_budget_bytes=1 << 50, queue_cap=8)  # 1 PiB of device memory
        assert e.value.status == oo.OO_ENOMEM
        oo.oo_serve_start(ctx, slots=2, hbm_budget_bytes=1 << 28, queue_cap=8)
        oo.oo_serve_stop(ctx)
    finally:
        oo.oo_destroy(ctx)


def test_ga_evaluation_time_limit(oo_mod):
    """A limit of 1 ns cuts every evaluation off after its first iteration,
    whatever the gene: every measured gene counts as infinitely slow."""
    oo = oo_mod
    ctx = oo.oo_create(0)
    try:
        r = oo.oo_ga_search(ctx, oo.jacobi(40, 37, 140, 40), 1, 6, 3, 0.9, 0.05, 5, 1e-6)
        seen = set(int(g) for g in r["history"].reshape(-1))
        assert all(np.isinf(r["gene_ms"][g]) for g in seen)
        assert np.isinf(r["best_ms"])
    finally:
        oo.oo_destroy(ctx)
