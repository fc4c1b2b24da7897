"""The allocation-free stencil entry point (for callers that cannot
allocate device memory when they call, e.g. on a fixed memory pool) must
give what the allocating entry point gives,
and what the oracle gives, and must report a bounded wait that ran out.

Runs last (file name) so a failure here cannot hide other results; it works
alone in a fresh process as well as after the other tests."""
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


def _pad(a, pitch):
    I, J, K = a.shape
    out = torch.zeros((I, J, pitch), dtype=torch.float32, device="cuda")
    out[:, :, :K] = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return out


def _inputs(shape, call):
    coef = np.stack([synth.field(300 + 17 * call + a, shape, -1.0, 1.0) for a in range(12)])
    coef[3] = synth.field(70 + call, shape, 0.1, 0.3)
    coef[10] = synth.field(80 + call, shape, 0.5, 1.5)
    p = synth.field(90 + call, shape, 0.0, 1.0)
    return coef, p


def _sweep_both(oo, ctx, shape, coef, p, omega):
    I, J, K = shape
    pitch = oo.oo_jacobi_pitch(K)
    dcoef = [_pad(coef[a], pitch) for a in range(12)]
    dp = _pad(p, pitch)
    w_ref = torch.full((I, J, pitch), -3.0, dtype=torch.float32, device="cuda")
    w_new = torch.full((I, J, pitch), -3.0, dtype=torch.float32, device="cuda")
    r_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    r_new = torch.zeros(1, dtype=torch.float64, device="cuda")
    # the inputs were written on torch's stream; the library runs on the
    # context's own stream, which does not wait for it
    torch.cuda.synchronize()
    oo.oo_stencil_dev(ctx, I, J, K, pitch, dcoef, dp, omega, w_ref, r_ref)
    oo.oo_stencil_noalloc_dev(ctx, I, J, K, pitch, dcoef, dp, omega, w_new, r_new)
    oo.oo_stencil_check(ctx)
    oo.oo_stencil_noalloc_check(ctx)
    return w_ref, w_new, r_ref.item(), r_new.item()


@pytest.mark.parametrize("shape", [(20, 21, 300), (33, 33, 65), (9, 40, 517)])
def test_static_scratch_matches_allocating_path_and_oracle(oo_mod, shape):
    I, J, K = shape
    ctx = oo_mod.oo_create(0)
    try:
        for call, omega in enumerate((0.8, 1.3)):   # two calls in a row share the static array
            coef, p = _inputs(shape, call)
            w_ref, w_new, r_ref, r_new = _sweep_both(oo_mod, ctx, shape, coef, p, omega)
            # same tile variant and work split as the allocating entry: same bits
            assert torch.equal(w_new, w_ref), call
            assert r_new == r_ref, (call, r_new, r_ref)
            # and the oracle's values: wrk2 within one float ulp where the
            # float-float result rounds the other way, residual to 1e-5
            w_or, r_or = oracle.stencil(coef, p.astype(np.float64), np.float32(omega))
            inner = (slice(1, -1),) * 3
            got = w_new[:, :, :K].cpu().numpy()[inner]
            ref32 = w_or.astype(np.float32)[inner]
            assert np.all(np.abs(got - ref32) <= np.spacing(np.abs(ref32))), call
            assert abs(r_new - r_or) <= 1e-5 * abs(r_or), (call, r_new, r_or)
    finally:
        oo_mod.oo_destroy(ctx)


def test_context_variant_option_applies(oo_mod):
    """Both entry points follow the context's tile-variant option."""
    shape = (12, 19, 140)
    ctx = oo_mod.oo_create(0)
    try:
        for v in (0, 3):
            oo_mod.oo_set_option(ctx, oo_mod.OO_OPT_STENCIL_VARIANT, v)
            coef, p = _inputs(shape, v)
            w_ref, w_new, r_ref, r_new = _sweep_both(oo_mod, ctx, shape, coef, p, 0.8)
            assert torch.equal(w_new, w_ref), v
            assert r_new == r_ref, (v, r_new, r_ref)
    finally:
        oo_mod.oo_destroy(ctx)


def test_wait_timeout_reported(oo_mod):
    """A sweep whose bounded wait runs out (the one-shot injection: the
    producer never issues its first p-tile copy) is reported by the check
    call, which clears the word; the next sweep is whole again."""
    shape = (20, 21, 300)
    I, J, K = shape
    pitch = oo_mod.oo_jacobi_pitch(K)
    ctx = oo_mod.oo_create(0)
    try:
        coef, p = _inputs(shape, 0)
        dcoef = [_pad(coef[a], pitch) for a in range(12)]
        dp = _pad(p, pitch)
        w = torch.zeros((I, J, pitch), dtype=torch.float32, device="cuda")
        r = torch.zeros(1, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        oo_mod.oo_inject_wait_timeout(ctx, oo_mod.OO_INJECT_STENCIL_LOAD)
        oo_mod.oo_stencil_noalloc_dev(ctx, I, J, K, pitch, dcoef, dp, 0.8, w, r)
        with pytest.raises(oo_mod.OOError) as e:
            oo_mod.oo_stencil_noalloc_check(ctx)
        assert e.value.status == oo_mod.OO_ETIMEOUT
        oo_mod.oo_stencil_noalloc_check(ctx)  # cleared
        oo_mod.oo_stencil_noalloc_dev(ctx, I, J, K, pitch, dcoef, dp, 0.8, w, r)
        oo_mod.oo_stencil_noalloc_check(ctx)
        _, r_or = oracle.stencil(coef, p.astype(np.float64), np.float32(0.8))
        assert abs(r.item() - r_or) <= 1e-5 * abs(r_or)
    finally:
        oo_mod.oo_destroy(ctx)


def test_rejects_grid_beyond_static_scratch(oo_mod):
    ctx = oo_mod.oo_create(0)
    try:
        I, J, K = 3, 8194 * 8 + 2, 130   # 2 k-tiles x 8194 j-tiles x 16 warps > 65536 slots
        pitch = oo_mod.oo_jacobi_pitch(K)
        dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
        res = torch.zeros(1, dtype=torch.float64, device="cuda")
        with pytest.raises(oo_mod.OOError) as e:
            oo_mod.oo_stencil_noalloc_dev(ctx, I, J, K, pitch, [dummy] * 12, dummy, 0.8, dummy, res)
        assert e.value.status == oo_mod.OO_EINVAL
        assert "static scratch" in str(e.value)
    finally:
        oo_mod.oo_destroy(ctx)
