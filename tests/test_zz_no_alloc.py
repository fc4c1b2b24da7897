"""The allocation-free stencil entry point (for callers that cannot
allocate device memory when they call, e.g. inside a CUDA-graph capture or
on a fixed memory pool) must give what the allocating entry point gives.

Runs last (file name) so a failure here cannot hide other results; it works
alone in a fresh process as well as after the other tests."""
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


def _pad(a, pitch):
    I, J, K = a.shape
    out = torch.zeros((I, J, pitch), dtype=torch.float32, device="cuda")
    out[:, :, :K] = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return out


@pytest.mark.parametrize("shape", [(20, 21, 300), (33, 33, 65), (9, 40, 517)])
def test_static_scratch_matches_allocating_path(oo_mod, shape):
    I, J, K = shape
    pitch = oo_mod.oo_jacobi_pitch(K)
    ctx = oo_mod.oo_create(0)
    try:
        for call, omega in enumerate((0.8, 1.3)):   # two calls in a row share the static array
            coef = np.stack([synth.field(300 + 17 * call + a, shape, -1.0, 1.0) for a in range(12)])
            coef[3] = synth.field(70 + call, shape, 0.1, 0.3)
            coef[10] = synth.field(80 + call, shape, 0.5, 1.5)
            p = synth.field(90 + call, shape, 0.0, 1.0)
            dcoef = [_pad(coef[a], pitch) for a in range(12)]
            dp = _pad(p, pitch)
            w_ref = torch.full((I, J, pitch), -3.0, dtype=torch.float32, device="cuda")
            w_new = torch.full((I, J, pitch), -3.0, dtype=torch.float32, device="cuda")
            r_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
            r_new = torch.zeros(1, dtype=torch.float64, device="cuda")
            oo_mod.oo_stencil_dev(ctx, I, J, K, pitch, dcoef, dp, omega, w_ref, r_ref)
            oo_mod.oo_stencil_noalloc_dev(ctx, I, J, K, pitch, dcoef, dp, omega, w_new, r_new)
            oo_mod.oo_sync(ctx)
            assert torch.equal(w_new, w_ref), call
            a, b = r_new.item(), r_ref.item()
            assert abs(a - b) <= 1e-11 * abs(b), (call, a, b)
    finally:
        oo_mod.oo_destroy(ctx)


def test_rejects_grid_beyond_static_scratch(oo_mod):
    ctx = oo_mod.oo_create(0)
    try:
        I, J, K = 3, 8194 * 8 + 2, 130   # 2 k-tiles x 8194 j-tiles x 8 warps > 65536 slots
        pitch = oo_mod.oo_jacobi_pitch(K)
        dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
        res = torch.zeros(1, dtype=torch.float64, device="cuda")
        with pytest.raises(oo_mod.OOError) as e:
            oo_mod.oo_stencil_noalloc_dev(ctx, I, J, K, pitch, [dummy] * 12, dummy, 0.8, dummy, res)
        assert e.value.status == oo_mod.OO_EINVAL
        assert "static scratch" in str(e.value)
    finally:
        oo_mod.oo_destroy(ctx)
