"""Generic loop programs (Sec. 4.3): the method applied to a second program,
a 2D five-point heat solver whose nests the caller supplies (numpy on the
CPU, torch on the GPU, on the caller's own buffers).  Every gene and both
transfer modes give the all-CPU result, the executed copies are the
oracle's transfer plan, and the GA's result gate rejects a wrong GPU nest."""
import math

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, ITERS = 192, 8
COEF, U, UNEW, RES = range(4)
# (name, level, parallelisable, reads, writes, partial)
NESTS = [
    dict(name="init_coef", level=0, parallelisable=1, reads=0, writes=1 << COEF, partial=0),
    dict(name="init_u", level=0, parallelisable=1, reads=0, writes=(1 << U) | (1 << UNEW), partial=0),
    dict(name="step", level=1, parallelisable=1, reads=(1 << U) | (1 << COEF), writes=(1 << UNEW) | (1 << RES),
         partial=(1 << UNEW) | (1 << RES)),
    dict(name="copy", level=1, parallelisable=1, reads=1 << UNEW, writes=1 << U, partial=1 << U),
    dict(name="edges", level=1, parallelisable=1, reads=0, writes=1 << U, partial=1 << U),
]
OUTPUTS = (1 << U) | (1 << RES)


@pytest.fixture(scope="module")
def oo_mod():
    from paper_2011_03602_gb300 import build as pkg_build
    from paper_2011_03602_gb300 import oo
    pkg_build.build()
    return oo


class Heat:
    """The program's state on both sides and its nest bodies."""

    def __init__(self, broken_copy=False):
        self.h = [np.zeros((N, N)), np.zeros((N, N)), np.zeros((N, N)), np.zeros(ITERS)]
        self.d = [torch.zeros((N, N), dtype=torch.float64, device="cuda") for _ in range(3)] + \
                 [torch.zeros(ITERS, dtype=torch.float64, device="cuda")]
        self.broken_copy = broken_copy
        i = np.arange(N)[:, None]
        j = np.arange(N)[None, :]
        self.coef0 = 0.1 + 0.01 * ((7 * i + 3 * j) % 11)
        self.u0 = ((13 * i + 5 * j) % 17) / 17.0

    def body(self, nest, on_gpu, it, stream):
        if on_gpu:
            with torch.cuda.stream(torch.cuda.ExternalStream(stream)):
                self._run(self.d, nest, it, lambda a: torch.from_numpy(a).cuda(), lambda x: torch.sum(x))
        else:
            self._run(self.h, nest, it, lambda a: a.copy(), lambda x: np.sum(x))

    def _run(self, v, nest, it, const, total):
        coef, u, unew, res = v
        if nest == 0:
            coef[...] = const(self.coef0)
        elif nest == 1:
            u[...] = const(self.u0)
            unew[...] = const(self.u0)
        elif nest == 2:
            c = u[1:-1, 1:-1]
            t = u[2:, 1:-1] + u[:-2, 1:-1]
            t = t + u[1:-1, 2:]
            t = t + u[1:-1, :-2]
            t = t - c * 4.0
            t = coef[1:-1, 1:-1] * t
            unew[1:-1, 1:-1] = c + t
            d = unew[1:-1, 1:-1] - c
            res[it] = total(d * d)
        elif nest == 3:
            if self.broken_copy and isinstance(u, torch.Tensor):
                u[1:-1, 1:-1] = unew[1:-1, 2:]  # a wrong GPU nest: shifted by one column
            else:
                u[1:-1, 1:-1] = unew[1:-1, 1:-1]
        else:
            u[0, :] = 1.0
            u[-1, :] = 0.0
            u[:, 0] = 0.5
            u[:, -1] = 0.25


def load(oo, ctx):
    return oo.oo_load_nests(ctx, NESTS, [N * N * 8] * 3 + [ITERS * 8], OUTPUTS,
                            ["coef", "u", "unew", "res"])


def test_every_gene_and_mode_matches_all_cpu(oo_mod):
    oo = oo_mod
    ctx = oo.oo_create(0)
    try:
        assert load(oo, ctx) == 5
        prog = Heat()
        oo.oo_run_program(ctx, 0, 1, ITERS, prog.body, prog.h, prog.d)
        u_ref, res_ref = prog.h[U].copy(), prog.h[RES].copy()
        assert np.all(np.isfinite(res_ref)) and res_ref[0] > 0
        var_bytes = [N * N * 8] * 3 + [ITERS * 8]
        for gene in range(32):
            for hoist in (1, 0):
                for a in prog.h:
                    a[...] = 0.0
                st = oo.oo_run_program(ctx, gene, hoist, ITERS, prog.body, prog.h, prog.d)
                assert np.array_equal(prog.h[U], u_ref), (gene, hoist)
                assert np.allclose(prog.h[RES], res_ref, rtol=1e-12, atol=0), (gene, hoist)
                xs, h2d, d2h = oracle.plan(NESTS, var_bytes, OUTPUTS, gene, hoist, ITERS)
                assert (st["n_xfers"], st["h2d_bytes"], st["d2h_bytes"]) == (len(xs), h2d, d2h), (gene, hoist)
                assert st["n_launches"] == bin(gene & 0b00011).count("1") + ITERS * bin(gene >> 2).count("1")
    finally:
        oo.oo_destroy(ctx)


def test_ga_gate_rejects_a_wrong_gpu_nest(oo_mod):
    oo = oo_mod
    ctx = oo.oo_create(0)
    try:
        L = load(oo, ctx)
        ref = Heat()
        oo.oo_run_program(ctx, 0, 1, ITERS, ref.body, ref.h, ref.d)
        u_ref = ref.h[U].copy()
        prog = Heat(broken_copy=True)
        r = oo.oo_ga_program(ctx, L, 1, ITERS, prog.body, prog.h, prog.d, 8, 6, 0.9, 0.05, 11,
                             check=lambda: np.array_equal(prog.h[U], u_ref))
        gm = r["gene_ms"]  # infinity: not measured, or failed the gate
        assert math.isfinite(r["best_ms"])
        assert not (r["best_gene"] >> 3) & 1          # the broken nest stays on the CPU
        assert any(math.isfinite(gm[g]) for g in range(32))
        for g in range(32):
            if (g >> 3) & 1:
                assert math.isinf(gm[g]), g           # every gene offloading it failed the gate
    finally:
        oo.oo_destroy(ctx)


def test_nest_failure_and_missing_buffers(oo_mod):
    oo = oo_mod
    ctx = oo.oo_create(0)
    try:
        load(oo, ctx)
        prog = Heat()

        def failing(nest, on_gpu, it, stream):
            if nest == 3:
                raise RuntimeError("nest failed")
            prog.body(nest, on_gpu, it, stream)
        with pytest.raises(oo.OOError) as e:
            oo.oo_run_program(ctx, 0b11111, 1, ITERS, failing, prog.h, prog.d)
        assert e.value.status == oo.OO_EUSER
        with pytest.raises(oo.OOError) as e:
            oo.oo_run_program(ctx, 0b00100, 1, ITERS, prog.body, prog.h, [None, None, None, None])
        assert e.value.status == oo.OO_EINVAL
    finally:
        oo.oo_destroy(ctx)
