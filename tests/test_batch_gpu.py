"""Batched uneven function blocks: grouped persistent kernels (and their
CUDA-graph replay) must give exactly what one call per request gives, and
both must match the FP64 oracle at the blocks' tolerances."""
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


def make_requests(seed, n_gemm, n_fft, gemm_range=(1, 300), fft_logn=(0, 15)):
    rng = np.random.default_rng(seed)
    reqs, host = [], []
    for i in range(n_gemm):
        m, n, k = (int(x) for x in rng.integers(gemm_range[0], gemm_range[1] + 1, 3))
        A = synth.gemm_matrix(10 * i + 1, m, k)
        B = synth.gemm_matrix(10 * i + 2, k, n)
        reqs.append(dict(kind="gemm", m=m, n=n, k=k, A=torch.from_numpy(A).cuda(), B=torch.from_numpy(B).cuda(),
                         C=torch.full((m, n), np.nan, dtype=torch.float64, device="cuda")))
        host.append((A, B))
    for i in range(n_fft):
        e = int(rng.integers(fft_logn[0], fft_logn[1] + 1))
        d = int(rng.choice([-1, 1]))
        x = synth.complex_normal(1000 + i, 1 << e) * 10.0 ** int(rng.integers(-3, 4))
        reqs.append(dict(kind="fft", n=1 << e, dir=d, x=torch.from_numpy(x.view(np.float64).copy()).cuda(),
                         X=torch.full((2 << e,), np.nan, dtype=torch.float64, device="cuda")))
        host.append((x, d))
    return reqs, host


def outputs(reqs):
    return [(r["C"] if r["kind"] == "gemm" else r["X"]).cpu().numpy().copy() for r in reqs]


def test_grouped_equals_per_call_and_oracle(oo_mod):
    ctx = oo_mod.oo_create(0)
    try:
        reqs, host = make_requests(5, 24, 18)
        b = oo_mod.oo_batch_create(ctx, reqs)
        try:
            got = {}
            for mode in (2, 0, 1, 1):
                for r in reqs:
                    (r["C"] if r["kind"] == "gemm" else r["X"]).fill_(np.nan)
                oo_mod.oo_batch_run(ctx, b, mode)
                oo_mod.oo_batch_check(ctx, b)
                got[mode] = outputs(reqs)
            info = oo_mod.oo_batch_info(b)
            assert info["n_gemm"] == 24 and info["n_fft"] == 18
        finally:
            oo_mod.oo_batch_destroy(b)
        for i in range(len(reqs)):
            assert np.array_equal(got[0][i], got[2][i]), i      # grouped == one call per request
            assert np.array_equal(got[1][i], got[2][i]), i      # graph replay == one call per request
        for r, h, out in zip(reqs, host, got[0]):
            if r["kind"] == "gemm":
                A, B = h
                ref = oracle.gemm(A, B)
                assert np.max(np.abs(out - ref) / (np.abs(A) @ np.abs(B))) <= 1e-4
            else:
                x, d = h
                X = out.view(np.complex128)
                ref = oracle.fft(x, d)
                assert np.linalg.norm(X - ref) / np.linalg.norm(ref) <= 1e-12
    finally:
        oo_mod.oo_destroy(ctx)


def test_only_ffts_and_only_gemms(oo_mod):
    ctx = oo_mod.oo_create(0)
    try:
        for ng, nf in ((0, 9), (7, 0)):
            reqs, host = make_requests(11 + ng, ng, nf, gemm_range=(16, 200), fft_logn=(8, 14))
            b = oo_mod.oo_batch_create(ctx, reqs)
            try:
                oo_mod.oo_batch_run(ctx, b, 1)
                oo_mod.oo_batch_check(ctx, b)
                a = outputs(reqs)
                oo_mod.oo_batch_run(ctx, b, 2)
                oo_mod.oo_batch_check(ctx, b)
                c = outputs(reqs)
                assert all(np.array_equal(x, y) for x, y in zip(a, c))
            finally:
                oo_mod.oo_batch_destroy(b)
    finally:
        oo_mod.oo_destroy(ctx)


def test_bad_requests(oo_mod):
    ctx = oo_mod.oo_create(0)
    try:
        x = torch.zeros(24, dtype=torch.float64, device="cuda")
        with pytest.raises(oo_mod.OOError):
            oo_mod.oo_batch_create(ctx, [dict(kind="fft", n=12, x=x, X=x)])
        with pytest.raises(oo_mod.OOError):
            oo_mod.oo_batch_create(ctx, [dict(kind="gemm", m=0, n=2, k=2, A=x, B=x, C=x)])
    finally:
        oo_mod.oo_destroy(ctx)


def test_full_size_batch_sampled(oo_mod):
    """The benchmark's batch (4096 GEMMs, m, n, k log-uniform in [16, 512];
    2048 FFTs, 2^8..2^16, alternating directions; same seeds): the CUDA-graph
    replay equals one call per request for every request, and sampled
    requests match the oracle."""
    n_gemm, n_fft = 4096, 2048
    dims = synth.log_uniform_int(4, 3 * n_gemm, 16, 512).reshape(n_gemm, 3)
    expo = 8 + np.floor(synth.uniform(5, n_fft) * 9).astype(int)
    ctx = oo_mod.oo_create(0)
    try:
        reqs = []
        for i, (m, n, k) in enumerate(dims.tolist()):
            reqs.append(dict(kind="gemm", m=m, n=n, k=k,
                             A=torch.from_numpy(synth.gemm_matrix(100 + i, m, k)).cuda(),
                             B=torch.from_numpy(synth.gemm_matrix(200000 + i, k, n)).cuda(),
                             C=torch.full((m, n), np.nan, dtype=torch.float64, device="cuda")))
        for i, e in enumerate(expo.tolist()):
            x = synth.complex_normal(400000 + i, 1 << e)
            reqs.append(dict(kind="fft", n=1 << e, dir=-1 if i % 2 == 0 else 1,
                             x=torch.from_numpy(x.view(np.float64).copy()).cuda(),
                             X=torch.full((2 << e,), np.nan, dtype=torch.float64, device="cuda")))
        b = oo_mod.oo_batch_create(ctx, reqs)
        try:
            oo_mod.oo_batch_run(ctx, b, 2)
            oo_mod.oo_batch_check(ctx, b)
            per_call = outputs(reqs)
            for r in reqs:
                (r["C"] if r["kind"] == "gemm" else r["X"]).fill_(np.nan)
            oo_mod.oo_batch_run(ctx, b, 1)
            oo_mod.oo_batch_check(ctx, b)
            graph = outputs(reqs)
        finally:
            oo_mod.oo_batch_destroy(b)
        for i in range(len(reqs)):
            assert np.array_equal(graph[i], per_call[i]), i
        rng = np.random.default_rng(7)
        for i in rng.choice(n_gemm, 48, replace=False):
            m, n, k = (int(v) for v in dims[i])
            A, B = synth.gemm_matrix(100 + int(i), m, k), synth.gemm_matrix(200000 + int(i), k, n)
            e = np.max(np.abs(graph[i] - oracle.gemm(A, B)) / (np.abs(A) @ np.abs(B)))
            assert e <= 1e-4, (i, e)
        for j in rng.choice(n_fft, 48, replace=False):
            x = synth.complex_normal(400000 + int(j), 1 << int(expo[j]))
            ref = oracle.fft(x, -1 if j % 2 == 0 else 1)
            X = graph[n_gemm + int(j)].view(np.complex128)
            assert np.linalg.norm(X - ref) <= 1e-12 * np.linalg.norm(ref), j
    finally:
        oo_mod.oo_destroy(ctx)


@pytest.mark.parametrize("gemm_range", [(1, 260), (400, 1100)])
def test_fp64_equivalent_requests_in_a_batch(oo_mod, gemm_range):
    """Both precision patterns in one batch: FP64-equivalent requests give
    exactly what oo_gemm_f64_dev gives for them alone (grouped, graph and
    per-call modes alike) and meet the 1e-12 bound; the split-BF16 requests
    around them are unaffected."""
    oo = oo_mod
    ctx = oo.oo_create(0)
    try:
        # (1, 260): the level schemes (k <= 512); (400, 1100) reaches the
        # pair scheme (k > 512), whose single products run their own kernel
        reqs, host = make_requests(17, 10, 6, gemm_range=gemm_range)
        eq = [i for i in range(10) if i % 3 != 1]
        for i in eq:
            reqs[i]["prec"] = oo.OO_PREC_FP64EQ
        alone = {}
        for i in range(10):
            r = reqs[i]
            C = torch.empty_like(r["C"])
            oo.oo_gemm_f64_dev(ctx, r["m"], r["n"], r["k"], r["A"], r["k"], r["B"], r["n"], C, r["n"],
                               prec=r.get("prec", oo.OO_PREC_SPLIT3_BF16))
            oo.oo_gemm_check(ctx, r["m"], r["n"], r["k"])
            alone[i] = C.cpu().numpy()
        b = oo.oo_batch_create(ctx, reqs)
        try:
            info = oo.oo_batch_info(b)
            assert info["n_gemm"] == 10
            assert info["gemm_flops"] == sum(2.0 * r["m"] * r["n"] * r["k"] for r in reqs[:10])
            for mode in (0, 1, 2, 1):
                for r in reqs:
                    (r["C"] if r["kind"] == "gemm" else r["X"]).fill_(np.nan)
                oo.oo_batch_run(ctx, b, mode)
                oo.oo_batch_check(ctx, b)
                out = outputs(reqs)
                for i in range(10):
                    assert np.array_equal(out[i], alone[i]), (mode, i)
        finally:
            oo.oo_batch_destroy(b)
        for i in eq:
            A, B = host[i]
            ref = oracle.gemm(A, B)
            err = np.max(np.abs(alone[i] - ref) / np.maximum(np.abs(A) @ np.abs(B), 1e-300))
            assert err <= 1e-12, (i, err)
    finally:
        oo.oo_destroy(ctx)
