"""The GA over genes (Sec. 4.2.2) with fitness from patterns measured on the
GPU: every pattern computes the same program, so every gene the GA measures
passes the result gate and has a finite time; the GA's answer is the
fastest gene it measured; genes it never measured report infinity.  The
same holds after a function-block trial ran on the same context (the
trial order of Sec. 4.2 shares one context between the two searches)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def oo_mod():
    from paper_2011_03602_gb300 import build as pkg_build
    from paper_2011_03602_gb300 import oo
    pkg_build.build()
    return oo


def check_ga(oo, ctx, shape, iters, seed):
    r = oo.oo_ga_search(ctx, oo.jacobi(*shape, iters), 1, 8, 8, 0.9, 0.05, seed)
    gm, seen = r["gene_ms"], set(int(g) for g in r["history"].reshape(-1))
    for g in range(64):
        if g in seen:
            assert np.isfinite(gm[g]) and gm[g] > 0, (g, gm[g])
        else:
            assert np.isinf(gm[g]), g
    assert r["best_gene"] in seen
    assert r["best_ms"] == gm[r["best_gene"]] == min(gm[g] for g in seen)
    return r


@pytest.mark.parametrize("shape,iters", [((33, 33, 65), 10), ((40, 37, 140), 6)])
def test_ga_measures_every_gene_it_visits(oo_mod, shape, iters):
    ctx = oo_mod.oo_create(0)
    try:
        check_ga(oo_mod, ctx, shape, iters, seed=7)
    finally:
        oo_mod.oo_destroy(ctx)


def test_ga_after_function_block_trial(oo_mod):
    oo = oo_mod
    ctx = oo.oo_create(0)
    try:
        sites = [("cblas_dgemm", oo.OO_LANG_C, 1, 256, 256, 300),
                 ("numpy.fft.fft", oo.OO_LANG_PYTHON, 2, 0, 1 << 14, 0)]
        oo.oo_fb_search(ctx, sites, prec=oo.OO_PREC_FP64EQ, tol=1e-10, seed=3)
        r = check_ga(oo, ctx, (40, 37, 140), 6, seed=11)
        # the all-GPU hoisted pattern, evaluated directly, passes the gate too
        I, J, K, it = 40, 37, 140, 6
        p = np.empty(I * J * K, np.float32)
        res = np.empty(it)
        oo.oo_run_pattern(ctx, 63, 1, oo.jacobi(I, J, K, it), p, res)
        p0, res0 = np.empty_like(p), np.empty_like(res)
        oo.oo_run_pattern(ctx, 0, 1, oo.jacobi(I, J, K, it), p0, res0)
        assert np.allclose(res, res0, rtol=1e-5, atol=0) and np.max(np.abs(p - p0)) <= 1e-5
        assert np.isfinite(r["best_ms"])
    finally:
        oo.oo_destroy(ctx)


def test_ga_resumes_from_a_saved_table(oo_mod):
    """Checkpoint / resume: a search stopped after 3 generations and resumed
    with its saved table for 6 makes the same first 3 generations without
    measuring those genes again, and every gene it visits has a time."""
    oo = oo_mod
    ctx = oo.oo_create(0)
    try:
        prob = oo.jacobi(33, 33, 65, 8)
        first = oo.oo_ga_search(ctx, prob, 1, 8, 3, 0.9, 0.05, 19)
        seen = set(int(g) for g in first["history"].reshape(-1))
        saved = np.array([first["gene_ms"][g] if g in seen else np.nan for g in range(64)])
        full = oo.oo_ga_search(ctx, prob, 1, 8, 6, 0.9, 0.05, 19, known_ms=saved)
        assert np.array_equal(full["history"][:3], first["history"])
        for g in seen:
            assert full["gene_ms"][g] == saved[g]
        for g in set(int(x) for x in full["history"].reshape(-1)):
            assert np.isfinite(full["gene_ms"][g])
    finally:
        oo.oo_destroy(ctx)
