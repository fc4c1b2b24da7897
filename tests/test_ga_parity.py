"""Library GA vs the oracle GA on injected time tables: identical
populations in every generation and the same answer (Sec. 4.2.2)."""
import numpy as np
import pytest

import oracle
from paper_2011_03602_gb300 import build as pkg_build
from paper_2011_03602_gb300 import oo


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg_build.build()


@pytest.mark.parametrize("L,pop,gens,pc,pm,seed", [
    (6, 16, 16, 0.9, 0.05, 1),
    (6, 16, 16, 0.9, 0.05, 12345),
    (6, 7, 5, 1.0, 0.5, 3),
    (10, 32, 8, 0.6, 0.1, 99),
    (1, 4, 4, 0.9, 0.05, 7),
    (6, 16, 4, 0.0, 0.0, 8),
])
def test_same_populations(L, pop, gens, pc, pm, seed):
    r = np.random.default_rng(seed)
    t = r.uniform(1, 50, 1 << L)
    t[r.random(1 << L) < 0.25] = np.inf
    h1, g1, t1 = oo.oo_ga_table(L, pop, gens, pc, pm, seed, t)
    h2, g2, t2 = oracle.ga(L, pop, gens, pc, pm, seed, t)
    assert np.array_equal(h1, h2)
    assert g1 == g2 and t1 == t2


def test_all_infinite():
    t = np.full(64, np.inf)
    h1, g1, t1 = oo.oo_ga_table(6, 16, 3, 0.9, 0.05, 4, t)
    h2, g2, t2 = oracle.ga(6, 16, 3, 0.9, 0.05, 4, t)
    assert np.array_equal(h1, h2) and g1 == g2 and np.isinf(t1)


def test_bad_arguments():
    with pytest.raises(oo.OOError):
        oo.oo_ga_table(6, 0, 3, 0.9, 0.05, 1, np.ones(64))
    with pytest.raises(oo.OOError):
        oo.oo_ga_table(6, 4, 3, 1.5, 0.05, 1, np.ones(64))


def test_resume_from_a_full_table_needs_no_gpu():
    """oo_ga_search_resume with every gene's time known measures nothing (a
    host-only context runs it) and makes the oracle GA's choices on that
    table; the returned table is the one given."""
    r = np.random.default_rng(21)
    t = r.uniform(1, 80, 64)
    t[r.random(64) < 0.2] = np.inf
    ctx = oo.oo_create(-1)
    try:
        res = oo.oo_ga_search(ctx, oo.jacobi(9, 9, 9, 2), 1, 16, 8, 0.9, 0.05, 77, known_ms=t)
    finally:
        oo.oo_destroy(ctx)
    h2, g2, t2 = oracle.ga(6, 16, 8, 0.9, 0.05, 77, t)
    assert np.array_equal(res["history"].reshape(-1), h2.reshape(-1))
    assert res["best_gene"] == g2 and res["best_ms"] == t2
    assert np.array_equal(res["gene_ms"], t)


def test_resume_arguments():
    ctx = oo.oo_create(-1)
    try:
        with pytest.raises(oo.OOError) as e:
            oo.oo_ga_search(ctx, oo.jacobi(9, 9, 9, 2), 1, 4, 2, 0.9, 0.05, 1, known_ms=np.zeros(64))
        assert e.value.status == oo.OO_EINVAL
        # a gene left to measure on a host-only context: no GPU to run it on
        t = np.full(64, 5.0)
        t[:] = np.nan
        with pytest.raises(oo.OOError) as e:
            oo.oo_ga_search(ctx, oo.jacobi(9, 9, 9, 2), 1, 4, 2, 0.9, 0.05, 1, known_ms=t)
        assert e.value.status == oo.OO_ESTATE
    finally:
        oo.oo_destroy(ctx)
