"""Function-block offload decision (Sec. 4.2.1) and trial order (Sec. 4.2):
the oracle's decision pinned by hand-made tables, the library's decision
against the oracle on random tables, and argument checks.  No GPU."""
import math

import numpy as np
import pytest

import oracle
from paper_2011_03602_gb300 import oo

INF = math.inf


def test_oracle_pins():
    # one block: offloading helps
    assert oracle.fb_best([10.0, 4.0]) == (1, 4.0)
    # one block: offloading slower (transfer-bound) -> keep the CPU code
    assert oracle.fb_best([4.0, 10.0]) == (0, 4.0)
    # result check failed for every offload -> the all-CPU program
    assert oracle.fb_best([7.0, INF, INF, INF]) == (0, 7.0)
    # two blocks: each helps alone, together best (combination measured)
    assert oracle.fb_best([10.0, 7.0, 6.0, 3.0]) == (3, 3.0)
    # two blocks: together worse than block 1 alone
    assert oracle.fb_best([10.0, 7.0, 6.0, 6.5]) == (2, 6.0)
    # ties keep the lower mask
    assert oracle.fb_best([5.0, 5.0, 5.0, 5.0]) == (0, 5.0)
    assert oracle.fb_best([9.0, 5.0, 5.0, 9.0]) == (1, 5.0)
    with pytest.raises(ValueError):
        oracle.fb_best([1.0, float("nan")])


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12])
def test_library_decision_matches_oracle(n):
    rng = np.random.default_rng(n)
    for trial in range(20):
        t = rng.integers(1, 6, 1 << n).astype(np.float64)  # many ties
        t[rng.random(t.size) < 0.3] = INF
        if trial % 5 == 0:
            t[1:] = INF
        assert oo.oo_fb_best(t) == oracle.fb_best(t)


def test_decision_rejects_bad_tables():
    with pytest.raises(oo.OOError):
        oo.oo_fb_best([1.0, float("nan")])
    with pytest.raises(ValueError):
        oo.oo_fb_best([1.0, 2.0, 3.0])


def test_trial_order_on_tables():
    """Sec. 4.2 order on given tables: the block decision, then the loop GA
    on the loop-time table; each step matches the oracle's."""
    fb = np.array([12.0, 5.0, 9.0, 4.0])
    loops = np.random.default_rng(3).uniform(1.0, 50.0, 64)
    loops[[5, 17, 40]] = INF
    assert oo.oo_fb_best(fb) == oracle.fb_best(fb)
    h1, g1, t1 = oo.oo_ga_table(6, 16, 16, 0.9, 0.05, 2011, loops)
    h2, g2, t2 = oracle.ga(6, 16, 16, 0.9, 0.05, 2011, loops)
    assert g1 == g2 and t1 == t2 and np.array_equal(h1, h2)


def test_fb_search_needs_a_device():
    ctx = oo.oo_create(-1)
    try:
        with pytest.raises(oo.OOError) as e:
            oo.oo_fb_search(ctx, [("cblas_dgemm", oo.OO_LANG_C, 1, 8, 8, 8)])
        assert e.value.status == oo.OO_ESTATE
    finally:
        oo.oo_destroy(ctx)
