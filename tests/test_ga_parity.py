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
