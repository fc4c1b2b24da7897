"""Library transfer planner vs the oracle's coherence walk: bit-exact
records and byte totals for every gene, both hoist modes."""
import numpy as np
import pytest

import oracle
from jacobi_table import NESTS, OUTPUTS, var_bytes
from paper_2011_03602_gb300 import build as pkg_build
from paper_2011_03602_gb300 import oo


@pytest.fixture(scope="module")
def ctx():
    pkg_build.build()
    c = oo.oo_create(-1)
    yield c
    oo.oo_destroy(c)


@pytest.mark.parametrize("iters", [0, 1, 3])
@pytest.mark.parametrize("hoist", [0, 1])
def test_jacobi_plans_match_oracle(ctx, iters, hoist):
    I, J, K = 7, 9, 11
    assert oo.oo_load_jacobi_nests(ctx, I, J, K, iters) == 6
    for gene in range(64):
        got = oo.oo_transfer_plan(ctx, gene, hoist, iters)
        exp = oracle.plan(NESTS, var_bytes(I, J, K, iters), OUTPUTS, gene, hoist, iters)
        assert got == exp, gene


def test_generic_tables_match_oracle(ctx):
    rng = np.random.default_rng(5)
    for trial in range(40):
        nv = int(rng.integers(1, 10))
        nn = int(rng.integers(1, 8))
        nests = []
        for n in range(nn):
            w = int(rng.integers(0, 1 << nv))
            nests.append(dict(level=int(rng.integers(0, 2)), parallelisable=int(rng.random() < 0.8),
                              reads=int(rng.integers(0, 1 << nv)), writes=w,
                              partial=w & int(rng.integers(0, 1 << nv))))
        vb = [int(x) for x in rng.integers(1, 1000, nv)]
        outputs = int(rng.integers(0, 1 << nv))
        L = oo.oo_load_nests(ctx, nests, vb, outputs)
        assert L == sum(n["parallelisable"] for n in nests)
        iters = int(rng.integers(0, 4))
        for gene in range(1 << L):
            for hoist in (0, 1):
                got = oo.oo_transfer_plan(ctx, gene, hoist, iters)
                exp = oracle.plan(nests, vb, outputs, gene, hoist, iters)
                assert got == exp, (trial, gene, hoist)


def test_gene_beyond_length_rejected(ctx):
    oo.oo_load_jacobi_nests(ctx, 5, 5, 5, 1)
    with pytest.raises(oo.OOError):
        oo.oo_transfer_plan(ctx, 64, 1, 1)
