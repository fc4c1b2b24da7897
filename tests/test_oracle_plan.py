"""Hand-derived transfer plans for chosen genes (Sec. 3.2.1 hoisting,
Sec. 4.2.2 transfer rules) pin the oracle's coherence walk."""
import pytest

import oracle
from jacobi_table import NESTS, OUTPUTS, V, var_bytes

I, J, K = 5, 6, 7
N4 = 4 * I * J * K


def plan(gene, hoist, iters):
    return oracle.plan(NESTS, var_bytes(I, J, K, iters), OUTPUTS, gene, hoist, iters)


@pytest.mark.parametrize("hoist", [0, 1])
def test_all_cpu_needs_no_copy(hoist):
    xs, h2d, d2h = plan(0, hoist, 5)
    assert xs == [] and h2d == 0 and d2h == 0


def test_all_gpu_hoisted_copies_results_once():
    iters = 7
    xs, h2d, d2h = plan(63, 1, iters)
    end = 2 + 4 * iters
    assert xs == [(end, V["p"], -1, N4), (end, V["res"], -1, 8 * iters)]
    assert h2d == 0 and d2h == N4 + 8 * iters


def test_stencil_only_hoisted():
    iters = 4
    xs, h2d, d2h = plan(1 << 2, 1, iters)
    expect = [(2, v, +1, N4) for v in range(14)]          # 12 coefficients, p, wrk2
    expect.append((3, V["wrk2"], -1, N4))                   # CPU copy-back reads wrk2
    for it in range(1, iters):
        expect.append((2 + 4 * it, V["p"], +1, N4))         # p changed on the host
        expect.append((3 + 4 * it, V["wrk2"], -1, N4))
    expect.append((2 + 4 * iters, V["res"], -1, 8 * iters))
    assert xs == expect
    assert h2d == (14 + iters - 1) * N4
    assert d2h == iters * N4 + 8 * iters


def test_coef_on_gpu_only_copies_coefficients_back_once():
    xs, h2d, d2h = plan(1, 1, 3)
    assert xs == [(2, v, -1, N4) for v in range(12)]
    assert h2d == 0 and d2h == 12 * N4


def test_all_gpu_unhoisted_copies_at_every_nest():
    iters = 2
    xs, h2d, d2h = plan(63, 0, iters)
    expect = [(1, v, -1, N4) for v in range(12)]            # N0 writes out
    expect += [(2, V["p"], -1, N4), (2, V["wrk2"], -1, N4)]  # N1 writes out
    for it in range(iters):
        q = 2 + 4 * it
        expect += [(q, v, +1, N4) for v in range(14)]
        expect += [(q + 1, V["wrk2"], -1, N4), (q + 1, V["res"], -1, 8 * iters)]
        expect += [(q + 1, V["p"], +1, N4), (q + 1, V["wrk2"], +1, N4), (q + 2, V["p"], -1, N4)]
        expect += [(q + 2, V["p"], +1, N4), (q + 3, V["p"], -1, N4)]
        expect += [(q + 3, V["p"], +1, N4), (q + 4, V["p"], -1, N4)]
    assert xs == expect
    assert h2d == sum(x[3] for x in expect if x[2] > 0)
    assert d2h == sum(x[3] for x in expect if x[2] < 0)


def test_gene_bits_skip_non_parallelisable_nests():
    nests = [dict(n) for n in NESTS]
    nests[1]["parallelisable"] = 0        # pinit stays on the CPU
    # gene bit 1 now belongs to the stencil nest
    a, _, _ = oracle.plan(nests, var_bytes(I, J, K, 3), OUTPUTS, 0b10, 1, 3)
    b, _, _ = plan(0b100, 1, 3)
    assert a == b


def test_hoisting_never_moves_more_bytes():
    for gene in range(64):
        _, h1, d1 = plan(gene, 1, 3)
        _, h0, d0 = plan(gene, 0, 3)
        assert h1 <= h0 and d1 <= d0, gene
