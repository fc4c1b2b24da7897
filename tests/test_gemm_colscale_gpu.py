"""Column scales of the split-BF16 matrix product (Sec. 3.2.2 function
block).  A column of B whose largest entry lies in [2^-20, 2^40) is split
unscaled in the same pass that finds its largest exponent; any other column
is split again with the power of two that brings its largest entry into
[1/2, 1).  Columns on both sides of that window go through every split path
-- the one-pass strips (even leading dimension), the two-pass fallback (odd
leading dimension), CTA pairs and single CTAs, the grouped batch -- and
must give the same bits in all of them and stay within the pattern's bound
(1e-4 of sum |a||b|) against the FP64 Dot2 oracle."""
import numpy as np
import pytest

import oracle
from paper_2011_03602_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPLIT3_TOL = 1e-4
# exponents e of the columns' largest entries (1.5 * 2^e): inside and
# outside [2^-20, 2^40), and on both edges
EDGES = [-300, -60, -25, -21, -20, -19, -1, 0, 1, 38, 39, 40, 41, 90, 700]


@pytest.fixture(scope="module")
def oo_mod():
    from paper_2011_03602_gb300 import build as pkg_build
    from paper_2011_03602_gb300 import oo
    pkg_build.build()
    return oo


@pytest.fixture(scope="module")
def ctxs(oo_mod):
    pair, single = oo_mod.oo_create(0), oo_mod.oo_create(0)
    oo_mod.oo_set_option(single, oo_mod.OO_OPT_GEMM_PAIR, 0)
    yield pair, single
    oo_mod.oo_destroy(pair)
    oo_mod.oo_destroy(single)


def edge_columns(seed, k, n, shift=0):
    """k x n uniform entries, column j rescaled so that its largest magnitude
    is 1.5 * 2^EDGES[(j + shift) mod len]."""
    B = synth.gemm_matrix(seed, k, n)
    e = np.array([EDGES[(j + shift) % len(EDGES)] for j in range(n)], dtype=float)
    return B / np.max(np.abs(B), axis=0) * (1.5 * np.exp2(e))


def err_metric(C, ref, A, B):
    return np.max(np.abs(C - ref) / np.maximum(np.abs(A) @ np.abs(B), 1e-300))


@pytest.mark.parametrize("m,n,k", [(64, 45, 300), (300, 257, 129), (513, 130, 1000)])
def test_window_edges_every_path(oo_mod, ctxs, m, n, k):
    pair, single = ctxs
    A = synth.gemm_matrix(m + 5, m, k)
    B = edge_columns(n + 7, k, n)
    ref = oracle.gemm(A, B)
    Cp = oo_mod.oo_gemm_f64(pair, A, B)      # one-pass strips, CTA pairs
    Cs = oo_mod.oo_gemm_f64(single, A, B)    # one-pass strips, single CTAs
    np.testing.assert_array_equal(Cp, Cs)
    assert err_metric(Cp, ref, A, B) <= SPLIT3_TOL
    # odd leading dimension of B: column maxima first, then the split
    ldb = n + 1 if n % 2 == 0 else n + 2
    ldb += 1 - ldb % 2  # odd
    dA = torch.from_numpy(A).cuda()
    dB = torch.zeros(k * ldb, dtype=torch.float64, device="cuda")
    dB.view(k, ldb)[:, :n] = torch.from_numpy(B).cuda()
    dC = torch.empty((m, n), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    oo_mod.oo_gemm_f64_dev(pair, m, n, k, dA, k, dB, ldb, dC, n)
    oo_mod.oo_gemm_check(pair, m, n, k)
    np.testing.assert_array_equal(dC.cpu().numpy(), Cp)


def test_nonfinite_column_among_edges(oo_mod, ctxs):
    """A column holding an infinity sits in a strip with in-window and
    out-of-window columns: its outputs are NaN, every other output is what
    the same product without that column gives."""
    pair, _ = ctxs
    m, n, k = 90, 48, 200
    A = synth.gemm_matrix(3, m, k)
    B = edge_columns(4, k, n, shift=3)
    C0 = oo_mod.oo_gemm_f64(pair, A, B)
    B[17, 5] = np.inf
    C1 = oo_mod.oo_gemm_f64(pair, A, B)
    assert np.all(np.isnan(C1[:, 5]))
    keep = [j for j in range(n) if j != 5]
    np.testing.assert_array_equal(C1[:, keep], C0[:, keep])


def test_grouped_batch_equals_single_calls(oo_mod, ctxs):
    """Split-BF16 requests with edge columns in one batch: grouped, graph
    and one-call-per-request runs all equal the single calls' bits."""
    pair, _ = ctxs
    oo = oo_mod
    rng = np.random.default_rng(5)
    reqs, alone = [], []
    for i in range(6):
        m, n, k = (int(x) for x in rng.integers(1, 300, 3))
        A = synth.gemm_matrix(40 + i, m, k)
        B = edge_columns(50 + i, k, n, shift=i)
        alone.append(oo.oo_gemm_f64(pair, A, B))
        assert err_metric(alone[-1], oracle.gemm(A, B), A, B) <= SPLIT3_TOL
        reqs.append(dict(kind="gemm", m=m, n=n, k=k, A=torch.from_numpy(A).cuda(), B=torch.from_numpy(B).cuda(),
                         C=torch.full((m, n), np.nan, dtype=torch.float64, device="cuda")))
    torch.cuda.synchronize()
    b = oo.oo_batch_create(pair, reqs)
    try:
        for mode in (0, 1, 2):
            for r in reqs:
                r["C"].fill_(np.nan)
            torch.cuda.synchronize()  # the fills ran on torch's stream, the batch runs on the context's
            oo.oo_batch_run(pair, b, mode)
            oo.oo_batch_check(pair, b)
            for i, r in enumerate(reqs):
                np.testing.assert_array_equal(r["C"].cpu().numpy(), alone[i], err_msg="mode %d req %d" % (mode, i))
    finally:
        oo.oo_batch_destroy(b)
