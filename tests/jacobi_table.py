"""The Jacobi loop-nest table as the tests describe it to both the oracle and
the library: 15 variables, 6 nests (all parallelisable)."""
VARS = ["a0", "a1", "a2", "a3", "b0", "b1", "b2", "c0", "c1", "c2", "bnd", "wrk1",
        "p", "wrk2", "res"]
V = {n: i for i, n in enumerate(VARS)}
COEF = (1 << 12) - 1
P, WRK2, RES = 1 << V["p"], 1 << V["wrk2"], 1 << V["res"]

NESTS = [
    dict(name="coef", level=0, parallelisable=1, reads=0, writes=COEF, partial=0),
    dict(name="pinit", level=0, parallelisable=1, reads=0, writes=P | WRK2, partial=0),
    dict(name="stencil", level=1, parallelisable=1, reads=COEF | P, writes=WRK2 | RES, partial=WRK2),
    dict(name="copyback", level=1, parallelisable=1, reads=WRK2, writes=P, partial=P),
    dict(name="bc_ij", level=1, parallelisable=1, reads=0, writes=P, partial=P),
    dict(name="bc_k", level=1, parallelisable=1, reads=0, writes=P, partial=P),
]
OUTPUTS = P | RES


def var_bytes(I, J, K, iters):
    n = I * J * K
    return [4 * n] * 14 + [8 * iters]
