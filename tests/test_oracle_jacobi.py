"""Pins for the Jacobi oracle (plain FP64 C): closed forms and hand values,
none of which re-types the oracle's own loop."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _zero_coef(I, J, K):
    return np.zeros((12, I, J, K), np.float32)


def test_hand_step_4x4x4():
    g = json.load(open(os.path.join(GOLDEN, "jacobi_4x4x4.json")))["exact_inputs"]
    coef, p = oracle.jacobi_setup(4, 4, 4)
    wrk2, res = oracle.stencil(coef, p.astype(np.float64), np.float32(0.8))
    assert res == pytest.approx(float(Fraction(g["res"])), rel=1e-6)
    assert wrk2[1, 1, 1] == pytest.approx(3.8 / 27, rel=1e-6)
    assert wrk2[2, 2, 2] == pytest.approx(12.8 / 27, rel=1e-6)
    # boundary points are untouched
    assert wrk2[0, 1, 1] == p[0, 1, 1]
    # the whole-program routine gives the same first residual
    r, _ = oracle.jacobi_run(4, 4, 4, 1)
    assert r[0] == res


@pytest.mark.parametrize("arr,delta", [(0, 1.0), (1, 10.0), (2, 100.0),
                                       (7, -1.0), (8, -10.0), (9, -100.0)])
def test_direct_terms_hit_the_right_neighbour(arr, delta):
    # p = i + 10 j + 100 k: each direct coefficient alone (a3 = bnd = 1) gives
    # ss = neighbour - p = +-1 (i), +-10 (j), +-100 (k).
    I, J, K = 5, 6, 7
    i, j, k = np.meshgrid(np.arange(I), np.arange(J), np.arange(K), indexing="ij")
    p = (i + 10 * j + 100 * k).astype(np.float32)
    coef = _zero_coef(I, J, K)
    coef[arr] = 1.0
    coef[3] = 1.0
    coef[10] = 1.0
    wrk2, res = oracle.stencil(coef, p.astype(np.float64), 0.5)
    nint = (I - 2) * (J - 2) * (K - 2)
    assert res == nint * delta * delta
    assert np.all(wrk2[1:-1, 1:-1, 1:-1] - p[1:-1, 1:-1, 1:-1] == 0.5 * delta)


@pytest.mark.parametrize("field,expect", [("ij", (4, 0, 0)), ("jk", (0, 4, 0)), ("ik", (0, 0, 4))])
def test_cross_terms_plane_and_sign(field, expect):
    # bilinear p = u v has cross difference exactly 4 in the (u, v) plane and 0
    # in the other two; wrk1 = p cancels the -p so ss = X.
    I, J, K = 6, 5, 7
    i, j, k = np.meshgrid(np.arange(I), np.arange(J), np.arange(K), indexing="ij")
    u, v = {"ij": (i, j), "jk": (j, k), "ik": (i, k)}[field]
    p = (u * v).astype(np.float32)
    nint = (I - 2) * (J - 2) * (K - 2)
    for b in range(3):
        coef = _zero_coef(I, J, K)
        coef[4 + b] = 1.0
        coef[3] = 1.0
        coef[10] = 1.0
        coef[11] = p
        _, res = oracle.stencil(coef, p.astype(np.float64), 1.0)
        assert res == nint * expect[b] ** 2, (field, b)


def test_bnd_and_omega_scale():
    I, J, K = 5, 5, 5
    i, j, k = np.meshgrid(np.arange(I), np.arange(J), np.arange(K), indexing="ij")
    p = (i + 10 * j + 100 * k).astype(np.float32)
    coef = _zero_coef(I, J, K)
    coef[0] = 1.0
    coef[3] = 1.0
    coef[10] = 2.0  # bnd doubles ss
    wrk2, res = oracle.stencil(coef, p.astype(np.float64), 0.25)
    assert res == 27 * 4.0
    assert np.all(wrk2[1:-1, 1:-1, 1:-1] - p[1:-1, 1:-1, 1:-1] == 0.5)


def _closed_form_first_residual(I, J, K):
    # p = g(k) depends on k only: s0 = 4 g(k) + g(k+1) + g(k-1) at every
    # interior point; evaluated in exact rationals from the float inputs.
    a3 = Fraction(float(np.float32(1.0 / 6.0)))
    g = [Fraction(float(np.float32(Fraction(kk * kk, (K - 1) ** 2)))) for kk in range(K)]
    tot = Fraction(0)
    for kk in range(1, K - 1):
        ss = a3 * (4 * g[kk] + g[kk + 1] + g[kk - 1]) - g[kk]
        tot += ss * ss
    return float(tot * (I - 2) * (J - 2))


@pytest.mark.parametrize("shape", [(4, 4, 4), (5, 7, 9), (33, 33, 65)])
def test_first_residual_closed_form(shape):
    res, _ = oracle.jacobi_run(*shape, iters=1, want_p=False)
    assert res[0] == pytest.approx(_closed_form_first_residual(*shape), rel=1e-10)


def test_first_residual_matches_continuum_value():
    # With exact 1/6 the residual is Nint / (9 (K-1)^4); the float a3 moves it
    # by ~2.4e-4 relative at 33x33x65 (measured here, stated in the design notes).
    I, J, K = 33, 33, 65
    cont = (I - 2) * (J - 2) * (K - 2) / (9.0 * (K - 1) ** 4)
    res, _ = oracle.jacobi_run(I, J, K, iters=1, want_p=False)
    assert res[0] == pytest.approx(cont, rel=5e-4)


def test_constant_field_fixed_point():
    I, J, K = 6, 7, 8
    coef, _ = oracle.jacobi_setup(I, J, K)
    c = 0.5
    p = np.full((I, J, K), c, np.float64)
    wrk2, res = oracle.stencil(coef, p, np.float32(0.8))
    # 6 c a3 - c is below half an ulp of c, so the stored value stays c
    assert np.all(wrk2.astype(np.float32) == np.float32(c))
    a3 = Fraction(float(np.float32(1.0 / 6.0)))
    ss = Fraction(c) * (6 * a3 - 1)
    assert res == pytest.approx(float(ss * ss * (I - 2) * (J - 2) * (K - 2)), rel=1e-12)


def test_program_keeps_dirichlet_faces():
    I, J, K = 7, 6, 9
    rng = np.random.default_rng(0)
    p0 = rng.random((I, J, K)).astype(np.float32)
    res, p = oracle.jacobi_run(I, J, K, iters=3, p0=p0)
    g = np.array([np.float32(kk * kk / (K - 1) ** 2) for kk in range(K)], np.float64)
    for face in (p[0], p[-1], p[:, 0], p[:, -1]):
        assert np.all(face == g[None, :])
    assert np.all(p[:, :, 0] == g[0]) and np.all(p[:, :, -1] == g[-1])


def test_float_store_mode_rounds_every_store():
    res32, p32 = oracle.jacobi_run(9, 8, 11, iters=4, mode=1)
    assert np.all(p32.astype(np.float32).astype(np.float64) == p32)
    res64, p64 = oracle.jacobi_run(9, 8, 11, iters=4, mode=0)
    assert not np.all(p64.astype(np.float32).astype(np.float64) == p64)
    np.testing.assert_allclose(res32, res64, rtol=1e-4)


def test_storage_modes_agree_at_small_config():
    # FP64 storage vs float storage at 33x33x65 x 50 iterations: the stated
    # float-residual tolerance is met between the two oracle modes.
    r32, _ = oracle.jacobi_run(33, 33, 65, 50, mode=1, want_p=False)
    r64, _ = oracle.jacobi_run(33, 33, 65, 50, mode=0, want_p=False)
    assert np.max(np.abs(r32 - r64) / r64) < 1e-5
