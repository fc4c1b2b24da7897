"""Pins for the matrix-product oracle (Sec. 3.2.2 function block)."""
import numpy as np

import oracle
from paper_2011_03602_gb300 import synth


def test_identity_and_permutation_are_exact():
    A = synth.gemm_matrix(1, 19, 23)
    assert np.array_equal(oracle.gemm(A, np.eye(23)), A)
    perm = np.random.default_rng(0).permutation(19)
    P = np.eye(19)[perm]
    assert np.array_equal(oracle.gemm(P, A), A[perm])


def test_small_integers_exact():
    r = np.random.default_rng(1)
    A = r.integers(-8, 9, (13, 40))
    B = r.integers(-8, 9, (40, 11))
    assert np.array_equal(oracle.gemm(A.astype(float), B.astype(float)), (A @ B).astype(float))


def test_compensation_recovers_cancelled_term():
    A = np.array([[1e16, 1.0, -1e16]])
    B = np.ones((3, 1))
    assert oracle.gemm(A, B)[0, 0] == 1.0          # a plain FP64 sum gives 0


def test_against_extended_precision_triple_loop():
    A = synth.gemm_matrix(2, 17, 29)
    B = synth.gemm_matrix(3, 29, 21)
    ref = A.astype(np.longdouble) @ B.astype(np.longdouble)
    C = oracle.gemm(A, B)
    err = np.abs(C.astype(np.longdouble) - ref)
    scale = np.abs(A) @ np.abs(B)
    assert np.all(err <= 2.3e-16 * np.abs(ref) + 1e-18 * scale)


def test_row_range():
    A = synth.gemm_matrix(4, 8, 5)
    B = synth.gemm_matrix(5, 5, 6)
    full = oracle.gemm(A, B)
    part = oracle.gemm(A, B, rows=(2, 5))
    assert np.array_equal(part[2:5], full[2:5]) and np.all(part[:2] == 0)
