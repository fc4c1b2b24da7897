"""Front-ends over the one C ABI (Sec. 4.3): the C client program builds on
the CPU; on a GPU it runs end to end (lookup, pattern, GEMM, FFT, serving
from three threads) and its numbers agree with the oracle."""
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2011_03602_gb300 import build as pkg_build

HERE = os.path.dirname(os.path.abspath(__file__))


def test_c_client_builds():
    exe = pkg_build.build_c_client()
    assert os.access(exe, os.X_OK)


def test_java_shim_sources_present():
    jdir = os.path.join(os.path.dirname(pkg_build.__file__), "frontends", "java")
    assert os.path.exists(os.path.join(jdir, "OoNative.java"))
    src = open(os.path.join(jdir, "oo_jni.c")).read()
    for fn in ("oo_create", "oo_gemm_f64", "oo_fft_c128", "oo_run_pattern", "oo_submit", "oo_wait"):
        assert fn in src


@pytest.mark.gpu
def test_c_client_runs():
    exe = pkg_build.build_c_client()
    out = subprocess.run([exe, "0"], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    lines = {l.split()[0]: l.split()[1:] for l in out.stdout.strip().splitlines()}
    assert lines["lookup"] == ["1", "2"]
    ref_res, _ = oracle.jacobi_run(33, 33, 65, 10, mode=1, want_p=False)
    assert abs(float(lines["pattern"][0]) - ref_res[0]) <= 1e-9 * ref_res[0]
    assert abs(float(lines["pattern"][1]) - ref_res[-1]) <= 1e-9 * ref_res[-1]
    assert float(lines["gemm_identity_maxerr"][0]) < 1e-4
    assert abs(float(lines["fft_tone"][0]) - 4096.0) < 1e-9 and float(lines["fft_tone"][1]) < 1e-9
    assert lines["serve"][0] == "1" and lines["serve"][1] == "24"
    assert "done" in lines


def test_c_load_generator_builds_and_exports():
    import ctypes
    lib = ctypes.CDLL(pkg_build.build_loadgen())
    assert hasattr(lib, "oo_load_run")


@pytest.mark.gpu
def test_c_load_generator_matches_ctypes_results():
    """The C serving client (run in-process, as the serve benchmark runs it)
    gets the same bits as the ctypes client for the same requests, tagged as
    the C front end."""
    import ctypes
    import time

    import bench
    from paper_2011_03602_gb300 import oo, synth
    cgen = ctypes.CDLL(pkg_build.build_loadgen())
    cgen.oo_load_run.restype = ctypes.c_int
    cgen.oo_load_run.argtypes = [ctypes.c_void_p, ctypes.POINTER(bench._CLoadPools),
                                 ctypes.POINTER(bench._CLoadItem), ctypes.c_int, ctypes.POINTER(bench._CLoadResult)]
    A, B = synth.gemm_matrix(1, 128, 128), synth.gemm_matrix(2, 128, 128)
    x = synth.complex_normal(3, 1 << 12)
    P = bench._CLoadPools()
    P.gemm_a[0], P.gemm_b[0], P.gemm_n[0] = A.ctypes.data, B.ctypes.data, 128
    P.fft_x[0], P.fft_log2[0] = x.ctypes.data, 12
    P.jac_i[0], P.jac_j[0], P.jac_k[0] = 9, 10, 11
    P.jac_iters, P.prec, P.client, P.max_in_flight = 5, oo.OO_PREC_FP64EQ, oo.OO_LANG_C, 4
    kinds = [oo.OO_BLOCK_GEMM, oo.OO_BLOCK_FFT, oo.OO_BLOCK_JACOBI] * 3
    items = (bench._CLoadItem * len(kinds))()
    now = time.perf_counter()
    for i, k in enumerate(kinds):
        items[i].kind, items[i].size, items[i].arrival = k, 0, now + 0.001 * i
    res = (bench._CLoadResult * len(kinds))()
    ctx = oo.oo_create(0)
    try:
        for start in (lambda: oo.oo_serve_start(ctx, slots=2, hbm_budget_bytes=512 << 20, queue_cap=64),
                      lambda: oo.oo_serve_start_resident(ctx, 512 << 20, 64)):
            start()
            assert cgen.oo_load_run(ctx, ctypes.byref(P), items, len(kinds), res) == 0
            C, X = np.empty((128, 128)), np.empty_like(x)
            p, r = np.empty(990, np.float32), np.empty(5)
            for kind, kw in (("gemm", dict(A=A, B=B, C=C)), ("fft", dict(x=x, X=X, dir=-1)),
                             ("jacobi", dict(I=9, J=10, K=11, iters=5, p=p, res=r))):
                oo.oo_wait(ctx, oo.oo_submit(ctx, oo.serve_request(kind, **kw)), 60000)
            want = [bench._digest64([C]), bench._digest64([X]), bench._digest64([p, r])]
            oo.oo_serve_stop(ctx)
            for i in range(len(kinds)):
                assert res[i].status == 0
                assert (res[i].digest_xor, res[i].digest_sum) == want[i % 3]
    finally:
        oo.oo_destroy(ctx)
