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
