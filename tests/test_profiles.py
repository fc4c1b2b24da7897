"""The committed ncu summaries stay usable: the stencil's recorded DRAM
traffic and the FFT's instruction count belong to the current sources (else
the benchmark line would carry no traffic figure or FFT roofline), and
every summary gives the ncu command that made it, with the GPU clocks left
alone."""
import glob
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_stencil_traffic_matches_current_sources():
    nbytes = bench.stencil_traffic()
    assert nbytes is not None, "stencil sources changed since the DRAM traffic was captured"
    algorithmic = bench.STENCIL_BYTES
    assert algorithmic <= nbytes <= 1.10 * algorithmic


def test_fft_instructions_match_current_sources():
    """The FFT's issue roofline takes its instruction count from the
    committed summary of the same sources."""
    r = bench.fft_issue_roofline(0.2, 152)
    assert r is not None, "FFT sources changed since the instruction count was captured"
    # two passes of 2^22 points, a few hundred thread instructions per point each
    assert 2 * 400 * (1 << 22) / 32 < r["warp_instructions_per_transform"] < 2 * 800 * (1 << 22) / 32


def test_every_summary_records_its_ncu_command():
    paths = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))
    assert paths
    for p in paths:
        text = open(p).read().replace("\\\n", " ")  # join continued lines
        cmds = [line for line in text.splitlines() if re.match(r"\s*ncu ", line)]
        assert cmds, p
        for c in cmds:
            assert "--clock-control none" in c, (p, c)
