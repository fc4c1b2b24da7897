"""Benchmark of the offload-pattern hot path on GB300.

Workload: the 19-point Jacobi program on a 257 x 257 x 513 float grid,
200 iterations, all six loop nests offloaded (gene 0b111111) with hoisted
transfers -- the configuration the GA search at scale runs on.  One step is
one whole pattern run (setup nests + 200 x [stencil, copy-back, two boundary
nests]).  Metric: effective HBM GB/s of the pattern = algorithmic bytes of
all nests / step time (stencil 56 B, copy-back 8 B per interior point and
iteration; setup 56 B per point; faces 4 B per face point and iteration).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 C oracle (test infrastructure) on the host
cores on a bounded sample of the same workload.
"""
import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

I, J, K, ITERS = 257, 257, 513, 200
GENE, HOIST = 0b111111, 1
METRIC = "stencil GB/s; GEMM/FFT solves/s; p50/p99 served vs plain offload at stated tol"
WORKLOAD = "jacobi19_257x257x513_it200_gene63_hoist"


def nint(i=None, j=None, k=None):
    i, j, k = i or I, j or J, k or K
    return (i - 2) * (j - 2) * (k - 2)


def pattern_bytes(i=None, j=None, k=None, iters=None):
    """Algorithmic bytes of one whole pattern run."""
    i, j, k = i or I, j or J, k or K
    iters = ITERS if iters is None else iters
    n = i * j * k
    faces = n - nint(i, j, k)
    setup = 48 * n + 8 * n
    per_iter = 56 * nint(i, j, k) + 8 * nint(i, j, k) + 4 * faces + 4 * 2 * i * j
    return setup + iters * per_iter


STENCIL_BYTES = 56 * nint()   # per stencil launch


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples (the JSON line carries their summary); directory from
        # OO_CLOCKS_DIR, else the system temporary directory
        import tempfile
        self.path = os.path.join(os.environ.get("OO_CLOCKS_DIR", tempfile.gettempdir()),
                                 "clocks_bench_%d.csv" % index)

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[4:]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        loaded = [r for r in rows if r[2] > 250.0] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in loaded for i, v in enumerate(r[3][1:5]) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(loaded), "reasons": reasons}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_max(pg, seconds, device):
    """Slowest rank's duration.  Every rank runs the same independent replica
    (patterns, GEMMs, FFTs and requests are independent problems: no
    data-path collective), so whole-job throughput is world_size x the
    per-rank work divided by this."""
    if pg is None:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def oracle_sample(iters):
    """The oracle as it stands on a bounded sample: the whole program at full
    grid size for `iters` iterations, single-threaded FP64 C."""
    import oracle
    t0 = time.perf_counter()
    oracle.jacobi_run(I, J, K, iters, mode=1, want_p=False)
    dt = time.perf_counter() - t0
    return pattern_bytes(iters=iters) / dt / 1e9, dt


def _oracle_replica(iters):
    """One process's share of the all-core baseline (0 iterations: only load
    the oracle library)."""
    import oracle
    if iters > 0:
        oracle.jacobi_run(I, J, K, iters, mode=1, want_p=False)
    return 0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def replica_procs():
    """Processes for the all-core baseline: one per host core, as many as fit
    in half the available memory (each holds the whole program, 2.3 GB)."""
    need = 68 * I * J * K + (1 << 28)  # the oracle: 13 float arrays and 2 double arrays
    avail = None
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    n = host_cores()
    if avail:
        n = max(1, min(n, avail // 2 // need))
    return n


class OraclePool:
    """All host cores running the oracle as it stands: independent replicas
    of the same bounded sample, one process each (started with spawn, so no
    process is forked from one that has touched the GPU).  Throughput = the
    replicas' algorithmic bytes / the wall time of the slowest."""

    def __init__(self, procs):
        import multiprocessing as mp
        self.procs = procs
        self.pool = mp.get_context("spawn").Pool(procs)
        self.pool.map(_oracle_replica, [0] * procs)

    def sample(self, iters):
        t0 = time.perf_counter()
        self.pool.map(_oracle_replica, [iters] * self.procs, chunksize=1)
        dt = time.perf_counter() - t0
        return self.procs * pattern_bytes(iters=iters) / dt / 1e9, dt

    def close(self):
        self.pool.close()
        self.pool.join()


def bench_config(ws):
    """The workload's config, the same in both arms of the benchmark."""
    return {"workload": WORKLOAD, "grid": [I, J, K], "iters": ITERS, "gene": GENE, "hoist": HOIST,
            "parallelism": "replicas" if ws > 1 else "single",
            "l2": "inputs larger than L2 (2 GB working set), no flush"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    iters = 2
    pool = OraclePool(replica_procs())
    try:
        for _ in range(args.warmup):
            pool.sample(iters)
        times = []
        for _ in range(args.steps):
            times.append(pool.sample(iters)[1])
    finally:
        pool.close()
    value = len(times) * pool.procs * pattern_bytes(iters=iters) / sum(times) / 1e9
    sample = ("%d independent replicas (one process per host core, %s) of the whole program on the %dx%dx%d "
              "grid for %d of %d iterations per step, FP64 C oracle" % (pool.procs, cpu_model(), I, J, K,
                                                                         iters, ITERS))
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * sum(times) / len(times), 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(ws),
            "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": pool.procs, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


STENCIL_SECTIONS = (  # (first line, line after) of the stencil's sources in csrc/jacobi.cu
    ("// ===================================================================== helpers",
     "// ============================================================ simple nests"),
    ("// ================================================================== stencil",
     "void attach_scratch("),
)


def stencil_sources_hash():
    """Hash of what the stencil kernel is built and launched from: ff.cuh and
    the helper and stencil sections of jacobi.cu (device helpers, kernel,
    tile variants, tensor maps, work split), so edits elsewhere in the file
    leave the recorded DRAM traffic valid."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2011_03602_gb300", "csrc")
    h = hashlib.sha256()
    with open(os.path.join(csrc, "ff.cuh"), "rb") as fh:
        h.update(fh.read())
    text = open(os.path.join(csrc, "jacobi.cu")).read()
    for first, after in STENCIL_SECTIONS:
        i = text.index(first)
        h.update(text[i:text.index(after, i)].encode())
    return h.hexdigest()[:16]


def stencil_traffic():
    """DRAM bytes (read + write) of one full-size stencil launch from the
    committed ncu summary, or None when the stencil sources have changed
    since that capture (the summary records stencil_sources_hash())."""
    import re
    path = os.path.join(ROOT, "profiles", "stencil_jacobi19_257x257x513.md")
    try:
        text = open(path).read()
        nbytes = int(re.search(r"dram_bytes_per_launch: (\d+)", text).group(1))
        want = re.search(r"sources_sha256_16: ([0-9a-f]+)", text).group(1)
        have = stencil_sources_hash()
    except (OSError, AttributeError, ValueError):
        return None
    return nbytes if have == want else None


def fft_sources_hash():
    """Hash of what the FFT pass kernels are built from: ff.cuh,
    fft_device.cuh and fft.cu."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2011_03602_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("ff.cuh", "fft_device.cuh", "fft.cu"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def fft_issue_roofline(ms, sms):
    """The 2^22 FFT against its bound, instruction issue: the warp
    instructions of one transform (both passes, from the committed ncu
    summary, or None when the FFT sources have changed since that capture)
    per second of the live time, against SMs x 4 schedulers x one warp
    instruction per clock at the 2070 MHz maximum SM clock."""
    import re
    path = os.path.join(ROOT, "profiles", "fft_c128_n2e22.md")
    try:
        text = open(path).read()
        inst = int(re.search(r"warp_instructions_per_transform: (\d+)", text).group(1))
        want = re.search(r"sources_sha256_16: ([0-9a-f]+)", text).group(1)
    except (OSError, AttributeError, ValueError):
        return None
    if want != fft_sources_hash():
        return None
    achieved = inst / (ms * 1e-3)
    peak = sms * 4 * 2.07e9
    return {"bound": "issue", "unit": "warp instructions/s", "achieved": round(achieved / 1e9, 1) * 1e9,
            "peak": peak, "frac": round(achieved / peak, 4), "warp_instructions_per_transform": inst,
            "instructions_from": "profiles/fft_c128_n2e22.md (ncu, same sources)",
            "peak_note": "SMs x 4 schedulers x 1 warp instruction per clock x 2070 MHz"}


def load_bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["bf16_tflops"]), float(pk.get("bf16_tflops_sustained", pk["bf16_tflops"])), "measured"
    except Exception:
        return 1900.0, 1700.0, "fallback"


def gemm_component(oo, ctx, torch, prec, A_h, B_h, A, B, C, with_errors):
    """One n x n x n product in precision pattern prec, timed with CUDA events
    on the context's stream (splits included); error against the oracle on
    sampled rows."""
    n = A_h.shape[0]
    for _ in range(3):
        oo.oo_gemm_f64_dev(ctx, n, n, n, A, n, B, n, C, n, prec=prec)
    oo.oo_sync(ctx)
    reps = 4 if prec == oo.OO_PREC_FP64EQ else 10
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx_stream_holder[0])
    for _ in range(reps):
        oo.oo_gemm_f64_dev(ctx, n, n, n, A, n, B, n, C, n, prec=prec)
    e1.record(ctx_stream_holder[0])
    e1.synchronize()
    oo.oo_gemm_check(ctx, n, n, n)
    ms = e0.elapsed_time(e1) / reps
    peak, peak_s, src = load_bf16_peak()
    products, beta, levels, kb = oo.oo_gemm_plan(prec, n)
    tensor = products * 2 * n ** 3 / (ms * 1e-3) / 1e12
    g = {"n": n, "ms": round(ms, 4), "solves_per_s": round(1e3 / ms, 2),
         "fp64_equiv_tflops": round(2 * n ** 3 / (ms * 1e-3) / 1e12, 2),
         "tensor_tflops": round(tensor, 1), "peak_source": src}
    if prec == oo.OO_PREC_SPLIT3_TF32:
        # TF32 peak: the measured BF16 peak x the nominal dense ratio 1.1 / 2.25 PFLOP/s
        tpeak = peak * 1.1 / 2.25
        g.update({"tf32_products": products, "peak_tf32_tflops": round(tpeak, 1),
                  "peak_note": "measured BF16 peak x nominal TF32/BF16 ratio (1.1 / 2.25)",
                  "frac_of_tf32_peak": round(tensor / tpeak, 4), "precision": "split3_tf32"})
    else:
        g.update({"bf16_products": products, "peak_bf16_tflops": peak, "frac_of_bf16_peak": round(tensor / peak, 4),
                  "precision": "split3_bf16" if prec == oo.OO_PREC_SPLIT3_BF16 else
                  "fp64eq_ozaki_bf16_beta%d_L%d_kblock%d" % (beta, levels, kb)})
    if with_errors:
        import oracle
        Ch = C.cpu().numpy()
        rows = [0, 1234, 4095]
        errs = []
        for r in rows:
            ref = oracle.gemm(A_h[r:r + 1], B_h)[0]
            errs.append(float(np.max(np.abs(Ch[r] - ref) / (np.abs(A_h[r]) @ np.abs(B_h)))))
        g["max_err_vs_oracle"] = max(errs)
        g["err_metric"] = "max |C-C*| / (|A||B|) over rows %s" % rows
    return g


def bench_blocks(oo, ctx, torch, with_errors=True):
    """Function blocks (Sec. 3.2.2): the GEMM at n = 4096 in both precision
    patterns (split-BF16 and FP64-equivalent) and the complex128 FFT at
    N = 2^22, device-resident inputs, CUDA events on the context's stream;
    errors against the oracle on a bounded sample."""
    from paper_2011_03602_gb300 import synth
    out = {}
    n = 4096
    A_h, B_h = synth.gemm_matrix(41, n, n), synth.gemm_matrix(42, n, n)
    A, B = torch.from_numpy(A_h).cuda(), torch.from_numpy(B_h).cuda()
    C = torch.empty(n, n, dtype=torch.float64, device="cuda")
    out["gemm"] = gemm_component(oo, ctx, torch, oo.OO_PREC_SPLIT3_BF16, A_h, B_h, A, B, C, with_errors)
    out["gemm"]["kernel"] = "CTA pairs (cta_group::2), 256-row tiles, width chosen per problem (224 at n = 4096)"
    # the same product on single CTAs (128x128 tiles), same inputs: context
    oo.oo_set_option(ctx, oo.OO_OPT_GEMM_PAIR, 0)
    single = gemm_component(oo, ctx, torch, oo.OO_PREC_SPLIT3_BF16, A_h, B_h, A, B, C, False)
    oo.oo_set_option(ctx, oo.OO_OPT_GEMM_PAIR, 1)
    out["gemm"]["single_cta_128x128"] = {k: single[k] for k in ("ms", "tensor_tflops", "frac_of_bf16_peak")}
    out["gemm_fp64eq"] = gemm_component(oo, ctx, torch, oo.OO_PREC_FP64EQ, A_h, B_h, A, B, C, with_errors)
    out["gemm_fp64eq"]["kernel"] = "CTA pairs (cta_group::2), 256x128 tiles"
    oo.oo_set_option(ctx, oo.OO_OPT_GEMM_PAIR, 0)
    single = gemm_component(oo, ctx, torch, oo.OO_PREC_FP64EQ, A_h, B_h, A, B, C, False)
    oo.oo_set_option(ctx, oo.OO_OPT_GEMM_PAIR, 1)
    out["gemm_fp64eq"]["single_cta_128x128"] = {k: single[k] for k in ("ms", "tensor_tflops", "frac_of_bf16_peak")}
    out["gemm_tf32"] = gemm_component(oo, ctx, torch, oo.OO_PREC_SPLIT3_TF32, A_h, B_h, A, B, C, with_errors)
    del A, B, C
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    logn = 22
    N = 1 << logn
    x_h = synth.complex_normal(43, N)
    x = torch.from_numpy(x_h.view(np.float64).copy()).cuda()
    y = torch.empty_like(x)
    for _ in range(3):
        oo.oo_fft_c128_dev(ctx, N, 1, -1, x, y)
    oo.oo_sync(ctx)
    reps = 20
    e0.record(ctx_stream_holder[0])
    for _ in range(reps):
        oo.oo_fft_c128_dev(ctx, N, 1, -1, x, y)
    e1.record(ctx_stream_holder[0])
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    f = {"n": N, "ms": round(ms, 4), "solves_per_s": round(1e3 / ms, 1),
         "GBps_two_pass_traffic": round(4 * 16 * N / (ms * 1e-3) / 1e9, 1), "precision": "float-float",
         # 5 N log2 N, the usual FFT operation count, against the FP64 rate
         # the float-float arithmetic stands in for (1.25 TFLOP/s nominal)
         "fp64_equiv_tflops": round(5.0 * N * logn / (ms * 1e-3) / 1e12, 3),
         "fp64_nominal_tflops": 1.25,
         "roofline": fft_issue_roofline(ms, torch.cuda.get_device_properties(0).multi_processor_count)}
    if with_errors:
        import oracle
        yh = y.cpu().numpy().view(np.complex128)
        ref = oracle.fft(x_h)
        f["rel_l2_err_vs_oracle"] = float(np.linalg.norm(yh - ref) / np.linalg.norm(ref))
    out["fft"] = f
    return out


ctx_stream_holder = [None]


def run_gpu(args):
    import torch
    from paper_2011_03602_gb300 import oo

    ws, rank, local = dist_env()
    dev = local if ws > 1 else 0
    torch.cuda.set_device(dev)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", dev))
        pg = dist
    stream = torch.cuda.Stream()
    ctx_stream_holder[0] = stream
    ctx = oo.oo_create(dev, stream)
    prob = oo.jacobi(I, J, K, ITERS)
    p_dev = torch.empty(I * J * K, dtype=torch.float32, device="cuda")
    r_dev = torch.empty(ITERS, dtype=torch.float64, device="cuda")

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    # warm-up (also allocates the workspace)
    for _ in range(max(args.warmup, 3)):
        oo.oo_run_pattern_dev(ctx, GENE, HOIST, prob, p_dev, r_dev)

    # ---- timed region: device-resident outputs
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(dev)
    with sampler:
        barrier()
        e0.record(stream)
        launches = 0
        for _ in range(args.steps):
            launches += oo.oo_run_pattern_dev(ctx, GENE, HOIST, prob, p_dev, r_dev)["n_launches"]
        e1.record(stream)
        barrier()
    ms = replica_max(pg, e0.elapsed_time(e1), "cuda")
    ms_step = ms / args.steps
    value = ws * pattern_bytes() / (ms_step * 1e-3) / 1e9
    res_check = r_dev.cpu().numpy()

    # ---- per-kernel durations with CUDA events on the launching stream
    st = oo.oo_run_pattern_dev(ctx, GENE, HOIST, oo.jacobi(I, J, K, ITERS, timing=True), p_dev, r_dev)
    stencil_ms = st["nest_ms"][2] / ITERS
    copy_ms = st["nest_ms"][3] / ITERS
    peak, peak_src = load_peaks()
    achieved = STENCIL_BYTES / (stencil_ms * 1e-3) / 1e9

    # ---- end to end through the C ABI with (pinned) host buffers
    p_pin = torch.empty(I * J * K, dtype=torch.float32, pin_memory=True)
    r_pin = torch.empty(ITERS, dtype=torch.float64, pin_memory=True)
    p_host, r_host = p_pin.numpy(), r_pin.numpy()
    oo.oo_run_pattern(ctx, GENE, HOIST, prob, p_host, r_host)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oo.oo_run_pattern(ctx, GENE, HOIST, prob, p_host, r_host)
    e2e_s = replica_max(pg, time.perf_counter() - t0, "cuda")
    e2e = ws * pattern_bytes() * args.steps / e2e_s / 1e9
    blocks = None
    if not args.no_blocks:
        blocks = bench_blocks(oo, ctx, torch, with_errors=(rank == 0 and not args.no_cpu_baseline))
    oo.oo_destroy(ctx)
    if blocks is not None and ws == 1 and not args.no_systems:
        blocks.update(bench_systems(args))

    if rank == 0:
        cpu = None
        if ws == 1 and not args.no_cpu_baseline:
            v1, dt1 = oracle_sample(2)
            pool = OraclePool(replica_procs())
            try:
                v, dt = pool.sample(2)
            finally:
                pool.close()
            cpu = {"value": round(v, 4), "unit": "GB/s", "cores": pool.procs, "kind": "oracle",
                   "sample": "%d independent replicas (one process per host core, %s) of the whole program on "
                             "the %dx%dx%d grid for 2 of %d iterations, FP64 C oracle, %.1f s"
                             % (pool.procs, cpu_model(), I, J, K, ITERS, dt),
                   "single_core": {"value": round(v1, 4), "unit": "GB/s", "cores": 1, "seconds": round(dt1, 2)}}
        traffic = stencil_traffic() if (I, J, K) == (257, 257, 513) else None
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": bench_config(ws),
            "roofline": {"bound": "hbm", "kernel": "stencil (nest N2)",
                         "achieved": round(achieved, 1), "peak": peak, "peak_source": peak_src,
                         "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                         "stencil_ms": round(stencil_ms, 5), "copyback_ms": round(copy_ms, 5)},
            "cpu_baseline": cpu,
            "e2e": {"value": round(e2e, 2), "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 4 * I * J * K + 8 * ITERS},
            "gpu_launches": launches,
            "clocks": sampler.summary(),
            "residual_last": float(res_check[-1]),
            "components": blocks,
        }
        print(json.dumps(line))
    if pg is not None:
        pg.destroy_process_group()
    return 0


def bench_systems(args):
    """The batched and served configurations in compact form, for the default
    line: the 4096 FP64-equivalent GEMMs + 2048 FFTs as one graph replay, as
    grouped launches and as one call per request (3 timed runs each, every
    16th result against the oracle), and the served mix at 2000 req/s
    offered for 0.5 s through both serving loops beside the plain one call
    per solve (first result of each kind and size against the oracle, every
    other result's digest against it).  A failure is reported in place of
    the figures."""
    out = {}
    try:
        b = measure_batched(4096, 2048, "fp64eq", [2, 0, 1], steps=3, warmup=2,
                            check=not args.no_cpu_baseline, check_stride=16)
        out["batched"] = {"workload": b["config"]["workload"], "precision": b["config"]["precision"],
                          "solves_per_s": b["value"], "modes": b["modes"],
                          "speedup_graph_vs_per_call": b["speedup_graph_vs_per_call"], "errors": b["errors"]}
    except Exception as e:  # reported, not hidden: the line names what failed
        out["batched"] = {"failed": repr(e)}
    try:
        ns = argparse.Namespace(**vars(args))
        ns.serve_rates, ns.serve_window, ns.serve_modes, ns.serve_prec = "2000", 0.5, "resident,host", "fp64eq"
        s = measure_serve(ns)
        out["serve"] = {"workload": s["config"]["workload"], "gemm_precision": s["config"]["gemm_precision"],
                        "offered_req_per_s": 2000, "window_s": 0.5,
                        "resident_loop": s["served"][0], "host_loop": s["served_other_loops"]["host"][0],
                        "plain_one_call_per_solve": s["plain_one_call_per_solve"],
                        "failed_requests": s["failed"],
                        "max_error_per_result_vs_oracle": s["max_error_per_result_vs_oracle"],
                        "java_share": s["config"]["front_ends"]["java_share_via_ctypes"]}
    except Exception as e:
        out["serve"] = {"failed": repr(e)}
    return out


def run_ga(args):
    """GA loop-offload search at scale (Sec. 4.2.2): the Jacobi program on the
    257 x 257 x 513 grid, 200 iterations, population 16, 16 generations,
    roulette selection, crossover 0.9, mutation 0.05; fitness from the
    measured run time with transfer hoisting on and off.  Evaluations slower
    than --ga-timeout-ms are cut off and count as failed (fitness 0)."""
    import torch
    from paper_2011_03602_gb300 import oo
    torch.cuda.set_device(0)
    ctx = oo.oo_create(0)
    prob = oo.jacobi(I, J, K, ITERS)
    out = {"metric": "GA offload-pattern search", "config": {"workload": WORKLOAD.replace("_gene63_hoist", ""),
           "grid": [I, J, K], "iters": ITERS, "pop": 16, "gens": 16, "pc": 0.9, "pm": 0.05,
           "seed": args.ga_seed, "eval_timeout_ms": args.ga_timeout_ms}}
    t0 = time.perf_counter()
    for hoist in (1, 0):
        t1 = time.perf_counter()
        r = oo.oo_ga_search(ctx, prob, hoist, 16, 16, 0.9, 0.05, args.ga_seed, args.ga_timeout_ms)
        gm = r["gene_ms"]
        measured = {int(g): float(gm[g]) for g in range(64) if np.isfinite(gm[g])}
        out["hoist_%s" % ("on" if hoist else "off")] = {
            "best_gene": int(r["best_gene"]), "best_gene_bits": format(int(r["best_gene"]), "06b"),
            "best_ms": float(r["best_ms"]), "distinct_genes_measured": int(np.sum(gm < np.inf)),
            "genes_cut_or_failed": int(len(set(int(x) for x in r["history"].reshape(-1))) - len(measured)),
            "all_gpu_ms": measured.get(63), "search_s": round(time.perf_counter() - t1, 1)}
    st = oo.oo_run_pattern(ctx, 0, 1, prob, np.empty(I * J * K, np.float32), np.empty(ITERS))
    out["all_cpu_ms"] = st["wall_ms"]
    out["total_s"] = round(time.perf_counter() - t0, 1)
    oo.oo_destroy(ctx)
    print(json.dumps(out))
    return 0


def run_fb(args):
    """Sec. 4.2 trial order at scale: function-block offload first (every
    combination of the known call sites of a C / Python / Java program,
    FP64-equivalent GEMM, result gate 1e-10), then the loop GA on the
    Jacobi program's nests (hoisting on).  Reports the measured table, the
    chosen pattern and the all-CPU time of the same program."""
    import torch
    from paper_2011_03602_gb300 import oo
    torch.cuda.set_device(0)
    ctx = oo.oo_create(0)
    sites = [("cblas_dgemm", oo.OO_LANG_C, 2, 2048, 2048, 2048),
             ("numpy.fft.fft", oo.OO_LANG_PYTHON, 4, 0, 1 << 20, 0),
             ("org.jtransforms.fft.DoubleFFT_1D.complexForward", oo.OO_LANG_JAVA, 8, 0, 1 << 16, 0),
             ("my_solver_step", oo.OO_LANG_C, 1, 64, 64, 64)]
    gI, gJ, gK, gIt = 129, 129, 257, 100
    prob = oo.jacobi(gI, gJ, gK, gIt)
    t0 = time.perf_counter()
    fb = oo.oo_fb_search(ctx, sites, prec=oo.OO_PREC_FP64EQ, tol=1e-10, seed=args.ga_seed)
    t_fb = time.perf_counter() - t0
    t1 = time.perf_counter()
    ga = oo.oo_ga_search(ctx, prob, 1, 16, 16, 0.9, 0.05, args.ga_seed, args.ga_timeout_ms)
    t_ga = time.perf_counter() - t1
    st = oo.oo_run_pattern(ctx, 0, 1, prob, np.empty(gI * gJ * gK, np.float32), np.empty(gIt))
    ms = fb["mask_ms"]
    table = {format(m, "04b"): (round(float(ms[m]), 2) if np.isfinite(ms[m]) else None) for m in range(ms.size)}
    all_cpu = float(ms[0]) + st["wall_ms"]
    best = float(fb["best_ms"]) + float(ga["best_ms"])
    out = {"metric": "function-block + loop offload trial (Sec. 4.2)", "unit": "ms",
           "config": {"workload": "fb_sites_gemm2048x2_fft2e20x4_fft2e16x8_unknown1+jacobi19_%dx%dx%d_it%d"
                      % (gI, gJ, gK, gIt), "prec": "fp64eq", "tol": 1e-10, "ga": "pop16 gens16 pc0.9 pm0.05",
                      "seed": args.ga_seed},
           "sites": [s[0] for s in sites], "block_ids": [int(b) for b in fb["block_ids"]],
           "mask_ms": table, "best_mask": format(int(fb["best_mask"]), "04b"), "fb_best_ms": float(fb["best_ms"]),
           "fb_all_cpu_ms": float(ms[0]), "loop_best_gene": format(int(ga["best_gene"]), "06b"),
           "loop_best_ms": float(ga["best_ms"]), "loop_all_cpu_ms": st["wall_ms"],
           "program_all_cpu_ms": round(all_cpu, 2), "program_best_ms": round(best, 2),
           "speedup_vs_all_cpu": round(all_cpu / best, 2), "fb_trial_s": round(t_fb, 1),
           "loop_ga_s": round(t_ga, 1),
           # every gene the GA measured: wall ms, or None where it failed the
           # result gate or ran past the evaluation time limit
           "loop_gene_ms": {format(int(g), "06b"): (round(float(ga["gene_ms"][g]), 3)
                                                    if np.isfinite(ga["gene_ms"][g]) else None)
                            for g in sorted(set(int(x) for x in ga["history"].reshape(-1)))}}
    oo.oo_destroy(ctx)
    print(json.dumps(out))
    return 0


def run_hoist(args):
    """Transfer hoisting (Sec. 3.2.1) measured: for a few genes, the pattern's
    wall time and CPU<->GPU traffic with copies hoisted to the outermost
    level each variable allows (lazy per-side validity) and with every GPU
    nest copying its data in and out at each invocation."""
    import torch
    from paper_2011_03602_gb300 import oo
    torch.cuda.set_device(0)
    ctx = oo.oo_create(0)
    genes = {"all_cpu": 0, "stencil_only": 4, "iteration_nests": 60, "all_gpu": 63}
    rows = []
    for (gI, gJ, gK, gIt) in ((65, 65, 129, 50), (129, 129, 257, 20)):
        prob = oo.jacobi(gI, gJ, gK, gIt)
        p = np.empty(gI * gJ * gK, np.float32)
        r = np.empty(gIt)
        for name, g in genes.items():
            for hoist in (1, 0):
                oo.oo_run_pattern(ctx, g, hoist, prob, p, r)  # warm-up
                best = None
                for _ in range(3):
                    st = oo.oo_run_pattern(ctx, g, hoist, prob, p, r)
                    if best is None or st["wall_ms"] < best["wall_ms"]:
                        best = st
                rows.append({"grid": [gI, gJ, gK], "iters": gIt, "gene": format(g, "06b"), "name": name,
                             "hoist": hoist, "wall_ms": round(best["wall_ms"], 3),
                             "h2d_bytes": int(best["h2d_bytes"]), "d2h_bytes": int(best["d2h_bytes"]),
                             "n_xfers": int(best["n_xfers"]), "xfer_ms": round(best["xfer_ms"], 3)})
    oo.oo_destroy(ctx)
    print(json.dumps({"metric": "pattern wall time with and without transfer hoisting", "unit": "ms",
                      "config": {"workload": "jacobi19_hoist_on_off", "timing": "best of 3 after 1 warm-up"},
                      "rows": rows}))
    return 0


def run_genes(args):
    """Every gene with and without hoisting on the small Jacobi configuration
    (33 x 33 x 65, 50 iterations; working set ~4 MB, resident in L2): wall
    time per pattern (best of 3 after a warm-up) and CPU<->GPU bytes, with
    each pattern's residuals checked against the all-CPU run."""
    import torch
    from paper_2011_03602_gb300 import oo
    torch.cuda.set_device(0)
    ctx = oo.oo_create(0)
    gI, gJ, gK, gIt = 33, 33, 65, 50
    prob = oo.jacobi(gI, gJ, gK, gIt)
    p = np.empty(gI * gJ * gK, np.float32)
    r = np.empty(gIt)
    oo.oo_run_pattern(ctx, 0, 1, prob, p, r)
    p_ref, r_ref = p.copy(), r.copy()
    table = {}
    worst = 0.0
    for hoist in (1, 0):
        for g in range(64):
            oo.oo_run_pattern(ctx, g, hoist, prob, p, r)
            best = None
            for _ in range(3):
                st = oo.oo_run_pattern(ctx, g, hoist, prob, p, r)
                best = st if best is None or st["wall_ms"] < best["wall_ms"] else best
            worst = max(worst, float(np.max(np.abs(r - r_ref) / np.abs(r_ref))))
            assert np.max(np.abs(p - p_ref)) <= 1e-5
            table.setdefault(format(g, "06b"), {})["on" if hoist else "off"] = [
                round(best["wall_ms"], 3), int(best["h2d_bytes"] + best["d2h_bytes"])]
    oo.oo_destroy(ctx)
    on = {g: v["on"][0] for g, v in table.items()}
    best_on = min(on, key=on.get)
    print(json.dumps({"metric": "per-gene pattern wall time, hoisting on / off", "unit": "ms",
                      "config": {"workload": "jacobi19_33x33x65_it50_all64genes", "timing": "best of 3 after 1 warm-up",
                                 "entry": "[wall_ms, h2d+d2h bytes]"},
                      "max_residual_rel_err_vs_all_cpu": worst, "fastest_gene_hoisted": best_on,
                      "fastest_ms": on[best_on], "all_cpu_ms": on["000000"], "genes": table}))
    return 0


def run_block(args):
    """Profiling helper: warm up and run one function block a few times
    (no oracle, no timing claims) so ncu can capture its kernels."""
    import torch
    from paper_2011_03602_gb300 import oo, synth
    torch.cuda.set_device(0)
    ctx = oo.oo_create(0)
    n = args.n
    if args.block == "gemm":
        A = torch.from_numpy(synth.gemm_matrix(1, n, n)).cuda()
        B = torch.from_numpy(synth.gemm_matrix(2, n, n)).cuda()
        C = torch.empty(n, n, dtype=torch.float64, device="cuda")
        prec = {"fp64eq": oo.OO_PREC_FP64EQ, "tf32": oo.OO_PREC_SPLIT3_TF32}.get(args.prec, oo.OO_PREC_SPLIT3_BF16)
        for _ in range(args.steps):
            oo.oo_gemm_f64_dev(ctx, n, n, n, A, n, B, n, C, n, prec=prec)
        oo.oo_gemm_check(ctx, n, n, n)
    else:
        batch = max(1, args.batch)
        x = torch.from_numpy(synth.complex_normal(3, n * batch).view(np.float64).copy()).cuda()
        y = torch.empty_like(x)
        for _ in range(args.steps):
            oo.oo_fft_c128_dev(ctx, n, batch, -1, x, y)
    oo.oo_sync(ctx)
    oo.oo_destroy(ctx)
    print(json.dumps({"block": args.block, "n": n, "runs": args.steps, "ok": True}))
    return 0


def run_blocks_sweep(args):
    """Function blocks over the workload's size ranges (device-resident
    inputs, CUDA events on the context's stream, splits included): the GEMM
    at n = 256, 1024, 4096 in every precision pattern (tensor TFLOP/s and
    error vs the oracle on sampled rows), and the FFT at N = 2^10..2^22 with
    batch max(1, 2^24 / N) (GB/s of one- or two-pass traffic against the
    measured HBM peak; error of the first transform vs the oracle)."""
    import torch
    import oracle
    from paper_2011_03602_gb300 import oo, synth
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    ctx_stream_holder[0] = stream
    ctx = oo.oo_create(0, stream.cuda_stream)
    hbm, hsrc = load_peaks()
    peak, _, psrc = load_bf16_peak()

    def timed(fn, reps):
        for _ in range(3):
            fn()
        oo.oo_sync(ctx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    gemm = []
    for n in (256, 1024, 4096):
        A_h, B_h = synth.gemm_matrix(61 + n, n, n), synth.gemm_matrix(62 + n, n, n)
        A, B = torch.from_numpy(A_h).cuda(), torch.from_numpy(B_h).cuda()
        C = torch.empty(n, n, dtype=torch.float64, device="cuda")
        rows = [0, n // 2, n - 1]
        refs = [(oracle.gemm(A_h[r:r + 1], B_h)[0], np.abs(A_h[r]) @ np.abs(B_h)) for r in rows]
        for name, prec in (("split3_bf16", oo.OO_PREC_SPLIT3_BF16), ("split3_tf32", oo.OO_PREC_SPLIT3_TF32),
                           ("fp64eq", oo.OO_PREC_FP64EQ)):
            ms = timed(lambda: oo.oo_gemm_f64_dev(ctx, n, n, n, A, n, B, n, C, n, prec=prec),
                       20 if n < 4096 else (4 if prec == oo.OO_PREC_FP64EQ else 10))
            oo.oo_gemm_check(ctx, n, n, n)
            products = oo.oo_gemm_plan(prec, n)[0]
            tensor = products * 2 * n ** 3 / (ms * 1e-3) / 1e12
            tpeak = peak * (1.1 / 2.25 if prec == oo.OO_PREC_SPLIT3_TF32 else 1.0)
            Ch = C.cpu().numpy()
            err = max(float(np.max(np.abs(Ch[r] - ref) / sc)) for r, (ref, sc) in zip(rows, refs))
            gemm.append({"n": n, "pattern": name, "ms": round(ms, 4), "solves_per_s": round(1e3 / ms, 1),
                         "tensor_tflops": round(tensor, 1), "frac_of_pattern_peak": round(tensor / tpeak, 4),
                         "max_err_vs_oracle": err})
        del A, B, C
    fft = []
    for e in range(10, 23):
        N = 1 << e
        batch = max(1, (1 << 24) // N)
        x_h = synth.complex_normal(63 + e, N * batch)
        x = torch.from_numpy(x_h.view(np.float64).copy()).cuda()
        y = torch.empty_like(x)
        ms = timed(lambda: oo.oo_fft_c128_dev(ctx, N, batch, -1, x, y), 10)
        passes = 1 if e <= 12 else 2
        gbps = passes * 32 * N * batch / (ms * 1e-3) / 1e9
        y0 = y[:2 * N].cpu().numpy().view(np.complex128)
        ref = oracle.fft(x_h[:N], -1)
        fft.append({"log2n": e, "batch": batch, "ms": round(ms, 4), "passes": passes,
                    "GBps": round(gbps, 1), "frac_of_hbm": round(gbps / hbm, 4),
                    "rel_l2_err_vs_oracle": float(np.linalg.norm(y0 - ref) / np.linalg.norm(ref))})
        del x, y
    oo.oo_destroy(ctx)
    print(json.dumps({"metric": "function blocks over the workload's size ranges", "data": "synthetic",
                      "peaks": {"hbm_gbs": hbm, "hbm_source": hsrc, "bf16_tflops": peak, "bf16_source": psrc,
                                "tf32_tflops_note": "measured BF16 peak x 1.1 / 2.25"},
                      "gemm": gemm, "fft": fft}))
    return 0


def run_vendor(args):
    """Context only, not the product path: the function blocks beside the
    FP64 library calls a function-block offload would otherwise make
    (cuBLAS DGEMM through torch.matmul, cuFFT Z2Z through torch.fft.fft), on
    the same stream, the same device-resident inputs (larger than L2 at the
    largest sizes; no flush) and CUDA-event timing.  max_rel_diff is
    max |ours - library| / max |library| per result."""
    import torch
    from paper_2011_03602_gb300 import oo, synth
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    ctx = oo.oo_create(0, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(max(args.warmup, 3)):
            fn()
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / args.steps

    out = {"gemm": {}, "fft": {}}
    with torch.cuda.stream(stream):
        for n in (1024, 4096):
            A = torch.from_numpy(synth.gemm_matrix(1, n, n)).cuda()
            B = torch.from_numpy(synth.gemm_matrix(2, n, n)).cuda()
            C = torch.empty(n, n, dtype=torch.float64, device="cuda")
            ref = torch.empty_like(C)
            t_lib = timed(lambda: torch.matmul(A, B, out=ref))
            row = {"cublas_dgemm_ms": round(t_lib, 4),
                   "cublas_dgemm_fp64_tflops": round(2 * n ** 3 / (t_lib * 1e-3) / 1e12, 2)}
            for name, prec in (("split3", oo.OO_PREC_SPLIT3_BF16), ("fp64eq", oo.OO_PREC_FP64EQ)):
                t = timed(lambda: oo.oo_gemm_f64_dev(ctx, n, n, n, A, n, B, n, C, n, prec=prec))
                oo.oo_gemm_check(ctx, n, n, n)
                d = float((C - ref).abs().max() / ref.abs().max())
                row[name] = {"ms": round(t, 4), "speedup_vs_cublas": round(t_lib / t, 2), "max_rel_diff": d}
            out["gemm"][str(n)] = row
            del A, B, C, ref
        for log2n, batch in ((22, 1), (20, 4), (10, 4096)):
            n = 1 << log2n
            xr = torch.from_numpy(synth.complex_normal(3, n * batch).view(np.float64).copy()).cuda()
            y = torch.empty_like(xr)
            xc = torch.view_as_complex(xr.view(-1, 2)).view(batch, n)
            ref = torch.empty_like(xc)
            t_lib = timed(lambda: ref.copy_(torch.fft.fft(xc, dim=-1)))
            t = timed(lambda: oo.oo_fft_c128_dev(ctx, n, batch, -1, xr, y))
            yc = torch.view_as_complex(y.view(-1, 2)).view(batch, n)
            d = float((yc - ref).abs().max() / ref.abs().max())
            out["fft"][f"2^{log2n}x{batch}"] = {"cufft_z2z_ms": round(t_lib, 4), "ours_ms": round(t, 4),
                                                "speedup_vs_cufft": round(t_lib / t, 2), "max_rel_diff": d}
            del xr, y, xc, ref
    oo.oo_sync(ctx)
    oo.oo_destroy(ctx)
    print(json.dumps({"mode": "vendor_context", "steps": args.steps, "warmup": max(args.warmup, 3),
                      "note": "library calls timed for context; not on the product path", **out}))
    return 0


def _batch_errors(job):
    """Errors of a slice of the batched requests against the oracle, in a
    worker process: GEMM max |C - C*| / (|A||B|), FFT relative L2."""
    import oracle
    from paper_2011_03602_gb300 import synth
    kind, idx, dims, out = job
    errs = []
    for i, d, y in zip(idx, dims, out):
        if kind == "gemm":
            m, n, k = d
            A, B = synth.gemm_matrix(100 + i, m, k), synth.gemm_matrix(200000 + i, k, n)
            errs.append(float(np.max(np.abs(y - oracle.gemm(A, B)) / (np.abs(A) @ np.abs(B)))))
        else:
            x = synth.complex_normal(400000 + i, 1 << d)
            ref = oracle.fft(x, -1 if i % 2 == 0 else 1)
            errs.append(float(np.linalg.norm(y.view(np.complex128) - ref) / np.linalg.norm(ref)))
    return errs


def run_batched(args):
    """Batched uneven function blocks: 4096 GEMMs with m, n, k log-uniform
    in [16, 512] (FP64-equivalent by default) and 2048 complex FFTs with
    lengths 2^8..2^16 (directions alternating), device-resident; grouped
    persistent kernels, the same as one CUDA-graph replay, and one library
    call per request.  Every result is then checked against the oracle on
    the host cores (worker processes)."""
    out = measure_batched(args.batch_gemms, args.batch_ffts, args.batch_prec,
                          [int(x) for x in args.batch_modes.split(",")], args.steps, args.warmup,
                          check=not args.no_cpu_baseline, check_stride=1)
    print(json.dumps(out))
    return 0


def measure_batched(n_gemm, n_fft, prec_name, modes, steps, warmup, check=True, check_stride=1):
    """The batched configuration as a dict (the --batched line, and the
    default line's "batched" component); results number check_stride apart
    are checked against the oracle after timing."""
    import multiprocessing as mp
    pool = mp.get_context("spawn").Pool(host_cores()) if check else None
    import torch
    from paper_2011_03602_gb300 import oo, synth
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    ctx = oo.oo_create(0, stream)
    prec = oo.OO_PREC_FP64EQ if prec_name == "fp64eq" else oo.OO_PREC_SPLIT3_BF16
    dims = synth.log_uniform_int(4, 3 * n_gemm, 16, 512).reshape(n_gemm, 3)
    expo = 8 + np.floor(synth.uniform(5, n_fft) * 9).astype(int)
    reqs = []
    with torch.cuda.stream(stream):
        for i, (m, n, k) in enumerate(dims.tolist()):
            A = torch.from_numpy(synth.gemm_matrix(100 + i, m, k)).to("cuda", non_blocking=False)
            B = torch.from_numpy(synth.gemm_matrix(200000 + i, k, n)).to("cuda", non_blocking=False)
            reqs.append(dict(kind="gemm", m=m, n=n, k=k, A=A, B=B, prec=prec,
                             C=torch.empty((m, n), dtype=torch.float64, device="cuda")))
        for i, e in enumerate(expo.tolist()):
            x = synth.complex_normal(400000 + i, 1 << e)
            reqs.append(dict(kind="fft", n=1 << e, dir=-1 if i % 2 == 0 else 1,
                             x=torch.from_numpy(x.view(np.float64).copy()).cuda(),
                             X=torch.empty(2 << e, dtype=torch.float64, device="cuda")))
    torch.cuda.synchronize()
    b = oo.oo_batch_create(ctx, reqs)
    info = oo.oo_batch_info(b)
    res = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    names = {2: "one_call_per_request", 0: "grouped_persistent", 1: "grouped_cuda_graph"}
    for mode in modes:
        for _ in range(max(warmup, 2)):
            oo.oo_batch_run(ctx, b, mode)
        oo.oo_batch_check(ctx, b)
        e0.record(stream)
        for _ in range(steps):
            oo.oo_batch_run(ctx, b, mode)
        e1.record(stream)
        e1.synchronize()
        oo.oo_batch_check(ctx, b)
        ms = e0.elapsed_time(e1) / steps
        res[names[mode]] = {"ms": round(ms, 3), "solves_per_s": round((n_gemm + n_fft) / (ms * 1e-3), 1),
                            "gemm_fp64_equiv_tflops": round(info["gemm_flops"] / (ms * 1e-3) / 1e12, 2)}
    # outputs of the last run (the headline mode) against the oracle
    errors = None
    if pool is not None:
        g_idx = list(range(0, n_gemm, check_stride))
        f_idx = list(range(0, n_fft, check_stride))
        outs = {i: reqs[i]["C"].cpu().numpy() for i in g_idx}
        outs.update({n_gemm + i: reqs[n_gemm + i]["X"].cpu().numpy() for i in f_idx})
        jobs = []
        for s in range(0, len(g_idx), 32):
            idx = g_idx[s:s + 32]
            jobs.append(("gemm", idx, [tuple(int(v) for v in dims[i]) for i in idx], [outs[i] for i in idx]))
        for s in range(0, len(f_idx), 32):
            idx = f_idx[s:s + 32]
            jobs.append(("fft", idx, [int(expo[i]) for i in idx], [outs[n_gemm + i] for i in idx]))
        t0 = time.perf_counter()
        res_e = pool.map(_batch_errors, jobs)
        pool.close()
        ge = [e for j, r in zip(jobs, res_e) if j[0] == "gemm" for e in r]
        fe = [e for j, r in zip(jobs, res_e) if j[0] == "fft" for e in r]
        errors = {"gemm_max_err_vs_oracle": max(ge) if ge else None,
                  "gemm_err_metric": "max |C-C*| / (|A||B|) per result",
                  "fft_max_rel_l2_vs_oracle": max(fe) if fe else None, "results_checked": len(ge) + len(fe),
                  "results_checked_how": ("every result" if check_stride == 1 else
                                          "every %dth GEMM and every %dth FFT" % (check_stride, check_stride)),
                  "oracle_seconds": round(time.perf_counter() - t0, 1), "oracle_processes": host_cores()}
    widths = oo.oo_get_gemm_tiles(ctx).tolist()
    oo.oo_batch_destroy(b)
    oo.oo_destroy(ctx)
    del reqs
    headline = res.get("grouped_cuda_graph") or res.get("grouped_persistent") or res["one_call_per_request"]
    out = {"metric": "batched GEMM/FFT solves/s", "unit": "solves/s",
           "value": headline["solves_per_s"], "higher_is_better": True,
           "steps": steps, "warmup": warmup, "data": "synthetic",
           "config": {"workload": "batched_%dgemm_logu16-512_%dfft_2e8-2e16" % (n_gemm, n_fft),
                      "gemm_flops_per_batch": info["gemm_flops"], "fft_points_per_batch": info["fft_points"],
                      "precision": ("fp64eq GEMM (Ozaki BF16 digit slices)" if prec == oo.OO_PREC_FP64EQ
                                    else "split3_bf16 GEMM") + ", float-float FFT",
                      "tile_widths_by_n_and_k_bucket": widths},
           "errors": errors,
           "modes": res,
           "speedup_graph_vs_per_call": (round(res["one_call_per_request"]["ms"] / res["grouped_cuda_graph"]["ms"], 2)
                                         if "one_call_per_request" in res and "grouped_cuda_graph" in res else None)}
    return out


def _serve_refs(job):
    """Oracle references for the served mix, in a worker process: sampled
    rows of a GEMM size, an FFT length, or a Jacobi grid's whole program."""
    import oracle
    from paper_2011_03602_gb300 import synth
    kind, a = job
    if kind == "gemm":
        A, B = synth.gemm_matrix(7 + a, a, a), synth.gemm_matrix(8 + a, a, a)
        rows = [0, a // 2, a - 1]
        ref = np.stack([oracle.gemm(A[r:r + 1], B)[0] for r in rows])
        scale = np.stack([np.abs(A[r]) @ np.abs(B) for r in rows])
        return (kind, a), (rows, ref, scale)
    if kind == "fft":
        return (kind, a), oracle.fft(synth.complex_normal(9 + a, 1 << a), -1)
    I, J, K = a
    res, p = oracle.jacobi_run(I, J, K, 100, mode=1)
    return (kind, a), (res, p.reshape(-1).astype(np.float32))


def _digest64(arrays):
    """XOR and sum (mod 2^64) of the whole 64-bit words of each array, as the
    C client (frontends/c/oo_loadgen.c) digests its outputs."""
    x, t = 0, 0
    for a in arrays:
        b = np.ascontiguousarray(a).reshape(-1).view(np.uint8)
        w = b[: (b.size // 8) * 8].view(np.uint64)
        if w.size:
            x ^= int(np.bitwise_xor.reduce(w))
            t = (t + int(np.sum(w, dtype=np.uint64))) & ((1 << 64) - 1)
    return x, t


class _CLoadPools(ctypes.Structure):
    _fields_ = [("gemm_a", ctypes.c_void_p * 16), ("gemm_b", ctypes.c_void_p * 16), ("gemm_n", ctypes.c_int32 * 16),
                ("fft_x", ctypes.c_void_p * 32), ("fft_log2", ctypes.c_int32 * 32),
                ("jac_i", ctypes.c_int32 * 8), ("jac_j", ctypes.c_int32 * 8), ("jac_k", ctypes.c_int32 * 8),
                ("jac_iters", ctypes.c_int32), ("prec", ctypes.c_int32), ("client", ctypes.c_int32),
                ("max_in_flight", ctypes.c_int32)]


class _CLoadItem(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("size", ctypes.c_int32), ("arrival", ctypes.c_double)]


class _CLoadResult(ctypes.Structure):
    _fields_ = [("latency_ms", ctypes.c_double), ("status", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("digest_xor", ctypes.c_uint64), ("digest_sum", ctypes.c_uint64)]


def run_serve(args):
    print(json.dumps(measure_serve(args)))
    return 0


def measure_serve(args):
    """Serving loop: Poisson arrivals at each offered rate, the stream split
    in thirds over client front ends that all submit through the C ABI: the
    C client (frontends/c/oo_loadgen.c, run in this process on its own
    thread; it allocates its own output buffers), a Python ctypes client,
    and the Java share -- no JDK exists on either machine, so a second
    ctypes client submits that third and the line says so.
    mix 50% GEMM (square, n log-uniform in [64, 2048], FP64-equivalent by
    default), 30% FFT (2^10..2^20), 20% Jacobi solves (65x65x129 or
    129x129x257, 100 iterations).  Reported: solves/s, p50/p99 latency of
    admitted requests, back-pressure counts, and the error of every result
    against the oracle (GEMM: sampled rows, max |C - C*| / (|A||B|); FFT:
    relative L2; Jacobi: residuals relative, p absolute), against the plain
    offload -- one synchronous call per solve in the same precision, in
    arrival order, on the same GPU and the same request stream."""
    import multiprocessing as mp
    import threading
    refs_pool = mp.get_context("spawn").Pool(host_cores())
    import torch
    from paper_2011_03602_gb300 import build as pkg_build
    from paper_2011_03602_gb300 import oo, synth
    torch.cuda.set_device(0)
    oo.lib()
    cgen = ctypes.CDLL(pkg_build.build_loadgen())
    cgen.oo_load_run.restype = ctypes.c_int
    cgen.oo_load_run.argtypes = [ctypes.c_void_p, ctypes.POINTER(_CLoadPools), ctypes.POINTER(_CLoadItem),
                                 ctypes.c_int, ctypes.POINTER(_CLoadResult)]
    rates = [int(x) for x in args.serve_rates.split(",")]
    window = args.serve_window
    # input pools: one operand set per size (results are still computed per request)
    gemm_sizes = [64, 128, 256, 512, 1024, 2048]
    pool_g = {n: (synth.gemm_matrix(7 + n, n, n), synth.gemm_matrix(8 + n, n, n)) for n in gemm_sizes}
    pool_f = {e: synth.complex_normal(9 + e, 1 << e) for e in range(10, 21)}
    grids = [(65, 65, 129), (129, 129, 257)]
    prec = oo.OO_PREC_FP64EQ if args.serve_prec == "fp64eq" else oo.OO_PREC_SPLIT3_BF16
    # oracle references: computed on the host cores after every timed phase
    # (the serving loops' host threads and copies need those cores)
    ref_jobs = [("gemm", n) for n in gemm_sizes] + [("fft", e) for e in range(10, 21)] + [("jacobi", g) for g in grids]
    worst = {"gemm": 0.0, "fft": 0.0, "jacobi_res": 0.0, "jacobi_p": 0.0}
    # the first result of every (kind, size) is kept and checked against the
    # oracle at the end; every other result's digest must equal the first's
    # (the blocks are deterministic), which keeps host memory bounded
    first, digests, n_checked, n_differ = {}, {}, [0], [0]
    first64, c_first, n_c_checked = {}, {}, [0]  # 64-bit-word digests (the C client's form)

    def draw(rng):
        u = rng.random()
        if u < 0.5:
            n = int(np.exp(np.log(64) + rng.random() * (np.log(2049) - np.log(64))))
            n = min(gemm_sizes, key=lambda g: abs(np.log(g) - np.log(n)))
            return ("gemm", n)
        if u < 0.8:
            return ("fft", int(rng.integers(10, 21)))
        return ("jacobi", int(rng.integers(0, 2)))

    def make(kind, a):
        if kind == "gemm":
            A, B = pool_g[a]
            return dict(A=A, B=B, C=np.empty((a, a)), prec=prec)
        if kind == "fft":
            x = pool_f[a]
            return dict(x=x, X=np.empty_like(x), dir=-1)
        I, J, K = grids[a]
        return dict(I=I, J=J, K=K, iters=100, p=np.empty(I * J * K, np.float32), res=np.empty(100))

    ctx = oo.oo_create(0)
    tuned = {"%dx%dx%d" % g: oo.oo_tune_stencil(ctx, *g)[0] for g in grids}  # stencil tile per grid
    # the C client's input pools: the same arrays as the ctypes clients'
    c_pools = _CLoadPools()
    for j, n in enumerate(gemm_sizes):
        c_pools.gemm_a[j], c_pools.gemm_b[j], c_pools.gemm_n[j] = (pool_g[n][0].ctypes.data, pool_g[n][1].ctypes.data, n)
    for e in range(10, 21):
        c_pools.fft_x[e - 10], c_pools.fft_log2[e - 10] = pool_f[e].ctypes.data, e
    for j, (I, J, K) in enumerate(grids):
        c_pools.jac_i[j], c_pools.jac_j[j], c_pools.jac_k[j] = I, J, K
    c_pools.jac_iters, c_pools.prec, c_pools.client, c_pools.max_in_flight = 100, prec, 0, 256
    modes = [m for m in args.serve_modes.split(",") if m]
    per_mode = {}
    for mode in modes:
        if mode == "resident":
            # the request loop resident on the device: persistent workers,
            # no kernel launch per request
            oo.oo_serve_start_resident(ctx, args.serve_budget_gb << 30, args.serve_queue, args.serve_tensor_ctas)
        else:
            # the host scheduler over slot streams
            oo.oo_serve_start(ctx, slots=args.serve_slots, hbm_budget_bytes=args.serve_budget_gb << 30,
                              queue_cap=args.serve_queue)
        first.clear()
        digests.clear()
        first64.clear()
        c_first.clear()
        # warm-up: one of each kind
        for kind, a in (("gemm", 2048), ("fft", 20), ("jacobi", 1)):
            kw = make(kind, a)
            oo.oo_wait(ctx, oo.oo_submit(ctx, oo.serve_request(kind, **kw)), 120000)
        results = []
        for rate in rates:
            rng = np.random.default_rng(rate)
            n_req = max(3, int(rate * window))
            arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
            kinds = [draw(rng) for _ in range(n_req)]
            lat, rejected, lock = [], [0], threading.Lock()
            lat_by = {"c": [], "python_ctypes": [], "java_share_via_ctypes": []}
            st0 = oo.oo_serve_stats(ctx)
            t0 = time.perf_counter() + 0.05

            def client(tag):
                mine, done = [], []
                fe = "python_ctypes" if tag == 1 else "java_share_via_ctypes"
                for i in range(tag, n_req, 3):
                    kind, a = kinds[i]
                    kw = make(kind, a)
                    dt = t0 + arrivals[i] - time.perf_counter()
                    if dt > 0:
                        time.sleep(dt)
                    st, t = oo.oo_submit_status(ctx, oo.serve_request(kind, client=tag, **kw))
                    if st == oo.OO_EBUSY:
                        with lock:
                            rejected[0] += 1
                        continue
                    if st != 0:
                        raise oo.OOError(st, oo.oo_last_error(ctx))
                    mine.append((t, kw, kinds[i]))
                    if len(mine) > 256:  # bound the client's host buffers in flight
                        t_old, kw_old, ka_old = mine.pop(0)
                        done.append(oo.oo_wait(ctx, t_old, 600000))
                        keep(ka_old, kw_old)
                got = done
                for t, kw, ka in mine:
                    got.append(oo.oo_wait(ctx, t, 600000))
                    keep(ka, kw)
                with lock:
                    lat.extend(got)
                    lat_by[fe].extend(got)

            c_idx = list(range(0, n_req, 3))
            c_items = (_CLoadItem * max(1, len(c_idx)))()
            for j, i in enumerate(c_idx):
                kind, a = kinds[i]
                c_items[j].kind = {"gemm": oo.OO_BLOCK_GEMM, "fft": oo.OO_BLOCK_FFT, "jacobi": oo.OO_BLOCK_JACOBI}[kind]
                c_items[j].size = gemm_sizes.index(a) if kind == "gemm" else (a - 10 if kind == "fft" else a)
                c_items[j].arrival = t0 + float(arrivals[i])
            c_res = (_CLoadResult * max(1, len(c_idx)))()

            def c_client():
                busy = cgen.oo_load_run(ctx, ctypes.byref(c_pools), c_items, len(c_idx), c_res)
                got = [c_res[j].latency_ms for j in range(len(c_idx)) if c_res[j].status == 0]
                with lock:
                    rejected[0] += max(0, busy)
                    lat.extend(got)
                    lat_by["c"].extend(got)

            def keep(ka, kw):
                kind, _ = ka
                outs = [kw["C"]] if kind == "gemm" else ([kw["X"]] if kind == "fft" else [kw["res"], kw["p"]])
                words = [o.reshape(-1).view(np.uint64 if o.dtype.itemsize == 8 else np.uint32) for o in outs]
                dg = tuple((int(np.bitwise_xor.reduce(w)), int(np.sum(w, dtype=np.uint64))) for w in words)
                with lock:
                    n_checked[0] += 1
                    if ka not in first:
                        first[ka] = [o.copy() for o in outs]
                        digests[ka] = dg
                        first64[ka] = _digest64(outs)
                    elif digests[ka] != dg:
                        n_differ[0] += 1

            ths = [threading.Thread(target=c_client)] + [threading.Thread(target=client, args=(tag,)) for tag in (1, 2)]
            start = time.perf_counter()
            for th in ths:
                th.start()
            for th in ths:
                th.join()
            elapsed = time.perf_counter() - start
            # the C client's results: every one's digest equals that of the
            # same request's result through ctypes (or, for a request kind
            # only the C client drew, that of its first C result)
            for j, i in enumerate(c_idx):
                r = c_res[j]
                if r.status == oo.OO_EBUSY:
                    continue
                if r.status != 0:
                    raise oo.OOError(r.status, "C client: " + oo.oo_status_str(r.status))
                ka = kinds[i]
                d = (int(r.digest_xor), int(r.digest_sum))
                ref = first64.get(ka) or c_first.setdefault(ka, d)
                n_checked[0] += 1
                n_c_checked[0] += 1
                if d != ref:
                    n_differ[0] += 1
            lat_a = np.array(lat) if lat else np.array([np.nan])
            st1 = oo.oo_serve_stats(ctx)
            dn = max(1, st1["completed"] - st0["completed"])
            stage = {k: round((st1["stage_ms"][k] * st1["completed"] - st0["stage_ms"][k] * st0["completed"]) / dn, 3)
                     for k in st1["stage_ms"]}
            results.append({"offered_req_per_s": rate, "requests": n_req, "admitted": len(lat),
                            "rejected_busy": rejected[0], "solves_per_s": round(len(lat) / elapsed, 1),
                            "p50_ms": round(float(np.percentile(lat_a, 50)), 3),
                            "p99_ms": round(float(np.percentile(lat_a, 99)), 3),
                            "mean_stage_ms": stage,
                            "by_front_end": {k: {"admitted": len(v),
                                                 "p50_ms": round(float(np.percentile(v, 50)), 3) if v else None,
                                                 "p99_ms": round(float(np.percentile(v, 99)), 3) if v else None}
                                             for k, v in lat_by.items()}})
        stats = oo.oo_serve_stats(ctx)
        oo.oo_serve_stop(ctx)
        per_mode[mode] = (results, stats, dict(first))
    # plain offload (no server running): the first rate's request stream, one
    # synchronous call per solve; latency from the queue the arrival process
    # would form in front of a one-at-a-time server
    rate = rates[0]
    rng = np.random.default_rng(rate)
    n_req = max(3, int(rate * window))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    kinds = [draw(rng) for _ in range(n_req)]
    prev, sim_end, lat_p = 0.0, 0.0, []
    tp0 = time.perf_counter()
    for i in range(n_req):
        kind, a = kinds[i]
        kw = make(kind, a)
        if kind == "gemm":
            oo.oo_gemm_f64(ctx, kw["A"], kw["B"], prec=prec, out=kw["C"])
        elif kind == "fft":
            oo.oo_fft_c128(ctx, kw["x"], -1, out=kw["X"])
        else:
            oo.oo_run_pattern(ctx, 63, 1, oo.jacobi(kw["I"], kw["J"], kw["K"], 100), kw["p"], kw["res"])
        now = time.perf_counter() - tp0
        sim_end = max(sim_end, arrivals[i]) + (now - prev)
        prev = now
        lat_p.append((sim_end - arrivals[i]) * 1e3)
    elapsed_p = time.perf_counter() - tp0
    plain = {"offered_req_per_s": rate, "requests": n_req, "solves_per_s": round(n_req / elapsed_p, 1),
             "p50_ms_if_arrivals_queue": round(float(np.percentile(lat_p, 50)), 3),
             "p99_ms_if_arrivals_queue": round(float(np.percentile(lat_p, 99)), 3)}
    oo.oo_destroy(ctx)
    refs = dict(refs_pool.map(_serve_refs, ref_jobs))
    refs_pool.close()
    checked = [(ka, outs) for m in per_mode.values() for ka, outs in m[2].items()]
    for (kind, a), outs in checked:
        if kind == "gemm":
            rows, ref, scale = refs[("gemm", a)]
            worst["gemm"] = max(worst["gemm"], float(np.max(np.abs(outs[0][rows] - ref) / scale)))
        elif kind == "fft":
            ref = refs[("fft", a)]
            worst["fft"] = max(worst["fft"], float(np.linalg.norm(outs[0] - ref) / np.linalg.norm(ref)))
        else:
            res_ref, p_ref = refs[("jacobi", grids[a])]
            res, p = outs
            worst["jacobi_res"] = max(worst["jacobi_res"], float(np.max(np.abs(res - res_ref) / np.abs(res_ref))))
            worst["jacobi_p"] = max(worst["jacobi_p"], float(np.max(np.abs(p.astype(np.float64) - p_ref))))
    results, stats, _ = per_mode[modes[0]]
    best = max(r["solves_per_s"] for r in results)
    out = {"metric": "served solves/s and p50/p99 latency", "unit": "solves/s", "value": best,
           "higher_is_better": True, "data": "synthetic",
           "config": {"workload": "serve_mix_50gemm64-2048_30fft2e10-2e20_20jacobi65-129_it100",
                      "gemm_precision": args.serve_prec,
                      "slots": args.serve_slots, "device_budget_gb": args.serve_budget_gb,
                      "resident_tensor_ctas": args.serve_tensor_ctas or "library default (an eighth of the SMs)",
                      "queue_cap": args.serve_queue, "window_s": window,
                      "front_ends": {"c": "frontends/c/oo_loadgen.c: C ABI calls from its own thread in this process, "
                                          "its own output buffers",
                                     "python_ctypes": "oo.py ctypes binding",
                                     "java_share_via_ctypes": "no JDK on either machine: the Java third of the "
                                                              "stream is submitted by a second ctypes client"}},
           "served": results, "served_loop": modes[0],
           "served_other_loops": {m: per_mode[m][0] for m in modes[1:]},
           "plain_one_call_per_solve": plain,
           "served_vs_plain_solves_per_s": round(results[0]["solves_per_s"] / plain["solves_per_s"], 2),
           "failed": {m: per_mode[m][1]["failed"] for m in modes}, "stencil_variant_by_grid": tuned,
           "max_error_per_result_vs_oracle": {
               "gemm": worst["gemm"], "gemm_metric": "max |C-C*| / (|A||B|) over rows 0, n/2, n-1",
               "fft_rel_l2": worst["fft"], "jacobi_residual_rel": worst["jacobi_res"],
               "jacobi_p_abs": worst["jacobi_p"], "results": n_checked[0],
               "results_differing_from_first_of_same_size": n_differ[0],
               "results_of_the_c_client_checked_by_digest": n_c_checked[0],
               "how": "first result of each kind and size against the oracle; every other result's "
                      "digest against that first result's"}}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-blocks", action="store_true", help="skip the GEMM / FFT component timings")
    ap.add_argument("--no-systems", action="store_true",
                    help="skip the batched and served components of the default line")
    ap.add_argument("--ga", action="store_true", help="run the GA search at scale instead of the step benchmark")
    ap.add_argument("--block", choices=["gemm", "fft"], default=None, help="profiling: run one function block")
    ap.add_argument("--fb", action="store_true", help="function-block + loop offload trial order")
    ap.add_argument("--hoist", action="store_true", help="pattern times with transfer hoisting on and off")
    ap.add_argument("--genes", action="store_true", help="all 64 genes x hoisting on/off, 33x33x65, 50 iterations")
    ap.add_argument("--batched", action="store_true", help="batched uneven GEMM/FFT configuration")
    ap.add_argument("--vendor", action="store_true",
                    help="context: function blocks beside cuBLAS DGEMM / cuFFT Z2Z on the same GPU")
    ap.add_argument("--serve", action="store_true", help="serving-loop configuration")
    ap.add_argument("--blocks-sweep", action="store_true",
                    help="GEMM at n = 256, 1024, 4096 in every pattern; FFT at 2^10..2^22, batch 2^24 / N")
    ap.add_argument("--serve-rates", default="2000,5000,10000,20000")
    ap.add_argument("--serve-prec", choices=["fp64eq", "split3"], default="fp64eq")
    ap.add_argument("--serve-modes", default="resident,host",
                    help="serving loops to run, the first is the headline: resident (persistent device workers), "
                         "host (scheduler thread over slot streams)")
    ap.add_argument("--serve-window", type=float, default=0.5, help="seconds of arrivals per rate")
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-tensor-ctas", type=int, default=0,
                    help="resident loop: SMs for the tensor-core worker (0: the library's default, an eighth)")
    ap.add_argument("--serve-budget-gb", type=int, default=16)
    ap.add_argument("--serve-queue", type=int, default=2048)
    ap.add_argument("--batch-gemms", type=int, default=4096)
    ap.add_argument("--batch-ffts", type=int, default=2048)
    ap.add_argument("--batch-prec", choices=["fp64eq", "split3"], default="fp64eq")
    ap.add_argument("--batch-modes", default="2,0,1",
                    help="batched: 2 one call per request, 0 grouped kernels, 1 the grouped CUDA graph")
    ap.add_argument("--n", type=int, default=4096, help="profiling: GEMM size or FFT length")
    ap.add_argument("--batch", type=int, default=1, help="profiling: FFT batch")
    ap.add_argument("--prec", choices=["split3", "tf32", "fp64eq"], default="split3", help="profiling: GEMM pattern")
    ap.add_argument("--ga-seed", type=int, default=2011)
    ap.add_argument("--ga-timeout-ms", type=float, default=3000.0)
    ap.add_argument("--grid", type=int, nargs=3, default=None,
                    help="profiling only: a smaller I J K than the benchmark workload")
    ap.add_argument("--iters", type=int, default=None, help="profiling only")
    args = ap.parse_args()
    global I, J, K, ITERS, STENCIL_BYTES, WORKLOAD
    if args.grid or args.iters:
        I, J, K = args.grid or (I, J, K)
        ITERS = args.iters or ITERS
        STENCIL_BYTES = 56 * nint(I, J, K)
        WORKLOAD = "jacobi19_%dx%dx%d_it%d_gene63_hoist" % (I, J, K, ITERS)
        args.no_cpu_baseline = True
        args.no_blocks = True
    if args.impl == "reference":
        return run_reference(args)
    if args.fb:
        return run_fb(args)
    if args.hoist:
        return run_hoist(args)
    if args.genes:
        return run_genes(args)
    if args.ga:
        return run_ga(args)
    if args.block:
        return run_block(args)
    if args.blocks_sweep:
        return run_blocks_sweep(args)
    if args.vendor:
        return run_vendor(args)
    if args.batched:
        return run_batched(args)
    if args.serve:
        return run_serve(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
