"""Benchmark: grouped pairwise tensordot on GB300 (tcgen05, bf16 operands,
float32 accumulation), 2048 random contraction specs in one launch.

Workload: 2048 specs from the seeded spec generator (seed 2): ranks 3-5,
dims uniform in {8,16,24,32,48,64}, 1-3 shared legs in random leg order,
every operand and result capped at 2^24 elements; float32 N(0,1) entries
drawn on the device (torch Philox, seeded). 2.01 TFLOP and 31.9 GB of
float32 operands and results per step, far larger than L2 (129 MB), so no
L2 flush is needed between steps.

One step = one tn_group_plan_run (pack, the GEMM on packed operands and the
fused GEMM of the thin contractions, plus a zeroing launch for the results
accumulated over split k ranges). The operands live in one device buffer
and the results in another (each tensor a view). The line also reports the
split-bf16x3 and plain-fp32 paths on the same workload, the end-to-end rate
through the public API from and to pinned host buffers (StagedGroupPlan: every
step copies all operands in and all results out, in 32 chunks whose copies and
kernels overlap; the single-copy form beside it), the roofline of
the dominant kernel, SM clocks sampled during the timed region, and the FP64
CPU oracle timed on a bounded sample (first 16 specs) on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "contraction TFLOP/s & % tensor peak; MPS fwd+bwd samples/s vs plain FP32 at tol"
N_SPECS = 2048
SEED = 2
CPU_SAMPLE_SPECS = 16     # cpu_baseline: first 16 specs (6.2 GFLOP)
REF_STEP_SPECS = 4        # --impl reference: first 4 specs per step


def workload_config(n=N_SPECS):
    """The workload's description; n < 2048 (--specs) is a smaller case of it
    for profiling, not the bench workload, and says so."""
    spec = ("2048 random specs" if n >= N_SPECS else "the first %d of the 2048 random specs" % n)
    return {"workload": "grouped tensordot: " + spec + " (rank 3-5, dims {8,16,24,32,48,64}, "
                        "1-3 shared legs in random order, 2^24-element cap), fp32 in/out, one launch",
            "specs": min(n, N_SPECS), "seed": SEED, "precision": "bf16 operands, fp32 accumulate (tcgen05)",
            "l2": ("inputs and results (31.9 GB) larger than L2; no flush needed" if n >= N_SPECS else
                   "a subset of the bench workload (profiling case)")}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured"
    return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 50 ms.

    start() returns once the first sample has arrived (so sampling is live
    when the timed region opens) and marks the time; stop() keeps the samples
    taken after that mark, or, when the region was shorter than one interval,
    the first sample after it."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 50

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []          # (monotonic time, line)
        self.first = threading.Event()
        self.t0 = 0.0

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", str(self.INTERVAL_MS)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.first.wait(timeout=5.0)
        self.t0 = time.monotonic()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))
            self.first.set()

    def stop(self):
        if self.proc is None:
            return None
        t1 = time.monotonic()
        # one more interval, so that a region shorter than it still has a sample
        time.sleep(self.INTERVAL_MS * 1.5e-3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        during = [ln for t, ln in self.lines if self.t0 <= t <= t1]
        if not during:
            during = [ln for t, ln in self.lines if t >= self.t0][:1]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in during:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm), "interval_ms": self.INTERVAL_MS}


def dist_env():
    from paper_1905_01330_gb300 import dist as tndist
    return tndist.env()


def cpu_oracle_sample(specs_h, count):
    """Times the FP64 oracle on the first `count` specs; returns (flop/s, seconds, flops, cores)."""
    import oracle
    from paper_1905_01330_gb300 import synth
    oracle.lib()
    data = []
    flops = 0.0
    for i, (sa, la, sb, lb) in enumerate(specs_h[:count]):
        A = synth.normal_f32(synth.substream(SEED, 2 * i), sa)
        B = synth.normal_f32(synth.substream(SEED, 2 * i + 1), sb)
        data.append((A, la, B, lb))
        flops += 2.0 * np.prod(synth.spec_sizes((sa, la, sb, lb)))
    t0 = time.perf_counter()
    for A, la, B, lb in data:
        oracle.tensordot(A, la, B, lb)
    dt = time.perf_counter() - t0
    return flops / dt, dt, flops, len(os.sched_getaffinity(0))


def cpu_oracle_rows():
    """The FP64 oracle on the host cores for the rows timed in the extras,
    each once on a stated case (a few seconds in all): node splitting (numpy's
    LAPACK SVD in float64), ncon of the N=20, chi=32 norm network, and the
    classifier with one MPS per label on a 64-sample subset."""
    import oracle
    from paper_1905_01330_gb300 import synth
    out = {}
    rng = np.random.default_rng(7)
    for name, shape, left, right, keep in (("split_node_two_site_chi128", (128, 2, 2, 128), [0, 1], [2, 3], 128),
                                           ("split_node_n1000_keep5", (1000, 1000), [0], [1], 5)):
        A = rng.standard_normal(shape).astype(np.float32)
        t0 = time.perf_counter()
        oracle.split_node(A, left, right, max_singular_values=keep)
        out[name] = {"ms": 1e3 * (time.perf_counter() - t0)}
    m = synth.random_mps(20, 2, 32, seed=1)
    net = []
    for base in (1000, 2000):
        for i in range(20):
            net.append((base + i if i > 0 else 0, 100 + i, base + i + 1 if i < 19 else 1))
    t0 = time.perf_counter()
    oracle.ncon(m + m, net)
    out["ncon_mps_norm_n20_chi32"] = {"ms": 1e3 * (time.perf_counter() - t0)}
    mps = synth.classifier_separate_mps(784, 32, 10, seed=122, eps_std=0.1)
    px = synth.pixels(64, 784, seed=3)
    t0 = time.perf_counter()
    oracle.classify_separate(mps, px)
    dt = time.perf_counter() - t0
    out["classifier_separate_chi32_L10"] = {"samples_per_s": 64 / dt, "sample": "first 64 of 4096 samples"}
    return out


def _time(fn, reps, warm, stream):
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _time_graph(fn, calls, replays, stream):
    """Per-call time of `fn` captured `calls` times into one CUDA graph, the
    graph replayed `replays` times (after one eager warm-up call)."""
    import torch
    fn()
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        fn()
    stream.wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(calls):
            fn()
    g.replay()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(replays):
        g.replay()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / (replays * calls)


def kernel_traffic(kernel, nbytes):
    """DRAM bytes per launch of `kernel` (a launch name of the plan: "pack",
    "gemm", "gemm_fused"), from the committed ncu capture, when that capture
    was taken of the kernel source as it is now (same SHA-256); else None. The
    capture ran a smaller case; its measured traffic over its algorithmic
    bytes scales to this launch's algorithmic bytes (the kernels move bytes in
    proportion to the operands and results)."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "packed_traffic.json")
    src = os.path.join(ROOT, "paper_1905_01330_gb300", "csrc", "packed.cu")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    with open(src, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    if d.get("source_sha256") != sha or kernel not in d.get("kernels", {}):
        return None
    return d["kernels"][kernel]["traffic_over_algorithmic"] * nbytes


def _score_err(ft, lam, ft_ref, lam_ref):
    ft = ft.double().cpu().numpy()
    got = ft * np.exp(lam.cpu().numpy() - lam_ref)[:, None]
    e = np.linalg.norm(got - ft_ref, axis=1) / np.linalg.norm(ft_ref, axis=1)
    return {"median": float(np.median(e)), "max": float(np.max(e))}


def _energy_golden():
    """The oracle's stored TFIM energies (tests/golden/energy_oracle.txt)."""
    rows = {}
    with open(os.path.join(ROOT, "tests", "golden", "energy_oracle.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, chi, n, seed, e, le, v, lv, _, _ = line.split()
            rows[k] = {"chi": int(chi), "n": int(n), "seed": int(seed), "energy": float(e) * np.exp(float(le)),
                       "norm": float(v) * np.exp(float(lv))}
    return rows


def _lc_mps_device(n, d, chi, seed, dev):
    """Left-canonical MPS built on the device (seeded normals, Householder QR,
    R's diagonal made positive), float64 then rounded to float32 once."""
    import torch
    from paper_1905_01330_gb300 import synth
    bonds = synth.mps_bonds(n, d, chi)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    cores = []
    for i in range(n):
        rows, cols = bonds[i] * d, bonds[i + 1]
        m = torch.randn(rows, cols, dtype=torch.float64, device=dev, generator=g)
        q, r = torch.linalg.qr(m)
        sgn = torch.sign(torch.diagonal(r))
        sgn[sgn == 0] = 1.0
        cores.append((q * sgn[None, :]).reshape(bonds[i], d, cols).float().contiguous())
    return cores


def _expect_flops(cores, W):
    f = 0.0
    d = cores[0].shape[1]
    for A, w in zip(cores, W):
        Da, Db = A.shape[0], A.shape[2]
        wa, wb = w.shape[0], w.shape[1]
        f += 2.0 * wa * Da * d * Db * Da          # (i)
        f += 2.0 * wb * d * Da * Db * wa * d      # (ii)
        f += 2.0 * wb * Db * Db * d * Da          # (iii)
        f += 2.0 * Da * d * Db * Da + 2.0 * Db * Db * Da * d  # norm sweep
    return f


def run_extras(tn, synth, dev, stream):
    """Secondary measurements of the other hot-path rows, on their own workloads:
    classifier forward (784 sites, batch 4096, chi 32/64/128) and training step
    (chi 64) in float32, bf16 and split bf16x3; the config-1 norm; the
    config-5 energies. Every reduced-precision result states its error against
    the FP64 oracle on a deterministic subset: the first 256 samples of the
    classifier batch, the oracle's stored energies of the workload chains
    (tests/golden/energy_oracle.txt). The oracle runs that produce those
    errors are timed and reported as CPU baselines (cpu_rows)."""
    import torch
    import oracle
    out, cpu_rows = {}, {}
    B, n, ls, L = 4096, 784, 392, 10
    SUB = 256
    px_h = synth.pixels(B, n, seed=3)
    px = torch.from_numpy(px_h).to(dev)
    y_h = synth.labels(B, L, seed=4)
    y = torch.from_numpy(y_h).to(dev)
    cls = {}
    for chi in (32, 64, 128):
        cores_h = synth.classifier_mps(n, chi, ls, L, seed=30 + chi, eps_std=0.1)
        cores = [torch.from_numpy(c).to(dev) for c in cores_h]
        flops = sum(4.0 * B * c.shape[0] * c.shape[-1] for i, c in enumerate(cores) if i != ls)
        entry = {"forward_gflop": flops / 1e9}
        t0 = time.perf_counter()
        ft_ref, lam_ref = oracle.classify(cores_h, ls, px_h[:SUB])
        dt = time.perf_counter() - t0
        cpu_rows["classifier_forward_chi%d" % chi] = {
            "samples_per_s": SUB / dt, "gflops": flops * SUB / B / dt / 1e9,
            "sample": "first %d of the 4096 samples (%.1f s)" % (SUB, dt)}
        ws = tn.classifier_workspace(cores, ls, L, B, 0)
        for prec in ("fp32", "bf16", "bf16x3"):
            fwd = lambda: tn.mps_classify(cores, ls, px, prec=prec, ckpt_every=0, workspace=ws)
            # device time from a CUDA graph (the eager figure includes the
            # binding's per-call marshalling of 784 cores, ~0.5 ms of host time)
            ms_eager = _time(fwd, 3, 1, stream)
            ms = _time_graph(fwd, 1, 5, stream)
            ft, lam, _ = fwd()
            entry[prec] = {"ms": ms, "ms_eager": ms_eager, "samples_per_s": B / (ms * 1e-3),
                           "tflops": flops / (ms * 1e-3) / 1e12,
                           "err_vs_oracle_first256": _score_err(ft[:SUB], lam[:SUB], ft_ref, lam_ref)}
        for prec in ("bf16", "bf16x3"):
            entry[prec + "_speedup_vs_fp32"] = entry["fp32"]["ms"] / entry[prec]["ms"]
        cls["chi%d" % chi] = entry
        if chi == 64:
            # training step: forward with checkpoints every 28 sites, loss head,
            # adjoint backward (fwd + bwd samples/s), and the gradient of the
            # first 256 samples against the oracle's
            ck = 28
            train = {"checkpoint_every": ck}
            for prec in ("fp32", "bf16", "bf16x3"):
                ws = tn.classifier_workspace(cores, ls, L, B, ck)

                def step():
                    ft, lam, _ = tn.mps_classify(cores, ls, px, prec=prec, ckpt_every=ck, workspace=ws)
                    loss, dft = tn.mps_classify_loss(ft, y)
                    tn.mps_classify_backward(cores, ls, px, dft, ws, prec=prec, ckpt_every=ck)
                ms_eager = _time(step, 3, 1, stream)
                # BF16 / BF16X3 from a CUDA graph; the FP32 backward builds and
                # uploads its grouped plans in the call, so it runs eagerly
                ms = ms_eager if prec == "fp32" else _time_graph(step, 1, 5, stream)
                train[prec] = {"ms": ms, "ms_eager": ms_eager, "samples_per_s": B / (ms * 1e-3),
                               "tflops": 4 * flops / (ms * 1e-3) / 1e12,
                               "timing": "eager" if prec == "fp32" else "CUDA graph"}
                del ws
            t0 = time.perf_counter()
            _, g_ref = oracle.classify_grad(cores_h, ls, px_h[:SUB], y_h[:SUB])
            dt = time.perf_counter() - t0
            cpu_rows["classifier_train_chi64"] = {"samples_per_s": SUB / dt,
                                                  "sample": "first %d of the 4096 samples (%.1f s)" % (SUB, dt)}
            ws = tn.classifier_workspace(cores, ls, L, SUB, ck)
            pxs, ys = px[:SUB].contiguous(), y[:SUB].contiguous()
            for prec in ("fp32", "bf16", "bf16x3"):
                ft, lam, _ = tn.mps_classify(cores, ls, pxs, prec=prec, ckpt_every=ck, workspace=ws)
                _, dft = tn.mps_classify_loss(ft, ys)
                g = tn.mps_classify_backward(cores, ls, pxs, dft, ws, prec=prec, ckpt_every=ck)
                errs = [float(np.linalg.norm(a.double().cpu().numpy() - r) / np.linalg.norm(r))
                        for a, r in zip(g, g_ref)]
                train[prec]["grad_err_vs_oracle_first256"] = {"median": float(np.median(errs)), "max": float(np.max(errs))}
            for prec in ("bf16", "bf16x3"):
                train[prec + "_speedup_vs_fp32"] = train["fp32"]["ms"] / train[prec]["ms"]
            cls["train_chi64"] = train
            del ws
        del cores
    out["classifier"] = cls

    # one MPS per label (Sec. IV.A): 10 MPS of 784 sites, batch 4096; scores
    # of the first 64 samples against the oracle
    sep = {}
    for chi in (32, 64):
        mps_h = synth.classifier_separate_mps(n, chi, L, seed=90 + chi, eps_std=0.1)
        mps = [[torch.from_numpy(c).to(dev) for c in m] for m in mps_h]
        flops = L * sum(4.0 * B * c.shape[0] * c.shape[-1] for c in mps[0])
        entry = {"forward_gflop": flops / 1e9}
        ft_ref, lam_ref = oracle.classify_separate(mps_h, px_h[:64])
        for prec in ("fp32", "bf16", "bf16x3"):
            ws = tn.classifier_separate_workspace(mps, B, 0)
            fwd = lambda: tn.mps_classify_separate(mps, px, prec=prec, ckpt_every=0, workspace=ws)
            ms_eager = _time(fwd, 2, 1, stream)
            ms = _time_graph(fwd, 1, 3, stream)  # device time (eager adds the marshalling of 10 x 784 cores)
            ft, lam, _ = fwd()
            entry[prec] = {"ms": ms, "ms_eager": ms_eager, "samples_per_s": B / (ms * 1e-3),
                           "tflops": flops / (ms * 1e-3) / 1e12,
                           "err_vs_oracle_first64": _score_err(ft[:64], lam[:64], ft_ref, lam_ref)}
            del ws
        if chi == 64:
            # training step: forward with checkpoints every 28 sites, loss head, adjoint backward of every MPS
            for prec in ("fp32", "bf16", "bf16x3"):
                ws = tn.classifier_separate_workspace(mps, B, 28)

                def sep_step():
                    ft, lam, _ = tn.mps_classify_separate(mps, px, prec=prec, ckpt_every=28, workspace=ws)
                    loss, dft = tn.mps_classify_loss(ft, y)
                    tn.mps_classify_separate_backward(mps, px, dft, ws, prec=prec, ckpt_every=28)
                ms_eager = _time(sep_step, 2, 1, stream)
                # BF16 / BF16X3 from a CUDA graph; the FP32 backward uploads plans in the call
                ms = ms_eager if prec == "fp32" else _time_graph(sep_step, 1, 3, stream)
                entry[prec]["train_step_ms"] = ms
                entry[prec]["train_step_ms_eager"] = ms_eager
                entry[prec]["train_samples_per_s"] = B / (ms * 1e-3)
                del ws
        sep["chi%d_L%d" % (chi, L)] = entry
        del mps
    out["classifier_separate"] = sep

    # large contractions: C[m, n] = sum_k A[m, k] B[k, n] at 8192^3 and
    # 16384^3, one-spec plans (pack + GEMM), each launch timed alone
    _, bf16_peak, _ = measured_peaks()
    big = {}
    for n in (8192, 16384):
        A = torch.randn(n, n, device=dev)
        B = torch.randn(n, n, device=dev)
        C = torch.empty(n, n, device=dev)
        f = 2.0 * n ** 3
        for prec in ("bf16", "bf16x3"):
            pl = tn.GroupPlan([(A, [1], B, [0], C)], prec=prec)
            pl.autotune()
            times = {}
            for i, name in enumerate(pl.launch_names()):
                times[name] = _time(lambda: pl.run_launch(i), 3, 1, stream)
            step = sum(times.values())
            big["n%d_%s" % (n, prec)] = {
                "ms": {k: round(v, 4) for k, v in times.items()},
                "gemm_tflops": f / (times["gemm"] * 1e-3) / 1e12,
                "gemm_frac_of_bf16_peak": f / (times["gemm"] * 1e-3) / 1e12 / bf16_peak,
                "step_tflops": f / (step * 1e-3) / 1e12,
                "step_frac_of_bf16_peak": f / (step * 1e-3) / 1e12 / bf16_peak}
            del pl
        del A, B, C
    out["large_contractions"] = big

    # node splitting (tn_split_node, one-sided Jacobi SVD): the two-site
    # tensor of an MPS sweep, (chi, 2, 2, chi) split between its sites with
    # chi values kept, and the (1000, 1000) node of Appendix A keeping 5
    spl = {}
    gen = torch.Generator(device=dev)
    gen.manual_seed(7)
    for name, shape, left, right, keep in (("two_site_chi128", (128, 2, 2, 128), [0, 1], [2, 3], 128),
                                           ("two_site_chi256", (256, 2, 2, 256), [0, 1], [2, 3], 256),
                                           ("n1000_keep5", (1000, 1000), [0], [1], 5)):
        A = torch.randn(shape, device=dev, generator=gen)
        info = {}
        tn.split_node(A, left, right, max_singular_values=keep, info=info)
        ms = _time(lambda: tn.split_node(A, left, right, max_singular_values=keep), 2, 1, stream)
        spl[name] = {"ms": ms, "jacobi_sweeps": info["sweeps"], "kept": keep}
        del A
    out["split_node"] = spl

    # config 1: <psi|psi>, N=20, chi=32 (one-CTA float32 sweep)
    m_h = synth.random_mps(20, 2, 32, seed=1)
    m = [torch.from_numpy(c).to(dev) for c in m_h]
    res = torch.empty(2, dtype=torch.float64, device=dev)
    us = 1e3 * _time(lambda: tn.mps_inner(m, m, prec="fp32", out=res), 50, 5, stream)
    us_graph = 1e3 * _time_graph(lambda: tn.mps_inner(m, m, prec="fp32", out=res), 20, 10, stream)
    r = res.cpu().numpy()
    out["mps_norm_n20_chi32"] = {"us_per_call_graph": us_graph, "us_per_call_eager": us,
                                 "log_norm": float(np.log(abs(r[0])) + r[1])}

    # ncon (Appendix B): the same <psi|psi> network written as ncon labels
    # (bra and ket cores, physical legs joined, boundary legs joined), 40 steps
    # of tn_contract in float32; no rescaling, so it is compared in value
    net = []
    for base in (1000, 2000):
        for i in range(20):
            net.append((base + i if i > 0 else 0, 100 + i, base + i + 1 if i < 19 else 1))
    ts = m + m
    val = float(tn.ncon(ts, net, prec="fp32"))
    ms_ncon = _time(lambda: tn.ncon(ts, net, prec="fp32"), 5, 2, stream)
    nplan = tn.NconPlan(ts, net, prec="fp32")
    ms_plan = _time(nplan.run, 10, 2, stream)
    nplan.capture()
    ms_graph = _time(nplan.replay, 20, 2, stream)
    out["ncon_mps_norm_n20_chi32"] = {"ms_per_call": ms_ncon, "ms_per_call_plan": ms_plan,
                                      "ms_per_call_plan_graph": ms_graph,
                                      "steps": len(tn.ncon_plan([t.shape for t in ts], net)[0]),
                                      "log_norm": float(np.log(abs(val))),
                                      "log_norm_diff_vs_tn_mps_inner": float(abs(np.log(abs(val)) -
                                                                               (np.log(abs(r[0])) + r[1])))}

    # config 5: TFIM energy, N=100, chi 256 / 512 / 1024, left-canonical.
    # |E| is small against the energy scale J(N-1)+hN of a random state, so
    # errors are stated relative to that scale (times <psi|psi>). Each
    # precision's error against the FP64 oracle comes from the oracle's stored
    # values (tests/golden/energy_oracle.txt): the whole chi = 256 chain and the
    # 20-full-bond-site subset chains of chi = 512 and 1024 (N = 38 and 40, the
    # N = 100 chain's per-site shapes), inputs regenerated from their seeds.
    golden = _energy_golden()

    def energy_err(cores_h, row, prec, grouped=False):
        cores = [torch.from_numpy(c).to(dev) for c in cores_h]
        Wg = [torch.from_numpy(w).to(dev) for w in synth.tfim_mpo(row["n"])]
        r = (tn.mps_expect_grouped([cores], Wg, prec=prec)[0] if grouped else tn.mps_expect(cores, Wg, prec=prec))
        r = r.cpu().numpy()
        e = r[0] * np.exp(r[1])
        return float(abs(e - row["energy"]) / ((2.0 * row["n"] - 1.0) * row["norm"]))

    W = [torch.from_numpy(w).to(dev) for w in synth.tfim_mpo(100)]
    for chi in (256, 512, 1024):
        row = golden["chain_chi%d_n%d" % (chi, 100 if chi == 256 else (38 if chi == 512 else 40))]
        sub_h = synth.left_canonical_mps(row["n"], 2, chi, seed=row["seed"])
        if chi == 256:
            cores = [torch.from_numpy(c).to(dev) for c in sub_h]  # the oracle's chain itself
            t0 = time.perf_counter()
            oracle.mpo_expect(sub_h, synth.tfim_mpo(100))
            dt = time.perf_counter() - t0
            cpu_rows["tfim_energy_n100_chi256"] = {"ms": 1e3 * dt, "sample": "the whole chain (energy sweep only)"}
        else:
            cores = _lc_mps_device(100, 2, chi, 5, dev)
        flops = _expect_flops(cores, W)
        en = {"gflop": flops / 1e9,
              "err_subset": "whole chain" if chi == 256 else "N=%d chain, 20 sites at the full bond" % row["n"]}
        res = torch.empty(4, dtype=torch.float64, device=dev)
        for prec in ("bf16x3", "fp32", "bf16"):
            ms_eager = _time(lambda: tn.mps_expect(cores, W, prec=prec, out=res), 2, 1, stream)
            # the whole sweep captured as one CUDA graph
            ms = _time_graph(lambda: tn.mps_expect(cores, W, prec=prec, out=res), 1, 3, stream)
            en[prec] = {"ms": ms, "ms_eager": ms_eager, "tflops": flops / (ms * 1e-3) / 1e12,
                        "err_vs_oracle_over_energy_scale": energy_err(sub_h, row, prec)}
        out["tfim_energy_n100_chi%d" % chi] = en
        del cores

    # config 5 batch: 64 left-canonical MPS, chi ~ U{64, 96, ..., 512} (seed 50), grouped launches;
    # errors on the batch's first four states (their oracle values stored), run as a grouped batch
    chis = synth.uneven_chis(64, seed=50)
    states = [_lc_mps_device(100, 2, chi, 500 + k, dev) for k, chi in enumerate(chis)]
    flops = sum(_expect_flops(c, W) for c in states)
    en = {"gflop": flops / 1e9, "states": len(states), "chi_min": min(chis), "chi_max": max(chis),
          "err_subset": "the batch's first 4 states (bonds %s), grouped" % chis[:4]}
    res = torch.empty(len(states), 4, dtype=torch.float64, device=dev)
    rows = [golden["batch%d_chi%d_n100" % (k, chis[k])] for k in range(4)]
    sub = [[torch.from_numpy(c).to(dev) for c in synth.left_canonical_mps(100, 2, r["chi"], seed=r["seed"])] for r in rows]
    for prec in ("bf16x3", "fp32", "bf16"):
        # planned once (host layout and tables), then each run only launches
        plan = tn.ExpectGroupedPlan(states, W, prec=prec)
        ms = _time(lambda: plan.run(out=res), 3, 1, stream)
        ms_oneshot = _time(lambda: tn.mps_expect_grouped(states, W, prec=prec, out=res), 2, 1, stream)
        del plan
        r4 = tn.mps_expect_grouped(sub, W, prec=prec).cpu().numpy()
        errs = [abs(r4[k, 0] * np.exp(r4[k, 1]) - row["energy"]) / (199.0 * row["norm"]) for k, row in enumerate(rows)]
        en[prec] = {"ms": ms, "ms_plan_and_run": ms_oneshot, "tflops": flops / (ms * 1e-3) / 1e12,
                    "max_err_vs_oracle_over_energy_scale": float(max(errs))}
    out["tfim_energy_batch64_n100_chi64_512"] = en
    del states, sub

    # config 1 and the oracle's own timing of it (the whole chain)
    m_h = synth.random_mps(20, 2, 32, seed=1)
    t0 = time.perf_counter()
    v, lg = oracle.mps_inner(m_h, m_h)
    cpu_rows["mps_norm_n20_chi32"] = {"us_per_call": 1e6 * (time.perf_counter() - t0), "sample": "the whole chain"}
    out["mps_norm_n20_chi32"]["err_vs_oracle"] = float(abs(out["mps_norm_n20_chi32"]["log_norm"] - (np.log(abs(v)) + lg)))
    out["cpu_rows"] = cpu_rows
    return out


def run_reference(args):
    """The FP64 CPU oracle on the host cores (rank 0 only), same metric and unit."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1905_01330_gb300 import synth
    specs_h = synth.contraction_specs(N_SPECS, seed=SEED)
    for _ in range(args.warmup):
        cpu_oracle_sample(specs_h, REF_STEP_SPECS)
    times, flops = [], 0.0
    cores = len(os.sched_getaffinity(0))
    for _ in range(args.steps):
        r, dt, fl, cores = cpu_oracle_sample(specs_h, REF_STEP_SPECS)
        times.append(dt)
        flops = fl
    total = sum(times)
    value = flops * args.steps / total / 1e12
    line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(),
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": "first %d of the 2048 specs per step (%.2f GFLOP)" % (REF_STEP_SPECS, flops / 1e9)},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0



def run_case(args):
    """One workload of the hot path, a warm-up call and one more, for profilers
    (ncu launch lists and captures); prints the device status, no bench line.
    Cases: classifier_forward, classifier_train, energy, energy_batch,
    mps_norm, grouped_tensordot (the first --specs specs of the bench workload)."""
    import torch
    from paper_1905_01330_gb300 import build, synth, tn
    build.build()
    tn.load()
    dev = torch.device("cuda", 0)
    B, n, ls, L = 4096, 784, 392, 10
    chi, prec = args.chi, args.prec
    if args.case in ("classifier_forward", "classifier_train"):
        px = torch.from_numpy(synth.pixels(B, n, seed=3)).to(dev)
        y = torch.from_numpy(synth.labels(B, L, seed=4)).to(dev)
        cores = [torch.from_numpy(c).to(dev) for c in synth.classifier_mps(n, chi, ls, L, seed=30 + chi, eps_std=0.1)]
        ck = 28 if args.case == "classifier_train" else 0
        ws = tn.classifier_workspace(cores, ls, L, B, ck)
        for _ in range(2):
            ft, lam, _ = tn.mps_classify(cores, ls, px, prec=prec, ckpt_every=ck, workspace=ws)
            if ck:
                loss, dft = tn.mps_classify_loss(ft, y)
                tn.mps_classify_backward(cores, ls, px, dft, ws, prec=prec, ckpt_every=ck)
    elif args.case == "energy":
        # N = 100 TFIM energy; random N(0, 1/chi) cores drawn on the device (the
        # sweep's work does not depend on the values: it rescales every site)
        W = [torch.from_numpy(w).to(dev) for w in synth.tfim_mpo(100)]
        bonds = synth.mps_bonds(100, 2, chi)
        g = torch.Generator(device=dev)
        g.manual_seed(5)
        cores = [torch.randn(bonds[i], 2, bonds[i + 1], device=dev, generator=g) / chi ** 0.5 for i in range(100)]
        res = torch.empty(4, dtype=torch.float64, device=dev)
        for _ in range(2):
            tn.mps_expect(cores, W, prec=prec, out=res)
    elif args.case == "energy_batch":
        # the 64-MPS batch (bonds U{64, ..., 512}, seed 50), random N(0, 1/chi) cores on the device
        W = [torch.from_numpy(w).to(dev) for w in synth.tfim_mpo(100)]
        g = torch.Generator(device=dev)
        g.manual_seed(50)
        states = []
        for c in synth.uneven_chis(64, seed=50):
            bonds = synth.mps_bonds(100, 2, c)
            states.append([torch.randn(bonds[i], 2, bonds[i + 1], device=dev, generator=g) / c ** 0.5
                           for i in range(100)])
        res = torch.empty(len(states), 4, dtype=torch.float64, device=dev)
        for _ in range(2):
            tn.mps_expect_grouped(states, W, prec=prec, out=res)
    elif args.case == "mps_norm":
        m = [torch.from_numpy(c).to(dev) for c in synth.random_mps(20, 2, 32, seed=1)]
        res = torch.empty(2, dtype=torch.float64, device=dev)
        for _ in range(3):
            tn.mps_inner(m, m, prec="fp32", out=res)
    elif args.case == "grouped_tensordot":
        specs_h = synth.contraction_specs(N_SPECS, seed=SEED)[:args.specs]
        gen = torch.Generator(device=dev)
        gen.manual_seed(SEED)
        specs = []
        for sa, la, sb, lb in specs_h:
            A = torch.randn(sa, device=dev, generator=gen)
            Bt = torch.randn(sb, device=dev, generator=gen)
            specs.append((A, list(la), Bt, list(lb), torch.empty(tn.result_shape(A, la, Bt, lb), device=dev)))
        plan = tn.GroupPlan(specs, prec=prec)
        for _ in range(2):
            plan.run()
    else:
        raise SystemExit("unknown case " + args.case)
    torch.cuda.synchronize()
    status = tn.sync_status()
    print("case %s chi %d prec %s status %d" % (args.case, chi, prec, status))
    return 0 if status == 0 else 1

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--specs", type=int, default=N_SPECS,
                    help="first N specs only (smaller case for profiling; not a bench line)")
    ap.add_argument("--variants", default="bf16x3,fp32", help="other paths to time, comma separated, or none")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the classifier, MPS-norm and energy measurements")
    ap.add_argument("--case", default=None,
                    help="run one workload twice for a profiler (classifier_forward, classifier_train, energy, "
                         "energy_batch, mps_norm, grouped_tensordot) instead of the bench")
    ap.add_argument("--chi", type=int, default=64, help="bond dimension of --case")
    ap.add_argument("--prec", default="bf16", help="precision of --case: fp32, bf16, bf16x3")
    args = ap.parse_args()
    if args.case:
        return run_case(args)
    if args.impl == "reference":
        return run_reference(args)

    import torch

    from paper_1905_01330_gb300 import build, synth, tn

    from paper_1905_01330_gb300 import dist as tndist
    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        tndist.init("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    build.build()
    tn.load()

    def barrier():
        tndist.barrier()

    # ---- inputs: spec shapes from SplitMix64, entries from a seeded device generator
    specs_h = synth.contraction_specs(N_SPECS, seed=SEED)[:args.specs]
    gen = torch.Generator(device=dev)
    gen.manual_seed(tndist.data_seed(SEED, rank))
    # all operands in one device buffer and all results in another (each
    # tensor a view starting on a 256-byte boundary), so a step's inputs and
    # results move between host and device as one copy each
    def layout(shapes):
        offs, n = [], 0
        for sh in shapes:
            offs.append(n)
            n += (int(np.prod(sh)) + 63) // 64 * 64
        return offs, n
    in_shapes = [sh for sa, _, sb, _ in specs_h for sh in (sa, sb)]
    out_shapes = [tuple(sa[p] for p in range(len(sa)) if p not in la) + tuple(sb[p] for p in range(len(sb)) if p not in lb)
                  for sa, la, sb, lb in specs_h]
    in_offs, n_in = layout(in_shapes)
    out_offs, n_out_all = layout(out_shapes)
    big_in = torch.empty(n_in, device=dev)
    big_out = torch.empty(n_out_all, device=dev)
    specs = []
    for i, (sa, la, sb, lb) in enumerate(specs_h):
        At = big_in[in_offs[2 * i]:in_offs[2 * i] + int(np.prod(sa))].view(sa)
        Bt = big_in[in_offs[2 * i + 1]:in_offs[2 * i + 1] + int(np.prod(sb))].view(sb)
        At.normal_(generator=gen)
        Bt.normal_(generator=gen)
        Ct = big_out[out_offs[i]:out_offs[i] + int(np.prod(out_shapes[i]))].view(out_shapes[i])
        assert tuple(Ct.shape) == tuple(tn.result_shape(At, la, Bt, lb))
        specs.append((At, list(la), Bt, list(lb), Ct))
    stream = torch.cuda.current_stream(dev)
    var_list = [] if args.variants == "none" else [v for v in args.variants.split(",") if v]
    plans = {p: tn.GroupPlan(specs, prec=p) for p in ["bf16"] + var_list}
    # setup, outside the timed region: the autotuner times the candidate GEMM
    # schedules on this workload and keeps the fastest
    schedules = {p: pl.autotune() for p, pl in plans.items() if p != "fp32"}
    plan = plans["bf16"]
    flops, nbytes = plan.flops, plan.bytes

    def timed(pl, steps, warmup, sampler=None):
        for _ in range(warmup):
            pl.run()
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if sampler:
            sampler.start()
        start.record(stream)
        for a, b in ev:
            a.record(stream)
            pl.run()
            b.record(stream)
        stop.record(stream)
        torch.cuda.synchronize(dev)
        clocks = sampler.stop() if sampler else None
        barrier()
        total_ms = start.elapsed_time(stop)
        per = [a.elapsed_time(b) for a, b in ev]
        return total_ms, per, clocks

    def timed_launches(pl, steps):
        """Average device time of each launch of a run, timed one at a time."""
        names = pl.launch_names()
        ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in names]
              for _ in range(steps)]
        torch.cuda.synchronize(dev)
        for row in ev:
            for i, (a, b) in enumerate(row):
                a.record(stream)
                pl.run_launch(i)
                b.record(stream)
        torch.cuda.synchronize(dev)
        return {n: float(np.mean([row[i][0].elapsed_time(row[i][1]) for row in ev])) for i, n in enumerate(names)}

    sampler = ClockSampler(dev.index if dev.index is not None else 0)
    total_ms, per, clocks = timed(plan, args.steps, args.warmup, sampler)
    status = tn.sync_status()
    if status != 0:
        raise RuntimeError("kernel status %d during the timed region" % status)
    ms_max = tndist.max_over_ranks(total_ms, dev)
    ms_per_step = ms_max / args.steps
    value = tndist.weak_scaling_value(flops, ms_per_step, world) / 1e12
    launch_ms = float(np.mean(per))

    # ---- same workload with the other two arithmetic paths (not the headline)
    variants = {}
    for p in var_list:
        tm, pp, _ = timed(plans[p], max(2, args.steps // 2), 1)
        variants[p] = {"ms_per_step": tm / max(2, args.steps // 2), "tflops": flops / (tm / max(2, args.steps // 2) * 1e-3) / 1e12}
    variants["bf16"] = {"ms_per_step": ms_per_step, "tflops": flops / (ms_per_step * 1e-3) / 1e12}
    if rank == 0 and not args.no_cpu_baseline:
        # each path's error against the FP64 oracle on five of the workload's
        # contractions (the smallest two and three from the middle of the
        # flop-sorted list), normwise against || |A||B| ||_F
        import oracle
        fl = [2.0 * np.prod(synth.spec_sizes(sp)) for sp in specs_h]
        order = np.argsort(fl)
        pick = [int(order[0]), int(order[1])] + [int(order[len(order) // 2 + i]) for i in range(3)]
        ref = {}
        for si in pick:
            At, la, Bt, lb, _ = specs[si]
            a, b = At.cpu().numpy(), Bt.cpu().numpy()
            ref[si] = (oracle.tensordot(a, la, b, lb), np.linalg.norm(oracle.tensordot(np.abs(a), la, np.abs(b), lb)))
        for p in ["bf16"] + var_list:
            plans[p].run()
            torch.cuda.synchronize(dev)
            errs = [float(np.linalg.norm(specs[si][4].double().cpu().numpy() - ref[si][0]) / ref[si][1]) for si in pick]
            variants[p]["err_vs_oracle_5_specs"] = {"max": max(errs), "normwise_against": "|| |A||B| ||_F"}

    # ---- end to end through the C ABI with pinned host buffers
    e2e = None
    if args.e2e_steps > 0:
        # one pinned host buffer for the operands, one for the results, laid
        # out like the device buffers
        host_in = big_in.cpu().pin_memory()
        host_out = torch.empty(big_out.shape, dtype=torch.float32, pin_memory=True)
        h2d = sum(A.numel() * 4 + B.numel() * 4 for A, _, B, _, _ in specs)
        d2h = sum(C.numel() * 4 for *_, C in specs)
        def e2e_time(step):
            step()
            torch.cuda.synchronize(dev)
            barrier()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            for _ in range(args.e2e_steps):
                step()
            s1.record(stream)
            torch.cuda.synchronize(dev)
            return tndist.max_over_ranks(s0.elapsed_time(s1) / args.e2e_steps, dev)

        def serial():
            big_in.copy_(host_in, non_blocking=True)
            plan.run()
            host_out.copy_(big_out, non_blocking=True)
        # the public staged plan: 32 chunks, host -> device copies, kernels and
        # device -> host copies of consecutive chunks overlapping
        staged = tn.StagedGroupPlan(specs, big_in, big_out, chunks=32, prec="bf16", schedule=schedules.get("bf16"))
        e_ms = e2e_time(lambda: staged.run(host_in, host_out))
        serial_ms = e2e_time(serial)
        e2e = {"value": tndist.weak_scaling_value(flops, e_ms, world) / 1e12, "unit": "TFLOP/s", "ms_per_step": e_ms,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "api": "StagedGroupPlan.run(host_in, host_out) = tn_staged_plan_run, 32 chunks",
               "serial_ms_per_step": serial_ms,
               "serial_value": tndist.weak_scaling_value(flops, serial_ms, world) / 1e12}
        del staged, host_in, host_out

    # ---- roofline of each launch of the step, timed one at a time; the
    # algorithmic bytes of each launch come from the plan (each operand
    # element read once, each result written once)
    hbm_peak, bf16_peak, peak_src = measured_peaks()
    algo = {n: b for n, b in zip(plan.launch_names(), plan.launch_bytes()) if n != "zero"}
    lt = timed_launches(plan, max(2, args.steps // 2))
    launches = {}
    for name, ms in lt.items():
        if name not in algo:   # the zeroing of split results: time only
            launches[name] = {"ms": ms}
            continue
        b = algo[name]
        launches[name] = {"ms": ms, "algorithmic_bytes": b, "gbs": b / (ms * 1e-3) / 1e9,
                          "frac_hbm": b / (ms * 1e-3) / 1e9 / hbm_peak}
    lt = {k: v for k, v in lt.items() if k in algo}
    dom = max(lt, key=lt.get)
    achieved_gbs = launches[dom]["gbs"]
    roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved_gbs / hbm_peak, "traffic": kernel_traffic(dom, launches[dom]["algorithmic_bytes"]),
                "kernel": dom, "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)",
                "algorithmic_bytes_per_launch": launches[dom]["algorithmic_bytes"],
                "launches": launches,
                "step_gbs": nbytes / (launch_ms * 1e-3) / 1e9,
                "step_frac": nbytes / (launch_ms * 1e-3) / 1e9 / hbm_peak,
                "tensor_tflops": flops / (launch_ms * 1e-3) / 1e12,
                "tensor_frac": flops / (launch_ms * 1e-3) / 1e12 / bf16_peak}

    # the large contractions of the workload (>= 1 GFLOP each): one grouped
    # plan of just those, its tensor-pipe fraction
    large = None
    if rank == 0 and not args.no_extras:
        big_idx = [i for i, sp in enumerate(specs_h) if 2.0 * np.prod(synth.spec_sizes(sp)) >= 1e9]
        if big_idx:
            lp = tn.GroupPlan([specs[i] for i in big_idx], prec="bf16")
            lp.autotune()
            lt_ms, _, _ = timed(lp, 5, 2)
            lflops = lp.flops
            large = {"specs": len(big_idx), "tflop": lflops / 1e12, "share_of_workload_flops": lflops / flops,
                     "ms": lt_ms / 5, "tflops": lflops / (lt_ms / 5 * 1e-3) / 1e12,
                     "tensor_frac": lflops / (lt_ms / 5 * 1e-3) / 1e12 / bf16_peak,
                     "hbm_gbs": lp.bytes / (lt_ms / 5 * 1e-3) / 1e9}
            del lp

    extras = None
    if rank == 0 and not args.no_extras:
        extras = run_extras(tn, synth, dev, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, dt, fl, cores = cpu_oracle_sample(synth.contraction_specs(N_SPECS, seed=SEED), CPU_SAMPLE_SPECS)
        cpu = {"value": r / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
               "sample": "first %d of the 2048 specs (%.2f GFLOP, %.1f s)" % (CPU_SAMPLE_SPECS, fl / 1e9, dt)}
        if not args.no_extras:
            cpu["other_rows"] = cpu_oracle_rows()
            cpu["other_rows"].update(extras.pop("cpu_rows", {}))

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16", "data": "synthetic", "config": workload_config(args.specs),
                "gpu_launches": args.steps * plan.launches, "clocks": clocks, "e2e": e2e, "roofline": roofline,
                "cpu_baseline": cpu, "variants": variants, "schedules": schedules,
                "tensor_peak_frac": value / world / bf16_peak, "large_contractions_subset": large,
                "extras": extras}
        print(json.dumps(line), flush=True)
    tndist.finish()
    return 0


if __name__ == "__main__":
    sys.exit(main())
