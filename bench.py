#!/usr/bin/env python
"""Benchmark: FFT GFLOP/s (5 n log2 n) and HBM-roofline fraction of the
plain FP32 path on the large workload, with parity against the FP64 oracle.

One step = one forward transform of each of the three large synthetic
complex64 inputs (seed 1, re/im ~ U[-1,1)): 1-D n = 2^24 (lifted to
4096 x 4096, two passes), 2-D 4096 x 4096 (two passes), 3-D 256^3 (three
axis passes).  Each input is 128 MiB, larger than the 126 MB L2, so no L2
flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl moa|reference]
Multi-GPU (torchrun, one rank per GPU): every rank runs its own replica of
the step (the transforms are independent problems; there is no exchange),
the time is the max over ranks and the value is the whole-job throughput.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FFT GFLOP/s (5n·log2n) & HBM-roofline fraction vs plain FP32 at rel-L2≤2e-6"
WORKLOAD = [("1d_2^24", (1 << 24,)), ("2d_4096^2", (4096, 4096)), ("3d_256^3", (256, 256, 256))]
WORKLOAD_NAME = ("complex64 forward FFT step: 1-D n=2^24 (r=c=4096 four-step) + 2-D 4096x4096 + 3-D 256^3, "
                 "seed 1, re/im ~ U[-1,1)")
TOL = 2e-6


def numel(shape):
    n = 1
    for s in shape:
        n *= s
    return n


def flops(shape):
    n = numel(shape)
    return 5.0 * n * math.log2(n)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def load_traffic(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            t = json.load(fh)
        ent = t.get("kernels", {}).get(kernel_key)
        if ent and ent.get("src_hash") == kernel_src_hash(kernel_key):
            return float(ent["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled in the background."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        loaded = [s for s in sm if smax and s > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, world: int) -> float:
    """Max of a per-rank scalar over all ranks (identity when world == 1)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gflops(flops_per_step: float, steps: int, world: int, max_ms: float) -> float:
    """Aggregate throughput: every rank runs its own step (replicas), the job
    time is the slowest rank's."""
    return world * flops_per_step * steps / (max_ms * 1e-3) / 1e9


def _code_only(src: str) -> str:
    """C/CUDA source without comments and blank lines (edits to comments do
    not change the kernels a capture was taken on)."""
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    lines = (re.sub(r"//.*", "", ln).rstrip() for ln in src.splitlines())
    return "\n".join(ln for ln in lines if ln.strip())


def kernel_src_hash(kernel: str) -> str:
    """Hash of the code of the source files a kernel is built from (its family)."""
    d = os.path.join(ROOT, "paper_0811_2535_gb300", "csrc")
    own = "pipe_kernels.cu" if kernel.startswith("pipe_") else "pass_kernels.cu"
    h = hashlib.sha256()
    for name in (own, "fft_core.cuh", "internal.h", "pdl.cuh"):
        with open(os.path.join(d, name), encoding="utf-8") as fh:
            h.update(name.encode())
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def oracle_step(shapes, seed):
    """Run the FP64 oracle on the given shapes; returns (seconds, outputs)."""
    import numpy as np

    import oracle
    from paper_0811_2535_gb300 import inputs
    oracle.build()
    outs, secs = [], 0.0
    for shape in shapes:
        x = inputs.uniform(shape, seed).astype(np.complex128)
        t0 = time.perf_counter()
        y = oracle.fft_radix2(x, -1) if len(shape) == 1 else oracle.fft_nd(x, len(shape), -1)
        secs += time.perf_counter() - t0
        outs.append(y)
    return secs, outs


def host_cpu() -> dict:
    """The host the CPU legs ran on: architecture, CPU model (lscpu), cores."""
    import platform
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"machine": platform.machine(), "model": model or platform.processor(), "nproc": os.cpu_count()}


def template_step(shapes, seed, reps: int = 2):
    """The paper's all-processor templates on every host core: Fig. 6.4 for
    the 1-D transform (m = the largest power of two <= the threads, at most
    sqrt(n), breakpoint log2(n/m) + 1) and Eq. B.6 with the lines of each axis
    in parallel for the others.  One untimed pass, then `reps` timed ones;
    returns (seconds per step, threads, m, whether every output equals the
    sequential oracle's bit for bit)."""
    import numpy as np

    import oracle
    from paper_0811_2535_gb300 import inputs
    oracle.build()
    threads = oracle.template_threads()
    xs = [inputs.uniform(shape, seed).astype(np.complex128) for shape in shapes]
    m_used = 1

    def one(keep):
        nonlocal m_used
        secs, outs = 0.0, []
        for shape, x in zip(shapes, xs):
            y = x.copy()
            t0 = time.perf_counter()
            if len(shape) == 1:
                n = shape[0]
                m = 1
                while m * 2 <= threads and (m * 2) * (m * 2) <= n:
                    m *= 2
                m_used = m
                y = oracle.template_partitioned(y, m, int(np.log2(n // m)) + 1, -1)
            else:
                oracle.template_nd(y, len(shape), -1, inplace=True)
            secs += time.perf_counter() - t0
            if keep:
                outs.append(y)
        return secs, outs

    one(False)
    secs, outs = 0.0, []
    for r in range(reps):
        s, o = one(r == reps - 1)
        secs += s
        outs = o or outs
    same = True
    for shape, x, y in zip(shapes, xs, outs):
        ref = oracle.fft_radix2(x, -1) if len(shape) == 1 else oracle.fft_nd(x, len(shape), -1)
        same = same and bool(np.array_equal(y, ref))
    return secs / reps, threads, m_used, same


def reference_shapes(scale_log2: int):
    """The large workload with every transform shrunk by 2^scale_log2 (at most
    2^11; every axis stays a power of two >= 2: the 3-D transform loses up to
    2^7 on its last axis, the rest on its middle axis)."""
    s = scale_log2
    a = min(s, 7)
    return [(1 << (24 - s),), (4096, 4096 >> s), (256, 256 >> (s - a), 256 >> a)]


def run_reference(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    import numpy as np  # noqa: F401
    from paper_0811_2535_gb300 import inputs
    # pick the sample so that (warmup + steps) oracle steps take about 2 minutes
    budget = 120.0 / max(1, args.steps + args.warmup)
    scale = 10
    probe, _ = oracle_step(reference_shapes(scale), inputs.SEED_LARGE)
    while scale > 0 and probe * 2.2 <= budget:
        scale -= 1
        probe *= 2.1
    shapes = reference_shapes(scale)
    for _ in range(args.warmup):
        oracle_step(shapes, inputs.SEED_LARGE)
    secs = 0.0
    for _ in range(args.steps):
        s, _ = oracle_step(shapes, inputs.SEED_LARGE)
        secs += s
    f = sum(flops(sh) for sh in shapes)
    value = f * args.steps / secs / 1e9
    sample = f"each step: 1-D 2^{24 - scale} + 2-D 4096x{4096 >> scale} + 3-D 256x256x{256 >> scale}, FP64 oracle"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD_NAME, "sample_scale_log2": scale},
            "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": 1, "kind": "oracle", "sample": sample,
                             "host": host_cpu()},
            "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0

def graph_time_ms(torch, fn, iters):
    """Mean time of `fn(stream)` replayed from a captured CUDA graph."""
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn(s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn(torch.cuda.current_stream())
    for _ in range(2):
        g.replay()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(iters):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / iters


def batched_report(torch, moafft, inputs, dev, iters):
    """Uneven batch (4096 transforms of 2^k points, k ~ U{6..16}, seed 2):
    the one persistent launch against the plain FP32 per-size baseline --
    the same transforms laid out grouped by length and run as one batched
    plan per distinct length (11 launches) -- both replayed from CUDA
    graphs."""
    import numpy as np
    lengths, vecs = inputs.uneven_batch(4096, inputs.SEED_UNEVEN)
    lengths = [int(n) for n in lengths]
    x = torch.from_numpy(np.concatenate(vecs)).to(dev)
    out = torch.empty_like(x)
    f = sum(flops((n,)) for n in lengths)
    alg = 16.0 * sum(lengths)
    bp = moafft.BatchedPlan(lengths, -1)
    choice = bp.choice()
    t_batch = graph_time_ms(torch, lambda st: bp.exec(x, out, stream=st), iters)
    bp.destroy()
    # per-size baseline: the transforms of each length contiguous, one plan each
    sizes = sorted(set(lengths))
    groups = {n: [v for v, m in zip(vecs, lengths) if m == n] for n in sizes}
    xg = torch.from_numpy(np.concatenate([np.concatenate(groups[n]) for n in sizes])).to(dev)
    og = torch.empty_like(xg)
    blocks, off = [], 0
    for n in sizes:
        cnt = len(groups[n])
        blocks.append((moafft.Plan([n], cnt, -1), off, n * cnt))
        off += n * cnt

    def per_size(st):
        for p, o, m in blocks:
            p.exec(xg[o:o + m], og[o:o + m], stream=st)
    t_size = graph_time_ms(torch, per_size, iters)
    for p, _, _ in blocks:
        if p.status() != 0:
            raise RuntimeError("device status word set in the per-size baseline")
        p.destroy()
    return {"workload": "4096 x 1-D 2^k, k ~ U{6..16} (seed 2), N(0,1), complex64 forward",
            "plan": choice, "algorithmic_bytes": alg,
            "persistent_graph_us": t_batch * 1e3, "persistent_GFLOPs": f / t_batch / 1e6,
            "persistent_algorithmic_GBps": alg / t_batch / 1e6,
            "per_size_graph_us": t_size * 1e3, "per_size_launches": len(blocks),
            "per_size_GFLOPs": f / t_size / 1e6, "per_size_algorithmic_GBps": alg / t_size / 1e6,
            "speedup_vs_per_size": t_size / t_batch}


def tensor_core_report(torch, moafft, inputs, dev, iters, with_oracle):
    """Precision workload 16384 x 4096 (U[-1,1) noise plus 5 complex
    sinusoids of amplitude 10 per row, seed 3): the plain FP32 row kernel against the
    tensor-core paths (radix-16 DFT blocks as FP16 hi/lo or BF16 hi/mid/lo
    products with FP32 accumulation), on tcgen05 and, as the legacy baseline,
    on mma.sync.  Errors: relative L2 per row against
    the FP64 oracle on 32 sampled rows (oracle leg only)."""
    import numpy as np
    n, batch = 4096, 16384
    x_h = inputs.sinusoids(batch, n, inputs.SEED_PRECISION)
    x = torch.from_numpy(x_h).to(dev)
    out = torch.empty_like(x)
    stream = torch.cuda.current_stream(dev)
    rows = np.random.default_rng(5).choice(batch, 32, replace=False)
    ref = None
    if with_oracle:
        import oracle
        ref = oracle.fft_radix2(x_h[rows].astype(np.complex128), -1)
    alg = 16.0 * n * batch
    rep = {"workload": "16384 x 1-D 4096, U[-1,1) + 5 sinusoids amp 10 (seed 3), complex64 forward"}
    for name, dt, kern in (("fp32", 0, ""), ("tc_fp16", 1, ""), ("tc_bf16", 2, ""), ("tc_fp16_mma_sync", 1, "sync"),
                           ("tc_bf16_mma_sync", 2, "sync")):
        os.environ["MOA_TC_KERNEL"] = kern
        p = moafft.Plan([n], batch, -1, dt)
        for _ in range(3):
            p.exec(x, out, stream=stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(iters):
            p.exec(x, out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) / iters * 1e3
        ent = {"kernel": p.pass_info(0)["kernel"], "us": us, "GFLOPs": flops((n,)) * batch / us / 1e3,
               "algorithmic_GBps": alg / us / 1e3}
        if ref is not None:
            y = out.cpu().numpy()[rows].astype(np.complex128)
            err = np.linalg.norm(y - ref, axis=-1) / np.linalg.norm(ref, axis=-1)
            ent["rel_l2_max"] = float(err.max())
            ent["rel_l2_median"] = float(np.median(err))
        if p.status() != 0:
            raise RuntimeError("device status word set in the tensor-core report")
        p.destroy()
        rep[name] = ent
    os.environ.pop("MOA_TC_KERNEL", None)
    return rep


def autograd_report(torch, moafft, inputs, dev, iters):
    """Differentiation workload: batch 256 x n = 2^18 (seed 4), loss =
    sum |H * F(x)|^2 with a fixed complex filter H, backward through the
    adjoint kernel (MoaFFTFunction).  Reports the whole forward + backward
    step and the two transforms alone (exec + exec_adjoint), each moving
    32n bytes per transform through HBM (two passes)."""
    n, batch = 1 << 18, 256
    H, x_h = inputs.spectral_filter(n, batch, inputs.SEED_GRADIENT)
    Hd = torch.from_numpy(H).to(dev)
    x = torch.from_numpy(x_h.reshape(batch, n)).to(dev).requires_grad_(True)
    plan = moafft.Plan([n], batch, -1)
    stream = torch.cuda.current_stream(dev)

    def fwd_bwd():
        x.grad = None
        y = moafft.fft_autograd(x, plan)
        loss = (Hd * y).abs().pow(2).sum()
        loss.backward()

    y0 = torch.empty_like(x.detach())
    g0 = torch.empty_like(y0)

    def transforms():
        plan.exec(x.detach(), y0, stream=stream)
        plan.exec_adjoint(y0, g0, stream=stream)

    out = {"workload": "256 x 1-D 2^18 (seed 4), loss sum|H*F(x)|^2, backward by the adjoint kernel",
           "passes": [plan.pass_info(i)["kernel"] for i in range(plan.info()["passes"])]}
    for name, fn in (("fwd_bwd_step", fwd_bwd), ("fft_plus_adjoint", transforms)):
        for _ in range(3):
            fn()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(iters):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) / iters * 1e3
        out[name + "_us"] = us
    t = out["fft_plus_adjoint_us"]
    out["fft_GFLOPs"] = 2 * batch * flops((n,)) / t / 1e3
    out["fft_algorithmic_GBps"] = 2 * 32.0 * n * batch / t / 1e3
    if plan.status() != 0:
        raise RuntimeError("device status word set in the autograd report")
    plan.destroy()
    return out


def small_report(torch, moafft, inputs, dev, iters):
    """n = 2^10, batch 1 (seed 0): one exec (a single 4096-point-tile
    launch) and the forward + inverse round trip, as latencies."""
    n = 1 << 10
    x = torch.from_numpy(inputs.uniform((n,), inputs.SEED_SMALL)).to(dev)
    y = torch.empty_like(x)
    z = torch.empty_like(x)
    plan = moafft.Plan([n], 1, -1)
    stream = torch.cuda.current_stream(dev)
    out = {"workload": "1-D 2^10, batch 1 (seed 0)", "kernel": plan.pass_info(0)["kernel"]}
    for name, fn in (("exec", lambda: plan.exec(x, y, stream=stream)),
                     ("round_trip", lambda: (plan.exec(x, y, stream=stream), plan.exec_adjoint(y, z, stream=stream)))):
        for _ in range(10):
            fn()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(iters):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        out[name + "_us"] = e0.elapsed_time(e1) / iters * 1e3
    zz = z.cpu().numpy() / n
    out["round_trip_rel_err"] = float(abs(zz - x.cpu().numpy()).max() / abs(x.cpu().numpy()).max())
    plan.destroy()
    return out


def schedules_report(torch, moafft, dev, iters, peak):
    """Radix schedules of the in-register stages (Sec. 4.8: any factorisation
    is valid) on batched rows of 2^25 points (256 MiB in, 256 MiB out):
    0 = radix 16 with the small radix first, 1 = small radix last, 2 =
    radix-8 stages, 3 = warp-shuffle kernel (cross-lane butterflies by
    shfl.xor, no shared-memory exchange); then what the autotuner keeps."""
    saved = {k: os.environ.get(k) for k in ("MOA_SCHED", "MOA_AUTOTUNE")}
    out = {}
    try:
        for L in (9, 11):
            n, batch = 1 << L, (1 << 25) >> L
            x = torch.randn(n * batch, dtype=torch.complex64, device=dev)
            y = torch.empty_like(x)
            stream = torch.cuda.current_stream(dev)
            res = {}
            os.environ["MOA_AUTOTUNE"] = "0"
            for v in (0, 1, 2, 3):
                os.environ["MOA_SCHED"] = str(v)
                plan = moafft.Plan([n], batch, -1)
                kern = plan.pass_info(0)["kernel"]
                if any(r["kernel"] == kern for r in res.values()):
                    plan.destroy()
                    continue   # the schedule does not exist for this length
                for _ in range(3):
                    plan.exec(x, y, stream=stream)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                for _ in range(iters):
                    plan.exec(x, y, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                us = e0.elapsed_time(e1) / iters * 1e3
                res[str(v)] = {"kernel": kern, "us": us, "frac": 16.0 * n * batch / (us * 1e3) / peak}
                plan.destroy()
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
            plan = moafft.Plan([n], batch, -1)
            res["autotuned"] = plan.choice()
            plan.destroy()
            out["2^%d x %d rows" % (L, batch)] = res
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return out


NOMINAL_HBM_GBPS = 8000.0   # GB300 HBM3e, nominal


def digest(line):
    """Headline figures of every report, a few hundred bytes."""
    def r(v, nd=3):
        return None if v is None else round(float(v), nd)
    rf, l1 = line["roofline"], line["lifted_1d"]
    d = {"step_us": r(line["ms_per_step"] * 1e3, 1), "TFLOPs": r(line["value"] / 1e3),
         "dominant": rf["kernel"], "dominant_frac": r(rf["frac"]), "dominant_frac_nominal": r(rf["frac_nominal"]),
         "1d_2^24_us": r(l1["time_us"], 1), "1d_2^24_frac": r(l1["frac"]),
         "1d_2^24_frac_nominal": r(l1["frac_nominal"]), "1d_2^24_in_step_us": r(l1["in_step_us"], 1),
         "1d_2^24_in_step_frac": r(l1["in_step_frac"]), "parity_ok": line["parity_ok"]}
    b = line.get("batched_uneven")
    if b:
        d["batched_us"] = r(b["persistent_graph_us"], 1)
        d["batched_per_size_us"] = r(b["per_size_graph_us"], 1)
        d["batched_frac"] = r(b["persistent_algorithmic_GBps"] / rf["peak"])
    t = line.get("tensor_core")
    if t:
        for k in ("fp32", "tc_fp16", "tc_bf16"):
            if k in t:
                d[k + "_us"] = r(t[k]["us"], 1)
                if "rel_l2_max" in t[k]:
                    d[k + "_rel_l2_max"] = float("%.2e" % t[k]["rel_l2_max"])
    sc = line.get("radix_schedules")
    if sc:
        for w, res in sc.items():
            d["sched_" + w.split()[0] + "_us"] = {k: r(v["us"], 1) for k, v in res.items() if k != "autotuned"}
    a = line.get("autograd")
    if a:
        d["autograd_fft_adjoint_us"] = r(a["fft_plus_adjoint_us"], 1)
        d["autograd_frac"] = r(a["fft_algorithmic_GBps"] / rf["peak"])
    if line.get("e2e"):
        d["e2e_GFLOPs"] = r(line["e2e"]["value"], 1)
    return d


def run_moa(args):
    import numpy as np
    import torch

    from paper_0811_2535_gb300 import build as _build
    from paper_0811_2535_gb300 import inputs, moafft

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        if local != 0:
            dist.barrier()   # local rank 0 builds (or finds built) the library first
    _build.build()
    if world > 1 and local == 0:
        torch.distributed.barrier()
    moafft.lib()

    plans, xs, outs, pass_kernels, pass_bytes, choices = [], [], [], {}, {}, {}
    for name, shape in WORKLOAD:
        p = moafft.Plan(list(shape), 1, -1)
        choices[name] = p.choice()   # which candidate the autotuner kept, and why
        pass_kernels[name] = [p.pass_info(i)["kernel"] for i in range(p.info()["passes"])]
        for i, kname in enumerate(pass_kernels[name]):
            # algorithmic bytes of one launch: 16 per element and pass it does
            pass_bytes[kname] = float(p.pass_info(i)["bytes"])
        plans.append(p)
        xs.append(torch.from_numpy(inputs.uniform(shape, inputs.SEED_LARGE)).to(dev))
        outs.append(torch.empty(numel(shape), dtype=torch.complex64, device=dev))
    stream = torch.cuda.current_stream(dev)
    npass = [len(pass_kernels[name]) for name, _ in WORKLOAD]
    launches_per_step = sum(npass)

    def step(events=None, ei=0):
        """One step through the public call: one exec per transform (its
        passes back to back, as a user runs them); events between transforms."""
        for p, x, o in zip(plans, xs, outs):
            p.exec(x, o, stream=stream)
            if events is not None:
                events[ei].record(stream)
                ei += 1
        return ei

    def pass_step(events, ei):
        """The same work pass by pass, with an event after every pass (for the
        per-kernel durations; the events keep consecutive passes from
        overlapping, so this is not the timed step)."""
        for p, x, o, k in zip(plans, xs, outs, npass):
            for i in range(k):
                p.exec_pass(i, x, o, stream=stream)
                events[ei].record(stream)
                ei += 1
        return ei

    for _ in range(args.warmup):
        step()
    pwarm = [torch.cuda.Event(enable_timing=True) for _ in range(launches_per_step + 1)]
    pass_step(pwarm, 0)
    torch.cuda.synchronize()

    # parity of the timed configuration (outputs of the last warm-up step)
    parity = {}
    cpu_baseline = None
    if rank == 0 and world == 1 and not args.no_oracle:
        secs, refs = oracle_step([s for _, s in WORKLOAD], inputs.SEED_LARGE)
        f = sum(flops(s) for _, s in WORKLOAD)
        cpu_baseline = {"value": f / secs / 1e9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                        "sample": "one full step (1-D 2^24 + 2-D 4096^2 + 3-D 256^3), FP64, 1 thread"}
        tsecs, threads, m, same = template_step([s for _, s in WORKLOAD], inputs.SEED_LARGE)
        cpu_baseline["parallel_template"] = {
            "value": f / tsecs / 1e9, "unit": "GFLOP/s", "cores": threads,
            "kind": "Fig. 6.4 / Eq. B.6 all-processor templates, OpenMP, FP64",
            "sample": f"one full step, mean of 2 after 1 untimed; 1-D on m = {m} processors",
            "bit_identical_to_oracle": same}
        cpu_baseline["host"] = host_cpu()
        for (name, shape), o, ref in zip(WORKLOAD, outs, refs):
            y = o.cpu().numpy().astype(np.complex128).reshape(-1)
            r = ref.reshape(-1)
            parity[name] = float(np.linalg.norm(y - r) / np.linalg.norm(r))

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    # a short untimed ramp so the sampler sees the clocks under load
    for _ in range(max(3, args.warmup)):
        step()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.nvtx.range("moafft: timed steps"):
        t0.record(stream)
        for _ in range(args.steps):
            step()
        t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    total_ms = t0.elapsed_time(t1)

    # per-transform durations: the same number of steps with an event between
    # transforms (an event between two kernels keeps the second from starting
    # early, so these add up to a little more than the timed steps)
    events = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps * len(WORKLOAD) + 1)]
    with torch.cuda.nvtx.range("moafft: per-transform steps"):
        events[0].record(stream)
        ei = 1
        for _ in range(args.steps):
            ei = step(events, ei)
        torch.cuda.synchronize()
    per_transform = {}
    k = 0
    for _ in range(args.steps):
        for name, _shape in WORKLOAD:
            per_transform.setdefault(name, []).append(events[k].elapsed_time(events[k + 1]))
            k += 1

    # the 1-D transform alone, execs back to back (how a caller running many
    # 2^24 transforms on one stream sees it)
    i1d = [name for name, _ in WORKLOAD].index("1d_2^24")
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nb2b = max(10, args.steps)
    with torch.cuda.nvtx.range("moafft: 1-D back to back"):
        b0.record(stream)
        for _ in range(nb2b):
            plans[i1d].exec(xs[i1d], outs[i1d], stream=stream)
        b1.record(stream)
    torch.cuda.synchronize()
    t1d_b2b = b0.elapsed_time(b1) / nb2b

    # per-kernel durations: the same number of steps, pass by pass
    pevents = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps * launches_per_step + 1)]
    with torch.cuda.nvtx.range("moafft: pass-by-pass steps"):
        pevents[0].record(stream)
        ei = 1
        for _ in range(args.steps):
            ei = pass_step(pevents, ei)
        torch.cuda.synchronize()
    clocks = sampler.stop()
    per_kernel = {}
    k = 0
    for _ in range(args.steps):
        for name, _shape in WORKLOAD:
            for kname in pass_kernels[name]:
                per_kernel.setdefault((name, kname), []).append(pevents[k].elapsed_time(pevents[k + 1]))
                k += 1
    total_ms = max_over_ranks(total_ms, world)
    ms_per_step = total_ms / args.steps
    f_step = sum(flops(s) for _, s in WORKLOAD)
    value = whole_job_gflops(f_step, args.steps, world, total_ms)

    # roofline of the dominant kernel (largest share of the step time)
    by_kernel = {}
    for (name, kname), ds in per_kernel.items():
        by_kernel.setdefault(kname, []).extend(ds)
    dom = max(by_kernel, key=lambda kn: sum(by_kernel[kn]))
    avg_ms = statistics.mean(by_kernel[dom])
    bytes_per_launch = 16.0 * (1 << 24)     # read + write of n = 2^24 complex64 per pass
    peak, peak_src = load_peaks()
    achieved = pass_bytes[dom] / (avg_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "frac_nominal": achieved / NOMINAL_HBM_GBPS,
                "traffic": load_traffic(dom), "kernel": dom, "peak_source": peak_src,
                "share": sum(by_kernel[dom]) / sum(sum(v) for v in by_kernel.values()),
                "timing": "CUDA events between passes, %d steps run pass by pass after the timed steps" % args.steps}
    kernels = {f"{name}:{kname}": {"avg_us": statistics.mean(ds) * 1e3,
                                   "GB_per_s": pass_bytes[kname] / (statistics.mean(ds) * 1e-3) / 1e9}
               for (name, kname), ds in per_kernel.items()}
    # the lifted 1-D transform as a whole (one exec in the timed steps, its two
    # passes back to back): 32n algorithmic bytes
    t1d = statistics.mean(per_transform["1d_2^24"])
    t1d_passes = sum(statistics.mean(ds) for (name, _k), ds in per_kernel.items() if name == "1d_2^24")
    lifted = {"time_us": t1d_b2b * 1e3, "algorithmic_bytes": 2 * bytes_per_launch,
              "achieved_GBps": 2 * bytes_per_launch / (t1d_b2b * 1e-3) / 1e9,
              "timing": "%d execs back to back on one stream between two events" % nb2b,
              "in_step_us": t1d * 1e3, "in_step_frac": 2 * bytes_per_launch / (t1d * 1e-3) / 1e9 / peak,
              "passes": pass_kernels["1d_2^24"], "sum_of_pass_times_us": t1d_passes * 1e3}
    lifted["frac"] = lifted["achieved_GBps"] / peak
    lifted["frac_nominal"] = lifted["achieved_GBps"] / NOMINAL_HBM_GBPS

    # end to end through the C ABI with host buffers (pinned), copies timed.
    # Each transform of the step has a stream of its own (as a caller with
    # several arrays would), so one transform's copies overlap another's
    # copies and kernels; the step is then bound by the host link with both
    # directions busy.
    e2e_steps = max(1, min(args.steps, 10))
    hin = [torch.from_numpy(inputs.uniform(s, inputs.SEED_LARGE).reshape(-1)).pin_memory() for _, s in WORKLOAD]
    hout = [torch.empty_like(h).pin_memory() for h in hin]
    dbuf = [torch.empty(numel(s), dtype=torch.complex64, device=dev) for _, s in WORKLOAD]
    xstreams = [torch.cuda.Stream(dev) for _ in WORKLOAD]

    def e2e_step():
        for p, a, b, d, xst in zip(plans, hin, hout, dbuf, xstreams):
            p.exec_host(a, b, d, stream=xst)

    e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.nvtx.range("moafft: end-to-end steps"):
        e0.record(stream)
        for xst in xstreams:
            xst.wait_event(e0)
        for _ in range(e2e_steps):
            e2e_step()
        for xst in xstreams:
            stream.wait_stream(xst)
        e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), world)
    io_bytes = sum(8 * numel(s) for _, s in WORKLOAD)
    e2e = {"value": whole_job_gflops(f_step, e2e_steps, world, e2e_ms), "unit": "GFLOP/s",
           "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes, "streams": len(xstreams)}

    for p in plans:
        if p.status() != 0:
            raise RuntimeError("device status word set after the benchmark")
    batched = None if args.no_batched else batched_report(torch, moafft, inputs, dev, max(3, min(args.steps, 20)))
    autograd = None if args.no_batched else autograd_report(torch, moafft, inputs, dev, max(3, min(args.steps, 20)))
    small = None if args.no_batched else small_report(torch, moafft, inputs, dev, 200)
    schedules = None if args.no_batched else schedules_report(torch, moafft, dev, 20, peak)
    tensor_core = None if args.no_batched else tensor_core_report(torch, moafft, inputs, dev, max(3, min(args.steps, 20)),
                                                                  not args.no_oracle)

    if rank == 0:
        # long sections first; a compact digest of every report last, so the
        # end of the line (what a log tail keeps) carries the headline figures
        line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD_NAME, "l2": "inputs larger than L2 (128 MiB each), no flush",
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "passes_per_step": launches_per_step},
                "plans": choices, "kernels": kernels, "tensor_core": tensor_core, "batched_uneven": batched, "autograd": autograd,
                "small_1d": small, "radix_schedules": schedules, "cpu_baseline": cpu_baseline, "e2e": e2e, "clocks": clocks,
                "gpu_launches": launches_per_step * args.steps, "rel_l2": parity or None,
                "parity_ok": (all(v <= TOL for v in parity.values()) if parity else None),
                "roofline": roofline, "lifted_1d": lifted}
        line["summary"] = digest(line)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["moa", "reference"], default="moa")
    ap.add_argument("--no-oracle", action="store_true", help="skip the CPU oracle parity/baseline leg")
    ap.add_argument("--no-batched", action="store_true", help="skip the uneven-batch, tensor-core, autograd and small-n reports")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_moa(args)


if __name__ == "__main__":
    sys.exit(main())
