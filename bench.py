#!/usr/bin/env python
"""Throughput of the Super Smoother periodogram on one GB300 (or N, weak).

Workload: one seasonal light curve of 3,000 points over 3,000 d with 100,000
trial frequencies in [0.01, 20) (the single-large-object configuration,
FP64 vs FP32-compensated).  One step = the whole hot path twice over that
input -- Super Smoother (Listing 1) and SuperSmootherSP (Sec. 3) -- through
the C ABI's device entry point in FP32C: fold, sort, smoother, chi2/power
and argmax.  Metric: point*frequency evaluations per second.

The JSON line also carries: FP64 throughput of the same work and its
agreement with FP32C, the oracle checked on sampled frequencies, e2e through
the host entry point from pinned memory, the roofline of the dominant
kernel (ALU-bound), the oracle timed on the host cores, and SM clocks
sampled during the timed region.

--impl reference times the plain FP64 C oracle (the only reference there is)
on the host cores over a bounded sample of the same workload per step.

--serve runs the serving workload instead: Poisson arrivals of single light
curves (2,000 objects/s for 60 s by default, n ~ logU(30, 3000), 10^4
frequencies, SS or SP per request) submitted through the C ABI's serving
entry points (ssp_server_*), and prints sustained objects/s and the
arrival-to-result latency percentiles as its own JSON line.

--matrix c1,c2,c3,c4 measures each configuration for SS and SP in FP32C and
FP64 through the device entry point (one JSON line per configuration and
variant): throughput, roofline fraction, FP32C agreement with FP64, and the
oracle on the host cores over a bounded sample.  C3 is autotuned first
(ssp_autotune; its time is reported, not counted).  C4's FP64 leg runs on a
subset of its objects.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "point·frequency evals/s (SS & SSSP), FP32-comp vs FP64 at tol, 1 GB300"
UNIT = "pt*f/s"
# Algorithmic FP operations per (point, frequency), counted on Friedman's
# updating-formula running line (one op per +, -, *, /): a window slide
# (remove + add) is 36 ops, a fit 4, a cross-validated residual 9 more.
# SS = 3 CV smooths + 3 residual smooths + span smooth + final smooth
#      + span choice/bass (8) + clamp/interpolation (8) + chi2 (3) = 366.
# SP = 3 fits + 3 generalized-validation residuals (3 each) + span choice (8)
#      + interpolation (8) + chi2 (3) = 148.
# SPG = 3 fits + 3 generalized-validation terms + chi2 (3) = 132: one span for
#      the whole fold, so no per-point choice or interpolation.
OPS_PER_PTF = {"ss": 3 * 49 + 3 * 40 + 40 + 40 + 8 + 8 + 3,
               "sp": 3 * 40 + 3 * 3 + 8 + 8 + 3,
               "spg": 3 * 40 + 3 * 3 + 3}


def ops_per_ptf(variant, n_per_object):
    """The smoothing ops above plus the sort, counted as compare/exchange
    steps at the same rate: log2 n per point, the comparison-sort bound,
    averaged over the catalog's points."""
    npo = np.asarray(n_per_object, dtype=np.float64)
    return OPS_PER_PTF[variant] + float(np.sum(npo * np.log2(npo)) / np.sum(npo))
FP32_LANES_PER_SM = 128
# DRAM bytes (read + write) per full-size launch of the FP32C periodogram
# kernels, from one ncu capture of this workload.  They apply only to the
# kernel sources they were taken on: bench.py reports them while the hash of
# those sources still matches, else null.
TRAFFIC_SOURCES = ("ssp_device.cuh", "ssp_kernels.cuh", "ssp_fold.h", "ssp_launch.h", "ssp_fp32.cu")
TRAFFIC = {"sha256": "82c63a68a2f9e2661cc3da8f30fd31d7712eb194ef6c69cc5dd4b84d2f65c77f",
           "ss": 2444032 + 799744, "sp": 1696768 + 15360}


def traffic_per_launch(variant):
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2111_07396_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return TRAFFIC[variant] if h.hexdigest() == TRAFFIC["sha256"] else None
L2_FLUSH_BYTES = 512 << 20


def max_over_ranks(dist, x, device="cpu"):
    """The largest of every rank's x (the job's time is its slowest rank's);
    x itself for a single process.  Any backend: NCCL on the GPUs, gloo in
    the tests."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank_step, steps, seconds):
    """Whole-job throughput: every rank processes its own replica of the
    workload (weak scaling), so the job does world x the units of one rank in
    the slowest rank's time."""
    return world * units_per_rank_step * steps / seconds


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--n-freq", type=int, default=100_000)
    ap.add_argument("--serve", action="store_true", help="serving workload (ssp_server_*)")
    ap.add_argument("--rate", type=float, default=2000.0, help="--serve: arrivals per second")
    ap.add_argument("--duration", type=float, default=60.0, help="--serve: seconds of arrivals")
    ap.add_argument("--serve-autotune", action="store_true",
                    help="--serve: tune the CTA sizes on a sample of the stream's objects first (not timed)")
    ap.add_argument("--serve-slots", type=int, default=0, help="--serve: batch slots (0: the server's default)")
    ap.add_argument("--serve-batch-ptf", type=float, default=0.0,
                    help="--serve: points x frequencies per batch at most (0: the server's default)")
    ap.add_argument("--serve-freq", type=int, default=10_000, help="--serve: trial frequencies")
    ap.add_argument("--matrix", default="", help="comma list of configurations (c1..c4)")
    ap.add_argument("--extras", action="store_true",
                    help="shared-fold and search-and-refine measurements")
    ap.add_argument("--subset-objects", type=int, default=0,
                    help="--matrix: keep the first K objects of each configuration")
    ap.add_argument("--subset-freq", type=int, default=0,
                    help="--matrix: keep F frequencies, evenly spaced over the grid")
    ap.add_argument("--no-oracle", action="store_true", help="--matrix, --serve: skip the oracle sample")
    ap.add_argument("--matrix-variants", default="ss,sp", help="--matrix: comma list of ss, sp, spg")
    return ap.parse_args()


def workload(n_freq):
    from paper_2111_07396_gb300 import synth
    cat = synth.config2(n_freq=n_freq)
    desc = {"workload": f"single seasonal object n={cat.points}, {cat.freq.size} freqs "
                        "in [0.01,20); SS + SP per step",
            "objects": 1, "points": cat.points, "n_freq": int(cat.freq.size),
            "variants": ["ss", "sp"], "precision": "fp32c",
            "l2": "flushed between timed steps (512 MiB write)"}
    return cat, desc


# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
def cpu_baseline(cat, p32=None, budget_s=12.0, max_freq=4096, obj=0, variants=("ss", "sp")):
    """The FP64 oracle, as it stands, on the host cores over a bounded sample
    of the workload's frequencies (both variants, or `variants`) for object
    `obj`; with p32 (this run's FP32C powers of that object) also the oracle
    at a few sampled frequencies against them."""
    import oracle
    t, y, dy = cat.obj(obj)
    n = t.size
    codes = [{"ss": oracle.SS, "sp": oracle.SP, "spg": oracle.SPG}[v] for v in variants]
    rng = np.random.default_rng(7)
    order = rng.permutation(cat.freq.size)
    cores = os.cpu_count() or 1
    done, used = 0, 0.0
    batch = max(cores, 16)
    while done < max_freq and used < budget_s:
        fq = cat.freq[order[done:done + batch]]
        t0 = time.perf_counter()
        for code in codes:
            oracle.periodogram(t, y, dy, [n], fq, code, n_threads=cores)
        used += time.perf_counter() - t0
        done += fq.size
    ptf = len(codes) * n * done
    out = {"value": ptf / used, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{done} of {cat.freq.size} frequencies (random), "
                     f"{'+'.join(v.upper() for v in variants)}, object {obj} (n={n}), "
                     f"{used:.1f} s wall"}
    if p32 is not None:
        from tests.parity import gate_error, oracle_powers, sample_freqs
        chk = {}
        for v, code in (("ss", oracle.SS), ("sp", oracle.SP)):
            if v not in p32:
                continue
            qs = sample_freqs(cat.freq.size, 12, seed=5, include=[int(np.argmax(p32[v]))])
            ref = oracle_powers(t, y, dy, cat.freq[qs], code)
            chk[v] = {"frequencies": int(qs.size), "max_gate_err": gate_error(p32[v][qs], ref)}
        out["oracle_check_fp32c"] = chk
    return out


def run_reference(args):
    """Reference arm: the plain FP64 C oracle on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    cat, desc = workload(args.n_freq)
    t, y, dy = cat.obj(0)
    n = t.size
    cores = os.cpu_count() or 1
    # 16 frequencies per core: about half a second a step on 16 cores, so the
    # default 3 + 10 steps take seconds and the rate is not dominated by the
    # threads' start-up
    per_step = min(cat.freq.size, max(16 * cores, 32))
    rng = np.random.default_rng(11)

    def step(k):
        fq = cat.freq[rng.choice(cat.freq.size, per_step, replace=False)]
        for code in (oracle.SS, oracle.SP):
            oracle.periodogram(t, y, dy, [n], fq, code, n_threads=cores)

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(k)
    dt = (time.perf_counter() - t0) / args.steps
    value = 2 * n * per_step / dt
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": desc, "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} random frequencies per step, SS+SP, n={n}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def run_ours(args):
    import torch

    from paper_2111_07396_gb300 import build as ssp_build
    from paper_2111_07396_gb300 import ssp
    from tests.parity import FLOOR, chi2_rel_error, gate_error

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or world == 1:
        ssp_build.build()
    if dist is not None:
        dist.barrier()
    ssp.lib()

    cat, desc = workload(args.n_freq)
    n, nf = cat.points, int(cat.freq.size)
    dev = torch.device("cuda", local)
    t = torch.from_numpy(cat.t).to(dev)
    y = torch.from_numpy(cat.y).to(dev)
    dy = torch.from_numpy(cat.dy).to(dev)
    fq = torch.from_numpy(cat.freq).to(dev)
    npo = cat.n_per_object
    out = {v: (torch.empty((1, nf), dtype=torch.float32, device=dev),
               torch.empty(1, dtype=torch.float64, device=dev)) for v in ("ss", "sp")}
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count

    def step(precision="fp32c", outs=out):
        for v in ("ss", "sp"):
            ssp.ssp_periodogram_device(t, y, dy, npo, fq, outs[v][0], outs[v][1], variant=v,
                                       precision=precision, stream=stream.cuda_stream)

    def timed_steps(profiled):
        # K steps between barriers, each bracketed by CUDA events on the
        # launching stream, L2 flushed before each (outside the events).  The
        # headline pass records nothing else; the profiled pass (same work,
        # right after) adds the library's per-launch event pairs, from which
        # the kernels' own durations come.
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        ssp.ssp_profile_read(reset=True)
        ssp.ssp_profile_enable(profiled)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            for k in range(args.steps):
                flush.fill_(float(k))
                ev[k][0].record(stream)
                step()
                ev[k][1].record(stream)
            torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        ssp.ssp_profile_enable(False)
        return [a.elapsed_time(b) for a, b in ev], clk.summary(), ssp.ssp_profile_read(reset=True)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        step_ms, clocks, _ = timed_steps(False)
        prof_step_ms, _, prof = timed_steps(True)
    total_ms = max_over_ranks(dist, float(sum(step_ms)), dev)
    ptf_step = 2 * n * nf
    value = job_rate(world, ptf_step, args.steps, total_ms / 1e3)

    # FP32C results of the last step, and the same work in FP64
    p32 = {v: out[v][0].cpu().numpy()[0].astype(np.float64) for v in out}
    b32 = {v: float(out[v][1].cpu().item()) for v in out}
    fp64 = None
    acc = {}
    if not args.no_fp64:
        out64 = {v: (torch.empty((1, nf), dtype=torch.float64, device=dev),
                     torch.empty(1, dtype=torch.float64, device=dev)) for v in ("ss", "sp")}
        with torch.cuda.stream(stream):
            step("fp64", out64)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ssp.ssp_profile_enable(True)
            e0.record(stream)
            step("fp64", out64)
            e1.record(stream)
            torch.cuda.synchronize()
            ssp.ssp_profile_enable(False)
            prof64 = ssp.ssp_profile_read(reset=True)
        ms64 = e0.elapsed_time(e1)
        fp64 = {"value": ptf_step / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64,
                "pgram_ms": {"ss": prof64["pgram_ss"][1], "sp": prof64["pgram_sp"][1]}}
        for v in ("ss", "sp"):
            ref = out64[v][0].cpu().numpy()[0]
            acc[v] = {"max_gate_err_vs_fp64": gate_error(p32[v], ref),
                      "max_chi2_rel_err_vs_fp64": chi2_rel_error(p32[v], ref),
                      "values_gated_by_floor": int(np.sum(np.abs(ref) < FLOOR)),
                      "max_abs_err_vs_fp64": float(np.max(np.abs(p32[v] - ref))),
                      # relative error without the floor, and how many values
                      # exceed the tolerance that way (powers near 0 make the
                      # unfloored ratio large while chi2 stays accurate)
                      "max_rel_err_unfloored": float(np.max(np.abs(p32[v] - ref) /
                                                            np.maximum(np.abs(ref), 1e-300))),
                      "values_rel_err_above_tol": int(np.sum(np.abs(p32[v] - ref) >
                                                             2e-4 * np.abs(ref))),
                      "best_index_same": bool(np.argmax(p32[v]) == np.argmax(ref)),
                      "tolerance": 2e-4}
        fp64["speedup_fp32c_over_fp64"] = fp64["ms_per_step"] / (total_ms / args.steps)

    # e2e through the host entry point from pinned host memory
    th = torch.from_numpy(cat.t).pin_memory()
    yh = torch.from_numpy(cat.y).pin_memory()
    dyh = torch.from_numpy(cat.dy).pin_memory()
    fh = torch.from_numpy(cat.freq).pin_memory()
    pw_h = {v: torch.empty((1, nf), dtype=torch.float32).pin_memory() for v in ("ss", "sp")}
    bp_h = {v: torch.empty(1, dtype=torch.float64).pin_memory() for v in ("ss", "sp")}

    def e2e_step():
        for v in ("ss", "sp"):
            ssp.ssp_periodogram(th, yh, dyh, npo, fh, variant=v, precision="fp32c",
                                out_power=pw_h[v], out_best_period=bp_h[v])

    for _ in range(max(1, args.warmup)):
        e2e_step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(dist, time.perf_counter() - t0, dev)
    h2d = 2 * (3 * 8 * n + 8 * nf)
    d2h = 2 * (4 * nf + 8)
    e2e = {"value": job_rate(world, ptf_step, args.steps, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "api": "ssp_periodogram (host pointers, pinned), SS + SP"}

    # roofline of the dominant kernel (SS periodogram kernel), ALU-bound
    ss_launches, ss_ms = prof["pgram_ss"]
    sp_launches, sp_ms = prof["pgram_sp"]
    clk_mhz = clocks["sm_mhz"] if clocks else 1432.0
    peak = FP32_LANES_PER_SM * sms * clk_mhz * 1e6 / 1e12
    ops_ss, ops_sp = ops_per_ptf("ss", [n]), ops_per_ptf("sp", [n])
    ach_ss = ops_ss * n * nf / (ss_ms / ss_launches / 1e3) / 1e12
    ach_sp = ops_sp * n * nf / (sp_ms / sp_launches / 1e3) / 1e12
    roof = {"bound": "alu", "kernel": "pgram_kernel<float,SS>", "achieved": ach_ss,
            "peak": peak, "unit": "TFLOP/s", "frac": ach_ss / peak,
            "traffic": traffic_per_launch("ss"),
            "ops_per_ptf": ops_ss, "avg_launch_ms": ss_ms / ss_launches,
            "peak_basis": f"{FP32_LANES_PER_SM} FP32 ops/clk/SM x {sms} SMs x "
                          f"{clk_mhz:.0f} MHz (median SM clock sampled during the timed region)",
            "sp": {"kernel": "pgram_kernel<float,SP>", "achieved": ach_sp,
                   "frac": ach_sp / peak, "ops_per_ptf": ops_sp,
                   "traffic": traffic_per_launch("sp"),
                   "avg_launch_ms": sp_ms / sp_launches}}

    try:
        f32, f64 = ssp.ssp_measure_alu_peaks()
        roof["measured_fma_tflops"] = {"fp32": f32, "fp64": f64,
                                       "how": "FMA-chain microbenchmark (2 flops per FMA)"}
    except ssp.SSPError:
        pass

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": desc, "e2e": e2e,
            "gpu_launches": sum(v[0] for v in prof.values()), "roofline": roof, "clocks": clocks,
            "profiled_pass_ms_per_step": float(sum(prof_step_ms)) / args.steps,
            "breakdown_ms_per_step": {k: v[1] / args.steps for k, v in prof.items()},
            "per_variant_ptf_s": {"ss": ptf_step / 2 / (ss_ms / ss_launches / 1e3),
                                  "sp": ptf_step / 2 / (sp_ms / sp_launches / 1e3)},
            "fp64": fp64, "accuracy_fp32c": acc,
            "best_period": b32}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cat, p32)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
def serve_oracle_check(objs, served, variants, freq, k=12):
    """The FP64 oracle at k sampled frequencies of each request in `served`
    ({request index: served power}), the served best frequency among them,
    against the served powers, under the parity gate."""
    import oracle
    from tests.parity import TOL, gate_error, oracle_powers, sample_freqs
    codes = (oracle.SS, oracle.SP)
    worst, n_f = 0.0, 0
    t0 = time.perf_counter()
    for i, p in sorted(served.items()):
        t, y, dy = objs[i]
        qs = sample_freqs(freq.size, k, seed=i, include=[int(np.argmax(p))])
        ref = oracle_powers(t, y, dy, freq[qs], codes[variants[i]])
        worst = max(worst, gate_error(p[qs], ref))
        n_f += qs.size
    return {"requests": len(served), "frequencies": n_f, "max_gate_err": worst,
            "tolerance": TOL["fp32c"], "oracle_s": time.perf_counter() - t0}


def run_serve(args):
    """Serving workload through ssp_server_*: a submitter thread replays the
    Poisson arrival times, a collector thread takes each finished ticket and
    its results.  Latency = result in hand minus scheduled arrival."""
    import threading

    from paper_2111_07396_gb300 import build as ssp_build
    from paper_2111_07396_gb300 import ssp, synth

    if int(os.environ.get("RANK", "0")) != 0:
        return
    ssp_build.build()
    ssp.lib()
    arrivals, cat, variants = synth.config5_arrivals(args.rate, args.duration, args.serve_freq)
    N, nf = int(arrivals.size), int(cat.freq.size)
    objs = [cat.obj(k) for k in range(N)]
    names = ("ss", "sp")
    tune = None
    if args.serve_autotune:
        # a sample of the stream (every 50th object) and of the grid; the choice
        # holds for the rest of the process, as for any later call
        t_tune = time.perf_counter()
        sub = cat.subset(list(range(0, N, 50)))
        tune = {v: ssp.ssp_autotune(sub.t, sub.y, sub.dy, sub.n_per_object, sub.freq, variant=v,
                                    budget_ptf=1e9).tolist() for v in names}
        tune["s"] = time.perf_counter() - t_tune
    srv = ssp.Server(cat.freq, precision="fp32c", slots=args.serve_slots,
                     max_batch_ptf=args.serve_batch_ptf)
    for k in range(8):                              # warm-up: plans, pools, pinned buffers
        t, y, dy = objs[k]
        srv.poll(srv.submit(t, y, dy, names[k % 2]), wait_ms=60000)
    first = srv.submit(*objs[0], "ss")              # tickets are sequential from here on
    srv.poll(first, wait_ms=60000)
    lat = np.full(N, np.nan)
    lat_srv = np.full(N, np.nan)
    best = np.zeros(N)
    t0 = time.perf_counter() + 0.1
    errors = []
    served = {}                                     # every 100th request's powers

    def submitter():
        for k in range(N):
            d = t0 + arrivals[k] - time.perf_counter()
            if d > 0:
                time.sleep(d)
            t, y, dy = objs[k]
            try:
                srv.submit(t, y, dy, names[variants[k]])
            except Exception as e:  # noqa: BLE001
                errors.append(repr(e))
                return

    def collector():
        got = 0
        while got < N and not errors:
            tk = srv.next(wait_ms=1000)
            if tk is None:
                continue
            k = tk - first - 1
            r = srv.poll(tk)
            lat[k] = (time.perf_counter() - (t0 + arrivals[k])) * 1e3
            lat_srv[k] = r[2]
            best[k] = r[1]
            if k % 100 == 0:
                served[k] = r[0].astype(np.float64)
            got += 1

    ts = threading.Thread(target=submitter)
    tc = threading.Thread(target=collector)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        ts.start()
        tc.start()
        ts.join()
        tc.join()
    end = float(np.nanmax(arrivals + lat / 1e3))    # first arrival to last result, s
    srv.close()
    ptf = float(np.sum(cat.n_per_object)) * nf
    # after the timed region: 1 % of the requests against the oracle
    check = None if args.no_oracle else serve_oracle_check(objs, served, variants, cat.freq)
    q = lambda a, p: float(np.nanpercentile(a, p))
    line = {"metric": "served objects/s (Poisson arrivals, single-object requests)",
            "value": N / end, "unit": "objects/s", "higher_is_better": True,
            "offered_rate": args.rate, "objects": N, "duration_s": args.duration,
            "ptf_per_s": ptf / end, "busy_s": end, "errors": errors[:3],
            "latency_ms": {"p50": q(lat, 50), "p90": q(lat, 90), "p99": q(lat, 99),
                           "max": float(np.nanmax(lat))},
            "server_latency_ms": {"p50": q(lat_srv, 50), "p99": q(lat_srv, 99)},
            "dtype": "f32", "data": "synthetic", "clocks": clk.summary(), "autotune": tune,
            "oracle_check_fp32c": check,
            "config": {"workload": f"Poisson arrivals {args.rate:g}/s for {args.duration:g} s, "
                                   f"n ~ logU(30, 3000), {nf} freqs in [0.05, 15), "
                                   "variant per request Bernoulli(0.5), FP32C",
                       "api": "ssp_server_submit / next / poll (host arrays)",
                       "slots": args.serve_slots or "default", "max_batch_ptf": args.serve_batch_ptf or "default"}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def run_matrix(args):
    """Per configuration and variant: FP32C and FP64 through the device entry
    point, agreement, roofline fraction and a bounded oracle sample."""
    import torch

    from paper_2111_07396_gb300 import build as ssp_build
    from paper_2111_07396_gb300 import ssp, synth
    from tests.parity import FLOOR, chi2_rel_error, gate_error

    if int(os.environ.get("RANK", "0")) != 0:
        return
    ssp_build.build()
    ssp.lib()
    dev = torch.device("cuda", 0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    gens = {"c1": synth.config1, "c2": synth.config2, "c3": synth.config3, "c4": synth.config4}
    stream = torch.cuda.Stream(device=dev)
    for name in [c for c in args.matrix.split(",") if c]:
        cat = gens[name]()
        if args.subset_objects:
            cat = cat.subset(list(range(min(args.subset_objects, cat.n_per_object.size))))
        if args.subset_freq and args.subset_freq < cat.freq.size:
            cat = cat.with_freq(cat.freq[::cat.freq.size // args.subset_freq][:args.subset_freq])
        N, nf = int(cat.n_per_object.size), int(cat.freq.size)
        put = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        fq = put(cat.freq)
        sub = cat if name != "c4" else cat.subset(list(range(min(N, 40))))
        for v in [v for v in args.matrix_variants.split(",") if v]:
            tune = None
            if name == "c3":
                t0 = time.perf_counter()
                g = ssp.ssp_autotune(cat.t, cat.y, cat.dy, cat.n_per_object, cat.freq, variant=v,
                                     budget_ptf=1e9)
                tune = {"seconds": time.perf_counter() - t0, "threads_per_range": g.tolist()}

            def timed(c, precision):
                tdev, ydev, dydev = put(c.t), put(c.y), put(c.dy)
                dt = torch.float64 if precision == "fp64" else torch.float32
                pw = torch.empty((c.n_per_object.size, nf), dtype=dt, device=dev)
                bp = torch.empty(c.n_per_object.size, dtype=torch.float64, device=dev)
                with torch.cuda.stream(stream):
                    ssp.ssp_periodogram_device(tdev, ydev, dydev, c.n_per_object, fq, pw, bp,
                                               variant=v, precision=precision, stream=stream)
                    stream.synchronize()
                    ssp.ssp_profile_read(True)
                    ssp.ssp_profile_enable(True)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    ssp.ssp_periodogram_device(tdev, ydev, dydev, c.n_per_object, fq, pw, bp,
                                               variant=v, precision=precision, stream=stream)
                    e1.record(stream)
                    stream.synchronize()
                    ssp.ssp_profile_enable(False)
                    prof = ssp.ssp_profile_read(True)
                ms = e0.elapsed_time(e1)
                return pw.cpu().numpy(), bp.cpu().numpy(), ms, prof

            with ClockSampler(0) as clk:
                p32, b32, ms32, prof32 = timed(cat, "fp32c")
            p64s, b64s, ms64, _ = timed(sub, "fp64")
            ptf = float(np.sum(cat.n_per_object)) * nf
            ptf_sub = float(np.sum(sub.n_per_object)) * nf
            ns = int(sub.n_per_object.size)
            p32s = p32[:ns]
            clocks = clk.summary()
            mhz = clocks["sm_mhz"] if clocks else 1432.0
            peak = FP32_LANES_PER_SM * sms * mhz * 1e6 / 1e12
            kname = "pgram_ss" if v == "ss" else "pgram_sp"   # SPG launches time as SP
            k_ms = prof32[kname][1]
            same = float(np.mean(np.argmax(p32s, axis=1) == np.argmax(p64s, axis=1)))
            big = int(np.argmax(cat.n_per_object))
            cpu = None if args.no_oracle else cpu_baseline(cat, budget_s=8.0, max_freq=512, obj=big,
                                                           variants=(v,))
            line = {"metric": "point*frequency evals/s", "config": name, "variant": v,
                    "objects": N, "points": int(np.sum(cat.n_per_object)), "n_freq": nf,
                    "fp32c": {"value": ptf / (ms32 / 1e3), "ms": ms32,
                              "kernel_ms": k_ms, "redo_ms": prof32["redo"][1]},
                    "fp64": {"value": ptf_sub / (ms64 / 1e3), "ms": ms64,
                             "objects": ns},
                    "fp32c_vs_fp64": {"max_gate_err": gate_error(p32s, p64s),
                                      "max_chi2_rel_err": chi2_rel_error(p32s, p64s),
                                      "values_gated_by_floor": int(np.sum(np.abs(p64s) < FLOOR)),
                                      "max_abs_err": float(np.max(np.abs(p32s - p64s))),
                                      "best_index_same": same,
                                      "best_period_same": float(np.mean(b32[:ns] == b64s))},
                    "roofline": {"bound": "alu", "ops_per_ptf": ops_per_ptf(v, cat.n_per_object),
                                 "achieved": ops_per_ptf(v, cat.n_per_object) * ptf / (k_ms / 1e3) / 1e12,
                                 "peak": peak, "unit": "TFLOP/s",
                                 "frac": ops_per_ptf(v, cat.n_per_object) * ptf / (k_ms / 1e3) / 1e12 / peak},
                    "autotune": tune, "clocks": clocks,
                    "cpu_baseline": cpu}
            print(json.dumps(line), flush=True)
            if name == "c3":
                ssp.ssp_autotune_clear()


def run_extras(args):
    """Two measurements through the host entry points, each after one warm-up
    call: (1) objects sharing one cadence, folded and sorted once per group,
    against the same work with jittered times; (2) search-and-refine (coarse
    SP, then SS on 64-frequency grids around the top 3 peaks) against SS over
    the whole coarse grid, on 2,000 sparse-catalog objects."""
    from paper_2111_07396_gb300 import build as ssp_build
    from paper_2111_07396_gb300 import ssp, synth

    if int(os.environ.get("RANK", "0")) != 0:
        return
    ssp_build.build()
    ssp.lib()

    def wall(fn):
        fn()
        t0 = time.perf_counter()
        out = fn()
        return time.perf_counter() - t0, out

    shared, jit = synth.shared_cadence(), synth.shared_cadence(jitter=True)
    for v in ("ss", "sp"):
        with ClockSampler(0) as clk:
            ts, (ps, _) = wall(lambda: ssp.ssp_periodogram(shared.t, shared.y, shared.dy,
                                                           shared.n_per_object, shared.freq,
                                                           variant=v))
            tj, (pj, _) = wall(lambda: ssp.ssp_periodogram(jit.t, jit.y, jit.dy, jit.n_per_object,
                                                           jit.freq, variant=v))
        print(json.dumps({
            "metric": "point*frequency evals/s", "unit": UNIT, "extra": "shared_fold", "variant": v,
            "shared": {"value": shared.pt_freq / ts, "s": ts},
            "separate": {"value": jit.pt_freq / tj, "s": tj}, "speedup": tj / ts,
            "max_abs_diff": float(np.max(np.abs(ps - pj))), "clocks": clk.summary(),
            "config": {"workload": "48 objects on one 3,000-point cadence, 4,000 freqs in "
                                   "[0.01, 20); separate = times jittered by k*1e-9 d",
                       "api": "ssp_periodogram (host arrays)", "precision": "fp32c"}}),
            flush=True)

    # launch plans: the single-object C1 workload (100 points, 2,000
    # frequencies), called again and again on device arrays; the device entry
    # point plans, allocates and launches each call, the plan replays a graph
    import torch
    c1 = synth.config1()
    put = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    dt_, dy_, dd_, df_ = put(c1.t), put(c1.y), put(c1.dy), put(c1.freq)
    for v in ("ss", "sp"):
        pw = torch.empty((1, c1.freq.size), dtype=torch.float32, device="cuda")
        bp = torch.empty(1, dtype=torch.float64, device="cuda")
        reps = 200
        res = {}
        with ssp.Plan(c1.n_per_object, c1.freq.size, variant=v) as plan:
            calls = {"device_entry": lambda: ssp.ssp_periodogram_device(
                         dt_, dy_, dd_, c1.n_per_object, df_, pw, bp, variant=v),
                     "plan": lambda: plan.execute(dt_, dy_, dd_, df_, pw, bp)}
            for name, fn in calls.items():
                for _ in range(5):
                    fn()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for _ in range(reps):
                    fn()
                torch.cuda.synchronize()
                res[name] = (time.perf_counter() - t0) / reps * 1e6
        print(json.dumps({
            "metric": "microseconds per call", "unit": "us", "extra": "launch_plan", "variant": v,
            "device_entry_us": res["device_entry"], "plan_us": res["plan"],
            "speedup": res["device_entry"] / res["plan"],
            "config": {"workload": "one 100-point object, 2,000 freqs in [0.1, 10), FP32C, "
                                   f"{reps} back-to-back calls on one stream",
                       "api": "ssp_periodogram_device vs ssp_plan_execute"}}), flush=True)

    cat = synth.config3(n_objects=2000, n_freq=20_000)
    step = float(cat.freq[1] - cat.freq[0])
    with ClockSampler(0) as clk:
        tr, (bp_r, _) = wall(lambda: ssp.ssp_search_refine(cat.t, cat.y, cat.dy, cat.n_per_object,
                                                           cat.freq, coarse_variant="sp",
                                                           fine_variant="ss", n_peaks=3,
                                                           n_fine=64))
        tf, (_, bp_f) = wall(lambda: ssp.ssp_periodogram(cat.t, cat.y, cat.dy, cat.n_per_object,
                                                         cat.freq, variant="ss"))
    near = np.abs(1.0 / bp_r - 1.0 / bp_f) <= step
    shapes = np.asarray(cat.shapes)
    truth = 1.0 / cat.periods
    by_shape = {}
    for sh in ("sin", "box", "noise"):
        m = shapes == sh
        by_shape[sh] = {"objects": int(m.sum()),
                        "refine_matches_full_grid": float(np.mean(near[m])),
                        "refine_finds_true_f": float(np.mean(np.abs(1.0 / bp_r[m] - truth[m]) <= step)),
                        "full_grid_finds_true_f": float(np.mean(np.abs(1.0 / bp_f[m] - truth[m]) <= step))}
    print(json.dumps({
        "metric": "objects/s", "unit": "objects/s", "extra": "search_refine",
        "refine": {"value": cat.n_per_object.size / tr, "s": tr},
        "ss_full_grid": {"value": cat.n_per_object.size / tf, "s": tf}, "speedup": tf / tr,
        "best_freq_within_one_step": float(np.mean(near)), "by_shape": by_shape,
        "clocks": clk.summary(),
        "config": {"workload": "2,000 sparse-catalog objects (n ~ logU(30, 500), 2,000 d), "
                               "coarse grid 20,000 freqs in [0.01, 10); SP coarse, SS on 3 x 64",
                   "api": "ssp_search_refine / ssp_periodogram (host arrays)",
                   "precision": "fp32c"}}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.serve:
        run_serve(args)
    elif args.matrix:
        run_matrix(args)
    elif args.extras:
        run_extras(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
