#!/usr/bin/env python3
"""Benchmark of the electron scattering self-energy Sigma^{<>} (Eq. 3) on one GB300.

One step = one evaluation of Sigma^> and Sigma^< for the medium FinFET-shaped workload
(Nkz=Nqz=5, NE=256, Nw=32, Na=512, Nb=4 chain neighbours, Norb=12, complex128,
seed 1): every row of the hot path (stage inputs, the q/w-independent products, the
(q, w) correlation, the FP64 reduction and the write of Sigma) runs inside the step.
Inputs (3.0 GB of G plus Dt) are larger than the 129 MB L2, so no flush is needed
between steps.

Beside the headline the default run measures, each with at least 20 timed repetitions
(p50/p99) and its own clock record:
  * the plain FP64 form on the same medium workload ("vs plain FP64");
  * the precision form: Na = 2048 (G about 6 GB per sign), mixed, complex128;
  * the batched form: 64 uneven instances (Na ~ U[64,1024], NE ~ U[64,512], Nkz=Nqz=3,
    Nw=16, 3..8 random neighbours, complex64) in one persistent, graph-captured launch;
  * the serving form: 2000 Poisson-arriving requests (the batched size distribution plus
    5 % Na=2048/NE=256 requests) over device-resident sessions, 120 GB budget, p50/p99.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--form mixed|fp64] [--impl ours|reference]
                  [--no-precision] [--no-batched] [--serving N]

Prints ONE JSON line on rank 0.  Under torchrun each rank evaluates its own replica of
the workload (replicas only: the single-instance path has no cross-GPU exchange), and
`value` is all ranks' points over the slowest rank's time.  `--impl reference` times
the CPU FP64 oracle on a bounded sample of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SSE atom-energy-kz points/s and fraction of roofline vs plain FP64; p50/p99"
UNIT = "points/s"
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 rate (no measured FP64 peak is recorded)
SPLIT_PRODUCTS = 3           # split-bf16 products per real product in the mixed form


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--form", choices=("auto", "mixed", "fp64"), default="auto")
    ap.add_argument("--workload", choices=("medium", "medium64", "tiny", "batched1"), default="medium",
                    help="medium: the benchmark workload; medium64: the same shape with Na=64 "
                         "(small case for profiling); tiny: the smallest workload; batched1: one "
                         "instance of the batched shape (Na=512, NE=256, Nkz=Nqz=3, Nw=16, 3..8 random "
                         "neighbours, complex64), for profiling the form the batched and served runs use")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=3,
                    help="timed steps of the plain FP64 form measured beside the mixed form")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the precision leg (Na = 2048, mixed, complex128)")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched leg (64 uneven instances, one persistent launch)")
    ap.add_argument("--serving", type=int, default=2000, metavar="N",
                    help="requests of the serving leg (Poisson arrivals; 0: skip the leg)")
    ap.add_argument("--leg-steps", type=int, default=20,
                    help="timed repetitions of each leg (p50/p99 need at least 20)")
    ap.add_argument("--no-pi", action="store_true",
                    help="skip the phonon self-energy leg (Pi, FP64; Nkz=Nqz=5, NE=256, Nw=32, Na=152)")
    return ap.parse_args()


BATCHED1_SPEC = dict(n_instances=1, na_range=(512, 512), ne_range=(256, 256))


def workload(name):
    from paper_1912_08810_gb300 import inputs
    small = inputs.Geometry(nkz=5, nqz=5, ne=256, nw=32, na=64, nb=4)
    one = inputs.Geometry(nkz=3, nqz=3, ne=256, nw=16, na=512, nb=8)
    return {"medium": (inputs.MEDIUM, 1), "medium64": (small, 1), "tiny": (inputs.TINY, 0),
            "batched1": (one, 3)}[name]


def make_workload(name):
    from paper_1912_08810_gb300 import inputs
    geo, seed = workload(name)
    if name == "batched1":
        return geo, inputs.make_batched(inputs.BatchedSpec(**BATCHED1_SPEC), seed)[0]
    return geo, inputs.make_instance(geo, seed)


def config_dict(geo, name, form):
    eb = 8 if name == "batched1" else 16
    in_bytes = eb * (2 * geo.nkz * geo.ne * geo.na * 144 + 2 * geo.nqz * geo.nw * geo.na * geo.nb * 9)
    nbr = "3..8 random" if name == "batched1" else "chain"
    dt = "complex64" if name == "batched1" else "complex128"
    return {"workload": f"{name} SSE: Nkz=Nqz={geo.nkz}, NE={geo.ne}, Nw={geo.nw}, Na={geo.na}, "
                        f"Nb={geo.nb} {nbr}, Norb=12, {dt}",
            "form": form, "nkz": geo.nkz, "nqz": geo.nqz, "ne": geo.ne, "nw": geo.nw, "na": geo.na,
            "nb": geo.nb, "norb": 12, "seed": workload(name)[1],
            "l2": f"inputs {in_bytes / 1e9:.2f} GB > 129 MB L2, no flush", "parallelism": "replicas"}


# --- clocks ------------------------------------------------------------------------------

class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid=None):
        self.proc = None
        self.path = None
        self.uuid = device_uuid

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"error": "nvidia-smi unavailable"}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, power, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"error": "no samples"}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


# --- profile-derived traffic -------------------------------------------------------------

def strip_comments(src):
    """C/C++/CUDA source without its comments and blank lines (string literals kept), so that
    a comment-only edit leaves a kernel's digest unchanged."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c == '"' or c == "'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return "\n".join(line.rstrip() for line in "".join(out).splitlines() if line.strip())


def source_digest(paths):
    h = hashlib.sha256()
    for p in paths:
        h.update(strip_comments(open(os.path.join(ROOT, p), encoding="utf-8").read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_tag, digest, workload):
    """DRAM bytes per launch recorded in profiles/<kernel_tag>_<workload>.md for this exact
    source."""
    fn = os.path.join(ROOT, "profiles", f"{kernel_tag}_{workload}.md")
    if os.path.exists(fn):
        txt = open(fn).read()
        m_d = re.search(r"source_digest:\s*([0-9a-f]+)", txt)
        m_t = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
        if m_d and m_t and m_d.group(1) == digest:
            return float(m_t.group(1))
    return None


KERNEL_SOURCES = {
    "fp64": ("sse_fp64_direct", ["paper_1912_08810_gb300/csrc/sse_fp64.cu"]),
    "mixed": ("sse_tc_kernel", ["paper_1912_08810_gb300/csrc/sse_mixed.cu", "paper_1912_08810_gb300/csrc/tc_ptx.h"]),
    "mixed_single_role": ("sse_mixed_kernel", ["paper_1912_08810_gb300/csrc/sse_mixed.cu",
                                               "paper_1912_08810_gb300/csrc/tc_ptx.h"]),
}


# --- our arm ---------------------------------------------------------------------------

def dist_setup(args=None):
    """Rank, world size and local rank from the launcher's environment; for N > 1 one
    process group over NCCL (one rank per GPU), or gloo where there is no GPU (the host-side
    logic is tested that way on CPU)."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(points_per_rank_step, steps, world, max_total_ms):
    """Points/s of the whole job: every rank runs its own replica of the workload, so the
    job evaluates world x points per step, timed by the slowest rank."""
    return points_per_rank_step * steps * world / (max_total_ms / 1e3)


def time_steps(step, steps, warmup, world, stream, clocks=None, before_timed=None):
    """W warm-up steps, then K timed steps bracketed by barrier + synchronize; CUDA events
    on the launching stream per step.  Returns (total_ms, per_step_ms)."""
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    if before_timed:
        before_timed()
    barrier(world)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    if clocks:
        clocks.start()
        time.sleep(0.3)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for a, b in evs:
        a.record(stream)
        step()
        b.record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    return t0.elapsed_time(t1), [a.elapsed_time(b) for a, b in evs], clk


def pct(xs, p):
    xs = sorted(xs)
    if not xs:
        return None
    i = min(len(xs) - 1, max(0, int(round(p / 100.0 * (len(xs) - 1)))))
    return xs[i]


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def tensor_peak(peaks, clk):
    """bf16 dense peak for a tensor-bound kernel, divided by the split products.  The burst
    figure applies when the clock record of the timed region shows the SM clock at its
    maximum and no power cap; otherwise the sustained (power-capped) figure."""
    burst = peaks.get("bf16_tflops")
    sustained = peaks.get("bf16_tflops_sustained")
    src = "measured" if burst else "fallback"
    burst = burst or 1900.0
    sustained = sustained or 1700.0
    full = (isinstance(clk, dict) and "sm_mhz" in clk and clk["sm_mhz"] >= 0.97 * clk["sm_max_mhz"]
            and "sw_power_cap" not in clk.get("reasons", []))
    bf16, kind = (burst, "burst") if full else (sustained, "sustained")
    return bf16 / SPLIT_PRODUCTS, f"{src} bf16 {kind} {bf16} TFLOP/s / {SPLIT_PRODUCTS} split products"


def leg_timing(step, steps, warmup, stream, uuid):
    """W untimed steps, then `steps` steps each bracketed by CUDA events on `stream`, with
    nvidia-smi sampling the clocks meanwhile.  Returns per-step ms and the clock record."""
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(uuid)
    clocks.start()
    time.sleep(0.3)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for e0, e1 in evs:
        e0.record(stream)
        step()
        e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    return [e0.elapsed_time(e1) for e0, e1 in evs], clk


def device_uuid():
    import torch
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
    except Exception:
        return None


def run_ours(args):
    import numpy as np
    import torch

    from paper_1912_08810_gb300 import inputs, sse

    world, rank, local = dist_setup(args)
    name = args.workload
    geo, inst = make_workload(name)
    dev = {k: torch.from_numpy(inst[k]).cuda().contiguous() for k in ("G_gt", "G_lt", "D_gt", "D_lt", "dH", "neigh")}
    S = {s: torch.empty_like(dev["G_gt"]) for s in ("gt", "lt")}
    stream = torch.cuda.current_stream()

    def make_plan(mode):
        return sse.Plan(dev["neigh"], dev["dH"], nkz=geo.nkz, nqz=geo.nqz, ne=geo.ne, nw=geo.nw, mode=mode)

    form = args.form
    plan = None
    if form in ("auto", "mixed"):
        try:
            plan = make_plan("mixed")
            form = "mixed"
        except sse.SSEError:
            if form == "mixed":
                raise
            form = "fp64"
    if plan is None:
        plan = make_plan("fp64")
    plan_keep = [plan]
    info = plan.info()
    points = geo.points()
    flops_step = 2 * info.flops_per_sign

    def step():
        plan.execute(dev["G_gt"], dev["G_lt"], dev["D_gt"], dev["D_lt"], S["gt"], S["lt"], stream=stream)

    uuid = device_uuid()
    clocks = ClockSampler(uuid)
    total_ms, per_step, clk = time_steps(step, args.steps, args.warmup, world, stream, clocks,
                                         before_timed=lambda: sse.sse_plan_set_timing(plan.handle, True))
    prep_ms, main_ms, timed_calls = sse.sse_plan_timing(plan.handle)
    sse.sse_plan_set_timing(plan.handle, False)
    plan.status()
    total_ms_max = max_over_ranks(total_ms, world)
    value = whole_job_value(points, args.steps, world, total_ms_max)
    # our kernels per step: the workspace pass (re-encoded G and slot tables, per sign) of
    # the Nkz = 5 tensor-core form, then the main kernel
    launches_per_step = 1 + (4 if (form == "mixed" and info.workspace_bytes > (1 << 20)) else 0)
    kern_ms = main_ms / timed_calls if timed_calls else statistics.mean(per_step)

    peaks = load_peaks()
    ws_form = form == "mixed" and info.workspace_bytes > (1 << 20)  # the warp-specialised form's workspace
    tag, srcs = KERNEL_SOURCES["mixed" if ws_form else ("mixed_single_role" if form == "mixed" else form)]
    digest = source_digest(srcs)
    traffic = profiled_traffic(tag, digest, name)
    if form == "mixed":
        peak, peak_src = tensor_peak(peaks, clk)
        roof = {"bound": "tensor", "unit": "TFLOP/s", "peak_source": peak_src}
    else:
        peak = FP64_NOMINAL_TFLOPS
        roof = {"bound": "alu", "unit": "TFLOP/s",
                "peak_source": "GB300 nominal FP64 1.25 TFLOP/s (DFMA pipe; no measured FP64 peak is recorded)"}
    achieved = flops_step / (kern_ms / 1e3) / 1e12
    roof.update({"kernel": tag, "kernel_ms": kern_ms,
                 "workspace_pass_ms": (prep_ms / timed_calls) if timed_calls else None,
                 "achieved": achieved, "peak": peak, "frac": achieved / peak,
                 "traffic": traffic, "algorithmic_flops_per_launch": flops_step,
                 "algorithmic_bytes_per_launch": 2 * info.bytes_per_sign, "source_digest": digest})

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps,
           "p50_ms": pct(per_step, 50), "p99_ms": pct(per_step, 99),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "bf16x3->f32->f64" if form == "mixed" else "f64",
           "data": "synthetic (seeded numpy; G anti-Hermitian, Dt Hermitian, chain neighbours)",
           "config": config_dict(geo, name, form), "roofline": roof, "clocks": clk,
           "gpu_launches": launches_per_step * args.steps}

    # the plain FP64 form on the same workload, for the "vs plain FP64" part of the metric
    if form == "mixed" and args.fp64_steps > 0:
        p64 = make_plan("fp64")

        def step64():
            p64.execute(dev["G_gt"], dev["G_lt"], dev["D_gt"], dev["D_lt"], S["gt"], S["lt"], stream=stream)

        t64, ps64, clk64 = time_steps(step64, args.fp64_steps, 1, world, stream, ClockSampler(uuid))
        t64 = max_over_ranks(t64, world)
        v64 = points * args.fp64_steps * world / (t64 / 1e3)
        a64 = flops_step / (statistics.mean(ps64) / 1e3) / 1e12
        out["fp64_form"] = {"value": v64, "unit": UNIT, "ms_per_step": t64 / args.fp64_steps,
                            "steps": args.fp64_steps, "roofline_frac": a64 / FP64_NOMINAL_TFLOPS,
                            "peak_source": "GB300 nominal FP64 1.25 TFLOP/s (not measured)",
                            "speedup_of_value": value / v64, "clocks": clk64}
        out["gpu_launches"] += args.fp64_steps + 1
        p64.close()

    hostin, hostout = {}, {}
    if not args.no_e2e:
        hostin = {k: torch.from_numpy(inst[k]).pin_memory() for k in ("G_gt", "G_lt", "D_gt", "D_lt")}
        hostout = {s: torch.empty(S[s].shape, dtype=S[s].dtype).pin_memory() for s in ("gt", "lt")}

        def step_e2e():
            plan.execute_host(hostin["G_gt"], hostin["G_lt"], hostin["D_gt"], hostin["D_lt"],
                              hostout["gt"], hostout["lt"], stream=stream)

        step_e2e()
        barrier(world)
        k_e2e = max(1, min(args.steps, 3 if form == "fp64" else args.steps))
        t = time.perf_counter()
        for _ in range(k_e2e):
            step_e2e()
        e2e_s = max_over_ranks(time.perf_counter() - t, world)
        h2d = sum(hostin[k].numel() * hostin[k].element_size() for k in hostin)
        d2h = sum(hostout[s].numel() * hostout[s].element_size() for s in hostout)
        out["e2e"] = {"value": points * k_e2e * world / e2e_s, "unit": UNIT, "steps": k_e2e,
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                      "api": "sse_execute_host (pinned host buffers)"}
        out["gpu_launches"] += (k_e2e + 1) * launches_per_step

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_sample(inst, geo)
    del hostin, hostout, dev, S, inst
    plan_keep.clear()
    plan = None
    torch.cuda.empty_cache()
    if not args.no_precision and form == "mixed":
        out["precision"] = run_precision(args, stream, peaks, uuid)
        out["gpu_launches"] += out["precision"]["gpu_launches"]
    if not args.no_batched and form == "mixed":
        out["batched"] = run_batched(args, stream, peaks, uuid)
        out["gpu_launches"] += out["batched"]["gpu_launches"]
    if not args.no_pi:
        out["pi"] = run_pi(args, stream, uuid)
        out["gpu_launches"] += out["pi"]["gpu_launches"]
    if args.serving and form == "mixed":
        out["serving"] = run_serving(args.serving, uuid)
        out["gpu_launches"] += out["serving"]["gpu_launches"]
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_precision(args, stream, peaks, uuid):
    """The precision workload: Nkz=Nqz=5, NE=256, Nw=32, Na=2048, Nb=4 chain neighbours,
    complex128 (G about 6 GB per sign), mixed form; inputs drawn on the device (seed 2).
    Its error against the oracle on the Na=128 slice is checked by the parity tests."""
    import torch

    from paper_1912_08810_gb300 import inputs, sse
    geo = inputs.PRECISION
    inst = inputs.make_instance_torch(geo, 2, dtype=torch.complex128)
    S = {s: torch.empty_like(inst["G_gt"]) for s in ("gt", "lt")}
    plan = sse.Plan(inst["neigh"], inst["dH"], nkz=geo.nkz, nqz=geo.nqz, ne=geo.ne, nw=geo.nw, mode="mixed")
    info = plan.info()
    flops = 2 * info.flops_per_sign

    def step():
        plan.execute(inst["G_gt"], inst["G_lt"], inst["D_gt"], inst["D_lt"], S["gt"], S["lt"], stream=stream)

    steps, warm = max(20, args.leg_steps), 3
    sse.sse_plan_set_timing(plan.handle, True)
    per, clk = leg_timing(step, steps, warm, stream, uuid)
    prep_ms, main_ms, calls = sse.sse_plan_timing(plan.handle)
    plan.status()
    ms = statistics.mean(per)
    kern_ms = main_ms / calls
    peak, peak_src = tensor_peak(peaks, clk)
    achieved = flops / (kern_ms / 1e3) / 1e12
    res = {"workload": "precision SSE: Nkz=Nqz=5, NE=256, Nw=32, Na=2048, Nb=4 chain, Norb=12, complex128, "
                       "seed 2 (drawn on device)",
           "points_per_step": geo.points(), "value": geo.points() / (ms / 1e3), "unit": UNIT,
           "ms_per_step": ms, "p50_ms": pct(per, 50), "p99_ms": pct(per, 99), "steps": steps, "warmup": warm,
           "gpu_launches": 5 * (steps + warm), "clocks": clk,
           "roofline": {"bound": "tensor", "kernel": "sse_tc_kernel", "kernel_ms": kern_ms,
                        "workspace_pass_ms": prep_ms / calls, "achieved": achieved, "peak": peak,
                        "unit": "TFLOP/s", "frac": achieved / peak, "peak_source": peak_src,
                        "algorithmic_flops_per_launch": flops}}
    plan.close()
    del inst, S
    torch.cuda.empty_cache()
    return res


def pi_flops(geo, neigh):
    """Algorithmic real flops of Pi per sign: per bond, the nine traces per (q, w, k, valid E)
    as 144-channel dot products of V_i = dH_i^+ G_aa and U_j = dH_j G_bb (formed once per
    (k, E) each: 6 products of 12^3), 8 flops per complex MAC."""
    bonds = int((neigh >= 0).sum())
    valid = sum(max(0, geo.ne - abs(w + geo.omega_first)) for w in range(geo.nw))
    cmacs = bonds * (geo.nqz * valid * geo.nkz * 9 * 144 + geo.nkz * geo.ne * 6 * 1728)
    return 8.0 * cmacs


def run_pi(args, stream, uuid):
    """The phonon self-energy Pi^> and Pi^< (Eqs. 4-5) in FP64 on Nkz=Nqz=5, NE=256, Nw=32,
    Na=152, Nb=4 chain neighbours, complex128 (seed 5, drawn on the device): one CTA per
    (atom, sign), two per SM.  FP64-pipe bound."""
    import torch

    from paper_1912_08810_gb300 import inputs, sse
    geo = inputs.Geometry(nkz=5, nqz=5, ne=256, nw=32, na=152, nb=4)
    inst = inputs.make_instance_torch(geo, 5, dtype=torch.complex128)
    plan = sse.Plan(inst["neigh"], inst["dH"], nkz=geo.nkz, nqz=geo.nqz, ne=geo.ne, nw=geo.nw, mode="fp64")
    shape = (geo.nqz, geo.nw, geo.na, geo.nb + 1, 3, 3)
    P = {s: torch.empty(shape, dtype=torch.complex128, device="cuda") for s in ("gt", "lt")}

    def step():
        plan.pi(inst["G_gt"], inst["G_lt"], P["gt"], P["lt"], stream=stream)

    steps, warm = 3, 1
    per, clk = leg_timing(step, steps, warm, stream, uuid)
    plan.status()
    ms = statistics.mean(per)
    flops = 2 * pi_flops(geo, inst["neigh"].cpu().numpy())
    achieved = flops / (ms / 1e3) / 1e12
    res = {"workload": "Pi (Eqs. 4-5), FP64: Nkz=Nqz=5, NE=256, Nw=32, Na=152, Nb=4 chain, complex128, seed 5",
           "value": geo.nqz * geo.nw * geo.na / (ms / 1e3), "unit": "(qz, w, atom) points/s",
           "ms_per_step": ms, "p50_ms": pct(per, 50), "steps": steps, "warmup": warm,
           "gpu_launches": steps + warm, "clocks": clk,
           "roofline": {"bound": "alu", "kernel": "sse_pi_kernel", "achieved": achieved,
                        "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_NOMINAL_TFLOPS,
                        "peak_source": "GB300 nominal FP64 1.25 TFLOP/s (not measured)",
                        "algorithmic_flops_per_launch": flops}}
    plan.close()
    del inst, P
    torch.cuda.empty_cache()
    return res


def run_batched(args, stream, peaks, uuid):
    """The batched workload: 64 instances (Na ~ U[64,1024], NE ~ U[64,512], Nkz=Nqz=3,
    Nw=16, 3..8 random neighbours within +-8 sites, complex64, seed 3), drawn on the device,
    evaluated by one persistent launch per step; the step is captured in a CUDA graph and
    replayed.  The first call runs the autotuner."""
    import torch

    from paper_1912_08810_gb300 import inputs, sse
    spec = inputs.BatchedSpec()
    insts = inputs.make_batched_torch(spec, 3)
    plans, ios, outs = [], [], []
    points = 0
    flops = 0.0
    for inst in insts:
        g = inst["geometry"]
        S = {s: torch.empty_like(inst["G_gt"]) for s in ("gt", "lt")}
        p = sse.Plan(inst["neigh"], inst["dH"], nkz=g.nkz, nqz=g.nqz, ne=g.ne, nw=g.nw, mode="mixed")
        ios.append(p._io(inst["G_gt"], inst["G_lt"], inst["D_gt"], inst["D_lt"], S["gt"], S["lt"]))
        plans.append(p)
        outs.append(S)
        points += g.points()
        flops += 2 * p.info().flops_per_sign
    handles = [p.handle for p in plans]
    side = torch.cuda.Stream()
    t0 = time.perf_counter()
    with torch.cuda.stream(side):
        sse.sse_execute_batch(handles, ios, side.cuda_stream)  # first call: autotune
    torch.cuda.synchronize()
    tune_s = time.perf_counter() - t0
    tuning = sse.sse_batch_tuning(handles, ios)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        sse.sse_execute_batch(handles, ios, side.cuda_stream)
    steps, warm = max(20, args.leg_steps), 3
    cur = torch.cuda.current_stream()
    per, clk = leg_timing(graph.replay, steps, warm, cur, uuid)
    plans[0].status()
    ms = statistics.mean(per)
    peak, peak_src = tensor_peak(peaks, clk)
    achieved = flops / (ms / 1e3) / 1e12
    res = {"workload": "64 instances, Na~U[64,1024], NE~U[64,512], Nkz=Nqz=3, Nw=16, Nb~U{3..8} "
                       "within +-8 sites, complex64, seed 3 (drawn on device)",
           "points_per_step": points, "value": points / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
           "p50_ms": pct(per, 50), "p99_ms": pct(per, 99), "steps": steps, "warmup": warm,
           "tiles_per_unit": tuning[0] if tuning else None, "longest_first": tuning[1] if tuning else None,
           "autotune_s": tune_s, "graph_captured": True, "gpu_launches": steps + warm + 12, "clocks": clk,
           "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "peak_source": peak_src,
                        "unit": "TFLOP/s", "frac": achieved / peak, "algorithmic_flops_per_launch": flops}}
    for p in plans:
        p.close()
    del insts, outs, graph
    torch.cuda.empty_cache()
    return res


def run_serving(n_requests, uuid, seed=4):
    """Serving workload: n_requests arriving as a Poisson stream over resident sessions
    drawn from the batched size distribution (95 %) plus large sessions (5 %: Na=2048,
    NE=256), each session an SCBA-style repeat (one request in flight per session, its
    buffers stay on the device), admitted against a 120 GB budget.  The arrival rate is
    calibrated to about 80 % of the measured service rate.  Latency = completion - arrival."""
    import numpy as np
    import torch

    from paper_1912_08810_gb300 import inputs, sse
    rng = np.random.default_rng(seed)
    spec = inputs.BatchedSpec(n_instances=24)
    sessions = []
    for inst in inputs.make_batched_torch(spec, seed):
        sessions.append(("normal", inst))
    big = inputs.Geometry(nkz=3, nqz=3, ne=256, nw=16, na=2048, nb=8)
    for j in range(2):
        nrng = np.random.default_rng([seed, 1000 + j])
        neigh = inputs.random_neighbours(nrng, big.na, 8)
        inst = inputs.make_instance_torch(big, 10_000 + j, neigh=neigh, hermitian_pairs=False)
        inst["geometry"] = big
        sessions.append(("large", inst))
    objs = []
    for kind, inst in sessions:
        g = inst["geometry"]
        S = {s: torch.empty_like(inst["G_gt"]) for s in ("gt", "lt")}
        p = sse.Plan(inst["neigh"], inst["dH"], nkz=g.nkz, nqz=g.nqz, ne=g.ne, nw=g.nw, mode="mixed")
        io = p._io(inst["G_gt"], inst["G_lt"], inst["D_gt"], inst["D_lt"], S["gt"], S["lt"])
        objs.append(dict(kind=kind, plan=p, io=io, S=S, points=g.points()))
    # calibration: each session alone, warm, with the split the server uses (no tuning)
    service = []
    old = os.environ.get("SSE_AUTOTUNE")
    os.environ["SSE_AUTOTUNE"] = "0"
    for o in objs:
        sse.sse_execute_batch([o["plan"].handle], [o["io"]], 0)
        torch.cuda.synchronize()
        t = time.perf_counter()
        sse.sse_execute_batch([o["plan"].handle], [o["io"]], 0)
        torch.cuda.synchronize()
        service.append(time.perf_counter() - t)
    if old is None:
        del os.environ["SSE_AUTOTUNE"]
    else:
        os.environ["SSE_AUTOTUNE"] = old
    normal = [i for i, o in enumerate(objs) if o["kind"] == "normal"]
    large = [i for i, o in enumerate(objs) if o["kind"] == "large"]
    mean_s = 0.95 * float(np.mean([service[i] for i in normal])) + 0.05 * float(np.mean([service[i] for i in large]))
    rate = 0.8 / mean_s
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    which = [int(rng.choice(large)) if rng.random() < 0.05 else int(rng.choice(normal)) for _ in range(n_requests)]
    server = sse.sse_server_create(120 << 30, 64, 30000)
    busy = {}
    waiting = {i: [] for i in range(len(objs))}
    lat, done_points, sizes = [], 0, []
    clocks = ClockSampler(uuid)
    clocks.start()
    t0 = time.perf_counter()
    nxt = 0
    inflight = {}
    try:
        while len(lat) < n_requests:
            now = time.perf_counter() - t0
            while nxt < n_requests and arrivals[nxt] <= now:
                waiting[which[nxt]].append((nxt, arrivals[nxt]))
                nxt += 1
            for sidx, q in waiting.items():
                if q and sidx not in busy:
                    rid, arr = q.pop(0)
                    o = objs[sidx]
                    tk = sse.sse_submit(server, o["plan"].handle, o["io"])
                    busy[sidx] = tk
                    inflight[tk] = (sidx, rid, arr)
            for tk in list(inflight):
                rc, r = sse.sse_poll(server, tk)
                if rc == sse.SSE_NOT_READY:
                    continue
                if rc != sse.SSE_OK:
                    raise RuntimeError(f"serving request failed: {sse.status_name(rc)}")
                sidx, rid, arr = inflight.pop(tk)
                del busy[sidx]
                lat.append((time.perf_counter() - t0 - arr) * 1e3)
                sizes.append(r.round_size)
                done_points += objs[sidx]["points"]
            time.sleep(0.0002)
        wall = time.perf_counter() - t0
        rounds, _, _ = sse.sse_server_stats(server)
    finally:
        sse.sse_server_destroy(server)
    clk = clocks.stop()
    for o in objs:
        o["plan"].close()
    torch.cuda.empty_cache()
    return {"requests": n_requests, "sessions": len(objs), "large_fraction": 0.05,
            "arrival_rate_per_s": rate, "budget_gb": 120, "value": done_points / wall, "unit": UNIT,
            "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "mean_ms": float(np.mean(lat)),
            "rounds": rounds, "requests_per_round": n_requests / max(rounds, 1),
            "mean_round_size_seen": float(np.mean(sizes)), "wall_s": wall, "clocks": clk,
            "gpu_launches": int(rounds) + 2 * len(objs),
            "latency": "completion minus Poisson arrival time, host clock"}


def cpu_sample(inst, geo, n_atoms=None):
    """Oracle on atoms [0, n) of the same workload, both signs; returns the baseline dict."""
    import oracle
    cores = oracle.num_threads()
    n = n_atoms or max(4, cores)
    t = time.perf_counter()
    for s in ("gt", "lt"):
        oracle.sigma_atoms(inst["G_" + s], inst["D_" + s], inst["dH"], inst["neigh"], 0, n)
    dt = time.perf_counter() - t
    pts = geo.nkz * geo.ne * n
    return {"value": pts / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"atoms 0..{n - 1} x all (kz, E), both signs ({pts} points, {dt:.1f} s)"}


# --- reference arm: the CPU FP64 oracle ---------------------------------------------------

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_1912_08810_gb300 import inputs
    name = args.workload
    geo, inst = make_workload(name)
    cores = oracle.num_threads()
    n = max(4, cores)

    def step():
        for s in ("gt", "lt"):
            oracle.sigma_atoms(inst["G_" + s], inst["D_" + s], inst["dH"], inst["neigh"], 0, n)

    for _ in range(args.warmup):
        step()
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        step()
        times.append(time.perf_counter() - t)
    pts = geo.nkz * geo.ne * n
    value = pts * len(times) / sum(times)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded numpy)", "config": config_dict(geo, name, "oracle"),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"atoms 0..{n - 1} x all (kz, E), both signs per step"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
