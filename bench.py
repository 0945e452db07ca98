#!/usr/bin/env python
"""Throughput of the self-gravity field solve on GB300.

One step = one pass of the whole hot path over one disc: ``sg_solve`` on a
2048 x 4096 log-polar grid (gas, h = 0.05, FP32 FFT path, outputs Phi, g_r
and g_phi), i.e. the row R2C, the fused column pass and the row C2R with
epilogue.  The kernel spectra are built once per plan (the paper
precomputes the kernel for the whole run) and are not part of a step; their
build time is reported separately.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: one process per GPU (torchrun); every rank solves its own
independent disc (no data exchange), so the job scales weakly; the time is
the maximum over ranks.  ``--impl reference`` times the FP64 CPU oracle on
the same workload on the host cores (rank 0 only).
"""
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SG field cells/s and HBM roofline fraction at rel-L2<=1e-5 vs FP64 oracle"
UNIT = "cells/s"
L2_FLUSH_BYTES = 256 << 20
PROFILE = os.path.join(ROOT, "profiles", "cols_2048x4096.md")
BIFLUID_PROFILE = os.path.join(ROOT, "profiles", "cols_bifluid_2048x4096.md")
BATCH_PROFILE = os.path.join(ROOT, "profiles", "batch_64discs.md")
BATCH_STREAMS_PROFILE = os.path.join(ROOT, "profiles", "batch_streams_64discs.md")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--nr", type=int, default=2048)
    ap.add_argument("--nphi", type=int, default=4096)
    ap.add_argument("--bifluid", action="store_true", help="gas + dust (St = 0.1) instead of gas only")
    ap.add_argument("--outputs", default="phi,gr,gphi",
                    help="components per fluid: phi,gr,gphi (default) or gr,gphi (accelerations only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--batch", action="store_true",
                    help="64 uneven gas + dust discs per step instead of one 2048 x 4096 disc")
    ap.add_argument("--batch-n", type=int, default=64, help="discs in the batch (the first n of the 64)")
    ap.add_argument("--batch-config", default="auto",
                    help="'auto' (autotune both engines), threads,ctas_per_sm,order,specialize for the persistent "
                         "kernel (e.g. 256,2,staged,1), or streams:K for the stream engine")
    ap.add_argument("--no-loop", action="store_true", help="batch mode: skip timing the per-disc loops")
    ap.add_argument("--direct", action="store_true",
                    help="the exact O(N^2) direct pair sum: GPU at 64 x 128 and 256 x 512, against the oracle's "
                         "direct sum on all host cores (full at 64 x 128, sampled targets and extrapolated above)")
    ap.add_argument("--semi", action="store_true",
                    help="the semi-spectral method (FFT in phi, direct sum in r) on a flaring disc, H/r = 0.05 r^0.25 "
                         "(1024 x 2048 gas unless --nr/--nphi are given)")
    ap.add_argument("--surrogate", action="store_true",
                    help="train the neural-operator surrogate on 512 x 1024 fields and report it against the exact path")
    ap.add_argument("--sur-steps", type=int, default=5000, help="surrogate training steps (2 fields each)")
    ap.add_argument("--engine", default="fft32",
                    choices=("fft32", "dft_fp16x3", "dft_bf16x3", "dft_fp16", "dft_bf16", "tc_bf16x3", "tc_tf32x3",
                             "tc_bf16", "tc_fp16x3"),
                    help="column-pass engine (tensor-core DFT stages for the precision study; gas-only discs)")
    args = ap.parse_args()
    outputs_of(args)          # reject a bad --outputs before any device work
    return args


def workload(args, rank=0):
    from paper_2506_10812_gb300 import inputs
    if args.bifluid:
        return inputs.lognormal_bifluid(args.nr, args.nphi, St=0.1, offset=3 + 1000 * rank)
    return inputs.lognormal_gas(args.nr, args.nphi, offset=2 + 1000 * rank)


_COMP_NAMES = {"phi": "Phi", "gr": "g_r", "gphi": "g_phi"}


def outputs_of(args):
    outs = tuple(x.strip() for x in args.outputs.split(",") if x.strip())
    if not outs or any(x not in _COMP_NAMES for x in outs) or len(set(outs)) != len(outs):
        raise SystemExit(f"--outputs: a comma list of distinct phi, gr, gphi (got {args.outputs!r})")
    return outs


def config_of(args, d):
    return {"workload": d.label + f", h_g={d.h_g}" + (f", h_d={d.h_d:.4g}" if d.h_d else "")
            + ", FFT path, outputs " + " + ".join(_COMP_NAMES[x] for x in outputs_of(args)) + " per fluid",
            "nr": d.nr, "nphi": d.nphi, "r_in": d.r_in, "r_out": d.r_out,
            "fluids": 2 if d.sigma_d is not None else 1,
            "l2": "flushed between timed steps (256 MiB write)",
            "kernel_spectra": "built once per plan, outside the timed steps"}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        self.t0 = time.time()

    def mark(self):
        return time.time()

    def stop(self, t_begin, t_end):
        if self.proc is None:
            return None
        time.sleep(0.12)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        # samples come every 50 ms from start(); keep those inside the timed window
        n0 = max(0, int((t_begin - self.t0) / 0.05) - 1)
        n1 = int((t_end - self.t0) / 0.05) + 2
        sel = rows[n0:n1] or rows
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for _, _, r in sel for i in range(4) if r[i].lower() == "active"})
        return {"sm_mhz": statistics.median(s for s, _, _ in sel), "sm_max_mhz": max(m for _, m, _ in sel),
                "reasons": reasons, "samples": len(sel)}


# -------------------------------------------------------------- roofline
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_hash(names=("sg_kernels.cu", "sg_cols.cuh", "sg_cols_steps.cu", "sg_fft.cuh", "sg_mem.cuh")):
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2506_10812_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(args):
    """DRAM bytes per column-pass launch from the committed ncu summary of this
    workload (2048 x 4096, all three components, gas only or gas + dust), if
    it was taken on the current kernel source."""
    if args.engine != "fft32" or (args.nr, args.nphi) != (2048, 4096) or args.outputs != "phi,gr,gphi":
        return None
    try:
        txt = open(BIFLUID_PROFILE if args.bifluid else PROFILE).read()
    except OSError:
        return None
    m = re.search(r"source_hash:\s*([0-9a-f]+)", txt)
    t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not (m and t) or m.group(1) != kernel_source_hash():
        return None
    return float(t.group(1))


def batch_profiled_ratio(streams=False):
    """DRAM bytes per model byte of a batch step, from the committed ncu
    summary of a smaller batch on the same sources: the persistent kernel's,
    or (streams) the sum over the per-disc launch chains of one step."""
    path, names = ((BATCH_STREAMS_PROFILE, ("sg_batch.cu", "sg_kernels.cu", "sg_rows.cu", "sg_cols.cuh",
                                            "sg_cols_steps.cu", "sg_fft.cuh", "sg_mem.cuh")) if streams
                   else (BATCH_PROFILE, ("sg_batch.cu", "sg_fft.cuh", "sg_mem.cuh")))
    try:
        txt = open(path).read()
    except OSError:
        return None
    m = re.search(r"source_hash:\s*([0-9a-f]+)", txt)
    t = re.search(r"dram_bytes_per_model_byte:\s*([0-9.eE+]+)", txt)
    if not (m and t) or m.group(1) != kernel_source_hash(names):
        return None
    return float(t.group(1))


# -------------------------------------------------------------- multi-GPU
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(x, world):
    """Maximum over ranks (identity for one process)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(cells_per_rank, world, total_ms_max, steps):
    """Cells/s of the whole job: every rank solves its own disc each step, and
    the job takes as long as its slowest rank."""
    return cells_per_rank * world / (total_ms_max / steps * 1e-3)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------ CPU oracle
def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the record."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def time_oracle(d, repeats):
    """Time the oracle's FP64 FFT convolution on the disc as the FP32 path sees
    it (inputs rounded to float32): on all host cores (scipy.fft, one worker
    per core; the reported baseline) and on one core (numpy, whose output is
    also the parity reference).  Kernel spectra are built outside the timing."""
    import os
    import oracle
    import copy
    d = copy.copy(d)
    d.sigma_g = d.sigma_g.astype(np.float32).astype(np.float64)
    if d.sigma_d is not None:
        d.sigma_d = d.sigma_d.astype(np.float32).astype(np.float64)
    g = oracle.Grid(d.nr, d.nphi, d.r_in, d.r_out)
    plan = oracle.fft64_plan(g, d.h_g, d.h_d if d.sigma_d is not None else None, d.G)
    ncpu = os.cpu_count() or 1

    def timed(workers, n):
        times, out = [], None
        for _ in range(n):
            t0 = time.perf_counter()
            out = oracle.fft64_apply(plan, d.sigma_g, d.sigma_d, workers=workers)
            times.append(time.perf_counter() - t0)
        return out, statistics.median(times)

    out, t1 = timed(None, repeats)
    timed(ncpu, 1)                       # thread pool start-up
    _, tn = timed(ncpu, max(repeats, 5))
    return out, {"value": d.cells / tn, "unit": UNIT, "cores": ncpu, "kind": "oracle",
                 "sample": f"median of {max(repeats, 5)} FP64 FFT-convolution solves of the full disc "
                           f"(scipy.fft, {ncpu} workers; kernel spectra precomputed), {tn:.3f} s each",
                 "single_core": {"value": d.cells / t1, "unit": UNIT, "cores": 1,
                                 "sample": f"median of {repeats} solves (numpy, one core), {t1:.3f} s each"},
                 "cpu_count": ncpu, "cpu_model": cpu_model()}


# ------------------------------------------------------------------ ours
def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else torch.cuda.current_device())
    torch.cuda.set_device(dev)
    from paper_2506_10812_gb300 import Plan
    d = workload(args, rank)
    t0 = time.perf_counter()
    plan = Plan(d.nr, d.nphi, d.r_in, d.r_out, d.h_g, d.h_d, G=d.G, device=dev)
    plan_build_ms = (time.perf_counter() - t0) * 1e3
    if args.engine != "fft32":
        plan.set_column_engine(args.engine)
    sg = torch.tensor(d.sigma_g, dtype=torch.float32, device=dev)
    sd = None if d.sigma_d is None else torch.tensor(d.sigma_d, dtype=torch.float32, device=dev)
    out = plan.solve(sg, sd, outputs=outputs_of(args))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    K, W = args.steps, args.warmup
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(K)]
    for e in ev:                     # torch creates the CUDA events on first record
        for x in e:
            x.record()
    import ctypes
    for _ in range(W):
        flush.fill_(1.0)
        plan.solve(sg, sd, out=out)
    torch.cuda.synchronize()
    # the timed steps: plain solves, as a caller runs them (L2 flushed before each)
    clocks = ClockSampler(dev.index)
    clocks.start()
    time.sleep(0.1)
    barrier(world)
    torch.cuda.synchronize()
    t_begin = time.time()
    for k in range(K):
        flush.fill_(1.0)
        ev[k][0].record()
        plan.solve(sg, sd, out=out)
        ev[k][5].record()
    torch.cuda.synchronize()
    barrier(world)
    t_end = time.time()
    clk = clocks.stop(t_begin, t_end)
    step_ms = [e[0].elapsed_time(e[5]) for e in ev]
    # the stage breakdown: a second pass with events between the launches (such
    # solves keep plain stream order, so each stage's events bracket its kernel)
    lib, handle = plan._lib, plan._h
    for k in range(K):
        flush.fill_(1.0)
        arr = (ctypes.c_void_p * 4)(*[x.cuda_event for x in ev[k][1:5]])
        if lib.sg_set_stage_events(handle, arr) != 0:
            raise RuntimeError("sg_set_stage_events failed")
        plan.solve(sg, sd, out=out)
    torch.cuda.synchronize()
    lib.sg_set_stage_events(handle, None)
    stage = {"rows_fwd": [], "cols": [], "rows_inv": []}
    ms3 = (ctypes.c_float * 3)()
    for e in ev:
        arr = (ctypes.c_void_p * 4)(*[x.cuda_event for x in e[1:5]])
        st = lib.sg_stage_times(arr, ms3)
        if st != 0:
            raise RuntimeError(f"sg_stage_times failed ({st})")
        for name, v in zip(stage, ms3):
            stage[name].append(float(v))
    total_ms = reduce_max(sum(step_ms), world)
    ms_per_step = total_ms / K
    cells_all = d.cells * world
    value = whole_job_rate(d.cells, world, total_ms, K)

    # ---- roofline of the dominant kernel (the column pass)
    nsrc = 2 if d.sigma_d is not None else 1
    ncomp = len(outputs_of(args))
    N, nr = d.nphi // 2, d.nr
    col_bytes, step_bytes, min_bytes = solve_model_bytes(nr, d.nphi, nsrc, ncomp)
    col_ms = statistics.mean(stage["cols"])
    peak, peak_kind = measured_peaks()
    achieved = col_bytes / (col_ms * 1e-3) / 1e9
    kname = "k_cols (fused column pass)" if args.engine == "fft32" else f"k_cols_mma ({args.engine} tensor-core DFT stages)"
    roofline = {"bound": "hbm", "kernel": kname, "achieved": round(achieved, 1),
                "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": profiled_traffic(args),
                "peak_source": f"{peak_kind} HBM copy bandwidth", "algorithmic_bytes_per_launch": col_bytes}
    # the column pass against the FP32 arithmetic peak (it is issue-bound, so neither fraction saturates):
    # nominal 5 L log2 L flops per length-L transform and 8 L per source-kernel product, against
    # 152 SMs x 128 FP32 lanes x 2 flops x the median SM clock sampled during the timed steps
    L = 2 * nr
    fft_flops = 5 * L * int(np.log2(L))
    col_flops = N * (nsrc * fft_flops + nsrc * ncomp * (fft_flops + 8 * nsrc * L))
    sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    compute = {"bound": "alu", "kernel": kname, "achieved": round(col_flops / (col_ms * 1e-3) / 1e12, 2),
               "peak": round(fp32_peak, 1), "unit": "TFLOP/s",
               "frac": round(col_flops / (col_ms * 1e-3) / 1e12 / fp32_peak, 4), "flops_per_launch": col_flops,
               "peak_source": "derived: 152 SMs x 128 FP32 FMA lanes x 2 flops x median SM clock",
               "model": "5 L log2 L per transform, 8 L per product"}
    # whole step against the 3-pass model traffic (60 B/cell gas-only with Phi)
    step_frac = step_bytes / (ms_per_step * 1e-3) / 1e9 / peak

    # ---- end to end through the C ABI with host buffers (pinned)
    hin_g = torch.from_numpy(d.sigma_g.astype(np.float32)).pin_memory()
    hin_d = None if d.sigma_d is None else torch.from_numpy(d.sigma_d.astype(np.float32)).pin_memory()
    hout = {k: torch.empty((d.nr, d.nphi), dtype=torch.float32).pin_memory() for k in out}
    plan.solve_host(hin_g, hin_d, out=hout)
    barrier(world)
    e2e_t = []
    for _ in range(args.e2e_steps):
        t0 = time.perf_counter()
        plan.solve_host(hin_g, hin_d, out=hout)
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = reduce_max(statistics.mean(e2e_t), world)
    h2d = 4 * nsrc * d.cells
    d2h = 4 * len(out) * d.cells

    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
              "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
              "dtype": "f32" if args.engine == "fft32" else f"f32 ({args.engine} tensor-core column DFTs)",
              "data": "synthetic (seeded log-normal disc, no dataset)",
              "config": dict(config_of(args, d), **({} if args.engine == "fft32" else {"column_engine": args.engine})),
              "roofline": roofline,
              "compute": compute,
              "step_roofline": {"model_bytes_per_step": step_bytes, "frac": round(step_frac, 4),
                                "compulsory_bytes_per_step": min_bytes,
                                "compulsory_frac": round(min_bytes / (ms_per_step * 1e-3) / 1e9 / peak, 4),
                                "note": "3-pass traffic model over the whole step; compulsory = sources + "
                                        "kernel spectra + outputs"},
              "stages_ms": {k: statistics.mean(v) for k, v in stage.items()},
              "plan_build_ms": plan_build_ms,
              "e2e": {"value": cells_all / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": d2h, "steps": args.e2e_steps},
              "gpu_launches": K * plan.launches_per_solve(),
              "clocks": clk}

    # ---- oracle: CPU baseline and parity of this very output (rank 0)
    if rank == 0 and not args.no_cpu_baseline:
        ref, cpu = time_oracle(d, 3)
        result["cpu_baseline"] = cpu
        import oracle
        got = {k: v.double().cpu().numpy() for k, v in out.items()}
        result["parity"] = {k: {"rel_l2": oracle.rel_l2(got[k], ref[k]), "rel_max": oracle.rel_max(got[k], ref[k])}
                            for k in got}
        result["parity_ok"] = all(v["rel_l2"] <= 1e-5 and v["rel_max"] <= 1e-4 for v in result["parity"].values())
    plan.close()
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------------- reference
def run_reference(args):
    """The oracle's FP64 FFT convolution on the machine's host cores (all of
    them; the single-core figure beside it), on this arm's workload."""
    import os
    world, rank, _ = dist_env()
    if rank != 0:
        return
    d = workload(args, 0)
    import oracle
    g = oracle.Grid(d.nr, d.nphi, d.r_in, d.r_out)
    plan = oracle.fft64_plan(g, d.h_g, d.h_d if d.sigma_d is not None else None, d.G)
    ncpu = os.cpu_count() or 1
    W = max(1, min(args.warmup, 3))
    K = max(1, min(args.steps, 20))
    for _ in range(W):
        oracle.fft64_apply(plan, d.sigma_g, d.sigma_d, workers=ncpu)
    t = []
    for _ in range(K):
        t0 = time.perf_counter()
        oracle.fft64_apply(plan, d.sigma_g, d.sigma_d, workers=ncpu)
        t.append(time.perf_counter() - t0)
    ms = 1e3 * sum(t) / K
    value = d.cells / (ms * 1e-3)
    t1 = []
    for _ in range(2):
        t0 = time.perf_counter()
        oracle.fft64_apply(plan, d.sigma_g, d.sigma_d)
        t1.append(time.perf_counter() - t0)
    ms1 = 1e3 * min(t1)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded log-normal disc, no dataset)", "config": config_of(args, d),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncpu, "kind": "oracle",
                         "sample": f"{K} FP64 FFT-convolution solves of the full disc (scipy.fft, {ncpu} workers; "
                                   f"kernel spectra precomputed); steps capped at 20 to bound the run",
                         "single_core": {"value": d.cells / (ms1 * 1e-3), "unit": UNIT, "cores": 1,
                                         "sample": f"best of 2 solves (numpy, one core), {ms1:.1f} ms each"},
                         "cpu_count": ncpu, "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}), flush=True)


def solve_model_bytes(nr, nphi, nsrc, ncomp):
    """Algorithmic HBM bytes of one FP32 FFT solve with `ncomp` components per
    target fluid: (column pass, whole 3-pass step, compulsory).  The column
    pass reads the row spectra and the kernel spectra (nsrc tables per
    output, (nphi/2 + 1) x nr complex each) and writes the column output;
    the step adds the sources, the row spectra written, the column output
    read back and the outputs; the compulsory traffic is the sources, the
    kernel spectra and the outputs.  Gas only with Phi: 28, 60 and 28 B/cell."""
    N, cells = nphi // 2, nr * nphi
    tables = 8 * nsrc * nsrc * ncomp * (N + 1) * nr
    col = 8 * nsrc * N * nr + tables + 8 * nsrc * ncomp * N * nr
    step = col + 8 * nsrc * N * nr + 4 * nsrc * cells + 8 * nsrc * ncomp * N * nr + 4 * nsrc * ncomp * cells
    compulsory = 4 * nsrc * cells + tables + 4 * nsrc * ncomp * cells
    return col, step, compulsory


def step_model_bytes(nr, nphi, nsrc, nout, esz=4):
    """Algorithmic HBM bytes of one FFT solve of one disc: the sources, the
    row spectra written and read back, the kernel spectra of every requested
    output, the column-pass output written and read back, the outputs."""
    N, c = nphi // 2, 2 * esz
    cells = nr * nphi
    return (esz * nsrc * cells + 2 * c * nsrc * N * nr + c * nsrc * nout * (N + 1) * (nr + 2)
            + 2 * c * nout * N * nr + esz * nout * cells)


def run_batch(args):
    """64 independent uneven gas + dust discs per step (FP32): the batched
    solve (one persistent launch replayed from a CUDA graph, launch shape
    autotuned) against the per-disc launch loop, from C and from Python."""
    import torch
    from paper_2506_10812_gb300 import Batch, Plan, inputs
    dev = torch.device("cuda", torch.cuda.current_device())
    discs = inputs.batch_discs()[:args.batch_n]
    t0 = time.perf_counter()
    plans = [Plan(d.nr, d.nphi, d.r_in, d.r_out, d.h_g, d.h_d, G=d.G, device=dev) for d in discs]
    build_ms = (time.perf_counter() - t0) * 1e3
    sg = [torch.tensor(d.sigma_g, dtype=torch.float32, device=dev) for d in discs]
    sd = [torch.tensor(d.sigma_d, dtype=torch.float32, device=dev) for d in discs]
    outs = [p.solve(g, x) for p, g, x in zip(plans, sg, sd)]
    t0 = time.perf_counter()
    if args.batch_config == "auto":
        batch = Batch(plans, sg, sd, outs, autotune=True)
    elif args.batch_config.startswith("streams:"):
        batch = Batch(plans, sg, sd, outs, streams=int(args.batch_config.split(":", 1)[1]))
    else:
        th, cps, order, spec = args.batch_config.split(",")
        batch = Batch(plans, sg, sd, outs, threads=int(th), ctas_per_sm=int(cps), order=order,
                      specialize=spec == "1")
    tune_ms = (time.perf_counter() - t0) * 1e3
    cfg = batch.config()
    tried = batch.tune_results()
    tile_trials = batch.tile_trials()
    # the other engine's fastest candidate, timed beside the tuned one
    other = None
    if args.batch_config == "auto":
        rest = [(c, m) for c, m in tried if ("streams" in c) != bool(cfg.get("streams", 0))]
        if rest:
            c, _ = min(rest, key=lambda x: x[1])
            other = (Batch(plans, sg, sd, outs, streams=c["streams"]) if "streams" in c else
                     Batch(plans, sg, sd, outs, threads=c["threads"], ctas_per_sm=c["ctas_per_sm"],
                           order=c["order"], specialize=c["specialize"]))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def py_loop():
        for p, g, x, o in zip(plans, sg, sd, outs):
            p.solve(g, x, out=o)

    def timed(fn, K, W, clocks=None):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        for _ in range(W):
            flush.fill_(1.0)
            fn()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
            time.sleep(0.1)
        t_begin = time.time()
        for a, e in ev:
            flush.fill_(1.0)
            a.record()
            fn()
            e.record()
        torch.cuda.synchronize()
        t_end = time.time()
        clk = clocks.stop(t_begin, t_end) if clocks else None
        return sum(a.elapsed_time(e) for a, e in ev) / K, clk

    K, W = args.steps, args.warmup
    ms_graph, clk = timed(batch.solve, K, W, ClockSampler(dev.index))
    batch.sync()
    ms_other = None
    if other is not None:
        ms_other, _ = timed(other.solve, K, W)
        other.sync()
    if args.no_loop:
        ms_loop_c = ms_loop_py = float("nan")
    else:
        ms_loop_c, _ = timed(batch.solve_loop, min(K, 50), W)
        ms_loop_py, _ = timed(py_loop, min(K, 20), W)
    batch.sync()
    cells = sum(d.cells for d in discs)
    model = sum(step_model_bytes(d.nr, d.nphi, 2, 6) for d in discs)
    peak, peak_kind = measured_peaks()
    achieved = model / (ms_graph * 1e-3) / 1e9
    streams = cfg.get("streams", 0)
    ratio = batch_profiled_ratio(streams=bool(streams))
    engine = (f"every disc's sg_solve launch chain on {streams} forked streams of one CUDA graph per step"
              if streams else "one persistent launch per step from a CUDA graph")
    from collections import Counter
    shapes = Counter(f"{d.nr}x{d.nphi}" for d in discs)

    def engine_line(c, ms):
        st = c.get("streams", 0)
        r = batch_profiled_ratio(streams=bool(st))
        a = model / (ms * 1e-3) / 1e9
        return {"config": c, "ms_per_step": ms, "value": cells / (ms * 1e-3),
                "roofline": {"bound": "hbm", "achieved": round(a, 1), "peak": peak, "unit": "GB/s",
                             "frac": round(a / peak, 4), "traffic": None if r is None else round(r * model)}}

    engines = {("streams" if cfg.get("streams", 0) else "persistent"): engine_line(cfg, ms_graph)}
    if other is not None:
        oc = other.config()
        engines["streams" if oc.get("streams", 0) else "persistent"] = engine_line(oc, ms_other)
    tiles_by_shape = {}
    for t in tile_trials:
        key = f"{t['nr']}x{t['nphi']}" + ("+dust" if t["nsrc"] == 2 else "")
        e = tiles_by_shape.setdefault(key, {"disc": t["disc"], "candidates": []})
        e["candidates"].append(dict(t["tiles"], ms=round(t["ms"], 4)))
        if t["chosen"]:
            e["chosen"] = t["tiles"]
    result = {"metric": METRIC, "value": cells / (ms_graph * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": K,
              "warmup": W, "ms_per_step": ms_graph, "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": "f32", "data": "synthetic (64 seeded log-normal gas + dust discs)",
              "config": {"workload": f"{len(discs)} independent gas + dust discs, grids drawn from 128x256..1024x2048, "
                                     "h_g in [0.03, 0.1], St in {0.01, 0.1, 1}, outputs Phi + g_r + g_phi "
                                     "per fluid; " + engine,
                         "shapes": dict(shapes), "cells": cells,
                         "l2": "flushed between timed steps (256 MiB write)",
                         "kernel_spectra": "built once per plan, outside the timed steps"},
              "batch_config": cfg,
              "autotune_candidates": [dict(c, ms=round(m, 4)) for c, m in tried],
              "engines": engines,
              "tile_trials": tiles_by_shape,
              "roofline": {"bound": "hbm",
                           "kernel": (f"per-disc solve chains on {streams} streams (whole step)" if streams
                                      else "k_batch (persistent, whole step)"),
                           "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                           "frac": round(achieved / peak, 4),
                           "traffic": None if ratio is None else round(ratio * model),
                           "traffic_note": "DRAM bytes of a 16-disc capture scaled by model bytes"
                                           + (" (sum over one step's launches, each on a flushed cache)"
                                              if streams else ""),
                           "peak_source": f"{peak_kind} HBM copy bandwidth",
                           "algorithmic_bytes_per_launch": model},
              "per_disc_loop": {"c_ms_per_step": ms_loop_c, "python_ms_per_step": ms_loop_py,
                                "launches_per_step": 3 * len(discs),
                                "speedup_vs_c_loop": ms_loop_c / ms_graph,
                                "speedup_vs_python_loop": ms_loop_py / ms_graph},
              "plan_build_ms": build_ms, "autotune_ms": tune_ms,
              "gpu_launches": K * (cfg["tasks"] if streams else 1), "clocks": clk}
    print(json.dumps(result), flush=True)
    batch.close()
    if other is not None:
        other.close()
    for p in plans:
        p.close()


def run_direct(args):
    """The direct pair sum (Sec. 2.2 kernel with its general-H form, the
    parity path): GPU FP32 and FP64 solves at the 64 x 128 gas disc and the
    256 x 512 gas + dust disc (St = 1, the hardest dust scale height), each
    checked against the FP64 oracle on seeded targets; and the oracle's own
    direct sum on all host cores: full at 64 x 128, a seeded target sample at
    256 x 512 and at the 2048 x 4096 gas disc, extrapolated by targets (each
    target's sum costs the same: all N sources).  Beside them, the FFT path on
    the same two discs: the GPU solve and the oracle's FP64 FFT convolution on
    all host cores and on one."""
    import os
    import torch
    import oracle
    from paper_2506_10812_gb300 import Plan, inputs
    dev = torch.device("cuda", torch.cuda.current_device())
    oracle.build()
    ncpu = os.cpu_count() or 1
    K, W = max(1, min(args.steps, 5)), max(1, min(args.warmup, 2))
    rng = np.random.default_rng(2506108120)
    cases = {"64x128 gas (C1)": inputs.small_gas(),
             "256x512 gas + dust, St = 1 (C2)": inputs.spiral_bifluid(St=1.0)}
    lines, parity = {}, {}
    for name, d in cases.items():
        g = oracle.Grid(d.nr, d.nphi, d.r_in, d.r_out)
        n = d.nr * d.nphi
        full = n <= 8192
        idx = np.arange(n) if full else np.sort(rng.choice(n, 1024, replace=False))
        nsrc = 2 if d.sigma_d is not None else 1
        per = {}
        # 64 x 128 in FP64 (its configuration) and FP32; 256 x 512 in FP32 (its configuration; an FP64 pair sum
        # there takes ~40 s on this GPU's FP64 units and is covered by the parity tests)
        for dtype in ((torch.float64, torch.float32) if full else (torch.float32,)):
            sg = torch.tensor(d.sigma_g, dtype=dtype, device=dev)
            sd = None if d.sigma_d is None else torch.tensor(d.sigma_d, dtype=dtype, device=dev)
            kk, ww = K, W
            with Plan(d.nr, d.nphi, d.r_in, d.r_out, d.h_g, d.h_d, G=d.G, dtype=dtype, method="direct",
                      device=dev) as plan:
                for _ in range(ww):
                    out = plan.solve(sg, sd)
                torch.cuda.synchronize()
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(kk)]
                for a, e in ev:
                    a.record()
                    out = plan.solve(sg, sd)
                    e.record()
                torch.cuda.synchronize()
                ms = sum(a.elapsed_time(e) for a, e in ev) / kk
            # the oracle on the same (rounded) inputs, at the sampled targets
            rd = lambda x: None if x is None else x.astype(np.float32).astype(np.float64) \
                if dtype == torch.float32 else x
            t0 = time.perf_counter()
            ref = oracle.direct(g, rd(d.sigma_g), rd(d.sigma_d), h_g=d.h_g, h_d=d.h_d, G=d.G,
                                targets=None if full else idx)
            t_or = time.perf_counter() - t0
            errs = {}
            for k, v in out.items():
                got = v.double().cpu().numpy().ravel()[idx]
                r = np.asarray(ref[k]).ravel()
                errs[k] = {"rel_l2": float(np.linalg.norm(got - r) / np.linalg.norm(r)),
                           "rel_max": float(np.max(np.abs(got - r)) / np.max(np.abs(r)))}
            key = "f32" if dtype == torch.float32 else "f64"
            per[key] = {"ms": ms, "steps": kk, "cells_per_s": n / (ms * 1e-3),
                        "pairs_per_s": float(n) * n * nsrc * nsrc / (ms * 1e-3)}
            parity[f"{name} {key}"] = errs
            if "oracle_direct" not in per:
                cpu_s = t_or * n / idx.size
                per["oracle_direct"] = {"cells_per_s": n / cpu_s, "cores": ncpu, "seconds_per_solve": cpu_s,
                                        "sample": ("full solve" if full else
                                                   f"{idx.size} seeded targets ({t_or:.1f} s), extrapolated "
                                                   f"by targets to all {n}")}
        # the FFT path on the same disc: the GPU solve in the configuration's dtype, and the oracle's FP64 FFT
        # convolution on all host cores and on one
        fdt = torch.float64 if full else torch.float32
        sg = torch.tensor(d.sigma_g, dtype=fdt, device=dev)
        sd = None if d.sigma_d is None else torch.tensor(d.sigma_d, dtype=fdt, device=dev)
        with Plan(d.nr, d.nphi, d.r_in, d.r_out, d.h_g, d.h_d, G=d.G, dtype=fdt, device=dev) as plan:
            for _ in range(3):
                plan.solve(sg, sd)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(20)]
            for a, e in ev:
                a.record()
                plan.solve(sg, sd)
                e.record()
            torch.cuda.synchronize()
            ms = sum(a.elapsed_time(e) for a, e in ev) / len(ev)
        per["gpu_fft"] = {"dtype": "f64" if full else "f32", "ms": ms, "cells_per_s": n / (ms * 1e-3), "steps": 20}
        fplan = oracle.fft64_plan(g, d.h_g, d.h_d if d.sigma_d is not None else None, d.G)
        tt = {}
        for wk in (None, ncpu):
            oracle.fft64_apply(fplan, d.sigma_g, d.sigma_d, workers=wk)
            ts = []
            for _ in range(5):
                t0 = time.perf_counter()
                oracle.fft64_apply(fplan, d.sigma_g, d.sigma_d, workers=wk)
                ts.append(time.perf_counter() - t0)
            tt[wk] = statistics.median(ts)
        per["oracle_fft64"] = {"cells_per_s": n / tt[ncpu], "cores": ncpu, "seconds_per_solve": tt[ncpu],
                               "single_core": {"cells_per_s": n / tt[None], "seconds_per_solve": tt[None]},
                               "sample": "median of 5 solves (kernel spectra precomputed)"}
        lines[name] = per
    # the 2048 x 4096 gas disc: the oracle's direct sum on a target sample, extrapolated
    d3 = inputs.lognormal_gas(2048, 4096, offset=2)
    g3 = oracle.Grid(d3.nr, d3.nphi, d3.r_in, d3.r_out)
    n3 = d3.nr * d3.nphi
    idx3 = np.sort(rng.choice(n3, 128, replace=False))
    t0 = time.perf_counter()
    oracle.direct(g3, d3.sigma_g, h_g=d3.h_g, G=d3.G, targets=idx3)
    t3 = time.perf_counter() - t0
    c3 = {"cells_per_s": n3 / (t3 * n3 / idx3.size), "seconds_per_solve": t3 * n3 / idx3.size, "cores": ncpu,
          "sample": f"{idx3.size} seeded targets ({t3:.1f} s), extrapolated by targets to all {n3}",
          "extrapolated": True}
    head = lines["256x512 gas + dust, St = 1 (C2)"]
    # each configuration's own dtype: FP64 at 64 x 128 (whose nearly axisymmetric g_phi sits at ~1.4e-5 in FP32,
    # reported beside it), FP32 at 256 x 512
    ok = all(v["rel_l2"] <= (1e-5 if "f32" in k else 1e-11) and v["rel_max"] <= (1e-4 if "f32" in k else 1e-10)
             for k, e in parity.items() if not k.startswith("64x128") or k.endswith("f64") for v in e.values())
    result = {"metric": "direct pair-sum cells/s at rel-L2<=1e-5 vs FP64 oracle (exact kernel, O(N^2))",
              "value": head["f32"]["cells_per_s"], "unit": "cells/s", "n_gpus": 1, "steps": K, "warmup": W,
              "ms_per_step": head["f32"]["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
              "dtype": "f32 (64 x 128 also in f64)", "data": "synthetic (seeded discs of the C1 and C2 recipes)",
              "config": {"workload": "256x512 gas + dust disc, St = 1 (h_d = 1.58e-3), direct pair sum, "
                                     "outputs Phi, g_r, g_phi per fluid", "l2": "inputs < L2; compute-bound"},
              "cases": lines, "parity": parity, "parity_ok": ok,
              "cpu_baseline": {"value": head["oracle_direct"]["cells_per_s"], "unit": "cells/s", "cores": ncpu,
                               "kind": "oracle", "sample": head["oracle_direct"]["sample"],
                               "cpu_count": ncpu, "cpu_model": cpu_model(),
                               "c1_full": lines["64x128 gas (C1)"]["oracle_direct"], "c3_2048x4096_gas": c3},
              "roofline": {"bound": "alu", "kernel": "k_direct (FP32)",
                           "achieved": round(head["f32"]["pairs_per_s"] / 1e9, 2), "unit": "Gpair/s",
                           "peak": None, "frac": None, "traffic": None,
                           "note": "each pair evaluates the scaled Bessel pair K0e, K1e - K0e by branch (series, "
                                   "quadrature or asymptotic), so no fixed flop count per pair exists"},
              "gpu_launches": sum(v["steps"] * (2 if "gas + dust" in c else 1)
                                  for c, per in lines.items() for k, v in per.items() if k in ("f32", "f64"))
                              + sum(per["gpu_fft"]["steps"] * 3 for per in lines.values())}
    print(json.dumps(result), flush=True)


def run_semi(args):
    """The semi-spectral method for scale heights that depend on r: a flaring
    log-normal gas disc, H = 0.05 r^1.25 (App. D's flaring form with p =
    0.25), FP32.  Timed as plain solves (L2 flushed before each), the
    per-mode products (k_semi_mv, which streams the plan's tables once) in a
    second pass with stage events; checked against the oracle's direct sum on
    seeded targets, whose time on all host cores, extrapolated by targets, is
    the CPU baseline (the same finite sum)."""
    import os
    import ctypes
    import torch
    import oracle
    from paper_2506_10812_gb300 import Plan, inputs
    dev = torch.device("cuda", torch.cuda.current_device())
    nr, nphi = (1024, 2048) if (args.nr, args.nphi) == (2048, 4096) else (args.nr, args.nphi)
    d = inputs.lognormal_gas(nr, nphi, offset=2)
    g = oracle.Grid(d.nr, d.nphi, d.r_in, d.r_out)
    R, _ = g.mesh()
    Hg = (0.05 * R ** 1.25).astype(np.float32)
    t0 = time.perf_counter()
    plan = Plan(d.nr, d.nphi, d.r_in, d.r_out, d.h_g, None, G=d.G, method="semispectral",
                H_g=torch.tensor(Hg, device=dev), device=dev)
    build_ms = (time.perf_counter() - t0) * 1e3
    sg = torch.tensor(d.sigma_g, dtype=torch.float32, device=dev)
    out = plan.solve(sg)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    K, W = args.steps, args.warmup
    for _ in range(W):
        flush.fill_(1.0)
        plan.solve(sg, out=out)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(K)]
    for e in ev:                     # torch creates the CUDA events on first record
        for x in e:
            x.record()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    clocks.start()
    time.sleep(0.1)
    t_begin = time.time()
    for k in range(K):
        flush.fill_(1.0)
        ev[k][0].record()
        plan.solve(sg, out=out)
        ev[k][5].record()
    torch.cuda.synchronize()
    clk = clocks.stop(t_begin, time.time())
    ms = sum(e[0].elapsed_time(e[5]) for e in ev) / K
    lib, handle = plan._lib, plan._h
    for k in range(K):
        flush.fill_(1.0)
        arr = (ctypes.c_void_p * 4)(*[x.cuda_event for x in ev[k][1:5]])
        if lib.sg_set_stage_events(handle, arr) != 0:
            raise RuntimeError("sg_set_stage_events failed")
        plan.solve(sg, out=out)
    torch.cuda.synchronize()
    lib.sg_set_stage_events(handle, None)
    stages = {"rows_fwd": [], "semi_mv": [], "rows_inv": []}
    ms3 = (ctypes.c_float * 3)()
    for e in ev:
        arr = (ctypes.c_void_p * 4)(*[x.cuda_event for x in e[1:5]])
        if lib.sg_stage_times(arr, ms3) != 0:
            raise RuntimeError("sg_stage_times failed")
        for name, v in zip(stages, ms3):
            stages[name].append(float(v))
    mv_ms = statistics.mean(stages["semi_mv"])
    N = d.nphi // 2
    table = 3 * N * d.nr * d.nr * 8
    mv_bytes = table + N * d.nr * 8 + 3 * N * d.nr * 8
    peak, peak_kind = measured_peaks()
    achieved = mv_bytes / (mv_ms * 1e-3) / 1e9
    # parity and the CPU baseline: the oracle's direct sum (same H field) on seeded targets
    rng = np.random.default_rng(2506108120)
    idx = np.sort(rng.choice(d.cells, 128, replace=False))
    t0 = time.perf_counter()
    ref = oracle.direct(g, d.sigma_g.astype(np.float32).astype(np.float64), H_g=Hg.astype(np.float64), G=d.G,
                        targets=idx)
    t_or = time.perf_counter() - t0
    parity = {}
    for k, v in out.items():
        got = v.double().cpu().numpy().ravel()[idx]
        r = np.asarray(ref[k])
        parity[k] = {"rel_l2": float(np.linalg.norm(got - r) / np.linalg.norm(r)),
                     "rel_max": float(np.max(np.abs(got - r)) / np.max(np.abs(r)))}
    ncpu = os.cpu_count() or 1
    cpu_s = t_or * d.cells / idx.size
    result = {"metric": METRIC, "value": d.cells / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": W,
              "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
              "data": "synthetic (seeded log-normal disc, no dataset)",
              "config": {"workload": f"{d.nr}x{d.nphi} log-normal gas disc, flaring H = 0.05 r^1.25, semi-spectral "
                                     "method (FFT in phi, direct sum in r), outputs Phi + g_r + g_phi",
                         "nr": d.nr, "nphi": d.nphi, "l2": "flushed between timed steps (256 MiB write)",
                         "tables": f"{table / 1e9:.2f} GB, built once per plan ({build_ms / 1e3:.1f} s), outside "
                                   "the timed steps"},
              "stages_ms": {k: statistics.mean(v) for k, v in stages.items()},
              "roofline": {"bound": "hbm", "kernel": "k_semi_mv (per-mode radial products)",
                           "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                           "frac": round(achieved / peak, 4), "traffic": None,
                           "peak_source": f"{peak_kind} HBM copy bandwidth", "algorithmic_bytes_per_launch": mv_bytes},
              "parity": parity,
              "parity_ok": all(v["rel_l2"] <= 1e-5 and v["rel_max"] <= 1e-4 for v in parity.values()),
              "cpu_baseline": {"value": d.cells / cpu_s, "unit": UNIT, "cores": ncpu, "kind": "oracle",
                               "sample": f"oracle direct sum (the same finite sum) at {idx.size} seeded targets "
                                         f"({t_or:.1f} s), extrapolated by targets to all {d.cells} cells",
                               "cpu_count": ncpu, "cpu_model": cpu_model(), "extrapolated": True},
              "plan_build_ms": build_ms, "gpu_launches": K * 3, "clocks": clk}
    plan.close()
    print(json.dumps(result), flush=True)


def surrogate_flops(nr, nphi, B, M1=16, K1=32):
    """Multiply-add work (x2) of one surrogate forward pass."""
    C, CIN, QH = 32, 7, 64
    n = B * nr * nphi
    per_layer = (2 * (2 * M1) * C * nphi * B * nr            # truncated phi-DFT
                 + 2 * (2 * K1) * (2 * M1 * C) * nr * B      # truncated radial DFT
                 + 2 * 2 * nr * (M1 * C) * (2 * K1) * B      # inverse radial DFT
                 + 2 * 2 * nphi * C * M1 * B * nr            # inverse phi-DFT
                 + 2 * n * C * C                             # pointwise channel mix
                 + 8 * B * K1 * M1 * C * C)                  # per-mode complex mix
    return 4 * per_layer + 2 * n * CIN * C + 2 * n * C * QH + 2 * n * QH * 2


def run_surrogate(args):
    """The spectral neural-operator surrogate on the 512 x 1024 gas + dust
    workload at two retained-mode sizes (16 azimuthal x 16 radial, and 16 x
    32): each trained on seeded fields the exact path labels, validated on
    held-out fields, its forward pass timed with the tcgen05 GEMMs and with
    the mma.sync ones, beside the exact FFT path; Surrogate.solve uses it
    only below the 1e-3 relative-error gate."""
    import torch
    from paper_2506_10812_gb300 import _native as N
    from paper_2506_10812_gb300.surrogate import GATE, Surrogate
    dev = torch.device("cuda", torch.cuda.current_device())
    lib = N.load()
    K, W = args.steps, args.warmup
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(fn):
        for _ in range(W):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        for a, e in ev:
            flush.fill_(1.0)
            a.record()
            fn()
            e.record()
        torch.cuda.synchronize()
        return sum(a.elapsed_time(e) for a, e in ev) / K

    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        peak_tf, peak_bw = float(pk["bf16_tflops"]), float(pk["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        peak_tf, peak_bw = 1900.0, 6800.0
    variants, exact, clk = {}, None, None
    for name, mp, mr in (("16x16", 16, 16), ("16x32", 16, 32)):
        S = Surrogate(nr=512, nphi=1024, batch=2, seed=0, device=dev, modes_phi=mp, modes_r=mr)
        t0 = time.perf_counter()
        hist = S.train(args.sur_steps, lr=2e-3, seed0=1000)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        rel = S.validate(list(range(10 ** 6, 10 ** 6 + 32)))
        N.check(lib.sg_nn_check(None), what="sg_nn_check")
        hs = S.load([10 ** 6 + 100, 10 ** 6 + 101])
        S.k.count = {}
        S.forward()
        count, S.k.count = S.k.count, None
        ms = {}
        for eng, code in (("tcgen05", N.SG_NN_GEMM_TCGEN05), ("mma_sync", N.SG_NN_GEMM_MMA_SYNC)):
            N.check(lib.sg_nn_set_gemm_engine(code), what="sg_nn_set_gemm_engine")
            if eng == "tcgen05" and clk is None:
                sampler = ClockSampler(dev.index)
                sampler.start()
                time.sleep(0.1)
                t_b = time.time()
                ms[eng] = timed(S.forward)
                clk = sampler.stop(t_b, time.time())
            else:
                ms[eng] = timed(S.forward)
        N.check(lib.sg_nn_set_gemm_engine(N.SG_NN_GEMM_TCGEN05), what="sg_nn_set_gemm_engine")
        N.check(lib.sg_nn_check(None), what="sg_nn_check")
        if exact is None:
            plans = [S._plan(h, St) for h, St in hs]
            outs = [{"gr_g": S.gr[b], "gphi_g": S.gphi[b]} for b in range(2)]
            ms_exact = timed(lambda: [p.solve(S.sg[b], S.sd[b], out=o)
                                      for b, (p, o) in enumerate(zip(plans, outs))])
            exact = {"ms": ms_exact, "cells_per_s": 2 * S.npix / (ms_exact * 1e-3)}
        fl = surrogate_flops(S.nr, S.nphi, 2, mp, mr)
        t = ms["tcgen05"] * 1e-3
        variants[name] = {
            "modes": {"azimuthal": mp, "radial": mr},
            "training": {"steps": args.sur_steps, "fields": 2 * args.sur_steps, "seconds": train_s,
                         "final_loss": hist[-1] if hist else None},
            "validation_rel_l2": {"gr_g": float(rel[0]), "gphi_g": float(rel[1]), "fields": 32},
            "gate": GATE, "surrogate_used": bool(S.val_error <= GATE),
            "forward_ms": {"tcgen05_gemm": ms["tcgen05"], "mma_sync_gemm": ms["mma_sync"]},
            "cells_per_s": 2 * S.npix / t,
            "launches_per_forward": count.get("launches", 0), "gemms_per_forward": count.get("gemms", 0),
            "roofline": {"bound": "hbm", "kernel": "surrogate forward (all launches)",
                         "achieved": round(count.get("gemm_bytes", 0) / t / 1e9, 1), "peak": peak_bw,
                         "unit": "GB/s", "frac": round(count.get("gemm_bytes", 0) / t / 1e9 / peak_bw, 4),
                         "traffic": None,
                         "algorithmic_bytes_per_forward": count.get("gemm_bytes", 0),
                         "bytes_note": "each GEMM operand read or written once; elementwise kernels not counted"},
            "tensor": {"achieved_tflops": round(fl / t / 1e12, 2), "peak": peak_tf,
                       "frac": round(fl / t / 1e12 / peak_tf, 5), "algorithmic_flops_per_forward": fl},
        }
        del S
        torch.cuda.empty_cache()
    head = variants["16x16"]
    result = {"metric": "surrogate cells/s and relative L2 vs the exact path (gate 1e-3)",
              "value": head["cells_per_s"], "unit": "cells/s", "n_gpus": 1, "steps": K, "warmup": W,
              "ms_per_step": head["forward_ms"]["tcgen05_gemm"], "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": "bf16 (FP32 accumulate)",
              "data": "synthetic (seeded log-normal + spiral + clump fields)",
              "config": {"workload": "2 gas + dust discs 512x1024, r in [0.1, 5], h_g in {0.03..0.1}, "
                                     "St in {0.01, 0.1, 1}; 4-layer width-32 spectral neural operator, "
                                     "16 x 16 retained modes (headline) and 16 x 32",
                         "l2": "flushed between timed steps (256 MiB write)"},
              "variants": variants, "exact_path": exact,
              "roofline": head["roofline"], "clocks": clk,
              "gpu_launches": K * head["launches_per_forward"]}
    print(json.dumps(result), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.surrogate:
        run_surrogate(args)
    elif args.direct:
        run_direct(args)
    elif args.semi:
        run_semi(args)
    elif args.batch:
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
