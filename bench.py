#!/usr/bin/env python
"""Throughput benchmark of the FC-DOM RTE solver (one JSON line on rank 0).

One bench step = one forward solve of the tomography workload: a 256 x 256
grid on [0,4]^2 cm, M = 32 ordinates, 16 single-beam sources (Transport
Sweep, 16 independent groups), 2000 AB4 steps, 32 detectors, fluence at the
last step: 16 * 256 * 256 * 32 * 2000 = 67.1e9 cell-ordinate-step updates.
The metric is updates/s (whole job); the adjoint gradient rate of the
Multiple-Staggered-Source workload (4 groups of 4 beams, 3000 steps,
checkpoints every 100) is reported beside it.

--impl reference times the FP64 CPU oracle (the method's reference
implementation here) on a bounded sample of the same workload.
Multi-GPU (torchrun): every rank solves the full workload on its own GPU
(weak scaling, no collective on the data path); the time is the max over
ranks and the value counts every rank's updates."""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RTE cell·ordinate·step updates/s and adjoint gradients/s vs plain FP32 GPU"
UNIT = "updates/s"
WORKLOAD_DESC = ("tomo256_M32: 256x256 grid on [0,4]^2 cm, M=32 ordinates, background "
                 "mua=0.1 mus=100 /cm with 3 seeded inclusions, g=0.9, n=1.4, 16 single-beam "
                 "sources (one group each), 2000 AB4 steps at dt=0.04 ps, 32 detectors")
# SIMT FP32 peak: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (max SM clock).
FP32_SIMT_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def load_peaks():
    """Measured peaks (generated MEASURED_PEAKS.json), else the fallback
    figures of one earlier GB300 measurement."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]), "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


PEAKS = load_peaks()

# DRAM traffic per launch from an ncu capture, valid only for the kernel
# source it was taken on.
NCU_TRAFFIC = {
    # dram__bytes_read.sum + dram__bytes_write.sum of one launch from ncu on
    # the tomography workload's per-launch size (16 groups x 256^2 x 32),
    # keyed by the kernel and the sha256 prefix of its sources; an entry
    # whose sources changed since its capture no longer matches.
    # TMA-fed x-pass (csrc/rte_tc_stream.cu + rte_tc_common.cuh) and the
    # one-tile y-pass (csrc/rte_tc.cu + rte_tc_common.cuh), schedule 4:
    # profiles/tc_stream_passes_tomo256_ncu.md
    # TMA-fed x-pass (csrc/rte_tc_stream.cu + rte_tc_common.cuh) and the
    # one-tile y-pass (csrc/rte_tc.cu + rte_tc_common.cuh), schedule 4:
    # profiles/tc_stream_passes_tomo256_ncu.md
    ("tc_pass_stream<x>", "1eb1154312966384"): 138.943232e6 + 90.579968e6,
    ("tc_pass_kernel<y>", "5ad975b3d17dce21"): 687.169280e6 + 188.580352e6,
    # tile-local fused step (csrc/rte_fused.cu), 16 x 16 parts:
    # profiles/fused_step_tomo256_ncu_full.md
    ("fused_step_kernel", "09d63ccdc8189d08"): 538.545920e6 + 231.291136e6,
    # its tensor-core form (csrc/rte_fused_tc.cu + rte_tc_common.cuh):
    # profiles/fused_step_tc_tomo256_ncu.md
    ("fused_step_tc_kernel", "36c1cad1904e669a"): 540.756736e6 + 231.811840e6,
}


def kernel_source_hash(name="tc_pass_ws"):
    """sha256 prefix of the sources a kernel is compiled from."""
    if name.startswith("tc_pass_ws"):
        srcs = ["rte_tc_ws.cu", "rte_tc_common.cuh"]
    elif name.startswith("tc_ypass_pipe"):
        srcs = ["rte_tc_pipe.cu", "rte_tc_common.cuh"]
    elif name.startswith("tc_pass_stream"):
        srcs = ["rte_tc_stream.cu", "rte_tc_common.cuh"]
    elif name.startswith("tc_pass"):
        srcs = ["rte_tc.cu", "rte_tc_common.cuh"]
    elif name.startswith("fused_step_tc"):
        srcs = ["rte_fused_tc.cu", "rte_tc_common.cuh"]
    elif name.startswith("fused_step"):
        srcs = ["rte_fused.cu"]
    else:
        srcs = ["rte_kernels.cu"]
    h = hashlib.sha256()
    for src in srcs:
        with open(os.path.join(ROOT, "paper_2202_09421_gb300", "csrc", src), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--time-steps", type=int, default=2000, help="AB4 steps per solve")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-steps", type=int, default=40)
    ap.add_argument("--schedule", default="auto",
                    choices=["auto", "one-tile", "persistent", "pipelined", "stream", "stream-xy"],
                    help="tensor-core pass schedule: autotuned, one tile per CTA (the default "
                         "configuration), persistent warp-specialised, one-tile x-pass with the "
                         "pipelined persistent y-pass, or the TMA-fed persistent x-pass")
    ap.add_argument("--no-autotune", action="store_true", help="same as --schedule one-tile")
    ap.add_argument("--inverse", type=int, default=10, metavar="ITERS",
                    help="also run the inverse solver (Algorithm 2) for ITERS L-BFGS-B iterations, "
                         "single sources against staggered groups (0: skip; about 7 s at 10)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the batched (48 media) and 512^2 M=64 precision measurements")
    return ap.parse_args()


def aggregate(updates_per_rank: int, local_ms: float, world: int, max_fn=None):
    """Whole-job rate over `world` ranks that each processed
    `updates_per_rank` updates: the job time is the max over ranks of the
    local time (max_fn reduces across ranks; identity on one rank)."""
    ms = max_fn(local_ms) if max_fn is not None else local_ms
    return updates_per_rank * world / (ms / 1e3), ms


# ---------------------------------------------------------------- oracle timing
_ORACLE_CHILD = """
import json, os, sys, time
sys.path.insert(0, %r)
from rte_inputs import workload_tomo256
from oracle.rte import Solver
n_steps, src, gate = %d, int(sys.argv[1]), sys.argv[2]
wl = workload_tomo256(n_steps=n_steps)
S = Solver(wl)
open(os.path.join(gate, "ready.%%d" %% src), "w").close()
while not os.path.exists(os.path.join(gate, "go")):
    time.sleep(0.001)
t0 = time.time()
S.forward(wl.groups[src %% len(wl.groups)], n_steps, wl.detectors)
t1 = time.time()
g = wl.grid
print(json.dumps({"start": t0, "end": t1, "updates": g.nx * g.ny * g.M * n_steps}))
"""


def oracle_rate(n_steps: int, procs: int | None = None):
    """Times the FP64 oracle on the machine's host cores: `procs` single-threaded
    interpreters (default: one per host core), each solving one source of the
    tomography workload (sources cycle over the 16) for n_steps AB4 steps.
    The sources are independent forward solves, so they run side by side;
    the oracle itself stays plain and single-threaded.  Every interpreter
    sets up its solver, then all start together.  Returns (updates/s over
    the wall time from the first start to the last end, that wall time in s,
    procs)."""
    procs = procs or os.cpu_count() or 1
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    code = _ORACLE_CHILD % (ROOT, n_steps)
    with tempfile.TemporaryDirectory() as gate:
        kids = [subprocess.Popen([sys.executable, "-c", code, str(k), gate], stdout=subprocess.PIPE,
                                 stderr=subprocess.PIPE, text=True, env=env) for k in range(procs)]
        deadline = time.time() + 600
        while sum(os.path.exists(os.path.join(gate, f"ready.{k}")) for k in range(procs)) < procs:
            if any(p.poll() not in (None, 0) for p in kids) or time.time() > deadline:
                for p in kids:
                    p.kill()
                raise RuntimeError("oracle timing: an interpreter failed to start")
            time.sleep(0.01)
        open(os.path.join(gate, "go"), "w").close()
        outs = []
        for p in kids:
            out, err = p.communicate()
            if p.returncode != 0:
                raise RuntimeError(f"oracle timing failed: {err[-500:]}")
            outs.append(json.loads(out.strip().splitlines()[-1]))
    wall = max(o["end"] for o in outs) - min(o["start"] for o in outs)
    return sum(o["updates"] for o in outs) / wall, wall, procs


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = args.cpu_sample_steps
    for _ in range(args.warmup):
        oracle_rate(max(2, n // 8))
    rates, secs = [], []
    procs = 1
    for _ in range(args.steps):
        r, sec, procs = oracle_rate(n)
        rates.append(r)
        secs.append(sec)
    value = statistics.median(rates)
    sample = (f"{procs} sources of the tomography workload side by side (one single-threaded FP64 oracle "
              f"interpreter per host core, sources cycling over the 16) x {n} AB4 steps per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.median(secs), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            self.proc.wait()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return None
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax.append(float(p[2]))
                except ValueError:
                    continue
                for k, nm in enumerate(names):
                    if p[5 + k].lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2202_09421_gb300 import binding as B
    from paper_2202_09421_gb300.solver import FCDOMSolver
    from rte_inputs import workload_mss256, workload_tomo256

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x: float) -> float:
        if world == 1:
            return x
        t = torch.tensor([x], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    wl = workload_tomo256(n_steps=args.time_steps)
    g = wl.grid
    updates = wl.updates
    a = torch.tensor(wl.mua, dtype=torch.float32, device=dev)
    b = torch.tensor(wl.mus, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def time_form(precision, steps, warmup, fc_parts=(1, 1), variant=None, instrument=True, flags=0):
        """Forward solve + detector readout per step; CUDA events on the
        launching stream; L2 flushed before every timed step.  The timed
        steps run without the library's per-kernel events; one more step with
        them on gives the per-pass times."""
        solver = FCDOMSolver(g, wl.optics, a, b, wl.c, wl.dt, ckpt_interval=0, precision=precision,
                             fc_parts=fc_parts, flags=flags)
        schedule = "one-tile" if args.no_autotune else args.schedule
        if variant is not None:
            B.rte_set_pass_variant(solver.ctx, variant)
            tuned = (variant, {})
        elif precision == B.RTE_PREC_FP32:
            tuned = (1, {})
        elif schedule == "auto":
            tuned = solver.autotune(wl.groups, 40)
        else:
            variant = {"persistent": 0, "one-tile": 1, "pipelined": 2, "stream": 4, "stream-xy": 5}[schedule]
            B.rte_set_pass_variant(solver.ctx, variant)
            tuned = (variant, {})

        def one_step():
            solver.forward(wl.groups, wl.n_steps, [wl.n_steps - 1])
            return solver.readout(wl.detectors)

        for _ in range(warmup):
            one_step()
            flush.fill_(1.0)
        barrier()
        launches0 = solver.kernel_launches()
        times = []
        for k in range(steps):
            flush.fill_(float(k))                  # evict the previous step from L2
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one_step()
            e1.record(stream)
            barrier()
            times.append(e0.elapsed_time(e1))
        launches = solver.kernel_launches() - launches0
        if not instrument:
            return solver, statistics.mean(times), [0.0, 0.0], [0, 0], launches, one_step, tuned
        # per-pass device times from one instrumented step (events on the
        # library's stream around every pass), outside the timed region
        flush.fill_(-1.0)
        barrier()
        B.rte_kernel_times(solver.ctx)
        B.rte_set_kernel_timing(solver.ctx, True)
        one_step()
        pass_ms, pass_cnt = B.rte_kernel_times(solver.ctx)
        B.rte_set_kernel_timing(solver.ctx, False)
        return solver, statistics.mean(times), pass_ms, pass_cnt, launches, one_step, tuned

    # Headline: tcgen05 tensor-core form with split 3xTF32 operands (FP32-level
    # accuracy; the forward parity tests hold it to 1e-5 against FP64).
    with ClockSampler(local) as clk:
        solver, ms_step, pass_ms, pass_cnt, launches, one_step, tuned = time_form(
            B.RTE_PREC_TF32X3, args.steps, args.warmup)
    value, ms_step = aggregate(updates, ms_step, world, max_over_ranks)

    # Rooflines.  The step: the method's algorithmic 24 B per update (read
    # u^k, L^{k-1..k-3}; write u^{k+1}, L^k) at the whole-step rate, against
    # HBM.  The dominant pass: y-pass 28 B per update (read u, R, L1..L3;
    # write u, L) against HBM; x-pass tensor-core flops (3 products x 2 flop
    # x (n + M) per update) against the TF32 peak, and its 8 B per update
    # against HBM.
    ncell_m = g.nx * g.ny * g.M * len(wl.groups)
    step_gbs = 24.0 * updates / (ms_step / 1e3) / 1e9
    # the configuration timed: schedule = choice % 6 (0 persistent
    # warp-specialised, 1 one tile per CTA, 2 pipelined y-pass, 4 TMA-fed
    # persistent x-pass, 5 TMA-fed persistent x- and y-passes), choice >= 6
    # tensor-core scattering
    sched = tuned[0] % 6
    names = {0: ["tc_pass_ws<x>", "tc_pass_ws<y>"], 1: ["tc_pass_kernel<x>", "tc_pass_kernel<y>"],
             2: ["tc_pass_kernel<x>", "tc_ypass_pipe<y>"], 4: ["tc_pass_stream<x>", "tc_pass_kernel<y>"],
             5: ["tc_pass_stream<x>", "tc_pass_stream<y>"]}[sched]
    per_launch = [pass_ms[k] / max(1, pass_cnt[k]) for k in range(2)]
    x_gbs = 8.0 * ncell_m / (per_launch[0] / 1e3) / 1e9
    x_tflops = 3 * 2 * (g.nx + g.M) * ncell_m / (per_launch[0] / 1e3) / 1e12
    y_gbs = 28.0 * ncell_m / (per_launch[1] / 1e3) / 1e9
    tf32_peak = PEAKS["bf16_tflops"] / 2.0
    passes = {
        names[0]: {"ms_per_launch": per_launch[0], "share": pass_ms[0] / sum(pass_ms),
                   "hbm": {"achieved": x_gbs, "bytes_per_update": 8, "frac": x_gbs / PEAKS["hbm_gbs"]},
                   "tensor": {"achieved": x_tflops, "unit": "TFLOP/s", "peak": tf32_peak,
                              "frac": x_tflops / tf32_peak,
                              "peak_source": "measured bf16 burst x 1/2 (tf32 nominal ratio)"},
                   "traffic": NCU_TRAFFIC.get((names[0], kernel_source_hash(names[0])))},
        names[1]: {"ms_per_launch": per_launch[1], "share": pass_ms[1] / sum(pass_ms),
                   "hbm": {"achieved": y_gbs, "bytes_per_update": 28, "frac": y_gbs / PEAKS["hbm_gbs"]},
                   "traffic": NCU_TRAFFIC.get((names[1], kernel_source_hash(names[1])))},
    }
    dom = 0 if per_launch[0] >= per_launch[1] else 1
    dom_gbs = x_gbs if dom == 0 else y_gbs
    roofline = {"step_frac": step_gbs / PEAKS["hbm_gbs"],
                "step": {"bytes_per_update": 24, "achieved": step_gbs, "unit": "GB/s",
                         "updates_per_s_ceiling": PEAKS["hbm_gbs"] * 1e9 / 24.0},
                "bound": "hbm", "achieved": dom_gbs, "peak": PEAKS["hbm_gbs"], "unit": "GB/s",
                "frac": dom_gbs / PEAKS["hbm_gbs"], "traffic": passes[names[dom]]["traffic"],
                "kernel": names[dom], "peak_source": f"{PEAKS['source']} (MEASURED_PEAKS.json hbm_gbs)",
                "passes": passes}

    # The other forms on the same workload: the plain FP32 SIMT form (the
    # metric's comparison) and the single-product TF32 reduced-precision form.
    forms = {}
    for name, prec, parts in (("plain_fp32_simt", B.RTE_PREC_FP32, (1, 1)), ("tf32_reduced", B.RTE_PREC_TF32, (1, 1)),
                              ("tf32x3_subdomains_4x4", B.RTE_PREC_TF32X3, (4, 4))):
        s2, ms2, _, _, _, _, _ = time_form(prec, 1, 1, fc_parts=parts, instrument=False)
        s2.close()
        ms2 = max_over_ranks(ms2)
        forms[name] = {"value": updates * world / (ms2 / 1e3), "unit": UNIT, "ms_per_step": ms2,
                       "headline_speedup": ms2 / ms_step}
    # The tile-local fused step (one kernel per step) of the decomposed
    # operator with 16 x 16 parts (16-point owned ranges), FP32 arithmetic;
    # its two-pass counterpart (same operator) beside it.  Roofline: the
    # one-pass algorithmic 24 B per update (read u, L1..L3; write u, L).
    s2, ms2, pm2, pc2, _, _, _ = time_form(B.RTE_PREC_FP32, 1, 1, fc_parts=(16, 16), variant=3)
    s2.close()
    ms2 = max_over_ranks(ms2)
    k_ms = pm2[1] / max(1, pc2[1])
    fused_gbs = 24.0 * ncell_m / (k_ms / 1e3) / 1e9
    forms["tile_local_fused_16x16"] = {
        "value": updates * world / (ms2 / 1e3), "unit": UNIT, "ms_per_step": ms2, "headline_speedup": ms2 / ms_step,
        "operator": "decomposed FC (Sec. 4.4), 16 x 16 parts, FP32",
        "roofline": {"bound": "hbm", "achieved": fused_gbs, "peak": PEAKS["hbm_gbs"], "unit": "GB/s",
                     "frac": fused_gbs / PEAKS["hbm_gbs"], "kernel": "fused_step_kernel",
                     "ms_per_launch": k_ms,
                     "traffic": NCU_TRAFFIC.get(("fused_step_kernel", kernel_source_hash("fused_step_kernel")))}}
    # The same step with its three contractions (x- and y-derivatives,
    # scattering) on the tensor cores, split 3xTF32 (FP32-level accuracy).
    s2, ms2, pm2, pc2, _, _, _ = time_form(B.RTE_PREC_TF32X3, 1, 1, fc_parts=(16, 16), variant=3,
                                           flags=B.RTE_FLAG_TC_FUSED_STEP)
    s2.close()
    ms2 = max_over_ranks(ms2)
    k_ms = pm2[1] / max(1, pc2[1])
    fused_gbs = 24.0 * ncell_m / (k_ms / 1e3) / 1e9
    forms["tile_local_fused_16x16_tc"] = {
        "value": updates * world / (ms2 / 1e3), "unit": UNIT, "ms_per_step": ms2, "headline_speedup": ms2 / ms_step,
        "operator": "decomposed FC (Sec. 4.4), 16 x 16 parts, tcgen05 3xTF32",
        "roofline": {"bound": "hbm", "achieved": fused_gbs, "peak": PEAKS["hbm_gbs"], "unit": "GB/s",
                     "frac": fused_gbs / PEAKS["hbm_gbs"], "kernel": "fused_step_tc_kernel",
                     "ms_per_launch": k_ms,
                     "traffic": NCU_TRAFFIC.get(("fused_step_tc_kernel",
                                                 kernel_source_hash("fused_step_tc_kernel")))}}
    s2, ms2, _, _, _, _, _ = time_form(B.RTE_PREC_TF32X3, 1, 1, fc_parts=(16, 16), variant=1, instrument=False)
    s2.close()
    ms2 = max_over_ranks(ms2)
    forms["tf32x3_subdomains_16x16_two_pass"] = {"value": updates * world / (ms2 / 1e3), "unit": UNIT,
                                                 "ms_per_step": ms2, "headline_speedup": ms2 / ms_step}

    # Photon balance at full size (eq. RTE integrated over angle and domain,
    # FP64 sums on the device, one extra reduction launch per step): the
    # residual (change in photons against the time integral of minus
    # absorption minus net outflux) of every group, relative to its peak
    # photon count, and the cost of recording it.
    sb = FCDOMSolver(g, wl.optics, a, b, wl.c, wl.dt, precision=B.RTE_PREC_TF32X3,
                     flags=B.RTE_FLAG_PHOTON_BALANCE)
    B.rte_set_pass_variant(sb.ctx, tuned[0] % 6)
    sb.forward(wl.groups, wl.n_steps)
    ms_bal = max_over_ranks(_timed(lambda: sb.forward(wl.groups, wl.n_steps), stream, flush, barrier))
    bal = sb.photon_balance().cpu().numpy()
    sb.close()
    resid = [float(((t[-1, 0] - t[0, 0]) - np.trapezoid(-t[:, 1] - t[:, 2], dx=wl.dt)) / np.abs(t[:, 0]).max())
             for t in bal]
    photon_balance = {"max_abs_rel_residual": max(abs(r) for r in resid),
                      "median_rel_residual": float(np.median(resid)),
                      "ms_per_step_with_balance": ms_bal, "overhead_vs_headline": ms_bal / ms_step - 1.0,
                      "definition": "((N(T) - N(t1)) - int(-absorption - net outflux) dt) / max N per group; "
                                    "N = int Phi / c, FP64 on the device"}

    # End to end through the public API with host buffers: copy the medium
    # from pinned host memory, solve, read the detector curves back.
    ha = torch.tensor(wl.mua, dtype=torch.float32).pin_memory()
    hb = torch.tensor(wl.mus, dtype=torch.float32).pin_memory()
    hc = torch.empty((len(wl.groups), len(wl.detectors), wl.n_steps), dtype=torch.float32).pin_memory()
    e2e_times = []
    for k in range(max(1, min(args.steps, 2))):
        flush.fill_(float(k))
        barrier()
        t0 = time.perf_counter()
        a.copy_(ha, non_blocking=True)
        b.copy_(hb, non_blocking=True)
        solver.set_medium(a, b)
        curves = one_step()
        hc.copy_(curves, non_blocking=True)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(statistics.mean(e2e_times))
    e2e = {"value": updates * world / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": ha.numel() * 4 + hb.numel() * 4, "d2h_bytes_per_step": hc.numel() * 4}
    solver.close()

    adjoint = None
    if not args.no_adjoint:
        wm = workload_mss256(n_steps=3000)
        tgt = workload_mss256(n_steps=3000, target=True)
        am = torch.tensor(wm.mua, dtype=torch.float32, device=dev)
        bm = torch.tensor(wm.mus, dtype=torch.float32, device=dev)
        st = FCDOMSolver(tgt.grid, tgt.optics, torch.tensor(tgt.mua, dtype=torch.float32, device=dev),
                         bm, tgt.c, tgt.dt, ckpt_interval=0, precision=B.RTE_PREC_TF32X3)
        st.forward(tgt.groups, tgt.n_steps)
        measured = st.readout(tgt.detectors)
        st.close()

        sched_box = {}

        def gradient_seconds(precision, discrete=False, reps=2):
            """Wall time of one gradient (forward + checkpoint recompute +
            adjoint march + gradient), the last of `reps` runs."""
            sa = FCDOMSolver(wm.grid, wm.optics, am, bm, wm.c, wm.dt, ckpt_interval=100, precision=precision)
            choice = sa.autotune(wm.groups, 40)[0] if precision != B.RTE_PREC_FP32 else None
            sched_box[precision] = choice                 # schedule for this workload's 4 groups
            out = []
            grads = None
            for k in range(reps):
                flush.fill_(float(k))
                barrier()
                t0 = time.perf_counter()
                sa.forward(wm.groups, wm.n_steps)
                fn = sa.discrete_adjoint_gradient if discrete else sa.adjoint_gradient
                J, ga, gb = fn(wm.detectors, measured)
                torch.cuda.synchronize()
                out.append(time.perf_counter() - t0)
                grads = (ga, gb)
            sa.close()
            return max_over_ranks(out[-1]), grads

        gs, _ = gradient_seconds(B.RTE_PREC_TF32X3)
        ds, _ = gradient_seconds(B.RTE_PREC_TF32X3, discrete=True)
        fs, _ = gradient_seconds(B.RTE_PREC_FP32, reps=1)
        adjoint = {"gradients_per_s": world / gs, "seconds_per_gradient": gs,
                   "plain_fp32_gradients_per_s": world / fs, "speedup_vs_plain_fp32": fs / gs,
                   "discrete_gradients_per_s": world / ds, "seconds_per_discrete_gradient": ds,
                   "form": "tcgen05 3xTF32 (headline) against plain FP32 SIMT",
                   "autotune_choice": sched_box.get(B.RTE_PREC_TF32X3),
                   "workload": "mss256_M32: 256x256, M=32, 4 MSS groups x 4 beams, 3000 steps, "
                               "checkpoint every 100, 32 detectors",
                   "update_equivalents_per_gradient": 3 * wm.updates}

    configs = None
    if not args.no_configs:
        configs = {"batched_48_media": measure_batched(args, dev, flush, barrier, max_over_ranks, world),
                   "precision512_M64": measure_precision512(args, dev, flush, barrier, max_over_ranks, world)}

    inverse = measure_inverse(dev, args.inverse) if args.inverse > 0 else None

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, secs, procs = oracle_rate(args.cpu_sample_steps + 20)
        cpu = {"value": rate, "unit": UNIT, "cores": procs, "kind": "oracle",
               "sample": f"{procs} sources of the tomography workload side by side (one single-threaded "
                         f"FP64 oracle interpreter per host core) x {args.cpu_sample_steps + 20} AB4 steps "
                         f"({secs:.1f} s wall)"}

    clocks = clk.summary()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC,
                       "form": "tcgen05 tensor cores, split 3xTF32 operands (FP32-level accuracy)",
                       "autotune": {"choice": tuned[0], "trial_ms_per_40_steps": tuned[1],
                                    "choices": "choice % 6: 0 persistent warp-specialised, 1 one tile per "
                                               "CTA, 2 pipelined y-pass, 4 TMA-fed persistent x-pass, 5 TMA-fed "
                                               "persistent x- and y-passes; choice >= 6: tensor-core scattering"},
                       "updates_per_step": updates * world, "l2": "flushed between timed steps "
                       "(256 MB write) and state > L2", "parallelism": f"replicas x{world}"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks, "forms": forms, "configs": configs, "inverse": inverse,
            "photon_balance": photon_balance, "adjoint": adjoint,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _timed(fn, stream, flush, barrier, reps=1):
    """Mean device time (ms) of fn over reps calls, CUDA events on the
    launching stream, L2 flushed before each."""
    import torch
    times = []
    for k in range(reps):
        flush.fill_(float(k))
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        barrier()
        times.append(e0.elapsed_time(e1))
    return statistics.mean(times)


def _rel(a, b):
    import torch
    return float(torch.linalg.norm((a - b).double()) / torch.linalg.norm(b.double()))


def measure_batched(args, dev, flush, barrier, max_over_ranks, world):
    """48 neck-like media on grids of 128..384 points per side (M = 32, one
    beam each, 1500 steps): plain FP32 kernels one medium after another
    against the batched tensor-core forms (one launch per pass per step over
    all media), and each form's detector curves against the FP32 run."""
    import torch
    from paper_2202_09421_gb300 import binding as B
    from paper_2202_09421_gb300.solver import FCDOMSolver, forward_batch
    from rte_inputs import workload_batched
    wls = workload_batched()
    n_steps = wls[0].n_steps
    updates = sum(w.updates for w in wls)
    stream = torch.cuda.current_stream()
    meds = [(torch.tensor(w.mua, dtype=torch.float32, device=dev),
             torch.tensor(w.mus, dtype=torch.float32, device=dev)) for w in wls]
    out, ref = {}, None
    forms = (("plain_fp32_per_medium", B.RTE_PREC_FP32, 0, False),
             ("tf32x3_batched_graph", B.RTE_PREC_TF32X3, B.RTE_FLAG_CUDA_GRAPH, True),
             ("bf16x3_batched_graph", B.RTE_PREC_BF16X3, B.RTE_FLAG_CUDA_GRAPH, True))
    for name, prec, flags, batched in forms:
        ss = [FCDOMSolver(w.grid, w.optics, a, b, w.c, w.dt, precision=prec, flags=flags)
              for w, (a, b) in zip(wls, meds)]

        def run():
            if batched:
                forward_batch(ss, [w.groups for w in wls], n_steps)
            else:
                for s_, w in zip(ss, wls):
                    s_.forward(w.groups, n_steps)
        run()
        l0 = ss[0].kernel_launches()
        ms = max_over_ranks(_timed(run, stream, flush, barrier))
        launches = ss[0].kernel_launches() - l0
        curves = torch.cat([s_.readout(w.detectors).flatten() for s_, w in zip(ss, wls)])
        if ref is None:
            ref = curves
        out[name] = {"value": updates * world / (ms / 1e3), "unit": UNIT, "ms_per_solve_set": ms,
                     "launches_first_medium": launches,
                     "curves_rel_l2_vs_plain_fp32": _rel(curves, ref)}
        for s_ in ss:
            s_.close()
    base = out["plain_fp32_per_medium"]["value"]
    for v in out.values():
        v["speedup_vs_plain_fp32"] = v["value"] / base

    # Gradients of all 48 media (forward + checkpoint recompute + continuous
    # adjoint, 3xTF32, checkpoints every 50 steps), data a 10 % weaker
    # signal: the batched adjoint (one launch per pass over all media)
    # against each medium's own adjoint after the same batched forward.
    from paper_2202_09421_gb300.solver import adjoint_gradient_batch
    ss = [FCDOMSolver(w.grid, w.optics, a, b, w.c, w.dt, precision=B.RTE_PREC_TF32X3, ckpt_interval=50)
          for w, (a, b) in zip(wls, meds)]
    forward_batch(ss, [w.groups for w in wls], n_steps)
    meas = [0.9 * s_.readout(w.detectors) for s_, w in zip(ss, wls)]
    dets = [w.detectors for w in wls]

    def grad_batched():
        forward_batch(ss, [w.groups for w in wls], n_steps)
        return adjoint_gradient_batch(ss, dets, meas)

    def grad_each():
        forward_batch(ss, [w.groups for w in wls], n_steps)
        return [s_.adjoint_gradient(w.detectors, m) for s_, w, m in zip(ss, wls, meas)]

    grads = {}
    for name, fn in (("batched", grad_batched), ("each_medium", grad_each)):
        flush.fill_(0.0)
        barrier()
        t0 = time.perf_counter()
        res = fn()
        torch.cuda.synchronize()
        grads[name] = (max_over_ranks(time.perf_counter() - t0), res)
    dmax = max(float((x[1] - y[1]).abs().max()) for x, y in zip(grads["batched"][1], grads["each_medium"][1]))
    for s_ in ss:
        s_.close()
    gradients = {"form": "tcgen05 3xTF32, checkpoints every 50 steps",
                 "batched_gradient_sets_per_s": world / grads["batched"][0],
                 "each_medium_gradient_sets_per_s": world / grads["each_medium"][0],
                 "speedup": grads["each_medium"][0] / grads["batched"][0],
                 "max_abs_diff_dJ_dmua_batched_vs_each": dmax,
                 "unit": "gradient sets (all 48 media) per s"}
    return {"workload": "48 neck-like media, grids from {128,192,256,384}^2 at dx = 4/255 cm, M = 32, "
                        f"one beam each, {n_steps} steps", "updates_per_solve_set": updates, "forms": out,
            "gradients": gradients}


def measure_precision512(args, dev, flush, barrier, max_over_ranks, world):
    """512 x 512, M = 64, g = 0.8 smooth random medium, one beam, 3000 steps:
    every precision form, timed, and its detector curves and final fluence
    against the plain FP32 run."""
    import torch
    from paper_2202_09421_gb300 import binding as B
    from paper_2202_09421_gb300.solver import FCDOMSolver
    from rte_inputs import workload_precision512
    wl = workload_precision512()
    stream = torch.cuda.current_stream()
    a = torch.tensor(wl.mua, dtype=torch.float32, device=dev)
    b = torch.tensor(wl.mus, dtype=torch.float32, device=dev)
    out, ref = {}, None
    for name, prec in (("plain_fp32_simt", B.RTE_PREC_FP32), ("tf32x3", B.RTE_PREC_TF32X3),
                       ("tf32", B.RTE_PREC_TF32), ("bf16x3", B.RTE_PREC_BF16X3), ("bf16", B.RTE_PREC_BF16)):
        s_ = FCDOMSolver(wl.grid, wl.optics, a, b, wl.c, wl.dt, precision=prec)
        box = {}

        def run():
            box["fl"] = s_.forward(wl.groups, wl.n_steps, [wl.n_steps - 1])
        run()
        ms = max_over_ranks(_timed(run, stream, flush, barrier))
        curves = s_.readout(wl.detectors)
        if ref is None:
            ref = (curves, box["fl"])
        out[name] = {"value": wl.updates * world / (ms / 1e3), "unit": UNIT, "ms_per_solve": ms,
                     "curves_rel_l2_vs_plain_fp32": _rel(curves, ref[0]),
                     "fluence_rel_l2_vs_plain_fp32": _rel(box["fl"], ref[1])}
        s_.close()
    base = out["plain_fp32_simt"]["value"]
    for v in out.values():
        v["speedup_vs_plain_fp32"] = v["value"] / base
    return {"workload": f"precision512_M64: 512x512 on [0,4]^2, M = 64, g = 0.8, smooth random mua/mus, "
                        f"1 beam, {wl.n_steps} steps", "updates_per_solve": wl.updates, "forms": out}


def measure_inverse(dev, iters):
    """Algorithm 2 on the 64 x 64, M = 32 inverse workload (a 1 cm square,
    two absorbing disks in a known background, 2000 steps): data from the
    target medium
    plus 10 % seeded noise, L-BFGS-B on the absorption within [0.1, 1]
    /cm from the background, with the 16 beams as single sources (TS) and
    as 4 staggered groups (MSS), the latter also driven by the exact
    discrete gradient instead of the paper's continuous adjoint.  Reports
    E(i), J and the wall time."""
    import torch
    from paper_2202_09421_gb300 import binding as B
    from paper_2202_09421_gb300.inverse import gpu_evaluator, node_areas, reconstruct
    from paper_2202_09421_gb300.solver import FCDOMSolver
    from rte_inputs import add_relative_noise, workload_inverse
    out = {}
    for mode, exact in (("ts", False), ("mss", False), ("mss_exact", True)):
        base = mode.split("_")[0]
        wl, tgt = workload_inverse(base), workload_inverse(base, target=True)
        mus = torch.tensor(wl.mus, dtype=torch.float32, device=dev)
        st = FCDOMSolver(tgt.grid, tgt.optics, torch.tensor(tgt.mua, dtype=torch.float32, device=dev), mus,
                         tgt.c, tgt.dt, precision=B.RTE_PREC_TF32X3)
        st.forward(tgt.groups, tgt.n_steps)
        clean = st.readout(tgt.detectors).cpu().numpy()
        st.close()
        meas = torch.tensor(add_relative_noise(clean, 0.10), dtype=torch.float32, device=dev)
        solver = FCDOMSolver(wl.grid, wl.optics, torch.tensor(wl.mua, dtype=torch.float32, device=dev), mus,
                             wl.c, wl.dt, ckpt_interval=100, precision=B.RTE_PREC_TF32X3)
        ev = gpu_evaluator(solver, wl.groups, wl.n_steps, wl.detectors, meas, mus, exact=exact)
        res = reconstruct(ev, wl.mua, 0.1, 1.0, max_iter=iters, a_true=tgt.mua, area=node_areas(wl.grid))
        solver.close()
        hist = res["history"]
        secs = hist[-1]["seconds"]
        out[mode] = {"groups": len(wl.groups), "gradient": "exact discrete adjoint" if exact else "continuous adjoint",
                     "iterations": len(hist) - 1, "objective_evaluations": res["nfev"],
                     "seconds": secs, "seconds_per_evaluation": secs / max(1, res["nfev"]),
                     "E": [h["E"] for h in hist], "J": [h["J"] for h in hist],
                     "seconds_at_iteration": [h["seconds"] for h in hist]}
    out["workload"] = ("inverse64: 64x64 on a 1 cm square, M = 32, background mua 0.1 / mus 100, two seeded "
                       "absorbing disks, 16 beams (TS: 16 sources; MSS: 4 staggered groups), 32 detectors, "
                       "2000 steps at dt 0.04 ps, 10 % noise, bounds [0.1, 1] /cm, 3xTF32, checkpoint every 100")
    out["mss_speedup_per_evaluation"] = (out["ts"]["seconds_per_evaluation"] /
                                         out["mss"]["seconds_per_evaluation"])
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
