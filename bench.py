#!/usr/bin/env python3
"""Benchmark of the lattice Boltzmann Maxwell hot path on GB300.

One benchmark step = the whole hot path over the metallo-dielectric Janus workload
(512 x 512, a = 32, lambda = 32 (T = 96), theta in {0, 30, ..., 180} deg, eps_r1 ~ U[2, 10],
30 periods each): for every instance re-rasterise the disc, reset the lattice, run
29 periods of fused stream-collide steps, one period with Fourier accumulation, and
the stress-tensor contour integral -> (F~x, F~y, M~z).  The metric is lattice
updates per second (MLUPS) over all steps of all instances.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
Under torchrun each rank runs its own seeded copy of the workload (weak scaling, no
collective on the data path) and rank 0 prints one JSON line.
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
sys.path.insert(0, ROOT)

METRIC = "MLUPS & HBM GB/s (% of peak) per precision form; design-map cells/sec at <=1e-3 force err"
WORKLOAD = "md_janus_512"
# algorithmic bytes per lattice update: the 11 stored planes read and written once, plus
# the 1-byte material id (FP16-deviation: 11 FP16 deviations + 3 FP32 fields each way)
BYTES_PER_LU = {"f64": 11 * 8 * 2 + 1, "f32": 11 * 4 * 2 + 1, "f16dev": 2 * (11 * 2 + 3 * 4) + 1,
                "f32x2": 11 * 8 * 2 + 1}
STEP_KERNEL = {"f64": "k_step<double, false, TM>", "f32": "k_step2_tma<false, TM> (two steps per launch)",
               "f16dev": "k_step2_f16_tma<false> (two steps per launch)"}
# step kernel of a form by steps per launch (polarization P)
KERNELS = {("f32", 1): "k_step<float, false, {P}>", ("f32", 2): "k_step2_tma<false, {P}> (TMA-staged 64 x 8 tiles)",
           ("f32", 3): "k_step3_tma<false, {P}> (TMA-staged 28 x 12 tiles)", ("f16dev", 1): "k_step_f16<false>",
           ("f16dev", 2): "k_step2_f16_tma<false> (TMA-staged 64 x 8 tiles)", ("f64", 1): "k_step<double, false, {P}>",
           ("f32", 4): "k_step4_stream<false, {P}> (row-streaming, 4 time levels in registers)",
           ("f16dev", 4): "k_step4_stream<true, TM> (row-streaming, 4 time levels in registers)",
           ("f32x2", 1): "k_step<df, false, {P}> (double-float)",
           ("f32x2", 2): "k_step2<df, false, {P}> (double-float)"}
# lattice steps one launch of that kernel advances (the default mode of each form)
STEPS_PER_LAUNCH = {"f64": 1, "f32": 2, "f16dev": 2}
# FP64 pipe operations per lattice update of the step kernel: 12 for the moments
# (sums of 5, 5 and 5 stored populations, one scaling), 16 for the equilibria and 2 f^eq - f
FP64_OPS_PER_LU = 28
SMS, FP64_OPS_PER_CLK_PER_SM = 152, 2


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--precision", default="f64", choices=["f64", "f32", "f16dev"])
    p.add_argument("--no-hbm-scale", action="store_true")
    p.add_argument("--no-design-map", action="store_true")
    p.add_argument("--design-map-instances", type=int, default=256)
    p.add_argument("--profile-case", action="store_true",
                   help="small case for ncu: two launches of each step kernel on a 2048^2 lattice and of the FP64 step on the 512^2 workload")
    p.add_argument("--profile-only", default="",
                   help="with --profile-case: only these form:mode[:acc] items and design maps (e.g. f32:four,f32:four:acc,batch4)")
    p.add_argument("--profile-n", type=int, default=2048, help="with --profile-only: the lattice size")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-forms", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=4.0,
                   help="target length of each of the four CPU-baseline samples")
    p.add_argument("--repeats", type=int, default=5, help="repeats of every secondary line (median and spread)")
    p.add_argument("--ncu-summary", metavar="CSV",
                   help="summarise an ncu --csv metrics capture of --profile-case into --ncu-out and exit")
    p.add_argument("--ncu-out", default=os.path.join(ROOT, "profiles", "counters.json"))
    p.add_argument("--ncu-command", default="", help="the command that made the capture (recorded in the summary)")
    return p.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_sha():
    """Hash of the sources of the FP64 step kernel (its counters go stale when they change)."""
    h = hashlib.sha256()
    for name in ("common.cuh", "step.cu"):
        with open(os.path.join(ROOT, "paper_2509_22308_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


COUNTERS = os.path.join(ROOT, "profiles", "counters.json")
FP64_OP_METRICS = ("sm__sass_thread_inst_executed_op_dadd_pred_on.sum",
                   "sm__sass_thread_inst_executed_op_dmul_pred_on.sum",
                   "sm__sass_thread_inst_executed_op_dfma_pred_on.sum")


def profiled_counters(kernel_prefix):
    """Per-launch counters of the FP64 step kernel on one 512^2 instance of the benchmark
    workload, from the machine-readable ncu summary (bench.py --ncu-summary), or None when
    it is missing or the kernel source changed since the capture."""
    try:
        with open(COUNTERS) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("source_sha256_16") != kernel_source_sha():
        return None
    for name, k in d.get("kernels", {}).items():
        if kernel_prefix in name and k.get("grid_sites") == 512 * 512:
            return k
    return None


def summarize_ncu(csv_path, out_path, command):
    """ncu --csv (metrics page) -> per-kernel mean of every metric per launch (JSON)."""
    import csv
    per = {}
    with open(csv_path, newline="") as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for row in csv.DictReader(lines):
        name = row.get("Kernel Name", "")
        grid = row.get("Grid Size", "")
        key = (name, grid, row.get("ID"))
        try:
            v = float(row["Metric Value"].replace(",", ""))
        except (KeyError, ValueError):
            continue
        per.setdefault(key, {})[row["Metric Name"]] = v
    kernels = {}
    for (name, grid, _), metrics in per.items():
        k = kernels.setdefault(f"{name} grid{grid}", {"launches": 0, "sum": {}})
        k["launches"] += 1
        for m, v in metrics.items():
            k["sum"][m] = k["sum"].get(m, 0.0) + v
    out = {"command": command, "source_sha256_16": kernel_source_sha(), "kernels": {}}
    for name, k in kernels.items():
        n = k["launches"]
        e = {"launches": n, "per_launch": {m: v / n for m, v in k["sum"].items()}}
        pl = e["per_launch"]
        if "dram__bytes_read.sum" in pl and "dram__bytes_write.sum" in pl:
            e["dram_bytes_per_launch"] = pl["dram__bytes_read.sum"] + pl["dram__bytes_write.sum"]
        if all(m in pl for m in FP64_OP_METRICS):
            e["fp64_ops_per_launch"] = sum(pl[m] for m in FP64_OP_METRICS)
        # the profile case's FP64 step kernels run on one 512^2 instance (grid of 16 x 16 x 1 blocks of 32 x 8)
        if "k_step<double" in name and "(16, 64, 1)" in name:
            e["grid_sites"] = 512 * 512
        out["kernels"][name] = e
    with open(out_path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
    print(f"wrote {out_path}: {len(out['kernels'])} kernels")


class ClockSampler:
    """nvidia-smi clock and throttle samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), max=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], pcap=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["max"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(r["power"] for r in rows)}


def max_over_ranks(value, dist=None):
    """Maximum of a per-rank float over all ranks (the job finishes with its slowest rank)."""
    if dist is None:
        return float(value)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def instance_lus(inst):
    return inst["nx"] * inst["ny"] * inst["periods"] * inst["period"]


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_sample(inst, threads, target_s, accumulate=True):
    """The oracle as it stands, on `threads` host cores: a bounded sample of one instance's
    hot path (plain steps, one accumulated period, the contour integral), or of its plain steps
    only (accumulate=False: for lattices where one period alone would take far longer than
    target_s)."""
    from oracle import geometry as G
    from oracle import lbm as OL
    from oracle import mst
    eps, pec, _ = G.janus_material(inst["nx"], inst["ny"], inst["a"], inst["phi0"], inst["eps1"],
                                   inst["eps2"], inst["pec2"])
    sim = OL.Simulation(eps, pec, period=inst["period"], ramp_steps=inst["ramp"], nthreads=threads)
    t0 = time.perf_counter()
    sim.advance(4)
    per_step = (time.perf_counter() - t0) / 4
    T = inst["period"] if accumulate else 0
    n_plain = max(1 if not accumulate else 0, int(target_s / per_step) - T)
    t0 = time.perf_counter()
    sim.advance(n_plain)
    if accumulate:
        sim.advance(T, accumulate=True)
        cx, cy = G.default_center(inst["nx"], inst["ny"])
        mst.force_torque(*sim.phasors(), cx, cy, inst["R"], mst.default_n_points(inst["R"]), inst["a"])
    el = time.perf_counter() - t0
    steps = n_plain + T
    return {"mlups": round(inst["nx"] * inst["ny"] * steps / el / 1e6, 2), "threads": threads,
            "steps": steps, "seconds": round(el, 2)}


def cpu_baseline(cfg1, cfg2, slice1024, target_s):
    """The oracle on the host: the 256^2 homogeneous workload and one 512^2 instance of the
    benchmark workload (whole hot path), and a 1024^2 instance of the 256-instance design map
    (plain steps), each on one thread and on every core; the headline value is the benchmark
    workload on every core."""
    threads = os.cpu_count() or 1
    runs = {}
    for cname, inst, acc in (("homogeneous_dielectric_256", cfg1, True), (WORKLOAD, cfg2, True),
                             ("design_map_1024_slice_plain_steps", slice1024, False)):
        for th in sorted({1, threads}):
            runs[f"{cname}_{th}_threads"] = oracle_sample(inst, th, target_s, accumulate=acc)
    main = runs[f"{WORKLOAD}_{threads}_threads"]
    return {"value": main["mlups"], "unit": "MLUPS", "cores": threads, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": (f"FP64 full-vector C oracle (OpenMP): bounded samples (~{target_s:.0f} s each) of one "
                       f"{cfg2['nx']}x{cfg2['ny']} instance of {WORKLOAD} and of the 256x256 homogeneous workload, "
                       "plain steps + 1 accumulated period + contour integral, and plain steps of a 1024x1024 "
                       "instance of the 256-instance design map, on 1 thread and on every core; "
                       f"value = {WORKLOAD} on {threads} threads"),
            "runs": runs}


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle on the host cores (bounded sample per step)."""
    if rank != 0:
        return
    from paper_2509_22308_gb300 import workloads as W
    from oracle import lbm as OL
    OL.build()
    inst = W.md_janus_512(1)[0]
    budget = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    threads = os.cpu_count() or 1
    vals, secs = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = oracle_sample(inst, threads, budget)
        if i >= args.warmup:
            vals.append(cb)
            secs.append(time.perf_counter() - t0)
    value = statistics.median(v["mlups"] for v in vals)
    sample = (f"FP64 full-vector C oracle, {threads} OpenMP threads: per step a bounded sample (~{budget:.0f} s) "
              f"of one 512x512 instance of {WORKLOAD} (plain steps + 1 accumulated period + contour integral)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * statistics.median(secs), 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": 512, "ny": 512, "instances_sampled": 1},
            "cpu_baseline": {"kind": "oracle", "cores": threads, "sample": sample, "value": value, "unit": "MLUPS",
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def profile_case(only="", n=2048):
    """Two launches of each step kernel (FP64; FP32 and FP16-deviation with two steps per
    launch, then with one; double-float; FP32 with three steps per launch; FP32 and
    FP16-deviation with four) on a 2048^2 lattice (state 0.3-0.7 GB per buffer, larger than
    L2, a few GB on the device in total), two launches of the FP64 step on one 512^2
    instance of the benchmark workload, then a 24-instance FP32 design map with two steps per
    launch and the same map with four.  `only` picks some of them: "form:mode" pairs for the
    lattice (of size n; "form:mode:acc" then also accumulates one period on the contour R), "batch2"
    and "batch4" for the design maps."""
    import torch
    from paper_2509_22308_gb300 import build as B
    B.build()
    from paper_2509_22308_gb300 import lbm_em as L
    from paper_2509_22308_gb300 import workloads as W
    if not only:
        n = 2048
    inst = dict(nx=n, ny=n, a=n / 16.0, phi0=0.5, eps1=4.0, eps2=1.0, pec2=True, period=240, periods=1,
                R=0.09375 * n, ramp=240)
    pairs = (("f64", "auto"), ("f32", "two"), ("f16dev", "two"), ("f32", "one"), ("f16dev", "one"),
             ("f32x2", "auto"), ("f32", "three"), ("f32", "four"), ("f16dev", "four"))
    maps = ("batch2", "batch4")
    if only:
        tokens = only.split(",")
        pairs = tuple(tuple(p.split(":")) for p in tokens if ":" in p)
        maps = tuple(p for p in tokens if ":" not in p)
    for fp, mode, *acc in pairs:
        with L.solver_for_instance(inst, fp, steps_per_launch=mode) as s:
            s.step({"two": 4, "three": 6, "four": 8}.get(mode, 2))
            if acc:
                s.force_torque(L.make_contour(inst["R"], inst["a"]))
            s.sync()
    if not only:
        # two launches of the benchmark's own 512^2 FP64 instance (theta = 0)
        with L.solver_for_instance(W.md_janus_512()[0], "f64") as s:
            s.step(2)
            s.sync()
    # a 24-instance FP32 design map (about 1 GB on the device): the two-step batch kernel with
    # its configuration fixed (no autotuning launches before it), then the four-step one
    # (whose tuning times three row-segment heights before the run)
    for m in maps:
        if m == "batch2":
            b = L.Batch(W.design_map_256(4, 24), "f32", tile_w=64, tile_h=8, ctas_per_sm=3)
        elif m == "batch4":
            b = L.Batch(W.design_map_256(4, 24), "f32", steps_per_launch=4)
        else:
            raise SystemExit(f"unknown profile case {m!r}")
        b.run()
        b.results()
        b.close()
    torch.cuda.synchronize()
    print("profile case done")


def spread(vals):
    """Median and spread of repeated measurements."""
    v = sorted(vals)
    return {"median": round(statistics.median(v), 3), "min": round(v[0], 3), "max": round(v[-1], 3),
            "n": len(v)}


def measure_fp64_peak(L, stream, torch, repeats=5):
    """FP64 pipe rate (FMAs per second, each one FP64 pipe operation) of the library's FMA-chain
    probe, CUDA events on the probe's stream: best of `repeats` launches of ~20 ms."""
    ev = lambda: torch.cuda.Event(enable_timing=True)
    L.probe_fp64_fma(stream, 64)
    rates = []
    for _ in range(repeats):
        a, b = ev(), ev()
        a.record(stream)
        n = L.probe_fp64_fma(stream, 4096)
        b.record(stream)
        b.synchronize()
        rates.append(n / (a.elapsed_time(b) / 1e3) / 1e12)
    return max(rates), statistics.median(rates)


# Single-domain step kernels on the 8192^2 lattice: (form, steps per launch, polarization)
SINGLE_DOMAIN_LINES = (("f32", "auto", "tm"), ("f32", "one", "tm"), ("f32", "two", "tm"), ("f32", "three", "tm"),
                       ("f32", "four", "tm"), ("f16dev", "auto", "tm"), ("f16dev", "one", "tm"),
                       ("f16dev", "four", "tm"), ("f32", "four", "te"), ("f64", "auto", "tm"),
                       ("f32x2", "auto", "tm"), ("f32x2", "two", "tm"), ("f32", "auto", "te"), ("f64", "auto", "te"))


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.ncu_summary:
        summarize_ncu(args.ncu_summary, args.ncu_out, args.ncu_command)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.profile_case:
        profile_case(args.profile_only, args.profile_n)
        return
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)

    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2509_22308_gb300 import build as B
    B.build()
    from paper_2509_22308_gb300 import lbm_em as L
    from paper_2509_22308_gb300 import workloads as W

    prec = args.precision
    instances = W.rank_workload(WORKLOAD, rank)
    n_inst = len(instances)
    # one stream per instance: the instances are independent, so their runs overlap and
    # fill the GPU (a 512^2 step alone is only 1.7 waves of thread blocks)
    main = torch.cuda.Stream()
    streams = [torch.cuda.Stream() for _ in instances]
    solvers = [L.solver_for_instance(inst, prec, st) for inst, st in zip(instances, streams)]
    janus = [L.make_janus(i["a"], i["phi0"], i["eps1"], i["eps2"], i["pec2"]) for i in instances]
    contours = [L.make_contour(i["R"], i["a"]) for i in instances]
    d_out = torch.zeros((n_inst, 3), dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    lus_per_step = sum(instance_lus(i) for i in instances)
    spl = STEPS_PER_LAUNCH[prec]
    launches_per_step = sum(2 + i["periods"] * i["period"] // spl for i in instances)
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def one_step(plain_events=None):
        """Whole hot path of every instance, all instances in flight; returns the
        (start, end) events on the main stream."""
        e_start, e_end = ev(), ev()
        e_start.record(main)
        for s, st, inst, j, c, k in zip(solvers, streams, instances, janus, contours, range(n_inst)):
            st.wait_event(e_start)
            s.set_janus(j)
            s.reset()
            n_plain = (inst["periods"] - 1) * inst["period"]
            a, b = ev(), ev()
            a.record(st)
            s.step(n_plain)
            b.record(st)
            if plain_events is not None:
                plain_events.append((a, b, n_plain, inst["nx"] * inst["ny"]))
            s.force_torque_device(c, d_out[k].data_ptr())
            done = ev()
            done.record(st)
            main.wait_event(done)
        e_end.record(main)
        return e_start, e_end

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    step_ms, plain, windows = [], [], []
    for _ in range(args.steps):
        with torch.cuda.stream(main):
            flush.fill_(1.0)
        n0 = len(plain)
        e0, e1 = one_step(plain)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        # the plain-step phase of this benchmark step: first start to last end over the streams
        starts = [e0.elapsed_time(a) for a, _, _, _ in plain[n0:]]
        ends = [e0.elapsed_time(b) for _, b, _, _ in plain[n0:]]
        windows.append(max(ends) - min(starts))
    torch.cuda.synchronize()
    results = d_out.cpu().numpy()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # the FP64 pipe's measured rate, inside the same clock record (the FP64 step's ceiling)
    fp64_peak, fp64_peak_median = measure_fp64_peak(L, main, torch)
    clocks = sampler.stop()
    total_ms = max_over_ranks(sum(step_ms), dist)
    value = lus_per_step * args.steps * world / (total_ms / 1e3) / 1e6

    # roofline of the dominant kernel, the plain step: its algorithmic work over the
    # window in which the plain steps of all instances ran (CUDA events on their streams)
    plain_ms = sum(windows)
    plain_launches = sum(n for _, _, n, _ in plain) // n_inst // spl
    plain_sites_steps = sum(n * sites for _, _, n, sites in plain)
    # a two-step kernel reads and writes the state once per launch, i.e. once per two steps
    plain_bytes = plain_sites_steps * BYTES_PER_LU[prec] // spl
    avg_launch_us = plain_ms * 1e3 / plain_launches
    achieved = plain_bytes / (plain_ms / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    prof = profiled_counters(STEP_KERNEL[prec].split("<")[0] + "<double") if prec == "f64" else None
    traffic = round(prof["dram_bytes_per_launch"]) if prof and "dram_bytes_per_launch" in prof else None
    if prec == "f64":
        # the FP64 step is bound by the FP64 pipe: operations per update x updates / time,
        # against the pipe's measured rate (FMA-chain probe, same run, same clock record)
        ops = plain_sites_steps * FP64_OPS_PER_LU
        achieved_t = ops / (plain_ms / 1e3) / 1e12
        derived_t = SMS * FP64_OPS_PER_CLK_PER_SM * sm_mhz * 1e6 / 1e12
        roofline = {"bound": "alu", "achieved": round(achieved_t, 4), "peak": round(fp64_peak, 4), "unit": "TFLOP/s",
                    "frac": round(achieved_t / fp64_peak, 4), "traffic": traffic, "kernel": STEP_KERNEL[prec],
                    "flop_convention": f"FP64 pipe operations (add, multiply or FMA = 1), {FP64_OPS_PER_LU} per "
                                       "lattice update",
                    "peak_source": "measured: the library's FP64 FMA-chain probe (lbm_em_probe_fp64_fma), best of "
                                   f"5 launches in this run (median {fp64_peak_median:.4f})",
                    "peak_derived": round(derived_t, 4),
                    "peak_derived_source": f"{SMS} SMs x {FP64_OPS_PER_CLK_PER_SM} FP64 ops/clk x median SM clock "
                                           f"{sm_mhz:.0f} MHz",
                    "algorithmic_ops_per_launch": 512 * 512 * FP64_OPS_PER_LU,
                    "avg_launch_us": round(avg_launch_us, 3),
                    "timing": f"{n_inst} instances on {n_inst} streams; avg_launch_us = plain-step window / "
                              "launches per instance, so one launch slot covers all instances",
                    "hbm_view": {"achieved_gbs": round(achieved, 1), "peak_gbs": peak,
                                 "frac": round(achieved / peak, 4),
                                 "algorithmic_bytes_per_launch": 512 * 512 * BYTES_PER_LU[prec]}}
        if prof and "fp64_ops_per_launch" in prof:
            roofline["fp64_ops_per_lu_measured"] = round(prof["fp64_ops_per_launch"] / (512 * 512), 3)
            roofline["counters_source"] = "profiles/counters.json (ncu, one 512^2 instance of the workload)"
    else:
        roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "traffic": traffic,
                    "kernel": STEP_KERNEL[prec], "peak_source": f"{peak_kind} copy bandwidth",
                    "algorithmic_bytes_per_launch": 512 * 512 * BYTES_PER_LU[prec],
                    "avg_launch_us": round(avg_launch_us, 3)}

    out = {"metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
           "config": {"workload": WORKLOAD, "nx": 512, "ny": 512, "instances": len(instances),
                      "a": 32, "period_steps": 96, "periods": 30,
                      "lattice_updates_per_step": lus_per_step,
                      "l2": "flushed (256 MiB write) between timed steps; a 512^2 lattice's ping-pong "
                            "state can stay L2-resident across the lattice time steps of one run",
                      "parallelism": f"replicas x{world} (independent instances per rank), "
                                     f"{n_inst} concurrent streams per GPU"},
           "roofline": roofline, "gpu_launches": launches_per_step * args.steps, "clocks": clocks,
           "forces_last_step": results.round(6).tolist()}

    if not args.no_e2e:
        # end to end through the C ABI with host buffers: create from host eps/PEC maps,
        # run, read the three results back, destroy; the bytes copied are counted by the
        # library (lbm_em_transfer_bytes) and by the one read-back of the results here
        maps = []
        for i, j in zip(instances, janus):
            reg = L.rasterize_janus(j, i["nx"], i["ny"])
            eps = np.ones((i["ny"], i["nx"]))
            eps[reg == 1] = i["eps1"]
            pec = (reg == 2).astype(np.uint8)
            maps.append((eps, pec))
        e2e_ms = []
        h2d = d2h = 0
        for k in range(args.steps + 1):
            torch.cuda.synchronize()
            c0 = L.transfer_bytes()
            t0 = time.perf_counter()
            hs, outs = [], torch.zeros((n_inst, 3), dtype=torch.float64, device="cuda")
            for inst, (eps, pec), st in zip(instances, maps, streams):
                hs.append(L.Solver(inst["nx"], inst["ny"], prec, eps_map=eps, pec_mask=pec,
                                   source=L.make_source(inst["period"], inst["ramp"]), stream=st))
            for kk, (h_, inst, c) in enumerate(zip(hs, instances, contours)):
                h_.step((inst["periods"] - 1) * inst["period"])
                h_.force_torque_device(c, outs[kk].data_ptr())
            torch.cuda.synchronize()
            host = outs.cpu().numpy()
            for h_ in hs:
                h_.close()
            c1 = L.transfer_bytes()
            if k > 0:
                e2e_ms.append((time.perf_counter() - t0) * 1e3)
                h2d += c1[0] - c0[0]
                d2h += c1[1] - c0[1] + host.nbytes
            assert np.allclose(host, results, rtol=1e-9, atol=1e-12)
        e2e_total = max_over_ranks(sum(e2e_ms), dist)
        out["e2e"] = {"value": round(lus_per_step * args.steps * world / (e2e_total / 1e3) / 1e6, 1),
                      "unit": "MLUPS", "h2d_bytes_per_step": int(h2d // args.steps),
                      "d2h_bytes_per_step": int(d2h // args.steps),
                      "bytes_source": "counted: the library's own host<->device copies (lbm_em_transfer_bytes) "
                                      "plus the read-back of the results"}

    if not args.no_forms and rank == 0:
        # every form on the benchmark workload, sequential on one stream (a 512^2 FP32 or FP16 state
        # stays resident in L2 across steps), repeated; force errors against the FP64 results
        forms = {}
        for fp in ("f32", "f16dev", "f32x2", "f64"):
            ss = [L.solver_for_instance(inst, fp, main) for inst in instances]
            for s, c in zip(ss, contours):  # warm-up (graphs, contour set-up)
                s.step(64)
                s.force_torque(c)
            smp = ClockSampler(local)
            smp.start()
            mlups, gbs_l = [], []
            for _ in range(args.repeats):
                ev_, res = [], []
                t0e, t1e = ev(), ev()
                t0e.record(main)
                for s, inst, c in zip(ss, instances, contours):
                    s.reset()
                    n_plain = (inst["periods"] - 1) * inst["period"]
                    a, b = ev(), ev()
                    a.record(main)
                    s.step(n_plain)
                    b.record(main)
                    ev_.append((a, b, n_plain))
                    res.append(s.force_torque(c))
                t1e.record(main)
                t1e.synchronize()
                ms = t0e.elapsed_time(t1e)
                pms = sum(a.elapsed_time(b) for a, b, _ in ev_)
                pn = sum(n for _, _, n in ev_)
                mlups.append(lus_per_step / (ms / 1e3) / 1e6)
                # one read and one write of the state per launch
                gbs_l.append(pn * 512 * 512 * BYTES_PER_LU[fp] / STEPS_PER_LAUNCH.get(fp, 1) / (pms / 1e3) / 1e9)
            fclk = smp.stop()
            res = np.array(res)
            ref = results if prec == "f64" else res
            drag = np.abs(ref[:, 0])
            err = np.abs(res - ref) / drag[:, None]
            g = statistics.median(gbs_l)
            forms[fp] = {"mlups": round(statistics.median(mlups), 1), "mlups_spread": spread(mlups),
                         "step_kernel_gbs": round(g, 1), "steps_per_launch": STEPS_PER_LAUNCH.get(fp, 1),
                         "frac_hbm": round(g / peak, 4),
                         "max_drag_err_rel": float(err[:, 0].max()),
                         "max_lift_torque_err_drag_scale": float(err[:, 1:].max()),
                         "clocks": fclk}
            for s in ss:
                s.close()
        out["forms"] = forms

    if not args.no_hbm_scale and rank == 0:
        # single-domain step kernel on an 8192^2 lattice (state far larger than the
        # 129 MB L2): algorithmic bytes per lattice update x updates / CUDA-event time, each
        # line repeated (96 steps, whole launches of every mode) with its own clock record.
        # Kernels that advance several steps per launch (temporal blocking) can exceed the
        # one-read-one-write-per-step roofline; their lines add the fraction at their own traffic.
        big = W.md_janus_8192()[0]
        sites = big["nx"] * big["ny"]
        hs = {}
        for fp, mode, pol in SINGLE_DOMAIN_LINES:
            key = fp + {"auto": "", "one": "_one_step_per_launch", "two": "_two_steps_per_launch",
                        "three": "_three_steps_per_launch", "four": "_four_steps_per_launch"}[mode]
            key += "_te" if pol == "te" else ""
            with L.solver_for_instance(big, fp, main, steps_per_launch=mode, polarization=pol) as s:
                s.step(4)
                smp = ClockSampler(local)
                smp.start()
                us_l = []
                for _ in range(args.repeats):
                    a, b = ev(), ev()
                    a.record(main)
                    s.step(96)
                    b.record(main)
                    b.synchronize()
                    us_l.append(a.elapsed_time(b) * 1e3 / 96)
                lclk = smp.stop()
                spl_l = s.steps_per_launch()
                kern = KERNELS[(fp, spl_l)].format(P=pol.upper())
            us = statistics.median(us_l)
            gbs = sites * BYTES_PER_LU[fp] / (us / 1e6) / 1e9
            hs[key] = {"kernel": kern, "steps_per_launch": spl_l, "us_per_step": round(us, 2),
                       "glups": round(sites / (us / 1e6) / 1e9, 2),
                       "glups_spread": spread([sites / (u / 1e6) / 1e9 for u in us_l]),
                       "achieved_gbs": round(gbs, 1), "frac_hbm": round(gbs / peak, 4),
                       "bytes_per_lu": BYTES_PER_LU[fp], "clocks": lclk}
            if spl_l > 1:
                # the state crosses HBM once per launch: 1/spl of the one-pass bytes per update
                hs[key]["own_bytes_per_lu"] = round(BYTES_PER_LU[fp] / spl_l, 2)
                hs[key]["own_frac_hbm"] = round(gbs / spl_l / peak, 4)
            if fp == "f64":
                ops = FP64_OPS_PER_LU + (1 if pol == "te" else 0)   # TE: 29 per update
                hs[key]["fp64_ops_per_lu"] = ops
                t_ops = sites * ops / (us / 1e6) / 1e12
                hs[key]["fp64_tops"] = round(t_ops, 4)
                hs[key]["frac_fp64_measured"] = round(t_ops / fp64_peak, 4)
        out["single_domain_8192"] = hs

    if not args.no_design_map and rank == 0:
        # batched design diagram: seeded dielectric Janus instances, uneven sizes
        # (a in {16, 32, 64}, grid 16 a) and run lengths (20 periods of T = 3 a),
        # one persistent kernel under a CUDA graph; FP32 lattice, FP64 accumulation,
        # force error against the same batch in FP64; FP32 repeated, the FP64 and
        # double-float comparisons twice
        dm = W.design_map_256(4, args.design_map_instances)
        res = {}
        for fp, reps in (("f32", args.repeats), ("f32x2", 2), ("f64", 2)):
            bt = L.Batch(dm, fp, stream=main)
            bt.run()                   # untimed first run (graph capture, first touch)
            bt.results()
            smp = ClockSampler(local)
            smp.start()
            ms_l = []
            for _ in range(reps):
                a, b = ev(), ev()
                a.record(main)
                bt.run()
                b.record(main)
                b.synchronize()
                ms_l.append(a.elapsed_time(b))
            dclk = smp.stop()
            F, _ = bt.results()
            res[fp] = (ms_l, F, bt.config() + (bt.steps_per_launch(),), dclk)
            bt.close()
        ms32, F32, cfg, clk32 = res["f32"]
        ms64, F64, _, _ = res["f64"]
        msx2, FX2, _, _ = res["f32x2"]
        errs = np.max(np.abs(F32 - F64), axis=1) / np.abs(F64[:, 0])
        lus = sum(instance_lus(i) for i in dm)
        m32 = statistics.median(ms32)
        out["design_map"] = {"instances": len(dm), "cells_per_s": round(len(dm) / (m32 / 1e3), 2),
                             "cells_per_s_spread": spread([len(dm) / (m / 1e3) for m in ms32]),
                             "mlups": round(lus / (m32 / 1e3) / 1e6, 1), "ms": round(m32, 1),
                             "fp64_cells_per_s": round(len(dm) / (statistics.median(ms64) / 1e3), 2),
                             "fp64_mlups": round(lus / (statistics.median(ms64) / 1e3) / 1e6, 1),
                             "f32x2_cells_per_s": round(len(dm) / (statistics.median(msx2) / 1e3), 2),
                             "f32x2_max_force_err_drag_scale":
                                 float((np.max(np.abs(FX2 - F64), axis=1) / np.abs(F64[:, 0])).max()),
                             "max_force_err_drag_scale": float(errs.max()),
                             "instances_within_1e-3": int(np.sum(errs <= 1e-3)),
                             "tile_w": cfg[0], "tile_h": cfg[1], "ctas_per_sm": cfg[2], "steps_per_launch": cfg[3],
                             "clocks": clk32,
                             "precision": "f32 lattice, f64 accumulation; error against the same batch in f64"}

    if not args.no_cpu_baseline and rank == 0 and world == 1:
        slice1024 = next(i for i in W.design_map_256(4, 256) if i["nx"] == 1024)
        out["cpu_baseline"] = cpu_baseline(W.homogeneous_dielectric_256()[0], instances[0], slice1024,
                                           args.cpu_seconds)

    for s in solvers:
        s.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
