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
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-forms", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="target length of the CPU-baseline sample")
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
    h = hashlib.sha256()
    for name in ("common.cuh", "step.cu"):
        with open(os.path.join(ROOT, "paper_2509_22308_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(precision):
    """DRAM bytes per launch of the step kernel from the committed ncu summary, or None
    when the summary is missing or the kernel source changed since it was taken."""
    path = os.path.join(ROOT, "profiles", f"k_step_{precision}_{WORKLOAD}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m_sha = re.search(r"source_sha256_16:\s*([0-9a-f]+)", text)
    m_b = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_b or m_sha.group(1) != kernel_source_sha():
        return None
    return float(m_b.group(1))


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


def cpu_baseline(inst, target_s):
    """The oracle as it stands, on the host cores: a bounded sample of one instance."""
    import numpy as np
    from oracle import geometry as G
    from oracle import lbm as OL
    from oracle import mst
    eps, pec, _ = G.janus_material(inst["nx"], inst["ny"], inst["a"], inst["phi0"], inst["eps1"],
                                   inst["eps2"], inst["pec2"])
    threads = os.cpu_count() or 1
    sim = OL.Simulation(eps, pec, period=inst["period"], ramp_steps=inst["ramp"], nthreads=threads)
    t0 = time.perf_counter()
    sim.advance(8)
    per_step = (time.perf_counter() - t0) / 8
    T = inst["period"]
    n_plain = max(0, int(target_s / per_step) - T)
    t0 = time.perf_counter()
    sim.advance(n_plain)
    sim.advance(T, accumulate=True)
    cx, cy = G.default_center(inst["nx"], inst["ny"])
    mst.force_torque(*sim.phasors(), cx, cy, inst["R"], mst.default_n_points(inst["R"]), inst["a"])
    el = time.perf_counter() - t0
    steps = n_plain + T
    return {"value": inst["nx"] * inst["ny"] * steps / el / 1e6, "unit": "MLUPS", "cores": threads,
            "kind": "oracle",
            "sample": (f"FP64 full-vector C oracle, {threads} OpenMP threads: one {inst['nx']}x{inst['ny']} "
                       f"instance of {WORKLOAD}, {n_plain} steps + 1 accumulated period ({T} steps) + "
                       f"contour integral, {el:.1f} s")}


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle on the host cores (bounded sample per step)."""
    if rank != 0:
        return
    from paper_2509_22308_gb300 import workloads as W
    from oracle import lbm as OL
    OL.build()
    inst = W.md_janus_512(1)[0]
    budget = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    vals, secs = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(inst, budget)
        if i >= args.warmup:
            vals.append(cb)
            secs.append(time.perf_counter() - t0)
    value = statistics.median(v["value"] for v in vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * statistics.median(secs), 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": 512, "ny": 512, "instances_sampled": 1},
            "cpu_baseline": {"kind": "oracle", "cores": vals[0]["cores"], "sample": vals[0]["sample"],
                             "value": value, "unit": "MLUPS"},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def profile_case():
    """Two launches of each step kernel (FP64; FP32 and FP16-deviation with two steps
    per launch, then with one; double-float; FP32 with three steps per launch) on a 2048^2 lattice (state 0.3-0.7 GB per
    buffer, larger than L2, a few GB on the device in total), two launches of the FP64 step
    on one 512^2 instance of the benchmark workload, then a 24-instance FP32 design map."""
    import torch
    from paper_2509_22308_gb300 import build as B
    B.build()
    from paper_2509_22308_gb300 import lbm_em as L
    inst = dict(nx=2048, ny=2048, a=128.0, phi0=0.5, eps1=4.0, eps2=1.0, pec2=True, period=240, periods=1,
                R=192.0, ramp=240)
    for fp, mode in (("f64", "auto"), ("f32", "two"), ("f16dev", "two"), ("f32", "one"), ("f16dev", "one"),
                     ("f32x2", "auto"), ("f32", "three")):
        with L.solver_for_instance(inst, fp, steps_per_launch=mode) as s:
            s.step({"two": 4, "three": 6}.get(mode, 2))
            s.sync()
    # and two launches of the benchmark's own 512^2 FP64 instance (theta = 0)
    from paper_2509_22308_gb300 import workloads as W
    with L.solver_for_instance(W.md_janus_512()[0], "f64") as s:
        s.step(2)
        s.sync()
    # then a 24-instance FP32 design map (about 1 GB on the device) with the batch kernel's
    # two-steps-per-launch configuration fixed (no autotuning launches before it)
    b = L.Batch(W.design_map_256(4, 24), "f32", tile_w=64, tile_h=8, ctas_per_sm=3)
    b.run()
    b.results()
    b.close()
    torch.cuda.synchronize()
    print("profile case done")


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.profile_case:
        profile_case()
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
    traffic = profiled_traffic(prec)
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    if prec == "f64":
        # the FP64 step is bound by the FP64 pipe: 2 FP64 operations per clock per SM
        ops = plain_sites_steps * FP64_OPS_PER_LU
        achieved_t = ops / (plain_ms / 1e3) / 1e12
        peak_t = SMS * FP64_OPS_PER_CLK_PER_SM * sm_mhz * 1e6 / 1e12
        roofline = {"bound": "alu", "achieved": round(achieved_t, 4), "peak": round(peak_t, 4), "unit": "TFLOP/s",
                    "frac": round(achieved_t / peak_t, 4), "traffic": traffic, "kernel": STEP_KERNEL[prec],
                    "flop_convention": f"FP64 pipe operations (add, multiply or FMA = 1), {FP64_OPS_PER_LU} per "
                                       "lattice update",
                    "peak_source": f"derived: {SMS} SMs x {FP64_OPS_PER_CLK_PER_SM} FP64 ops/clk x median SM clock "
                                   f"{sm_mhz:.0f} MHz",
                    "algorithmic_ops_per_launch": 512 * 512 * FP64_OPS_PER_LU,
                    "avg_launch_us": round(avg_launch_us, 3),
                    "timing": f"{n_inst} instances on {n_inst} streams; avg_launch_us = plain-step window / "
                              "launches per instance, so one launch slot covers all instances",
                    "hbm_view": {"achieved_gbs": round(achieved, 1), "peak_gbs": peak,
                                 "frac": round(achieved / peak, 4),
                                 "algorithmic_bytes_per_launch": 512 * 512 * BYTES_PER_LU[prec]}}
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
        # run, read the three results back, destroy
        maps = []
        for i, j in zip(instances, janus):
            reg = L.rasterize_janus(j, i["nx"], i["ny"])
            eps = np.ones((i["ny"], i["nx"]))
            eps[reg == 1] = i["eps1"]
            pec = (reg == 2).astype(np.uint8)
            maps.append((eps, pec))
        e2e_ms = []
        for k in range(args.steps + 1):
            torch.cuda.synchronize()
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
            if k > 0:
                e2e_ms.append((time.perf_counter() - t0) * 1e3)
            assert np.allclose(host, results, rtol=1e-9, atol=1e-12)
        e2e_total = max_over_ranks(sum(e2e_ms), dist)
        h2d = 0
        for i in instances:
            pitch = (i["nx"] + 31) // 32 * 32
            n_pts = 2 * int(np.ceil(2 * np.pi * i["R"]))
            # material ids, material table, phase table, contour slot map, contour points
            h2d += i["nx"] * i["ny"] + 256 * 32 + i["period"] * 16 + pitch * i["ny"] * 4 + n_pts * 64
        out["e2e"] = {"value": round(lus_per_step * args.steps * world / (e2e_total / 1e3) / 1e6, 1),
                      "unit": "MLUPS", "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(len(instances) * (3 * 8 + 4))}

    if not args.no_forms and rank == 0:
        forms = {}
        for fp in ("f32", "f16dev", "f32x2", "f64"):
            if fp == prec:
                forms[fp] = {"mlups": out["value"] / world, "step_kernel_gbs": round(achieved, 1),
                             "steps_per_launch": spl,
                             "frac_hbm": round(achieved / peak, 4)}
                continue
            # sequential on one stream: a 512^2 FP32/FP16 state stays resident in L2 across steps
            ss = [L.solver_for_instance(inst, fp, main) for inst in instances]
            for s, c in zip(ss, contours):  # warm-up (graphs, contour set-up)
                s.step(64)
                s.force_torque(c)
                s.reset()
            ev_ = []
            res = []
            t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0e.record(main)
            for s, inst, c in zip(ss, instances, contours):
                n_plain = (inst["periods"] - 1) * inst["period"]
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
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
            # state bytes per update: one read and one write per launch (two steps for FP32 and
            # FP16-deviation, one for double-float and FP64)
            gbs = pn * 512 * 512 * BYTES_PER_LU[fp] / STEPS_PER_LAUNCH.get(fp, 1) / (pms / 1e3) / 1e9
            res = np.array(res)
            ref = results if prec == "f64" else res
            drag = np.abs(ref[:, 0])
            err = np.abs(res - ref) / drag[:, None]
            forms[fp] = {"mlups": round(lus_per_step / (ms / 1e3) / 1e6, 1), "step_kernel_gbs": round(gbs, 1),
                         "steps_per_launch": STEPS_PER_LAUNCH.get(fp, 1),
                         "frac_hbm": round(gbs / peak, 4),
                         "max_drag_err_rel": float(err[:, 0].max()),
                         "max_lift_torque_err_drag_scale": float(err[:, 1:].max())}
            for s in ss:
                s.close()
        out["forms"] = forms

    if not args.no_hbm_scale and rank == 0:
        # single-domain step kernel on an 8192^2 lattice (state far larger than the
        # 129 MB L2): algorithmic bytes per lattice update x updates / CUDA-event time.
        # The FP32 and FP16-deviation kernels advance two steps per launch (temporal
        # blocking), so they can exceed the one-read-one-write-per-step roofline.
        big = W.md_janus_8192()[0]
        hs = {}
        # TE^z lines: the same lattice and kernels with the TE moments and collision
        for fp, mode, pol in (("f32", "auto", "tm"), ("f32", "one", "tm"), ("f32", "two", "tm"), ("f16dev", "auto", "tm"),
                              ("f16dev", "one", "tm"), ("f64", "auto", "tm"), ("f32x2", "auto", "tm"),
                              ("f32x2", "two", "tm"), ("f32", "auto", "te"), ("f64", "auto", "te")):
            key = fp + {"auto": "", "one": "_one_step_per_launch", "two": "_two_steps_per_launch",
                        "three": "_three_steps_per_launch"}[mode]
            key += "_te" if pol == "te" else ""
            P = "TE" if pol == "te" else "TM"
            kern = {("f32", "auto"): f"k_step3_tma<false, {P}> (three steps per launch, TMA-staged tiles)",
                    ("f32", "two"): f"k_step2_tma<false, {P}> (two steps per launch, TMA-staged tiles)",
                    ("f32", "one"): f"k_step<float, false, {P}>", ("f16dev", "one"): "k_step_f16<false>",
                    ("f32", "three"): f"k_step3_tma<false, {P}> (three steps per launch, TMA-staged tiles)",
                    ("f16dev", "auto"): "k_step2_f16_tma<false> (two steps per launch, TMA-staged tiles)",
                    ("f64", "auto"): f"k_step<double, false, {P}>",
                    ("f32x2", "auto"): f"k_step<df, false, {P}> (double-float)",
                    ("f32x2", "two"): f"k_step2<df, false, {P}> (double-float, two steps per launch)"}[(fp, mode)]
            with L.solver_for_instance(big, fp, main, steps_per_launch=mode, polarization=pol) as s:
                s.step(4)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                n = 15 if "three steps" in kern else 16  # whole launches only
                a.record(main)
                s.step(n)
                b.record(main)
                b.synchronize()
                us = a.elapsed_time(b) * 1e3 / n
                sites = big["nx"] * big["ny"]
                gbs = sites * BYTES_PER_LU[fp] / (us / 1e6) / 1e9
                hs[key] = {"kernel": kern, "us_per_step": round(us, 2),
                          "glups": round(sites / (us / 1e6) / 1e9, 2), "achieved_gbs": round(gbs, 1),
                          "frac_hbm": round(gbs / peak, 4), "bytes_per_lu": BYTES_PER_LU[fp]}
                if "two steps per launch" in kern:
                    # the state crosses HBM once per two steps: half the one-pass bytes per update
                    hs[key]["two_step_bytes_per_lu"] = BYTES_PER_LU[fp] / 2
                    hs[key]["two_step_frac_hbm"] = round(gbs / 2 / peak, 4)
                if "three steps per launch" in kern:
                    hs[key]["three_step_bytes_per_lu"] = round(BYTES_PER_LU[fp] / 3, 2)
                    hs[key]["three_step_frac_hbm"] = round(gbs / 3 / peak, 4)
                if fp == "f64":
                    ops = FP64_OPS_PER_LU + (1 if pol == "te" else 0)   # TE: 29 per update
                    hs[key]["fp64_ops_per_lu"] = ops
                    t_ops = sites * ops / (us / 1e6) / 1e12
                    hs[key]["fp64_tops"] = round(t_ops, 4)
                    hs[key]["frac_fp64_pipe"] = round(t_ops / (SMS * FP64_OPS_PER_CLK_PER_SM * sm_mhz * 1e6 / 1e12), 4)
        out["single_domain_8192"] = hs

    if not args.no_design_map and rank == 0:
        # batched design diagram: seeded dielectric Janus instances, uneven sizes
        # (a in {16, 32, 64}, grid 16 a) and run lengths (20 periods of T = 3 a),
        # one persistent kernel under a CUDA graph; FP32 lattice, FP64 accumulation,
        # force error against the same batch in FP64
        dm = W.design_map_256(4, args.design_map_instances)
        res = {}
        for fp in ("f32", "f32x2", "f64"):
            bt = L.Batch(dm, fp, stream=main)
            if fp == "f32":            # untimed first run (graph capture, first touch)
                bt.run()
                bt.results()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(main)
            bt.run()
            b.record(main)
            b.synchronize()
            F, _ = bt.results()
            res[fp] = (a.elapsed_time(b), F, bt.config())
            bt.close()
        ms32, F32, cfg = res["f32"]
        ms64, F64, _ = res["f64"]
        msx2, FX2, _ = res["f32x2"]
        errs = np.max(np.abs(F32 - F64), axis=1) / np.abs(F64[:, 0])
        lus = sum(instance_lus(i) for i in dm)
        out["design_map"] = {"instances": len(dm), "cells_per_s": round(len(dm) / (ms32 / 1e3), 2),
                             "mlups": round(lus / (ms32 / 1e3) / 1e6, 1), "ms": round(ms32, 1),
                             "fp64_cells_per_s": round(len(dm) / (ms64 / 1e3), 2),
                             "fp64_mlups": round(lus / (ms64 / 1e3) / 1e6, 1), "fp64_ms": round(ms64, 1),
                             "f32x2_cells_per_s": round(len(dm) / (msx2 / 1e3), 2),
                             "f32x2_max_force_err_drag_scale":
                                 float((np.max(np.abs(FX2 - F64), axis=1) / np.abs(F64[:, 0])).max()),
                             "max_force_err_drag_scale": float(errs.max()),
                             "instances_within_1e-3": int(np.sum(errs <= 1e-3)),
                             "tile_w": cfg[0], "tile_h": cfg[1], "ctas_per_sm": cfg[2],
                             "precision": "f32 lattice, f64 accumulation; error against the same batch in f64"}

    if not args.no_cpu_baseline and rank == 0 and world == 1:
        out["cpu_baseline"] = cpu_baseline(instances[0], args.cpu_seconds)

    for s in solvers:
        s.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
