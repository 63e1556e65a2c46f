#!/usr/bin/env python
"""Throughput of the DVM Boltzmann step on the GB300.

Metric: phase-space cell updates per second (cells x |V| / s) of one explicit
step (upwind transport over the octree faces, FP64-finished moments,
conservative BGK relaxation), on the Mach-5 sphere flow with ~1.01M kinetic
cells and a 24^3 velocity grid (1.40e10 f values, FP32 storage).  Also
reported: the fraction of the measured HBM roofline reached by the step
kernel, the same metric end to end through the C ABI with host buffers,
the FP64 CPU oracle on the host cores (a bounded sample of the workload),
and the SM clocks seen during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 (torchrun, one process per GPU) every rank steps its own replica of
the workload; the ranks exchange nothing (value = all ranks' updates / the
slowest rank's time).
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "phase-space cell updates/s (cells x |V| / s)"
UNIT = "cell-updates/s"
CPU_SAMPLE_CONFIG = "c3_sphere_m5_small"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", default="c3_sphere_m5")
    ap.add_argument("--precision", choices=["f32", "bf16"], default="f32")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def workload_desc(name, cfg, ncells, nv, prec):
    return ("%s: %dD octree levels %d-%d around a sphere r=%g (%d kinetic cells), %d^3 velocities "
            "on [%g,%g]^3, Mach %.1f inflow, outflow, specular wall, BGK Kn=%g, %s storage"
            % (name, cfg["dim"], cfg["base_level"], cfg["max_level"], cfg["r"], ncells, cfg["n"][0],
               cfg["lo"][0], cfg["hi"][0], cfg["fs_u"][0] / math.sqrt(W.GAMMA), cfg["kn"], prec))


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
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
                rows.append((float(parts[1]), float(parts[2]), parts[5], parts[6], parts[7], parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        smax = max(r[1] for r in rows)
        loaded = [r for r in rows if r[0] > 0.5 * smax] or rows
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            for nm, v in zip(names, r[2:]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------- oracle leg
def oracle_rate(steps, warmup=0, threads=None):
    """FP64 oracle on the 17.7k-cell tree of the same Mach-5 sphere flow with the
    same 24^3 velocity grid: returns (updates/s, cores, sample text, seconds)."""
    import oracle as O
    cores = threads or len(os.sched_getaffinity(0))
    os.environ["OMP_NUM_THREADS"] = str(cores)
    c = W.CONFIGS[CPU_SAMPLE_CONFIG]
    o = O.Problem(O.make_spec(c["dim"], c["base_level"], c["max_level"], c["pred"], c["c"], c["r"],
                              c["beta"], c["solid"], c["bc"]), c["n"], c["lo"], c["hi"])
    o.set_freestream(c["fs_rho"], c["fs_u"], c["fs_T"])
    xyz, _ = o.centres()
    o.init_maxwellian(*W.initial_state(c, xyz))
    dt = o.dt_cfl(c["cfl"])
    if warmup:
        o.step(warmup, dt, O.COLL_BGK, c["kn"])
    t0 = time.perf_counter()
    o.step(steps, dt, O.COLL_BGK, c["kn"])
    el = time.perf_counter() - t0
    cores = O.threads()
    sample = ("%d step(s) of the Mach-5 sphere flow on the %s tree (%d cells x %d velocities, "
              "FP64, BGK), OpenMP over cells" % (steps, CPU_SAMPLE_CONFIG, o.ncells, o.nv))
    return o.ncells * o.nv * steps / el, cores, sample, el


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    rate, cores, sample, el = oracle_rate(args.steps, warmup=args.warmup)
    cfg = W.CONFIGS[args.config]
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_desc(args.config, cfg, -1, cfg["n"][0] ** 3, args.precision),
                   "reference_sample": sample, "parallelism": "host cores"},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our arm
def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _profiled_traffic(kernel_file, key):
    """DRAM bytes per launch from the committed ncu summary, valid only while
    the kernel source is unchanged."""
    src = os.path.join(ROOT, "paper_1503_00707_gb300", "csrc", kernel_file)
    rec = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(rec):
        return None
    d = json.load(open(rec)).get(key)
    if not d:
        return None
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return d["bytes_per_launch"] if d.get("source_sha") == h else None


def run_ours(args):
    import numpy as np
    import torch
    import paper_1503_00707_gb300 as D
    from paper_1503_00707_gb300 import _build

    rank, local, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        _build.build()
    if world > 1:
        torch.distributed.barrier()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, cores, sample, _ = oracle_rate(1)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    cfg = W.CONFIGS[args.config]
    prec = {"f32": D.F32, "bf16": D.BF16}[args.precision]
    stream = torch.cuda.Stream()
    s = D.solver_from_config(cfg, prec, D.COLL_BGK, stream=stream)
    xyz, _ = s.centres()
    s.init_maxwellian(*W.initial_state(cfg, xyz))
    dt = s.dt_cfl(cfg["cfl"])
    ncells, nv = s.ncells, s.nv
    bytes_per_update = {"f32": 8, "bf16": 4}[args.precision]

    s.step(args.warmup, dt)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = D.Solver.launch_count()
    e0.record(stream)
    s.step(args.steps, dt)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = D.Solver.launch_count() - l0
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.barrier()
        ms = float(t.item())
    value = world * ncells * nv * args.steps / (ms / 1e3)
    per_launch_s = ms / 1e3 / args.steps
    peak, peak_kind = _peaks()
    achieved = bytes_per_update * ncells * nv / per_launch_s / 1e9
    key = "k_step_bgk_%s_%s" % (args.config, args.precision)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": _profiled_traffic("k_step.cu", key), "peak_source": peak_kind,
            "algorithmic_bytes_per_update": bytes_per_update}

    # end to end through the C ABI: pinned host f -> device, step, moments -> host
    e2e = None
    if not args.no_e2e:
        fbytes = s.f_bytes()
        avail = 0
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                avail = int(line.split()[1]) * 1024
        if avail > 2.5 * fbytes:
            host = torch.empty(fbytes, dtype=torch.uint8, pin_memory=True)
            s.download_f(host.data_ptr(), fbytes)
            mom = (np.zeros(ncells), np.zeros((ncells, 3)), np.zeros(ncells))
            s.upload_f(host.data_ptr(), fbytes)
            s.step(1, dt)
            s.step_moments(mom)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.e2e_steps):
                s.upload_f(host.data_ptr(), fbytes)
                s.step(1, dt)
                s.step_moments(mom)
            el = time.perf_counter() - t0
            e2e = {"value": world * ncells * nv * args.e2e_steps / el, "unit": UNIT,
                   "h2d_bytes_per_step": fbytes, "d2h_bytes_per_step": ncells * 5 * 8,
                   "steps": args.e2e_steps}
            del host
        else:
            e2e = {"value": None, "unit": UNIT, "h2d_bytes_per_step": fbytes, "d2h_bytes_per_step": ncells * 40,
                   "skipped": "host memory available (%d GB) below 2.5x the f buffer" % (avail >> 30)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_desc(args.config, cfg, ncells, nv, args.precision),
                       "cells": ncells, "velocities": nv, "f_values": ncells * nv,
                       "storage": args.precision, "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (f is %.1f GB)" % (s.f_bytes() / 1e9)},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    s.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
