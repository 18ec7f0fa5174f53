#!/usr/bin/env python
"""Throughput of the FETD-PIC particle step on GB300: particle-steps/s.

One step = Faraday update (+ per-triangle field record), the fused
gather / push / walk / deposit particle kernel, the Ampere update (C^T H b - i
and the SPAI SpMV) and, every K steps (K autotuned), the counting sort by
triangle.

Workload (default): magnetized electron-positron pair plasma on a 200,978-
triangle jittered Delaunay mesh with PEC walls, 20 particles per species per
triangle (8.04 M), 2-D Maxwell-Juttner momenta kT/mc^2 = 0.1, omega_c/omega_p
= 0.5, Vay pusher.  The headline runs the FP32 path (cell-local barycentric
positions); the plain FP64 path runs the same workload beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 (one rank per GPU; started through torch.distributed.run, which
bench.py does itself when launched without it) every rank advances its own
replica (weak scaling), or, for the batched form, its share of the 64
instances split by estimated cost (strong scaling); no collective is on the
data path, the time is the max over ranks and the value counts all ranks'
particle-steps.  The headline is the median of 5 timed repeats of K steps.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (gather+push+walk+deposit), FP32/batched vs FP64 plain"
UNIT = "particle-steps/s"
CPU_SAMPLE = 250_000          # oracle particles per host process, in both CPU legs
FP64_FLOP_PER_PARTICLE = 243.6  # FP64 flops per particle-step of the plain FP64 kernel (ncu count)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="pair", choices=["pair", "beam", "batched", "cyclotron"],
                    help="pair: 200k-triangle pair plasma (default); beam: 1M-triangle high-gamma beam; "
                         "batched: 64 uneven pair plasmas in one launch; cyclotron: 64 electrons")
    ap.add_argument("--side", type=int, default=317, help="jittered grid side (about 2 side^2 triangles)")
    ap.add_argument("--ppc", type=int, default=20, help="particles per species per triangle")
    ap.add_argument("--pusher", default=None)
    ap.add_argument("--sort-interval", type=int, default=16)
    ap.add_argument("--fp64-steps", type=int, default=0, help="0 = min(steps, 100)")
    ap.add_argument("--e2e-steps", type=int, default=0, help="0 = min(steps, 10)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=CPU_SAMPLE,
                    help="particles of the oracle's sample per host process")
    ap.add_argument("--cpu-procs", type=int, default=0, help="oracle processes (0 = every host core)")
    ap.add_argument("--repeats", type=int, default=5, help="timed repeats of K steps (median reported)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched and high-gamma beam workloads of the default line")
    ap.add_argument("--variant", type=int, default=0, help="FP32 particle-kernel variant (0 = autotuned)")
    ap.add_argument("--no-tune", action="store_true", help="keep the library defaults instead of autotuning")
    ap.add_argument("--dry-ranks", action="store_true", help=argparse.SUPPRESS)
    a = ap.parse_args()
    a.pusher_given = a.pusher is not None
    if a.pusher is None:
        a.pusher = "vay"
    return a


def workload(args):
    """The seeded workload(s): a list of instances (one for all but the batched form)."""
    from paper_1707_04333_gb300 import inputs
    if args.workload == "beam":
        if not args.pusher_given:
            args.pusher = "hc"
        return [inputs.high_gamma_beam(707, 50_000_000, seed=4, pusher=args.pusher)]
    if args.workload == "batched":
        return inputs.batched_pair_plasmas(n_inst=64, seed=5)
    if args.workload == "cyclotron":
        args.pusher = args.pusher if args.pusher_given else "boris"
        return [inputs.cyclotron(gamma=2.0, n=64, nx=32, seed=1, pusher=args.pusher)]
    return [inputs.pair_plasma(args.side, args.ppc, kT=0.1, wc_over_wp=0.5, seed=2, pusher=args.pusher)]


def describe(ws, args, precision):
    nf = sum(len(w.mesh.triangles) for w in ws)
    npart = sum(w.n_particles for w in ws)
    if args.workload == "beam":
        return (f"high-gamma beam {nf} triangles, {npart} electrons, gamma log-uniform [10, 1000], "
                f"E_x = 0.5 c B_z, {args.pusher}, {precision}")
    if args.workload == "batched":
        return (f"batched pair plasmas: {len(ws)} instances, {nf} triangles, {npart} particles in one launch "
                f"per stage, {args.pusher}, {precision}")
    if args.workload == "cyclotron":
        return f"cyclotron {nf} triangles, {npart} electrons, gamma 2, B_z 1 T, {args.pusher}, {precision}, graphs"
    return (f"pair-plasma {nf} triangles, {npart} particles (e+p, {args.ppc}/species/triangle), "
            f"{args.pusher}, {precision}")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id):
        self.dev = device_id
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.06)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons, n = [], [], set(), 0
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            n += 1
            for nm, v in zip(names[1:], f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": n}


def host_cpu():
    """CPU model, architecture and the cores this process may run on."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"model": model or platform.processor() or "unknown", "arch": platform.machine(), "cores": cores}


def _oracle_worker(job):
    """One host process: the FP64 oracle as it stands (single-threaded) on one seeded particle
    sample, full steps (Faraday, particles, Ampere with the level-2 SPAI) on the full mesh.
    Returns (particles, seconds, steps); with target_s one calibration step sets the step count
    for about target_s seconds."""
    nodes, tris, dt, b0, e0, ext, species, pusher, warmup, steps, target_s = job
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from oracle import oracle
    from paper_1707_04333_gb300 import inputs
    sim = oracle.OracleSim(nodes, tris, dt, eps0=inputs.EPS0, mu0=inputs.MU0, c=inputs.C_LIGHT, spai_level=2,
                           b0=b0, e0=e0, ext=ext)
    n = 0
    for q, m, x, u, hint in species:
        sim.load(q, m, x, u, hint)
        n += len(x)
    for _ in range(warmup):
        sim.step(pusher)
    if target_s:
        t0 = time.perf_counter()
        sim.step(pusher)
        steps = int(max(2, min(200, target_s / max(time.perf_counter() - t0, 1e-3))))
    t0 = time.perf_counter()
    for _ in range(steps):
        sim.step(pusher)
    return n, time.perf_counter() - t0, steps


def cpu_oracle(w, sample, steps, warmup=0, procs=1, target_s=None, seed=5):
    """Time the oracle on `procs` host processes at once (spawned, so no GPU state is inherited),
    each on its own seeded sample of `sample` particles (split over the species) with the full mesh
    and field update.  Returns (rate, particles, seconds, steps): all processes' particle-steps per
    second of the slowest process's step time; one process gives the single-core rate."""
    from oracle import oracle
    oracle.build()
    rng = np.random.default_rng(seed)
    per = max(1, sample // len(w.species))
    jobs = []
    for _ in range(max(1, procs)):
        sp = []
        for s in w.species:
            idx = np.sort(rng.choice(len(s.x), min(per, len(s.x)), replace=False))
            sp.append((s.q, s.m, s.x[idx], s.u[idx], s.hint[idx]))
        jobs.append((w.mesh.nodes, w.mesh.triangles, w.dt, w.b0, w.e0, w.ext, sp, w.pusher, warmup, steps,
                     target_s))
    if len(jobs) == 1:
        res = [_oracle_worker(jobs[0])]
    else:
        with mp.get_context("spawn").Pool(len(jobs)) as pool:
            res = pool.map(_oracle_worker, jobs)
    n = sum(r[0] for r in res)
    per_step = max(r[1] / r[2] for r in res)
    nsteps = min(r[2] for r in res)
    return n / per_step, n, per_step * nsteps, nsteps


def cpu_baseline_record(w, args, steps=0, warmup=0, target_s=None):
    """The oracle on every host core (one process per core) and on one core, same sample size per
    process in both; the all-core figure is the value."""
    host = host_cpu()
    procs = args.cpu_procs or host["cores"]
    v1, n1, t1, s1 = cpu_oracle(w, args.cpu_sample, steps, warmup=warmup, procs=1, target_s=target_s)
    va, na, ta, sa = cpu_oracle(w, args.cpu_sample, steps, warmup=warmup, procs=procs, target_s=target_s)
    return {"value": va, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": (f"{procs} host processes (one per core), each the single-threaded oracle on its own seeded "
                       f"sample of {args.cpu_sample} of the {w.n_particles} particles, full "
                       f"{len(w.mesh.triangles)}-triangle mesh and field update, {sa} steps"),
            "single_core": {"value": v1, "particles": n1, "steps": s1, "seconds": t1},
            "cpu": host}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    ws = workload(args)
    w = max(ws, key=lambda x: x.n_particles)
    cpu = cpu_baseline_record(w, args, steps=args.steps, warmup=args.warmup)
    val = cpu["value"]
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * args.cpu_sample * cpu["cores"] / val,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": describe(ws, args, "fp64 CPU oracle"),
                                        "sample_particles_per_process": args.cpu_sample},
        "cpu_baseline": cpu,
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def launcher_argv(argv, n, port):
    """Command that runs this benchmark as n local ranks, one per GPU (torch.distributed.run)."""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
            "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__), *argv]


def _free_port():
    import socket
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def dry_ranks(args):
    """--dry-ranks: the multi-rank host path without a GPU (gloo): the batched form's instances
    split over the ranks by estimated cost, the end-of-run reductions, one JSON line from rank 0."""
    import torch.distributed as dist
    from paper_1707_04333_gb300 import inputs, ranks
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        dist.init_process_group("gloo")
    ws = inputs.batched_pair_plasmas(n_inst=64, seed=5, scale=0.02)
    costs = [ranks.instance_cost(x.n_particles, len(x.mesh.triangles)) for x in ws]
    mine = ranks.shard_instances(costs, world)[rank]
    units = ranks.sum_over_ranks(sum(ws[i].n_particles for i in mine))
    slowest = ranks.max_over_ranks(float(rank + 1))
    count = ranks.sum_over_ranks(len(mine))
    if rank == 0:
        print(json.dumps({"dry_ranks": True, "n_gpus": world, "instances": int(count),
                          "particles": int(units), "max_over_ranks": slowest}), flush=True)
    if world > 1:
        dist.destroy_process_group()


TRAFFIC_SUMMARY = os.path.join(ROOT, "profiles", "k_particles32_pair200k_traffic.json")


def kernel_label(variant):
    """Name of the FP32 particle kernel a variant launches (0 = the library's default, which takes
    two particles per thread; the hybrids 17, 18, 21 and 22 switch kernels a few steps after a sort)."""
    two = variant == 0 or variant >= 8
    hybrids = {17: (12, 6, 14), 18: (12, 4, 14), 21: (19, 6, 14), 22: (19, 6, 20)}
    if variant in hybrids:
        early, steps, late = hybrids[variant]
        return (f"k_particles32x2 (gather+push+walk+deposit, variant {variant}: variant {early} for the first "
                f"{steps} steps after a sort, then variant {late})")
    return (f"{'k_particles32x2' if two else 'k_particles32'} (gather+push+walk+deposit, "
            f"variant {variant if variant else 'default'})")


def measured_traffic(workload, pbytes, variant=None):
    """DRAM bytes (read + write) of one particle-kernel launch from the committed ncu summary, or
    None when the summary is for another workload or kernel variant, or the kernel's sources
    changed since the capture (their SHA-256 is stored with the figure)."""
    import hashlib
    try:
        with open(TRAFFIC_SUMMARY) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None, "no ncu summary"
    if t.get("workload_flag") != workload or t.get("bytes_per_launch") != pbytes:
        return None, "ncu summary is for another workload"
    if variant is not None and t.get("variant") != variant:
        return None, f"ncu summary is for variant {t.get('variant')}, the run used variant {variant}"
    h = hashlib.sha256()
    for rel in t["sources"]:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    if h.hexdigest() != t["source_sha256"]:
        return None, "kernel sources changed since the ncu capture"
    return t["dram_bytes_per_launch"], f"ncu, one launch (variant {t['variant']}): {os.path.relpath(TRAFFIC_SUMMARY, ROOT)}"


def timed_steps(fetdpic, sim, steps, warmup, pusher, stream, barrier, repeats=1):
    """Warm-up, then `repeats` timed regions of exactly `steps` steps, each bracketed by a barrier
    and a device synchronisation, timed with CUDA events on the context stream.  Returns the ms
    of each region."""
    import torch
    sim.step(warmup, pusher).sync()
    out = []
    for _ in range(repeats):
        barrier()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        fetdpic.fetdpic_step(sim.h, steps, pusher)
        ev1.record(stream)
        fetdpic.fetdpic_sync(sim.h)
        torch.cuda.synchronize()
        barrier()
        out.append(ev0.elapsed_time(ev1))
    return out


def workload_line(fetdpic, ws, args, stream, barrier, name, steps, warmup, cache):
    """Headline-style numbers of one more workload form: FP32 graph replay (median of 3), the
    particle kernel's event-timed share and HBM fraction, and the plain FP64 path beside it."""
    from paper_1707_04333_gb300 import ranks
    pusher = args.pusher
    sim = fetdpic.Simulation(ws, precision="fp32", spai_level=2, sort_interval=args.sort_interval,
                             stream=stream, use_graphs=True)
    sim.load()
    tuned = sim.autotune(pusher, trial_steps=32, cache=cache)
    ms = statistics.median(timed_steps(fetdpic, sim, steps, warmup, pusher, stream, barrier, repeats=3))
    pbytes, npart = fetdpic.fetdpic_particle_bytes(sim.h)
    sim.close()
    st_sim = fetdpic.Simulation(ws, precision="fp32", spai_level=2, sort_interval=tuned[1], stream=stream,
                                kernel_variant=tuned[0], time_stages=True)
    st_sim.load()
    timed_steps(fetdpic, st_sim, steps, warmup, pusher, stream, barrier)
    st, _ = fetdpic.fetdpic_stage_times(st_sim.h)
    st_sim.close()
    part_ms = st[1] / max(st[3], 1)
    peak, _ = peaks()
    k64 = min(steps, 20)
    sim64 = fetdpic.Simulation(ws, precision="fp64", spai_level=2, sort_interval=tuned[1], stream=stream,
                               time_stages=True)
    sim64.load()
    ms64 = timed_steps(fetdpic, sim64, k64, min(warmup, 3), pusher, stream, barrier)[0]
    st64, _ = fetdpic.fetdpic_stage_times(sim64.h)
    sim64.close()
    value = ranks.aggregate_rate(npart, steps, ms)
    v64 = ranks.aggregate_rate(npart, k64, ms64)
    return {"workload": describe(ws, argparse.Namespace(**{**vars(args), "workload": name}), "fp32"),
            "value": value, "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
            "particles": npart, "triangles": sum(len(w.mesh.triangles) for w in ws), "instances": len(ws),
            "tuning": {"kernel_variant": tuned[0], "sort_interval": tuned[1]},
            "particle_kernel": {"ms": part_ms, "achieved_gbs": pbytes / (part_ms / 1e3) / 1e9 if part_ms > 0 else None,
                                "frac_of_measured_hbm": pbytes / (part_ms / 1e3) / 1e9 / peak if part_ms > 0 else None},
            "stages_ms_per_step": {"faraday_ms": st[0] / max(st[3], 1), "particles_ms": part_ms,
                                   "ampere_ms": st[2] / max(st[3], 1), "sort_ms_per_step": st[4] / max(st[3], 1)},
            "fp64_plain": {"value": v64, "ms_per_step": ms64 / k64, "particles_ms": st64[1] / max(st64[3], 1),
                           "speedup_fp32_over_fp64": value / v64}}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # one process per GPU: start the ranks ourselves
        sys.exit(subprocess.call(launcher_argv(sys.argv[1:], args.gpus, _free_port())))
    if args.dry_ranks:
        dry_ranks(args)
        return
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_1707_04333_gb300 import build_lib, fetdpic
    if rank == 0:
        build_lib.build()
    barrier()
    build_lib.build()

    from paper_1707_04333_gb300 import ranks
    ws = workload(args)
    sharded = args.workload == "batched" and world > 1
    if sharded:
        # independent instances: split them over the ranks by estimated cost (no exchange per step)
        costs = [ranks.instance_cost(x.n_particles, len(x.mesh.triangles)) for x in ws]
        ws = [ws[i] for i in ranks.shard_instances(costs, world)[rank]]
    w = max(ws, key=lambda x: x.n_particles)     # the instance the CPU baseline samples
    stream = torch.cuda.Stream()          # explicit stream: the context's kernels and the timing events
    cache = os.path.join(ROOT, "paper_1707_04333_gb300", "_build", "tuning.json")

    dev_id = local
    try:
        dev_id = str(torch.cuda.get_device_properties(local).uuid)
        if not dev_id.startswith("GPU-"):
            dev_id = "GPU-" + dev_id
    except Exception:
        pass
    clocks = ClockSampler(dev_id)

    # ---- headline: FP32 path, steps replayed from captured graphs, median of the repeats
    sim = fetdpic.Simulation(ws, precision="fp32", spai_level=2, sort_interval=args.sort_interval, stream=stream,
                             kernel_variant=args.variant, use_graphs=True)
    sim.load()
    if args.variant == 0 and not args.no_tune:
        tuned = sim.autotune(args.pusher, trial_steps=32, cache=cache)
    else:
        tuned = (args.variant, args.sort_interval)
    fetdpic.fetdpic_stage_times(sim.h)                # launch counts start here
    clocks.start()
    reps = timed_steps(fetdpic, sim, args.steps, args.warmup, args.pusher, stream, barrier, repeats=args.repeats)
    clk = clocks.stop()
    _, launches = fetdpic.fetdpic_stage_times(sim.h)
    launches_per_region = launches * args.steps // max(1, args.steps * args.repeats + args.warmup)
    reps = [ranks.max_over_ranks(x, device="cuda") for x in reps]
    ms = statistics.median(reps)
    pbytes, npart = fetdpic.fetdpic_particle_bytes(sim.h)
    npart_all = ranks.sum_over_ranks(npart, device="cuda")
    K = args.steps
    value = ranks.aggregate_rate(npart_all, K, ms)
    # ---- the same workload and tuning with CUDA events between stages (breakdown, roofline)
    ks = min(args.steps, 500)
    sim_st = fetdpic.Simulation(ws, precision="fp32", spai_level=2, sort_interval=tuned[1], stream=stream,
                                kernel_variant=tuned[0], time_stages=True)
    sim_st.load()
    ms_st = timed_steps(fetdpic, sim_st, ks, args.warmup, args.pusher, stream, barrier)[0]
    st, _ = fetdpic.fetdpic_stage_times(sim_st.h)
    sim_st.close()
    part_ms = st[1] / max(st[3], 1) if st[3] > 0 else 0.0
    peak, peak_kind = peaks()
    achieved = pbytes / (part_ms / 1e3) / 1e9 if part_ms > 0 else None
    traffic, traffic_note = measured_traffic(args.workload, pbytes, tuned[0])
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "traffic": traffic,
                "kernel": kernel_label(tuned[0]), "peak_kind": peak_kind,
                "bytes_per_launch": pbytes, "traffic_source": traffic_note}
    stages = {"faraday_ms": st[0] / max(st[3], 1), "particles_ms": part_ms,
              "ampere_ms": st[2] / max(st[3], 1), "sort_ms_per_step": st[4] / max(st[3], 1),
              "run": f"{ks} plain-launch steps with CUDA events between stages, "
                     f"{ms_st / ks:.4f} ms per step (the headline replays captured graphs)"}

    # ---- end to end through the C ABI with page-locked host buffers
    e2e = None
    if not args.no_e2e:
        ke = args.e2e_steps or min(args.steps, 10)
        hx, hu, hc = [], [], []
        for k, (inst, sid, n) in enumerate(sim.species):
            g = sim.read_species(sid)
            hx.append(torch.from_numpy(g["x"]).pin_memory().numpy())
            hu.append(torch.from_numpy(g["u"]).pin_memory().numpy())
            hc.append(torch.from_numpy(g["cell"]).pin_memory().numpy())
        ox = [torch.empty(a.shape, dtype=torch.float64).pin_memory().numpy() for a in hx]
        ou = [torch.empty(a.shape, dtype=torch.float64).pin_memory().numpy() for a in hu]
        oc = [torch.empty(a.shape, dtype=torch.int32).pin_memory().numpy() for a in hc]
        L = fetdpic.lib()
        P = fetdpic._ptr
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # every step: write both species from page-locked host buffers, step, read both species
        # back asynchronously (the device-to-host copy of one step's result overlaps the
        # host-to-device copy of the next step's input); one fetdpic_sync at the end waits for all
        for _ in range(ke):
            for k, (inst, sid, n) in enumerate(sim.species):
                rc = L.fetdpic_write_particles(sim.h, sid, P(hx[k]), P(hu[k]), P(hc[k]))
                assert rc == 0, rc
            fetdpic.fetdpic_step(sim.h, 1, args.pusher)
            for k, (inst, sid, n) in enumerate(sim.species):
                rc = L.fetdpic_read_particles_async(sim.h, sid, P(ox[k]), P(ou[k]), P(oc[k]))
                assert rc == 0, rc
        rc = L.fetdpic_sync(sim.h)
        assert rc == 0, rc
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        te = ranks.max_over_ranks(te, device="cuda")
        e2e = {"value": ranks.aggregate_rate(npart_all, ke, te * 1e3), "unit": UNIT, "h2d_bytes_per_step": int(npart * 36),
               "d2h_bytes_per_step": int(npart * 36), "steps": ke,
               "how": "per step: fetdpic_write_particles of every species from page-locked host buffers, "
                      "fetdpic_step, fetdpic_read_particles_async of every species; one fetdpic_sync "
                      "at the end, inside the timed region"}
    sim.close()
    del sim

    # ---- measured arithmetic peaks (the FP64 path is bound by the FP64 rate)
    arith = None
    if rank == 0 and not args.no_fp64:
        arith = {"fp32_tflops": fetdpic.fetdpic_fma_rate(False), "fp64_tflops": fetdpic.fetdpic_fma_rate(True),
                 "how": "FMA chains filling every SM, CUDA events, best launch of >= 20 ms"}

    # ---- plain FP64 path on the same workload
    fp64 = None
    if not args.no_fp64:
        k64 = args.fp64_steps or min(args.steps, 100)
        sim64 = fetdpic.Simulation(ws, precision="fp64", spai_level=2, sort_interval=tuned[1], stream=stream,
                                   time_stages=True)
        sim64.load()
        ms64 = timed_steps(fetdpic, sim64, k64, min(args.warmup, 3), args.pusher, stream, barrier)[0]
        st64, _ = fetdpic.fetdpic_stage_times(sim64.h)
        pb64, np64 = fetdpic.fetdpic_particle_bytes(sim64.h)
        sim64.close()
        ms64 = ranks.max_over_ranks(ms64, device="cuda")
        v64 = ranks.aggregate_rate(ranks.sum_over_ranks(np64, device="cuda"), k64, ms64)
        p64 = st64[1] / max(st64[3], 1)
        fp64 = {"value": v64, "ms_per_step": ms64 / k64, "steps": k64, "particles_ms": p64,
                "particle_kernel_gbs": pb64 / (p64 / 1e3) / 1e9 if p64 > 0 else None,
                "speedup_fp32_over_fp64": value / v64,
                "note": "the FP64 path is the bit-exact reference: no FMA contraction, IEEE division and "
                        "square root, so part of the speed-up is that choice"}
        if arith and p64 > 0:
            tf = FP64_FLOP_PER_PARTICLE * np64 / (p64 / 1e3) / 1e12
            fp64["particle_kernel_fp64_tflops"] = tf
            fp64["frac_of_measured_fp64"] = tf / arith["fp64_tflops"] if arith["fp64_tflops"] else None

    # ---- the batched (64 uneven instances) and high-gamma beam forms, N = 1 only
    extra = None
    if rank == 0 and world == 1 and not args.no_extra and args.workload == "pair":
        extra = {}
        for name in ("batched", "beam"):
            a2 = argparse.Namespace(**{**vars(args), "workload": name, "pusher_given": False})
            ws2 = workload(a2)
            try:
                extra[name] = workload_line(fetdpic, ws2, a2, stream, barrier, name, args.steps, args.warmup, cache)
            except Exception as ex:          # report, do not lose the headline
                extra[name] = {"error": f"{type(ex).__name__}: {ex}"}
            del ws2

    # ---- CPU oracle baseline (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_record(w, args, steps=0, warmup=0, target_s=12.0)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True,
            "scaling": "strong" if sharded else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": describe(ws, args, "fp32 cell-local barycentric"),
                       "tuning": {"kernel_variant": tuned[0], "sort_interval": tuned[1]},
                       "triangles": sum(len(x.mesh.triangles) for x in ws), "particles_per_gpu": npart,
                       "instances": len(ws),
                       "l2": f"inputs larger than L2 (particle state 2 x {pbytes / 2e6:.0f} MB per step, L2 129 MB)",
                       "parallelism": (f"instances sharded over {world} ranks" if sharded
                                       else f"replicas x{world}")},
            "repeats_ms": reps,
            "roofline": roofline,
            "stages_ms_per_step": stages,
            "fp64_plain": fp64,
            "arith_peaks": arith,
            "workloads": extra,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches_per_region),
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
