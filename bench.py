#!/usr/bin/env python
"""Benchmark of the coupled electrophoresis time step on GB300.

One step is Algorithm 1 of the paper on the GPU: particle mapping, the
multigrid Debye-Hueckel solve to the residual tolerance, EDL field and body
force, the fused stream-collide sweep, momentum-exchange forces and the
rigid-body update.  Workload: a 512^3 periodic suspension of 2,880 charged
spheres of radius 5 (the per-GPU weak-scaling shape), MIXED32 form.

Prints one JSON line.  Under torchrun every rank runs an independent replica
on its own GPU (the step has no exchange across GPUs here); the timed region
is bracketed by barriers and the slowest rank's time is used.
"""
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "coupled-step MLUPS & %HBM roofline at 512^3; served runs/s, p99 latency mixed vs FP64"
UNIT = "MLUPS"
# algorithmic bytes per fluid cell of the stream-collide kernel in the MIXED32
# form: 19 FP32 populations read + 19 written, the FP32 potential (the body
# force is formed in the kernel from psi at the cell and, from cache, its
# neighbours), 1 flag byte; obstacle cells only read their flag byte
LBM_BYTES_FLUID = 2 * 19 * 4 + 4 + 1
LBM_BYTES_SOLID = 1


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=512, help="cells per axis")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-form measurement")
    ap.add_argument("--no-channel", action="store_true", help="skip the 128^3 channel measurement")
    ap.add_argument("--e2e-steps", type=int, default=0, help="steps of the host-buffer run (default: --steps)")
    ap.add_argument("--serving", action="store_true",
                    help="serving mode: a stream of independent runs, MIXED32 continuous batching "
                         "against FP64 one run at a time")
    ap.add_argument("--requests", type=int, default=24, help="serving: number of requests")
    ap.add_argument("--slots", type=int, default=8, help="serving: resident runs (MIXED32 server)")
    ap.add_argument("--max-run-steps", type=int, default=1000, help="serving: step cap per run")
    ap.add_argument("--max-edge", type=int, default=96, help="serving: largest grid edge of the request mix")
    ap.add_argument("--no-serving", action="store_true", help="skip the short serving measurement")
    ap.add_argument("--smoother", choices=["fused", "two_pass"], default="two_pass",
                    help="execution of a red-black sweep (same arithmetic)")
    ap.add_argument("--mg-storage", choices=["native", "fp16"], default="native",
                    help="storage of the finest level's multigrid correction")
    ap.add_argument("--fine-layout", choices=["auto", "natural"], default="auto",
                    help="finest-level layout of the multigrid correction and right-hand side")
    ap.add_argument("--staging", choices=["registers", "bulk"], default="registers",
                    help="operand staging of the finest level's half sweep")
    ap.add_argument("--nu", type=int, nargs=2, default=None, metavar=("NU1", "NU2"),
                    help="pre- and post-smoothing sweeps of the V-cycle (default: the workload's 2, 2)")
    ap.add_argument("--lbm-block", type=int, nargs=2, default=(0, 0), metavar=("X", "Y"),
                    help="thread-block shape of the stream-collide (0 0: the library default)")
    return ap.parse_args()


def rank_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def max_over_ranks(value, dist=None, device=None):
    """Largest value over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(cells, steps, world, seconds):
    """Whole-job MLUPS of `world` replicas that each advanced `cells` cells
    by `steps` steps, timed by the slowest rank."""
    return cells * steps * world / seconds / 1e6


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def _oracle_mlups(wl, steps, warmup, omp):
    """MLUPS of the FP64 oracle as it stands on wl: `warmup` untimed steps,
    then `steps` timed ones."""
    import oracle

    o = oracle.Oracle(wl, omp=omp)
    for _ in range(warmup):
        o.step()
    t0 = time.perf_counter()
    for _ in range(steps):
        o.step()
    dt = time.perf_counter() - t0
    return wl.n_cells * steps / dt / 1e6, dt


def cpu_baseline(n=128):
    """The FP64 oracle as it stands (plain C, -O3, no FMA contraction) on the
    host cores, bounded to ~15 s of CPU work:
    * value: the all-core OpenMP build (same source and bits, independent
      cells shared out) on an n^3 sub-box of the suspension (same sphere
      density, radius, charges, Debye length and field), 1 untimed + 5 timed
      steps;
    * single_thread: the serial build on the same sub-box, 1 + 2 steps;
    * c1_full: the 32^3 single-sphere case in full (100 steps), serial."""
    import oracle
    from paper_1708_08741_gb300 import workloads as W

    nproc = os.cpu_count() or 1
    wl = W.suspension_sample(n)
    v_all, dt_all = _oracle_mlups(wl, 5, 1, omp=True)
    v_one, dt_one = _oracle_mlups(wl, 2, 1, omp=False)
    c1 = W.single_sphere()
    v_c1, dt_c1 = _oracle_mlups(c1, 100, 0, omp=False)
    return {"value": v_all, "unit": UNIT, "cores": oracle.threads(True), "kind": "oracle",
            "sample": f"{n}^3 periodic sub-box of the suspension, {wl.n_particles} spheres R=5 (the density of "
                      f"2,880 in 512^3), FP64 C oracle built with OpenMP (all host cores), 5 timed steps after 1 "
                      f"untimed step",
            "seconds": dt_all, "nproc": nproc,
            "single_thread": {"value": v_one, "unit": UNIT, "cores": 1, "seconds": dt_one,
                              "sample": f"the same {n}^3 sub-box, serial build, 2 timed steps after 1 untimed"},
            "c1_full": {"value": v_c1, "unit": UNIT, "cores": 1, "seconds": dt_c1,
                        "sample": "32^3 periodic box, one zeta sphere R=4, 3-level V-cycles to 1e-10, "
                                  "all 100 steps, serial build"}}


def workload_name(n, n_spheres, levels, res_rf):
    """The benchmark workload as both arms name it in `config` (the
    arithmetic form is the line's `dtype`)."""
    return (f"suspension {n}^3 periodic, {n_spheres} charged spheres R=5, lambda_D=4, E=1e-3, "
            f"{levels}-level V(2,2) to RES_RF {res_rf:g}")


def run_reference(args):
    """The oracle as it stands, on the host cores (OpenMP build), each step
    one oracle step of an n^3 sub-box of the suspension; rank 0 only."""
    rank, _, world = rank_info()
    if rank != 0:
        return
    import oracle
    from paper_1708_08741_gb300 import workloads as W

    n = 128 if (args.steps + args.warmup) <= 24 else 64
    wl = W.suspension_sample(n)
    value, dt = _oracle_mlups(wl, args.steps, args.warmup, omp=True)
    cores = oracle.threads(True)
    full = W.suspension(n=args.n, n_spheres=int(round(2880 * (args.n / 512) ** 3)),
                        levels=6 if args.n % 32 == 0 else 4)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.n, full.n_particles, full.levels, full.res_rf),
                   "cells": full.n_cells, "parallelism": f"host cores x{cores}",
                   "sample": f"{n}^3 periodic sub-box, {wl.n_particles} spheres R=5 (the same density)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"each step one oracle step of the {n}^3 sub-box (OpenMP build, all host cores)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    import paper_1708_08741_gb300 as es
    from paper_1708_08741_gb300 import workloads as W

    rank, local, world = rank_info()
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if dist is not None:
            dist.barrier()

    wl = W.suspension(n=args.n, n_spheres=int(round(2880 * (args.n / 512) ** 3)),
                      levels=6 if args.n % 32 == 0 else 4)
    smoother = es.ES_SMOOTH_FUSED if args.smoother == "fused" else es.ES_SMOOTH_TWO_PASS
    mg = es.ES_MG_FP16 if args.mg_storage == "fp16" else es.ES_MG_NATIVE
    lay = es.ES_LAYOUT_NATURAL if args.fine_layout == "natural" else es.ES_LAYOUT_AUTO
    sim = es.Simulation(wl, es.ES_MIXED32, device=str(dev),
                        overrides=dict(smoother=smoother, mg_storage=mg, fine_layout=lay,
                                       lbm_block=tuple(args.lbm_block),
                                       **({"nu1": args.nu[0], "nu2": args.nu[1]} if args.nu else {}),
                                       sweep_staging=1 if args.staging == "bulk" else 0))
    stream = sim.stream
    N = wl.n_cells

    for _ in range(max(args.warmup, 0)):
        sim.step()
    torch.cuda.synchronize(dev)
    barrier()
    torch.cuda.synchronize(dev)

    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    start, stop = ev(), ev()
    lbm_ev = [(ev(), ev()) for _ in range(args.steps)]
    phase_ev = [[ev() for _ in range(5)] for _ in range(args.steps)]
    cycles = []
    start_ratio = []  # residual norm at the start of each solve / tolerance
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = sim.kernel_launches()
    # timed region 1: the steps themselves (a handful of phase events per
    # step, no per-kernel instrumentation)
    with torch.cuda.stream(stream):
        start.record(stream)
        for k in range(args.steps):
            pe = phase_ev[k]
            pe[0].record(stream)
            sim.map_particles()
            pe[1].record(stream)
            info = sim.solve()
            cycles.append(info["cycles"])
            start_ratio.append(info["r0"] / info["tol"] if info["tol"] > 0 else 0.0)
            pe[2].record(stream)
            lbm_ev[k][0].record(stream)
            sim.lbm_step()
            lbm_ev[k][1].record(stream)
            pe[3].record(stream)
            sim.forces_device()
            sim.advance()
            pe[4].record(stream)
        stop.record(stream)
    torch.cuda.synchronize(dev)
    launches = sim.kernel_launches() - launches0
    barrier()
    torch.cuda.synchronize(dev)
    # timed region 2: the same number of further steps with every grid-sized
    # launch bracketed by CUDA events on the library's stream (per-kernel
    # durations for the roofline; the event records cost host time, which
    # is why the step time comes from region 1)
    sim.profile_start()
    pcycles = 0
    for k in range(args.steps):
        pcycles += sim.step()["cycles"]
    prof = sim.profile_stop()
    barrier()
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    t = start.elapsed_time(stop) / 1e3
    t_all = max_over_ranks(t, dist, dev)
    lbm_ms = statistics.mean(a.elapsed_time(b) for a, b in lbm_ev)
    phases = {name: statistics.mean(pe[i].elapsed_time(pe[i + 1]) for pe in phase_ev)
              for i, name in enumerate(["map", "solve_and_body_force", "lbm", "forces_advance"])}
    vcycles = sum(cycles)

    own = torch.empty(N, dtype=torch.int32, device=dev)
    sim.field_device(es.FIELD_OWNER, own)
    n_solid = int((own >= 0).sum().item())
    del own
    n_fluid = N - n_solid
    lbm_bytes = LBM_BYTES_FLUID * n_fluid + LBM_BYTES_SOLID * n_solid
    peak, peak_kind = measured_peaks()
    kernels = kernel_table(prof, lbm_bytes, peak)
    top = kernels[0]

    # end to end through the C ABI with host buffers: the particle state comes
    # in from host memory each step and the new state and forces go back
    e2e_steps = args.e2e_steps or args.steps
    parts = es.pack_particles(wl.x, wl.v, wl.w, wl.R, wl.kind, wl.zeta, wl.q)
    sim.lib.es_get_particles(sim.h, parts, wl.n_particles)
    F = np.zeros(3 * wl.n_particles)
    T = np.zeros(3 * wl.n_particles)
    info_c = es.SolveInfo()
    torch.cuda.synchronize(dev)
    barrier()
    t0 = time.perf_counter()
    e2e_cycles = 0
    for _ in range(e2e_steps):
        sim._check(sim.lib.es_set_particles(sim.h, parts, wl.n_particles), "es_set_particles")
        sim._check(sim.lib.es_map_particles(sim.h), "es_map_particles")
        sim._check(sim.lib.es_potential_solve(sim.h, -1, info_c), "es_potential_solve")
        e2e_cycles += info_c.cycles
        sim._check(sim.lib.es_lbm_step(sim.h), "es_lbm_step")
        sim._check(sim.lib.es_forces(sim.h, F.ctypes.data, T.ctypes.data, 0), "es_forces")
        sim._check(sim.lib.es_advance(sim.h), "es_advance")
        sim._check(sim.lib.es_get_particles(sim.h, parts, wl.n_particles), "es_get_particles")
    torch.cuda.synchronize(dev)
    t_e2e = max_over_ranks(time.perf_counter() - t0, dist, dev)
    psize = ctypes_sizeof_particle(es)
    h2d = wl.n_particles * psize
    d2h = wl.n_particles * (psize + 48)

    levels = sim.params.levels
    sim.close()
    del sim
    torch.cuda.synchronize(dev)
    fp64 = None
    if not args.no_fp64:
        fp64 = measure_fp64(args, dev, barrier)
    chan = None if args.no_channel else measure_channel(dev)
    serv = None
    if rank == 0 and world == 1 and not args.no_serving:
        serv = serving_measure(12, 8, 600, (32, 64), str(dev))
    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline()
    if rank != 0:
        return
    value = aggregate_throughput(N, args.steps, world, t_all)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_all / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(args.n, wl.n_particles, levels, wl.res_rf)
                               + (", FP16 finest-level correction" if mg == es.ES_MG_FP16 else ""),
                   "cells": N, "fluid_cells": n_fluid, "parallelism": f"replicas x{world}",
                   "l2_policy": "inputs larger than L2 (PDF fields 20 GB)"},
        "mflups": n_fluid * args.steps * world / t_all / 1e6,
        "vcycles_per_step": vcycles / args.steps,
        **vcycle_stats(prof, pcycles),
        "start_residual_over_tol": sorted(round(x, 1) for x in start_ratio),
        "phases_ms": phases,
        "roofline": {"kernel": top["kernel"], "bound": "hbm", "achieved": top["gbs"], "peak": peak,
                     "unit": "GB/s", "frac": top["frac"], "traffic": TRAFFIC.get(top["kernel"]),
                     "peak_source": peak_kind, "bytes_per_launch": top["bytes_per_launch"],
                     "ms_per_launch": top["ms_per_launch"], "launches": top["launches"],
                     "share_of_timed_kernels": top["share"]},
        "kernels": kernels,
        "lbm_step_ms": lbm_ms,
        "e2e": {"value": aggregate_throughput(N, e2e_steps, world, t_e2e), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * t_e2e / e2e_steps,
                "vcycles_per_step": e2e_cycles / e2e_steps},
        "gpu_launches": launches,
        "clocks": clk,
        "cpu_baseline": base,
        "fp64_form": fp64,
        "channel128": chan,
        "serving": serv,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# kernels that can lead the table, from one ncu capture of each kernel in its
# current form, by kernel key; a kernel missing here has no capture of its
# current code (traffic null).
# (ncu --set full of the 320^3 workload, scaled to 512^3 by the cell count)
TRAFFIC = {"smooth_half L0": 194.1e6 * 4.096, "lbm": 5220.8e6 * 4.096}


def kernel_table(prof, lbm_bytes, peak):
    """Per kernel and level, from the library's event timing over the timed
    steps: launches, mean device time, algorithmic bytes per launch, achieved
    GB/s and its fraction of the measured peak, share of the kernel time;
    sorted by total time.  The stream-collide's bytes count fluid cells only
    (obstacle cells move their flag byte), hence lbm_bytes from the caller."""
    rows = []
    total = sum(r["ms"] for r in prof) or 1.0
    for r in prof:
        n = max(r["launches"], 1)
        b = lbm_bytes if r["name"] == "lbm" else r["bytes"] / n
        ms = r["ms"] / n
        gbs = b / (ms / 1e3) / 1e9 if ms > 0 else 0.0
        key = r["name"] if r["level"] < 0 else f"{r['name']} L{r['level']}"
        rows.append({"kernel": key, "launches": r["launches"], "ms_per_launch": ms, "bytes_per_launch": b,
                     "gbs": gbs, "frac": gbs / peak, "share": r["ms"] / total})
    rows.sort(key=lambda x: -x["share"])
    return rows


# kernels that make up a V-cycle (per level)
VCYCLE_KERNELS = ("smooth_half", "smooth_near", "smooth_fused", "restrict", "prolong", "coarse_solve")
# floating-point operations of the stream-collide per interior fluid cell,
# counted from k_lbm with an FMA as two: moments 45, modified velocity, u.u,
# u.f and constants 23, rest population 10, nine TRT pairs with Luo forcing
# 264 (axis pairs 28 each, diagonal pairs 30)
LBM_FLOPS = 342


def vcycle_stats(prof, cycles):
    """Device time of one V-cycle (all levels) from the per-kernel event
    timing of a region that ran `cycles` V-cycles."""
    ms = sum(r["ms"] for r in prof if r["name"] in VCYCLE_KERNELS)
    if cycles <= 0 or ms <= 0:
        return {"vcycle_ms": None, "vcycles_per_s": None}
    v = ms / cycles
    return {"vcycle_ms": v, "vcycles_per_s": 1e3 / v, "vcycle_kernel_ms_total": ms, "vcycles_profiled": cycles}


def measure_fp64(args, dev, barrier):
    """The FP64 form on the same workload: step time, V-cycle time, and the
    stream-collide against the measured FP64 FMA peak (the form is bound by
    GB300's FP64 pipe, not by HBM)."""
    import torch

    import paper_1708_08741_gb300 as es
    from paper_1708_08741_gb300 import workloads as W

    wl = W.suspension(n=args.n, n_spheres=int(round(2880 * (args.n / 512) ** 3)),
                      levels=6 if args.n % 32 == 0 else 4)
    peak = es.alu_peak(es.ES_FP64)
    sim = es.Simulation(wl, es.ES_FP64, device=str(dev))
    for _ in range(2):
        sim.step()
    torch.cuda.synchronize(dev)
    barrier()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    a, b = ev(), ev()
    steps = 3
    cyc = 0
    with torch.cuda.stream(sim.stream):
        a.record(sim.stream)
        for _ in range(steps):
            cyc += sim.step()["cycles"]
        b.record(sim.stream)
    torch.cuda.synchronize(dev)
    t = a.elapsed_time(b) / 1e3
    sim.profile_start()
    pc = 0
    for _ in range(2):
        pc += sim.step()["cycles"]
    prof = sim.profile_stop()
    own = torch.empty(wl.n_cells, dtype=torch.int32, device=dev)
    sim.field_device(es.FIELD_OWNER, own)
    n_fluid = int((own < 0).sum().item())
    del own
    sim.close()
    lbm = [r for r in prof if r["name"] == "lbm"][0]
    lbm_ms = lbm["ms"] / max(lbm["launches"], 1)
    achieved = LBM_FLOPS * n_fluid / (lbm_ms / 1e3) / 1e9
    top = sorted(prof, key=lambda r: -r["ms"])[:6]
    return {"ms_per_step": t / steps * 1e3, "mlups": wl.n_cells * steps / t / 1e6, "steps": steps,
            "vcycles_per_step": cyc / steps, **vcycle_stats(prof, pc),
            "roofline": {"kernel": "lbm", "bound": "alu", "achieved": achieved, "peak": peak, "unit": "GFLOP/s",
                         "frac": achieved / peak, "flops_per_fluid_cell": LBM_FLOPS, "ms_per_launch": lbm_ms,
                         "peak_source": "es_alu_peak FP64 FMA probe, CUDA events"},
            "top_kernels_ms": {(r["name"] if r["level"] < 0 else f"{r['name']} L{r['level']}"):
                               r["ms"] / max(r["launches"], 1) for r in top}}


def measure_channel(dev, steps=20, warmup=3):
    """The channel configuration at its own size (128^3, walls at the z
    faces, 64 charged spheres R=6, lambda_D=3, E=2e-3, 4-level V-cycles to
    1e-8) in the FP64 and MIXED32 forms: ms per step and MLUPS with CUDA
    events over `steps` steps after `warmup`."""
    import torch

    import paper_1708_08741_gb300 as es
    from paper_1708_08741_gb300 import workloads as W

    out = {}
    for prec, name in ((es.ES_FP64, "fp64"), (es.ES_MIXED32, "mixed32")):
        wl = W.channel()
        sim = es.Simulation(wl, prec, device=str(dev))
        for _ in range(warmup):
            sim.step()
        ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
        a, b = ev(), ev()
        cyc = 0
        torch.cuda.synchronize(dev)
        with torch.cuda.stream(sim.stream):
            a.record(sim.stream)
            for _ in range(steps):
                cyc += sim.step()["cycles"]
            b.record(sim.stream)
        torch.cuda.synchronize(dev)
        t = a.elapsed_time(b) / 1e3
        sim.close()
        out[name] = {"ms_per_step": t / steps * 1e3, "mlups": wl.n_cells * steps / t / 1e6,
                     "vcycles_per_step": cyc / steps, "steps": steps}
    return out


def ctypes_sizeof_particle(es):
    import ctypes

    return ctypes.sizeof(es.Particle)


def serving_measure(n_requests, slots, max_steps, edge_range, device, seed=5):
    """One seeded request stream (Poisson arrivals at 20/s, grid edges
    log-uniform in edge_range per axis, 1-200 spheres of radius 3-8, Debye
    length 2-8, field 5e-4..3e-3, zeta 0.5-2, periodic; a run ends when its
    mean particle velocity changes by < 1e-4 relative per 100 steps, or at
    the step cap) served four ways, so that batching and precision are seen
    apart: MIXED32 with `slots` runs resident (each on its own host thread
    and stream), MIXED32 with `slots` runs stepped in lockstep and their
    stream-collides batched into one launch, MIXED32 one run at a time, and
    FP64 one run at a time.  Accuracy: every server's final mean particle
    velocities against FP64's."""
    from paper_1708_08741_gb300 import serving as S

    reqs = S.request_stream(n_requests, rate=20.0, seed=seed, edge_range=edge_range)
    kw = dict(check_every=100, rel_tol=1e-4, max_steps=max_steps)
    import paper_1708_08741_gb300 as es

    servers = {
        f"mixed32_{slots}_slots": S.gpu_server(es.ES_MIXED32, slots=slots, device=device, **kw),
        f"mixed32_{slots}_slots_batched": S.gpu_batch_server(es.ES_MIXED32, slots=slots, device=device, **kw),
        "mixed32_1_slot": S.gpu_server(es.ES_MIXED32, slots=1, device=device, **kw),
        "fp64_1_slot": S.gpu_server(es.ES_FP64, slots=1, device=device, **kw),
    }
    results = {name: srv.serve(reqs) for name, srv in servers.items()}
    ref = results["fp64_1_slot"]
    out = {}
    for name, res in results.items():
        summ = S.summarize(res)
        errs = []
        for a, b in zip(res, ref):
            if a.steps == b.steps and a.error is None and b.error is None:
                errs.append(float(np.linalg.norm(a.v_mean - b.v_mean) / max(np.linalg.norm(b.v_mean), 1e-300)))
        summ["v_mean_rel_err_vs_fp64"] = {"median": float(np.median(errs)) if errs else None,
                                          "max": max(errs) if errs else None, "compared_runs": len(errs)}
        summ["peak_resident"] = servers[name].peak_resident
        out[name] = summ
    base = out["fp64_1_slot"]
    for name, summ in out.items():
        summ["runs_per_s_over_fp64"] = summ["runs_per_s"] / base["runs_per_s"]
        summ["p99_fp64_over_this"] = base["p99_latency_s"] / summ["p99_latency_s"]
    return {"config": {"requests": n_requests, "rate_per_s": 20.0, "grid_edges": list(edge_range),
                       "spheres": "1-200, R 3-8 (<= 5 % solid)", "lambda_D": "2-8", "E": "5e-4..3e-3",
                       "zeta": "0.5-2", "steady": "1e-4 per 100 steps", "step_cap": max_steps, "res_rf": 1e-8,
                       "seed": seed},
            "servers": out}


def run_serving(args):
    """Serving mode: one JSON line with the four servers of serving_measure."""
    import torch

    rank, local, world = rank_info()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    m = serving_measure(args.requests, args.slots, args.max_run_steps, (32, args.max_edge), f"cuda:{local}")
    best = m["servers"][f"mixed32_{args.slots}_slots"]
    line = {
        "metric": "served runs/s and p50/p99 time to steady velocity, MIXED32 continuous batching vs FP64 "
                  "one run at a time",
        "value": best["runs_per_s"], "unit": "runs/s", "higher_is_better": True, "n_gpus": 1,
        "data": "synthetic", **m,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.serving:
        run_serving(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
