"""Serving independent electrophoresis runs on one GPU with continuous batching.

A request is a complete run: a seeded workload (grid, spheres, Debye length,
field) stepped until the mean particle velocity is steady.  The server keeps
a fixed number of slots; a request is admitted as soon as a slot is free and
the device memory the library reports for it (``es_device_bytes``) fits in
the budget next to the runs already resident, so requests that arrive while
others run join them.  Each admitted run lives in its own library context on
its own CUDA stream, driven by its own host thread (the library releases
Python's lock while it waits on the GPU), so the kernels of all resident runs
overlap on the device.  Runs are independent and deterministic, so a run's
result does not depend on what else is resident (tested).

Request mix (the serving configuration): Poisson arrivals; grid edges
log-uniform per axis; 1-200 spheres of one radius in [3, 8] (capped at 5 %
solid volume so that the non-overlapping placement exists); Debye length in
[2, 8]; field in [5e-4, 3e-3] along x; one zeta potential in [0.5, 2] per run
(equal spheres drift together; the method has no collision response, so a
run whose spheres meet stops with ES_EOVERLAP and is reported as failed);
periodic boundaries.  Steady: the mean particle velocity changes by less than
``rel_tol`` of its magnitude over ``check_every`` steps, capped at
``max_steps``.  The potential is solved to RES_RF 1e-8 (the configuration
names none): looser solves leave potential errors of cond(A) x RES_RF, which
at 1e-6 already move particle velocities by ~1e-4 between two correct runs.

The scheduler, admission and statistics are plain Python and take a
simulation factory, so they are tested on the CPU with a stand-in simulation.
"""
from __future__ import annotations

import math
import threading
import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np

from . import workloads as W


@dataclass
class Request:
    rid: int
    arrival: float  # seconds after the start of the stream
    wl: W.Workload


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    steps: int
    steady: bool
    v_mean: np.ndarray
    v: np.ndarray = field(repr=False, default=None)
    x: np.ndarray = field(repr=False, default=None)
    error: Optional[str] = None  # the run stopped with an error (e.g. two spheres overlapped)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def _round_edge(e: float, mult: int, lo: int, hi: int) -> int:
    v = int(round(e / mult)) * mult
    return max(lo, min(hi, v))


def request_workload(rid: int, seed: int = 5, edge_range=(32, 192), max_spheres: int = 200,
                     radius_range=(3.0, 8.0), debye_range=(2.0, 8.0), field_range=(5e-4, 3e-3),
                     zeta_range=(0.5, 2.0), max_solid: float = 0.05, res_rf: float = 1e-8) -> W.Workload:
    """The workload of request ``rid`` (its own PCG32 stream)."""
    rng = W.PCG32(seed, stream=1000 + rid)
    lo, hi = edge_range
    raw = [math.exp(rng.uniform_range(math.log(lo), math.log(hi))) for _ in range(3)]
    levels = 3 if min(raw) < 64 else 4
    mult = 1 << levels  # every extent stays even on the coarsest level
    dims = [_round_edge(e, mult, lo, hi) for e in raw]
    radius = rng.uniform_range(*radius_range)
    n = 1 + int(rng.uniform() * max_spheres)
    vol = dims[0] * dims[1] * dims[2]
    n = max(1, min(n, int(max_solid * vol / (4.0 / 3.0 * math.pi * radius ** 3))))
    debye = rng.uniform_range(*debye_range)
    E = rng.uniform_range(*field_range)
    periodic = (1, 1, 1)
    centres = W.place_spheres(n, radius, dims, periodic, rng)
    zeta = np.full(n, rng.uniform_range(*zeta_range))  # one zeta per run: the spheres keep their spacing
    wl = W.Workload(name=f"req{rid}_{dims[0]}x{dims[1]}x{dims[2]}_{n}xR{radius:.2f}", dims=dims,
                    periodic=periodic, tau=1.0, kappa=1.0 / debye, eps=1.0, E_ext=(E, 0.0, 0.0),
                    levels=levels, res_rf=res_rf, steps=0)
    return W._set_particles(wl, centres, np.full(n, radius), np.full(n, W.KIND_ZETA), zeta, np.zeros(n))


def request_stream(n: int = 256, rate: float = 20.0, seed: int = 5, **kw) -> List[Request]:
    """``n`` requests with Poisson arrivals at ``rate`` per second."""
    rng = W.PCG32(seed, stream=7)
    t = 0.0
    out = []
    for i in range(n):
        t += -math.log(1.0 - rng.uniform()) / rate
        out.append(Request(i, t, request_workload(i, seed=seed, **kw)))
    return out


def percentile(values: Sequence[float], p: float) -> float:
    """Linear-interpolation percentile (p in [0, 100])."""
    v = sorted(values)
    if not v:
        return float("nan")
    k = (len(v) - 1) * p / 100.0
    f = int(math.floor(k))
    c = min(f + 1, len(v) - 1)
    return v[f] + (v[c] - v[f]) * (k - f)


def run_to_steady(sim, check_every: int = 100, rel_tol: float = 1e-4, max_steps: int = 20000):
    """Steps ``sim`` until the mean particle velocity changes by less than
    rel_tol of its magnitude over check_every steps (or max_steps)."""
    steps = 0
    prev = None
    while True:
        for _ in range(check_every):
            sim.step()
        steps += check_every
        p = sim.particles()
        vm = np.mean(p["v"], axis=0)
        if prev is not None:
            if np.linalg.norm(vm - prev) <= rel_tol * max(np.linalg.norm(vm), 1e-300):
                return steps, True, vm, p
        if steps >= max_steps:
            return steps, False, vm, p
        prev = vm


class Server:
    """Continuous-batching scheduler.

    sim_factory(workload, stream_index) -> simulation with step(),
    particles() and close(); bytes_of(workload) -> device bytes of a run.
    """

    def __init__(self, sim_factory: Callable, bytes_of: Callable, slots: int, budget_bytes: int,
                 check_every: int = 100, rel_tol: float = 1e-4, max_steps: int = 20000,
                 clock: Callable[[], float] = time.perf_counter):
        if slots < 1:
            raise ValueError("slots must be >= 1")
        self.sim_factory = sim_factory
        self.bytes_of = bytes_of
        self.slots = slots
        self.budget = budget_bytes
        self.check_every = check_every
        self.rel_tol = rel_tol
        self.max_steps = max_steps
        self.clock = clock
        self.peak_resident = 0
        self.peak_bytes = 0

    def serve(self, requests: Sequence[Request], time_scale: float = 1.0) -> List[Result]:
        """Replays the arrivals (times multiplied by time_scale) and returns
        one Result per request, in request order."""
        for r in requests:
            if self.bytes_of(r.wl) > self.budget:
                raise ValueError(f"request {r.rid} needs more device memory than the budget")
        lock = threading.Condition()
        pending: List[Request] = []
        results: Dict[int, Result] = {}
        state = {"resident": 0, "bytes": 0, "errors": []}
        free_slots = list(range(self.slots))
        t0 = self.clock()

        def worker(req: Request, slot: int, need: int, admitted: float):
            try:
                sim = self.sim_factory(req.wl, slot)
            except Exception as e:  # cannot run at all: reported after the stream
                sim, res = None, None
                with lock:
                    state["errors"].append((req.rid, e))
            if sim is not None:
                try:
                    steps, steady, vm, p = run_to_steady(sim, self.check_every, self.rel_tol, self.max_steps)
                    res = Result(req.rid, req.arrival * time_scale, admitted, self.clock() - t0, steps, steady,
                                 vm, p["v"], p["x"])
                except Exception as e:  # the run itself failed (e.g. overlap): a failed result
                    res = Result(req.rid, req.arrival * time_scale, admitted, self.clock() - t0, -1, False,
                                 np.full(3, np.nan), error=f"{type(e).__name__}: {e}")
                finally:
                    sim.close()
            with lock:
                if res is not None:
                    results[req.rid] = res
                state["resident"] -= 1
                state["bytes"] -= need
                free_slots.append(slot)
                lock.notify_all()

        def admit_ready():
            # first fit in arrival order among the requests that have arrived
            i = 0
            while i < len(pending) and free_slots:
                need = self.bytes_of(pending[i].wl)
                if state["bytes"] + need <= self.budget:
                    req = pending.pop(i)
                    slot = free_slots.pop(0)
                    state["resident"] += 1
                    state["bytes"] += need
                    self.peak_resident = max(self.peak_resident, state["resident"])
                    self.peak_bytes = max(self.peak_bytes, state["bytes"])
                    th = threading.Thread(target=worker, args=(req, slot, need, self.clock() - t0), daemon=True)
                    th.start()
                else:
                    i += 1

        queue = sorted(requests, key=lambda r: r.arrival)
        k = 0
        with lock:
            while k < len(queue) or pending or state["resident"] > 0:
                now = self.clock() - t0
                while k < len(queue) and queue[k].arrival * time_scale <= now:
                    pending.append(queue[k])
                    k += 1
                admit_ready()
                if k < len(queue):
                    wait = queue[k].arrival * time_scale - (self.clock() - t0)
                    if wait > 0:
                        lock.wait(timeout=wait)
                elif pending or state["resident"] > 0:
                    lock.wait(timeout=0.05)
        if state["errors"]:
            rid, e = state["errors"][0]
            raise RuntimeError(f"request {rid} failed: {e}") from e
        return [results[r.rid] for r in requests]


class BatchServer:
    """Continuous batching in lockstep: the resident runs advance one time
    step together, and their stream-collides go to the GPU as one persistent
    launch (es_lbm_step_batch) over a work table of the runs' tiles.  Each
    step: every run's particle mapping (its own stream), every run's
    potential solve (host threads, so that the solves' norm reads overlap),
    one batched stream-collide, every run's forces and rigid-body update;
    every check_every steps of a run its mean particle velocity is compared
    (the steady-state rule of run_to_steady) and a finished run leaves,
    freeing its slot and memory for the requests that wait.

    sim_factory(workload, slot) -> es.Simulation; bytes_of(workload) ->
    device bytes of a run; batch_step(sims) -> one batched stream-collide.
    """

    def __init__(self, sim_factory: Callable, bytes_of: Callable, batch_step: Callable, slots: int,
                 budget_bytes: int, check_every: int = 100, rel_tol: float = 1e-4, max_steps: int = 20000,
                 clock: Callable[[], float] = time.perf_counter):
        if slots < 1:
            raise ValueError("slots must be >= 1")
        self.sim_factory = sim_factory
        self.bytes_of = bytes_of
        self.batch_step = batch_step
        self.slots = slots
        self.budget = budget_bytes
        self.check_every = check_every
        self.rel_tol = rel_tol
        self.max_steps = max_steps
        self.clock = clock
        self.peak_resident = 0
        self.launches = 0  # batched stream-collide launches

    def serve(self, requests: Sequence[Request], time_scale: float = 1.0) -> List[Result]:
        from concurrent.futures import ThreadPoolExecutor

        for r in requests:
            if self.bytes_of(r.wl) > self.budget:
                raise ValueError(f"request {r.rid} needs more device memory than the budget")
        queue = sorted(requests, key=lambda r: r.arrival)
        pending: List[Request] = []
        results: Dict[int, Result] = {}
        resident = []  # dicts: req, sim, slot, need, admitted, steps, prev
        free_slots = list(range(self.slots))
        used = 0
        k = 0
        t0 = self.clock()
        pool = ThreadPoolExecutor(max_workers=self.slots)

        def retire(run, res):
            nonlocal used
            run["sim"].close()
            results[run["req"].rid] = res
            free_slots.append(run["slot"])
            used -= run["need"]
            resident.remove(run)

        def failed(run, e):
            retire(run, Result(run["req"].rid, run["req"].arrival * time_scale, run["admitted"],
                               self.clock() - t0, -1, False, np.full(3, np.nan),
                               error=f"{type(e).__name__}: {e}"))

        try:
            while k < len(queue) or pending or resident:
                now = self.clock() - t0
                while k < len(queue) and queue[k].arrival * time_scale <= now:
                    pending.append(queue[k])
                    k += 1
                i = 0
                while i < len(pending) and free_slots:
                    need = self.bytes_of(pending[i].wl)
                    if used + need <= self.budget:
                        req = pending.pop(i)
                        slot = free_slots.pop(0)
                        sim = self.sim_factory(req.wl, slot)
                        used += need
                        resident.append({"req": req, "sim": sim, "slot": slot, "need": need,
                                         "admitted": self.clock() - t0, "steps": 0, "prev": None})
                        self.peak_resident = max(self.peak_resident, len(resident))
                    else:
                        i += 1
                if not resident:
                    if k < len(queue):
                        time.sleep(max(0.0, queue[k].arrival * time_scale - (self.clock() - t0)))
                    continue
                # one lockstep step of every resident run
                for run in list(resident):
                    try:
                        run["sim"].map_particles()
                    except Exception as e:
                        failed(run, e)
                futs = [(run, pool.submit(run["sim"].solve)) for run in resident]
                for run, f in futs:
                    try:
                        f.result()
                    except Exception as e:
                        failed(run, e)
                if not resident:
                    continue
                self.batch_step([run["sim"] for run in resident])
                self.launches += 1
                for run in list(resident):
                    try:
                        run["sim"].forces_device()
                        run["sim"].advance()
                    except Exception as e:
                        failed(run, e)
                        continue
                    run["steps"] += 1
                    if run["steps"] % self.check_every:
                        continue
                    try:
                        p = run["sim"].particles()
                    except Exception as e:
                        failed(run, e)
                        continue
                    vm = np.mean(p["v"], axis=0)
                    prev = run["prev"]
                    steady = prev is not None and np.linalg.norm(vm - prev) <= self.rel_tol * max(
                        np.linalg.norm(vm), 1e-300)
                    if steady or run["steps"] >= self.max_steps:
                        retire(run, Result(run["req"].rid, run["req"].arrival * time_scale, run["admitted"],
                                           self.clock() - t0, run["steps"], steady, vm, p["v"], p["x"]))
                    else:
                        run["prev"] = vm
        finally:
            pool.shutdown(wait=True)
            for run in list(resident):
                run["sim"].close()
        return [results[r.rid] for r in requests]


def summarize(results: Sequence[Result]) -> dict:
    """runs/s counts the completed runs (failed ones are listed apart)."""
    ok = [r for r in results if r.error is None]
    lat = [r.latency for r in ok]
    makespan = max(r.finished for r in results) - min(r.arrival for r in results)
    return {"runs": len(ok), "failed": len(results) - len(ok),
            "runs_per_s": len(ok) / makespan if makespan > 0 else float("nan"),
            "p50_latency_s": percentile(lat, 50), "p99_latency_s": percentile(lat, 99),
            "makespan_s": makespan, "steady": sum(1 for r in ok if r.steady),
            "steps_total": sum(r.steps for r in ok)}


def gpu_server(precision: int, slots: int, device: str = "cuda:0", budget_fraction: float = 0.8,
               overrides: Optional[dict] = None, tuner=None, **kw) -> Server:
    """A Server whose runs are library contexts on their own CUDA streams.
    With a tuner (autotune.Autotuner), each run takes the smoothing schedule
    chosen for its workload class (tuned once per class, at admission)."""
    import torch

    import paper_1708_08741_gb300 as es

    dev = torch.device(device)
    streams = [torch.cuda.Stream(dev) for _ in range(slots)]
    free, _ = torch.cuda.mem_get_info(dev)
    tune_lock = threading.Lock()

    def factory(wl, slot):
        torch.cuda.set_device(dev)
        ov = dict(overrides or {})
        if tuner is not None:
            with tune_lock:
                ov.update(tuner.tune(wl))
        return es.Simulation(wl, precision, device=device, stream=streams[slot], overrides=ov)

    def bytes_of(wl):
        return es.device_bytes(wl, precision, overrides)

    return Server(factory, bytes_of, slots, int(budget_fraction * free), **kw)


def gpu_batch_server(precision: int, slots: int, device: str = "cuda:0", budget_fraction: float = 0.8,
                     overrides: Optional[dict] = None, tuner=None, **kw) -> BatchServer:
    """A BatchServer of library contexts, each on its own CUDA stream, whose
    stream-collides are launched together (es_lbm_step_batch)."""
    import torch

    import paper_1708_08741_gb300 as es

    dev = torch.device(device)
    streams = [torch.cuda.Stream(dev) for _ in range(slots)]
    free, _ = torch.cuda.mem_get_info(dev)

    def factory(wl, slot):
        torch.cuda.set_device(dev)
        ov = dict(overrides or {})
        if tuner is not None:
            ov.update(tuner.tune(wl))
        return es.Simulation(wl, precision, device=device, stream=streams[slot], overrides=ov)

    def bytes_of(wl):
        return es.device_bytes(wl, precision, overrides)

    return BatchServer(factory, bytes_of, es.lbm_step_batch, slots, int(budget_fraction * free), **kw)
