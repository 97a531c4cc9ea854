"""Autotuner for the multigrid smoothing schedule and the stream-collide's
block shape of a workload.

The V-cycle's pre- and post-smoothing sweep counts (nu1, nu2) and the way a
red-black sweep is executed (two in-place passes, or one fused pass on
levels whose x extent is a multiple of 128) trade cycles per step against
time per cycle.  Every candidate solves to the same tolerance (the
workload's RES_RF), so the fastest candidate per step is chosen at equal
accuracy.  Then, with that schedule, the stream-collide's thread-block
shape (es_params.lbm_block: cells along x by rows along y) is timed: the
best shape depends on the grid's row length and on how much of the
potential's neighbour rows a block finds in its own cache; every shape
gives the same bits.  Each candidate runs ``warmup``
untimed steps and ``steps`` timed steps from the same initial state on the
GPU, timed with CUDA events on the run's stream.  Results are cached per
grid shape, level count and sphere count class, so a server tunes a request
class once.
"""
from __future__ import annotations

import itertools
import math
from typing import Callable, Dict, Iterable, Optional, Sequence, Tuple

DEFAULT_NU = ((1, 1), (2, 1), (1, 2), (2, 2), (3, 3))


def candidates(wl, nus: Sequence[Tuple[int, int]] = DEFAULT_NU) -> list:
    """The schedules worth trying for a workload: every (nu1, nu2) with the
    two-pass sweep, and with the fused sweep where the finest level's x
    extent is a multiple of 128 (the fused kernel's tile)."""
    import paper_1708_08741_gb300 as es

    smoothers = [es.ES_SMOOTH_TWO_PASS]
    if int(wl.dims[0]) % 128 == 0:
        smoothers.append(es.ES_SMOOTH_FUSED)
    return [dict(nu1=a, nu2=b, smoother=s) for (a, b), s in itertools.product(nus, smoothers)]


# stream-collide block shapes (x cells, y rows); (0, 0) is the library default 32 x 4
DEFAULT_SHAPES = ((0, 0), (128, 1), (64, 2), (32, 8))


def block_shapes(wl, shapes: Sequence[Tuple[int, int]] = DEFAULT_SHAPES) -> list:
    """The stream-collide block shapes worth trying for a workload (those no
    wider than its x extent rounded up to a warp, plus the default)."""
    nx = int(wl.dims[0])
    return [dict(lbm_block=tuple(s)) for s in shapes if s == (0, 0) or s[0] <= max(32, ((nx + 31) // 32) * 32)]


def choose(times: Dict[int, float]) -> int:
    """Index of the fastest finite time (ties: the earlier candidate)."""
    best, best_t = None, math.inf
    for i in sorted(times):
        t = times[i]
        if t < best_t:
            best, best_t = i, t
    if best is None:
        raise ValueError("no candidate completed")
    return best


def class_key(wl) -> tuple:
    """Workloads that share a schedule: same level count, cell count within a
    factor of two, sphere count within a factor of two, same fused-sweep
    eligibility."""
    n = wl.n_particles
    return (int(wl.levels), int(round(math.log2(wl.n_cells))), 0 if n == 0 else int(math.log2(n)) + 1,
            int(wl.dims[0]) % 128 == 0)


class Autotuner:
    """Chooses and caches a smoothing schedule per workload class.

    measure(wl, overrides) -> seconds per step (or raises when the candidate
    fails, e.g. does not converge within max_cycles).
    """

    def __init__(self, measure: Callable, cands: Optional[Callable] = None, shapes: Optional[Callable] = None):
        self.measure = measure
        self.cands = cands or candidates
        self.shapes = shapes if shapes is not None else block_shapes
        self.cache: Dict[tuple, dict] = {}
        self.log: Dict[tuple, list] = {}

    def _best(self, wl, cs, log):
        times = {}
        for i, ov in enumerate(cs):
            try:
                times[i] = float(self.measure(wl, ov))
            except Exception:
                times[i] = math.inf
            log.append((cs[i], times[i]))
        return cs[choose(times)]

    def tune(self, wl) -> dict:
        """The schedule first, then (with it) the block shape."""
        key = class_key(wl)
        if key in self.cache:
            return self.cache[key]
        log: list = []
        best = self._best(wl, self.cands(wl), log)
        shapes = self.shapes(wl) if self.shapes else []
        if len(shapes) > 1:
            best = self._best(wl, [{**best, **sh} for sh in shapes], log)
        self.cache[key] = best
        self.log[key] = log
        return best


def gpu_measure(precision: int, steps: int = 8, warmup: int = 4, device: str = "cuda:0") -> Callable:
    """A measure function that times steps of a fresh context per candidate."""
    import torch

    import paper_1708_08741_gb300 as es

    def measure(wl, overrides):
        sim = es.Simulation(wl, precision, device=device, overrides=overrides)
        try:
            for _ in range(warmup):
                sim.step()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            sim.synchronize()
            a.record(sim.stream)
            for _ in range(steps):
                sim.step()
            b.record(sim.stream)
            b.synchronize()
            return a.elapsed_time(b) / 1e3 / steps
        finally:
            sim.close()

    return measure
