"""Serving host logic on the CPU: the request mix, the percentile, the
steady-velocity stop and the continuous-batching scheduler (slots, memory
admission, arrivals joining a running mix), driven by a stand-in simulation
whose particles approach a terminal velocity exponentially."""
import math
import threading
import time

import numpy as np
import pytest

from paper_1708_08741_gb300 import serving as S
from paper_1708_08741_gb300 import workloads as W


def test_request_mix_follows_the_serving_configuration():
    reqs = S.request_stream(48, rate=20.0, seed=5)
    again = S.request_stream(48, rate=20.0, seed=5)
    assert [r.wl.dims for r in reqs] == [r.wl.dims for r in again]
    t = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(t) > 0)
    # Poisson(20/s): mean gap 0.05 s (loose bound for 48 draws)
    assert 0.025 < np.mean(np.diff(t)) < 0.1
    for r in reqs:
        wl = r.wl
        mult = 1 << wl.levels
        assert all(32 <= d <= 192 and d % mult == 0 for d in wl.dims)
        assert 1 <= wl.n_particles <= 200
        R = wl.R[0]
        assert 3.0 <= R <= 8.0 and np.all(wl.R == R)
        solid = wl.n_particles * 4.0 / 3.0 * math.pi * R ** 3 / wl.n_cells
        assert solid <= 0.05 + 1e-12 or wl.n_particles == 1
        assert 2.0 <= 1.0 / wl.kappa <= 8.0
        assert 5e-4 <= wl.E_ext[0] <= 3e-3
        assert np.all((wl.zeta >= 0.5) & (wl.zeta <= 2.0))
        # non-overlapping with the placement gap (minimum image, periodic)
        x = wl.x
        for i in range(len(x)):
            d = x[i + 1:] - x[i]
            for a in range(3):
                L = wl.dims[a]
                d[:, a] -= L * np.round(d[:, a] / L)
            assert np.all(np.linalg.norm(d, axis=1) >= 2 * R + 2 - 1e-9)


def test_percentile_matches_numpy_linear():
    rng = np.random.Generator(np.random.PCG64(1))
    v = rng.random(37)
    for p in (0, 10, 50, 90, 99, 100):
        assert abs(S.percentile(v, p) - np.percentile(v, p)) < 1e-15


class FakeSim:
    """Particles approach v_t = (E, 0, 0) with a time constant set by the
    grid size; each step takes a little wall time, as a GPU step does."""

    live = 0
    peak = 0
    lock = threading.Lock()

    def __init__(self, wl, slot, step_time=2e-5):
        self.wl = wl
        self.t = 0
        self.tau = 20.0 + wl.dims[0] / 8.0
        self.vt = np.array([wl.E_ext[0] * 1e3, 0.0, 0.0])
        self.step_time = step_time
        with FakeSim.lock:
            FakeSim.live += 1
            FakeSim.peak = max(FakeSim.peak, FakeSim.live)

    def step(self):
        self.t += 1
        time.sleep(self.step_time)

    def particles(self):
        v = self.vt * (1.0 - math.exp(-self.t / self.tau))
        n = self.wl.n_particles
        return {"v": np.tile(v, (n, 1)), "x": self.wl.x.copy(), "w": np.zeros((n, 3))}

    def close(self):
        with FakeSim.lock:
            FakeSim.live -= 1


def _expected_steps(tau, check=100, tol=1e-4, cap=20000):
    # first check k where |v(k c) - v((k-1) c)| <= tol |v(k c)|
    k = 1
    while True:
        k += 1
        a, b = 1 - math.exp(-(k - 1) * check / tau), 1 - math.exp(-k * check / tau)
        if abs(b - a) <= tol * abs(b) or k * check >= cap:
            return k * check


def test_run_to_steady_stops_at_the_first_quiet_interval():
    wl = S.request_workload(3)
    sim = FakeSim(wl, 0, step_time=0.0)
    steps, steady, vm, _ = S.run_to_steady(sim)
    assert steady and steps == _expected_steps(sim.tau)
    sim.close()
    sim = FakeSim(wl, 0, step_time=0.0)
    steps, steady, _, _ = S.run_to_steady(sim, max_steps=300)
    assert not steady and steps == 300
    sim.close()


@pytest.mark.parametrize("slots", [1, 3])
def test_scheduler_slots_memory_and_arrivals(slots):
    reqs = S.request_stream(10, rate=200.0, seed=9, edge_range=(32, 64))
    FakeSim.live = FakeSim.peak = 0
    need = {r.rid: r.wl.n_cells * 100 for r in reqs}
    budget = int(2.5 * max(need.values()))
    srv = S.Server(lambda wl, slot: FakeSim(wl, slot), lambda wl: wl.n_cells * 100, slots=slots,
                   budget_bytes=budget, check_every=50, max_steps=2000)
    res = srv.serve(reqs, time_scale=1.0)
    assert [r.rid for r in res] == [r.rid for r in reqs]
    assert srv.peak_resident <= slots and FakeSim.peak <= slots
    assert srv.peak_bytes <= budget
    for r in res:
        assert r.admitted >= r.arrival - 1e-9 and r.finished >= r.admitted
        assert r.steady
    if slots > 1:
        # requests that arrived while others ran were admitted into the mix
        assert srv.peak_resident > 1
    s = S.summarize(res)
    assert s["runs"] == 10 and s["p99_latency_s"] >= s["p50_latency_s"] > 0


def test_scheduler_rejects_a_request_larger_than_the_budget():
    reqs = S.request_stream(2, seed=9, edge_range=(32, 48))
    srv = S.Server(lambda wl, slot: FakeSim(wl, slot), lambda wl: 10 ** 12, slots=2, budget_bytes=10 ** 9)
    with pytest.raises(ValueError):
        srv.serve(reqs)


def test_result_alone_equals_result_in_the_mix_for_a_deterministic_run():
    reqs = S.request_stream(5, rate=500.0, seed=4, edge_range=(32, 48))
    mk = lambda wl, slot: FakeSim(wl, slot, step_time=0.0)  # noqa: E731
    mix = S.Server(mk, lambda wl: 1, slots=5, budget_bytes=10, check_every=50).serve(reqs)
    for r in reqs:
        alone = S.Server(mk, lambda wl: 1, slots=1, budget_bytes=10, check_every=50).serve([r])[0]
        m = mix[r.rid]
        assert alone.steps == m.steps and np.array_equal(alone.v, m.v)


class FakeLockstepSim(FakeSim):
    """FakeSim driven through the calls of one time step, as the lockstep
    server issues them; advance() moves time on.  fail_at: the solve of that
    step raises (a run that fails, e.g. on overlapping spheres)."""

    def __init__(self, wl, slot, fail_at=None):
        super().__init__(wl, slot, step_time=0.0)
        self.fail_at = fail_at
        self.calls = []

    def map_particles(self):
        self.calls.append("map")

    def solve(self):
        if self.fail_at is not None and self.t + 1 == self.fail_at:
            raise RuntimeError("planted failure")
        self.calls.append("solve")

    def forces_device(self):
        self.calls.append("forces")

    def advance(self):
        self.t += 1


@pytest.mark.parametrize("slots", [1, 3])
def test_lockstep_batch_server_matches_the_threaded_server(slots):
    """The lockstep scheduler steps the resident runs together (one batched
    stream-collide per step for all of them), admits by slots and memory as
    runs finish, and gives every run the same steps and result as the
    threaded scheduler."""
    reqs = S.request_stream(10, rate=200.0, seed=9, edge_range=(32, 64))
    FakeSim.live = FakeSim.peak = 0
    budget = int(2.5 * max(r.wl.n_cells * 100 for r in reqs))
    batches = []
    srv = S.BatchServer(lambda wl, slot: FakeLockstepSim(wl, slot), lambda wl: wl.n_cells * 100,
                        lambda sims: batches.append(len(sims)), slots=slots, budget_bytes=budget,
                        check_every=50, max_steps=2000)
    res = srv.serve(reqs)
    ref = S.Server(lambda wl, slot: FakeSim(wl, slot, step_time=0.0), lambda wl: 1, slots=1, budget_bytes=10,
                   check_every=50, max_steps=2000).serve(reqs)
    assert [r.rid for r in res] == [r.rid for r in reqs]
    assert srv.peak_resident <= slots and FakeSim.peak <= slots
    assert max(batches) <= slots and srv.launches == len(batches)
    if slots > 1:
        assert max(batches) > 1  # runs shared a batched launch
    for a, b in zip(res, ref):
        assert a.steps == b.steps and a.steady and np.array_equal(a.v, b.v)
        assert a.finished >= a.admitted >= a.arrival - 1e-9


def test_lockstep_batch_server_reports_a_failed_run_and_serves_the_rest():
    reqs = S.request_stream(4, rate=500.0, seed=4, edge_range=(32, 48))
    bad = reqs[1].rid
    mk = lambda wl, slot: FakeLockstepSim(wl, slot, fail_at=30 if wl is reqs[1].wl else None)  # noqa: E731
    res = S.BatchServer(mk, lambda wl: 1, lambda sims: None, slots=4, budget_bytes=10, check_every=50).serve(reqs)
    assert res[bad].error is not None and "planted failure" in res[bad].error
    assert all(r.error is None and r.steady for r in res if r.rid != bad)
