"""The seeded input generator shared by both sides: PCG32 against its
published reference outputs, and the placement rules of the workloads."""
import os

import numpy as np

from paper_1708_08741_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_pcg32_reference_stream():
    with open(os.path.join(GOLDEN, "pcg32_reference.txt")) as f:
        line = [l for l in f if not l.startswith("#")][0]
    expect = [int(t, 16) for t in line.split()]
    rng = W.PCG32(42, 54)
    assert [rng.next_u32() for _ in range(6)] == expect


def test_uniform_and_normal_moments():
    rng = W.PCG32(5)
    u = np.array([rng.uniform() for _ in range(20000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01
    n = np.array([rng.normal() for _ in range(20000)])
    assert abs(n.mean()) < 0.03 and abs(n.std() - 1.0) < 0.03


def _min_gap(wl):
    x = wl.x
    best = np.inf
    for i in range(len(x)):
        d = x - x[i]
        for a in range(3):
            if wl.periodic[a]:
                L = wl.dims[a]
                d[:, a] -= L * np.round(d[:, a] / L)
        r = np.sqrt((d * d).sum(1))
        r[i] = np.inf
        best = min(best, r.min())
    return best


def test_channel_and_suspension_placement():
    wl = W.channel()
    assert wl.n_particles == 64 and np.all(wl.R == 6.0)
    assert _min_gap(wl) >= 2 * 6.0 + 2.0
    assert np.all(wl.x[:, 2] >= 7.0) and np.all(wl.x[:, 2] <= 128 - 7.0)
    assert np.all((wl.q >= 0.5) & (wl.q <= 1.5))
    s = W.suspension_sample(128)
    assert s.n_particles == 45 and _min_gap(s) >= 12.0
    # determinism: same seed, same workload
    s2 = W.suspension_sample(128)
    np.testing.assert_array_equal(s.x, s2.x)
    np.testing.assert_array_equal(s.q, s2.q)


def test_full_suspension_counts():
    wl = W.suspension()
    assert wl.n_particles == 2880 and wl.dims == [512, 512, 512]
    assert _min_gap(wl) >= 12.0
    assert abs(wl.q.mean() - 1.0) < 0.01 and abs(wl.q.std() - 0.1) < 0.01
