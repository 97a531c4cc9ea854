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


def test_paper_node_problem():
    """One node's problem of the paper's scaling runs (Sec. 7): 2 x 4 x 2
    blocks of 144^3 cells, each with 64 spheres of radius 6 on a lattice of
    spacing 36 whose first centre is (19, 19, 19), periodic in y only.  With
    the centres on lattice points, the cell-in-sphere rule (cell centre
    within R) takes 912 cells a sphere, 1.955 % of the domain: the paper's
    "about 1.95 %" of obstacle cells (the spheres' volume would be 1.94 %)."""
    wl = W.paper_node()
    assert wl.dims == [288, 576, 288] and tuple(wl.periodic) == (0, 1, 0)
    assert wl.n_particles == 1024 and np.all(wl.R == 6.0) and np.all(wl.kind == W.KIND_ZETA)
    for a in range(3):
        np.testing.assert_array_equal(np.unique(wl.x[:, a]), 19.0 + 36.0 * np.arange(wl.dims[a] // 36))
    blocks, per_block = np.unique((wl.x // 144).astype(int), axis=0, return_counts=True)
    assert len(blocks) == 16 and np.all(per_block == 64)
    assert _min_gap(wl) == 36.0
    # clearance from the x and z walls
    for a in (0, 2):
        assert wl.x[:, a].min() - 6.0 >= 1.0 and wl.dims[a] - (wl.x[:, a].max() + 6.0) >= 1.0
    h = np.arange(-8, 8) + 0.5
    X, Y, Z = np.meshgrid(h, h, h, indexing="ij")
    per_sphere = int((X * X + Y * Y + Z * Z <= 36.0).sum())
    assert per_sphere == 912
    assert abs(100.0 * per_sphere * wl.n_particles / wl.n_cells - 1.95) < 0.01
