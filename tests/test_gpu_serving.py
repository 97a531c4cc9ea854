"""Serving on the GPU: a run's result is the same alone and in a mix of runs
that share the device (separate contexts, streams and host threads), and
the MIXED32 server's results match the FP64 server's within 1e-4."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_08741_gb300 import build

    build.build()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _disp(x, wl):
    """Displacement from the request's initial positions (minimum image on
    the periodic axes): absolute coordinates of tens of cells would hide
    errors of a few thousandths of a cell."""
    d = np.asarray(x, dtype=np.float64).reshape(-1, 3) - np.asarray(wl.x, dtype=np.float64).reshape(-1, 3)
    for a in range(3):
        if wl.periodic[a]:
            d[:, a] -= wl.dims[a] * np.round(d[:, a] / wl.dims[a])
    return d


def test_alone_equals_in_the_mix_and_mixed_matches_fp64():
    import paper_1708_08741_gb300 as es
    from paper_1708_08741_gb300 import serving as S

    reqs = S.request_stream(5, rate=200.0, seed=21, edge_range=(32, 56), max_spheres=8)
    # rel_tol = 0: every run takes exactly max_steps, so that runs compare step for step
    kw = dict(check_every=50, rel_tol=0.0, max_steps=300)
    srv = S.gpu_server(es.ES_MIXED32, slots=5, **kw)
    mix = srv.serve(reqs)
    assert srv.peak_resident > 1  # the runs overlapped on the device
    for r in reqs:
        alone = S.gpu_server(es.ES_MIXED32, slots=1, **kw).serve([r])[0]
        m = mix[r.rid]
        assert alone.steps == m.steps == 300
        np.testing.assert_array_equal(alone.v, m.v)
        np.testing.assert_array_equal(alone.x, m.x)
    ref = S.gpu_server(es.ES_FP64, slots=1, **kw).serve(reqs[:3])
    for r, a, b in zip(reqs[:3], ref, mix[:3]):
        assert _rel(b.v, a.v) < 1e-4
        assert _rel(_disp(b.x, r.wl), _disp(a.x, r.wl)) < 1e-4


def test_autotuner_on_the_gpu_picks_a_schedule_that_meets_the_tolerance():
    import paper_1708_08741_gb300 as es
    from paper_1708_08741_gb300 import autotune as A
    from paper_1708_08741_gb300 import workloads as W

    wl = W.suspension_sample(64)
    tuner = A.Autotuner(A.gpu_measure(es.ES_MIXED32, steps=3, warmup=2))
    best = tuner.tune(wl)
    schedule = {k: v for k, v in best.items() if k != "lbm_block"}
    assert schedule in A.candidates(wl)
    assert "lbm_block" in best and {"lbm_block": best["lbm_block"]} in A.block_shapes(wl)
    times = [t for _, t in tuner.log[A.class_key(wl)]]
    assert all(t > 0 for t in times) and min(times) < float("inf")
    sim = es.Simulation(wl, es.ES_MIXED32, overrides=best)
    for _ in range(3):
        info = sim.step()
        assert info["r"] < info["tol"]
    sim.close()


def _runs(precision):
    """Three resident runs of uneven size (a ragged walled box, a periodic
    sphere box, a suspension sample), all without free-slip faces."""
    import paper_1708_08741_gb300 as es
    from paper_1708_08741_gb300 import workloads as W

    return [W.mixed_box(), W.single_sphere(n=32), W.suspension_sample(48, levels=3)]


@pytest.mark.parametrize("prec_name", ["fp64", "mixed32", "mixed16"])
def test_batched_stream_collide_equals_single_runs(prec_name):
    """es_lbm_step_batch steps the stream-collide of several resident runs
    (different grid sizes, walls, spheres) in one launch: every run's
    populations and particles after 5 coupled steps are the same bits as
    when each run steps alone."""
    import paper_1708_08741_gb300 as es

    precision = {"fp64": es.ES_FP64, "mixed32": es.ES_MIXED32, "mixed16": es.ES_MIXED16}[prec_name]
    alone = [es.Simulation(wl, precision) for wl in _runs(precision)]
    batch = [es.Simulation(wl, precision) for wl in _runs(precision)]
    for _ in range(5):
        for g in alone:
            g.step()
        for g in batch:
            g.map_particles()
            g.solve()
        es.lbm_step_batch(batch)
        for g in batch:
            g.forces_device()
            g.advance()
    for a, b in zip(alone, batch):
        np.testing.assert_array_equal(a.field(es.FIELD_PDF), b.field(es.FIELD_PDF))
        np.testing.assert_array_equal(a.particles()["x"], b.particles()["x"])
        a.close()
        b.close()


def test_stream_collide_block_shapes_give_the_same_bits():
    """The stream-collide's block shape (es_params.lbm_block, a tuning knob)
    does not change the result."""
    import paper_1708_08741_gb300 as es
    from paper_1708_08741_gb300 import workloads as W

    out = []
    for shape in ((0, 0), (32, 4), (64, 2), (256, 1)):
        g = es.Simulation(W.mixed_box(), es.ES_MIXED32, overrides=dict(lbm_block=shape))
        for _ in range(3):
            g.step()
        out.append(g.field(es.FIELD_PDF))
        g.close()
    for o in out[1:]:
        np.testing.assert_array_equal(out[0], o)


def test_batch_rejects_mixed_precisions_and_duplicates():
    import paper_1708_08741_gb300 as es
    from paper_1708_08741_gb300 import workloads as W

    a = es.Simulation(W.single_sphere(n=16, radius=3.0, levels=2), es.ES_MIXED32)
    b = es.Simulation(W.single_sphere(n=16, radius=3.0, levels=2), es.ES_FP64)
    for sims in ([a, b], [a, a]):
        with pytest.raises(es.EsError) as e:
            es.lbm_step_batch(sims)
        assert e.value.code == es.ES_EINVAL
    a.close()
    b.close()
