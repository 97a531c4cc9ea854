"""Autotuner selection logic on the CPU (a stand-in timing function)."""
import math

import pytest

from paper_1708_08741_gb300 import autotune as A
from paper_1708_08741_gb300 import workloads as W


def test_choose_takes_the_fastest_and_skips_failures():
    assert A.choose({0: 3.0, 1: 1.0, 2: math.inf, 3: 1.0}) == 1
    with pytest.raises(ValueError):
        A.choose({0: math.inf})


def test_candidates_offer_the_fused_sweep_only_on_128_wide_grids():
    import paper_1708_08741_gb300 as es

    narrow = A.candidates(W.single_sphere())
    wide = A.candidates(W.mixed_box(dims=(128, 28, 32), periodic=(1, 0, 0)))
    assert {c["smoother"] for c in narrow} == {es.ES_SMOOTH_TWO_PASS}
    assert {c["smoother"] for c in wide} == {es.ES_SMOOTH_TWO_PASS, es.ES_SMOOTH_FUSED}
    assert len(wide) == 2 * len(narrow) == 2 * len(A.DEFAULT_NU)


def test_tuner_caches_per_class_and_treats_failures_as_slow():
    calls = []

    def measure(wl, ov):
        calls.append(ov)
        if ov["nu1"] == 1 and ov["nu2"] == 1:
            raise RuntimeError("did not converge")
        return 1.0 / (ov["nu1"] + ov["nu2"])  # more smoothing is faster here

    t = A.Autotuner(measure, shapes=lambda wl: [])
    wl = W.single_sphere()
    best = t.tune(wl)
    assert (best["nu1"], best["nu2"]) == (3, 3)
    n = len(calls)
    assert t.tune(W.single_sphere()) is best and len(calls) == n  # cached
    assert dict(t.log[A.class_key(wl)][0][0]) == {"nu1": 1, "nu2": 1, "smoother": 0}
    assert t.log[A.class_key(wl)][0][1] == math.inf


def test_tuner_then_times_block_shapes_with_the_chosen_schedule():
    """Stage two: with the fastest schedule fixed, the stream-collide block
    shapes are timed and the fastest kept; the default shape is always a
    candidate and shapes wider than the grid are skipped."""
    seen = []

    def measure(wl, ov):
        seen.append(ov)
        t = 1.0 / (ov["nu1"] + ov["nu2"])
        shape = ov.get("lbm_block", (0, 0))
        return t * (0.5 if shape == (32, 8) else 1.0)

    wl = W.single_sphere()  # nx = 32
    shapes = A.block_shapes(wl)
    assert {tuple(s["lbm_block"]) for s in shapes} == {(0, 0), (32, 8)}
    best = A.Autotuner(measure).tune(wl)
    assert best["lbm_block"] == (32, 8) and (best["nu1"], best["nu2"]) == (3, 3)
    stage2 = [ov for ov in seen if "lbm_block" in ov]
    assert len(stage2) == len(shapes) and all((o["nu1"], o["nu2"]) == (3, 3) for o in stage2)
