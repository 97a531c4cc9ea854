"""The Henry-validation drivers on the GPU against the oracle: the sphere
dragged through a free-slip box by a constant force on top of its
hydrodynamic force (the Stokes half of the validation, Sec. 6.4), and the
electrophoretic sphere itself, on short runs of a 64^3 box."""
import math

import numpy as np
import pytest

import oracle
import paper_1708_08741_gb300 as es
from paper_1708_08741_gb300 import validation as V

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_08741_gb300 import build

    build.build()


def _oracle_dragged(wl, f0, steps, every):
    o = oracle.Oracle(wl, omp=True)
    out = []
    for s in range(1, steps + 1):
        o.map_particles()
        o.solve()
        o.body_force()
        o.lbm_step()
        F, T = o.forces()
        F = F.copy()
        F[0, 0] += f0
        o.set_forces(F, T)
        o.advance()
        if s % every == 0:
            out.append(o.particles()["v"][0, 0])
    return np.array(out)


@pytest.mark.parametrize("precision,tol", [(es.ES_FP64, 1e-12), (es.ES_MIXED32, 1e-4)])
def test_dragged_sphere_against_oracle(precision, tol):
    """64^3 box with free-slip walls on all faces, an uncharged sphere of
    radius 4 (tau = 6, the paper's value) dragged by F_0 = 6 pi mu R U for a
    U near the validation's Henry velocity, 300 steps: the sampled sphere
    velocities of the library's driver match the oracle's."""
    tau, R, n = 6.0, 4.0, 64
    mu = (tau - 0.5) / 3.0
    f0 = 6.0 * math.pi * mu * R * 1e-3
    wl = V._box(n, R, tau, 0.5 / R, 0.0, 0.0, (0.0, 0.0, 0.0), 4, walls=True)
    got = V.dragged_velocity(wl, f0, 300, sample_every=50, precision=precision)
    ref = _oracle_dragged(wl, f0, 300, 50)
    g = np.array(got["U_samples"])
    assert g.shape == ref.shape
    assert np.max(np.abs(g - ref)) <= tol * np.max(np.abs(ref))
    assert ref[-1] > ref[0] > 0.0  # the sphere is still speeding up towards U


def test_electrophoretic_sphere_against_oracle():
    """The electrophoretic half: a zeta = 1 sphere of radius 4, kappa R =
    0.5, E = 2.5e-3 in a free-slip 64^3 box, 200 steps in MIXED32 against the
    oracle: sphere velocity, fluid velocity and potential within 1e-4."""
    from _pair import Pair

    wl = V._box(64, 4.0, 6.0, 0.5 / 4.0, 2.5e-3, 1.0, (0.0, 0.0, 0.0), 4, walls=True)
    p = Pair(wl, es.ES_MIXED32, omp=True)
    for _ in range(200):
        _, ginfo, _, _ = p.step(forced=False)
        assert ginfo["status"] == es.ES_OK
    r = p.compare()
    assert r["owner_equal"]
    for k in ("psi", "u", "v", "disp"):
        assert r[k] < 1e-4, (k, r[k])
    assert p.o.particles()["v"][0, 0] > 0.0  # moving with the field (zeta > 0)
