"""Pins of the oracle's lattice Boltzmann step (Sec. 4.1) against closed forms
and invariants that the paper and the mathematics fix.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_1708_08741_gb300 import workloads as W


def _box(dims, periodic, tau=1.0, accel=(0.0, 0.0, 0.0), levels=1):
    wl = W.Workload(name="box", dims=list(dims), periodic=periodic, tau=tau, kappa=0.0, eps=1.0,
                    E_ext=(0.0, 0.0, 0.0), accel=accel, levels=levels, coarse_sweeps=1)
    return wl


def _equilibrium(c, w, rho, u):
    """Incompressible equilibrium of Sec. 4.1 written out for the test input."""
    cu = np.einsum("qa,a...->q...", c.astype(float), u)
    uu = (u * u).sum(0)
    return w[:, None, None, None] * (rho + 3.0 * cu + 4.5 * cu ** 2 - 1.5 * uu)


def test_lattice_is_d3q19():
    c, w = oracle.lattice()
    assert c.shape == (19, 3)
    # isotropy conditions of D3Q19 with c_s^2 = 1/3
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(np.einsum("q,qa->a", w, c), 0.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("q,qa,qb->ab", w, c, c), np.eye(3) / 3.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("q,qa,qb,qc->abc", w, c, c, c), 0.0, atol=1e-16)
    # every direction has its opposite
    for q in range(19):
        assert any((c[k] == -c[q]).all() for k in range(19))


def test_rest_state_is_fixed_point():
    o = oracle.Oracle(_box((6, 4, 8), (1, 1, 0)))
    o.map_particles()
    for _ in range(5):
        o.body_force()
        o.lbm_step()
    c, w = oracle.lattice()
    f = o.field(oracle.FIELD_PDF)
    np.testing.assert_allclose(f, np.broadcast_to(w[:, None, None, None], f.shape), rtol=0, atol=1e-16)
    np.testing.assert_array_equal(o.field(oracle.FIELD_U), 0.0)


def test_equilibrium_is_fixed_point_of_collision():
    """A uniform equilibrium state with any velocity is left unchanged by the
    TRT collision (its non-equilibrium parts vanish) and by streaming."""
    dims = (4, 4, 4)
    o = oracle.Oracle(_box(dims, (1, 1, 1), tau=0.73))
    c, w = oracle.lattice()
    u = np.zeros((3,) + dims[::-1])
    u[0], u[1], u[2] = 0.02, -0.013, 0.007
    feq = _equilibrium(c, w, 1.01, u)
    o.set_field(oracle.FIELD_PDF, feq)
    o.map_particles()
    o.body_force()
    o.lbm_step()
    np.testing.assert_allclose(o.field(oracle.FIELD_PDF), feq, rtol=0, atol=2e-16)


@pytest.mark.parametrize("tau", [1.0, 0.7, 1.9])
def test_collision_moments_single_cell(tau):
    """On a 1x1x1 periodic lattice streaming maps each population onto itself,
    so one step is one collision.  Mass is conserved and the momentum grows
    by exactly the body force f_b (Sec. 4.1: momentum density defined with
    the forcing term, Eq. modified_velocity)."""
    rng = np.random.Generator(np.random.PCG64(7))
    c, w = oracle.lattice()
    fb = np.array([3e-3, -2e-3, 1e-3])
    o = oracle.Oracle(_box((1, 1, 1), (1, 1, 1), tau=tau, accel=tuple(fb)))
    f0 = (w * (1.0 + 0.05 * rng.standard_normal(19))).reshape(19, 1, 1, 1)
    o.set_field(oracle.FIELD_PDF, f0)
    o.map_particles()
    o.body_force()
    o.lbm_step()
    f1 = o.field(oracle.FIELD_PDF).reshape(19)
    f0 = f0.reshape(19)
    assert abs(f1.sum() - f0.sum()) < 1e-15
    np.testing.assert_allclose(c.T @ f1, c.T @ f0 + fb, rtol=0, atol=2e-16)


def test_mass_conservation_walls_sphere_forcing():
    """Bounce-back at resting walls and at a resting sphere, collision and the
    forcing term all conserve mass exactly: sum over fluid cells of all
    populations is invariant to round-off."""
    wl = W.single_sphere(n=16, radius=3.0, zeta=0.5, debye=3.0, E=5e-3, levels=1)
    wl.periodic = (1, 1, 0)
    wl.accel = (1e-4, 2e-5, 0.0)
    o = oracle.Oracle(wl)
    rng = np.random.Generator(np.random.PCG64(3))
    c, w = oracle.lattice()
    f = w[:, None, None, None] * (1.0 + 0.01 * rng.standard_normal((19, 16, 16, 16)))
    o.set_field(oracle.FIELD_PDF, f)
    o.map_particles()
    fluid = o.owner() < 0
    m0 = o.field(oracle.FIELD_PDF)[:, fluid].sum()
    for _ in range(10):
        o.solve(forced_cycles=2)
        o.body_force()
        o.lbm_step()
    m1 = o.field(oracle.FIELD_PDF)[:, fluid].sum()
    assert abs(m1 - m0) / m0 < 1e-13


@pytest.mark.parametrize("tau,H", [(1.0, 16), (0.8, 12), (1.7, 10)])
def test_poiseuille_exact_with_half_way_walls(tau, H):
    """Body-force-driven channel between resting no-slip walls half-way outside
    the first and last layer.  With the TRT odd rate of Sec. 4.1 the walls sit
    exactly half-way (Ginzburg), so the steady profile is the parabola
    u(z) = g/(2 nu) (z + 1/2)(H - 1/2 - z), nu = (tau - 1/2)/3 (Eq. kinVisc)."""
    g = 1e-6
    o = oracle.Oracle(_box((1, 1, H), (1, 1, 0), tau=tau, accel=(g, 0.0, 0.0)))
    o.map_particles()
    nu = (tau - 0.5) / 3.0
    z = np.arange(H) + 0.0
    exact = g / (2.0 * nu) * (z + 0.5) * (H - 0.5 - z)
    steps = int(40 * H * H / nu) + 2000
    for _ in range(steps):
        o.lbm_step()
    u = o.field(oracle.FIELD_U)[0, :, 0, 0]
    assert np.max(np.abs(u / exact - 1.0)) < 1e-10
    np.testing.assert_allclose(o.field(oracle.FIELD_U)[1:], 0.0, atol=1e-15)


def test_shear_wave_decay_sets_viscosity():
    """A periodic shear wave u_x = U sin(k z) decays as exp(-nu k^2 t) in the
    Stokes limit; the decay rate pins nu = (tau - 1/2) c_s^2 (Eq. kinVisc)."""
    L, tau, U = 32, 0.9, 1e-5
    dims = (1, 1, L)
    o = oracle.Oracle(_box(dims, (1, 1, 1), tau=tau))
    c, w = oracle.lattice()
    z = np.arange(L) + 0.5
    k = 2.0 * np.pi / L
    u = np.zeros((3, L, 1, 1))
    u[0, :, 0, 0] = U * np.sin(k * z)
    o.set_field(oracle.FIELD_PDF, _equilibrium(c, w, 1.0, u))
    o.map_particles()
    amps = []
    for t in range(400):
        o.lbm_step()
        if t >= 100:
            ux = o.field(oracle.FIELD_U)[0, :, 0, 0]
            amps.append(2.0 / L * np.sum(ux * np.sin(k * z)))
    rate = -np.polyfit(np.arange(len(amps)), np.log(amps), 1)[0]
    nu = (tau - 0.5) / 3.0
    assert abs(rate / (nu * k * k) - 1.0) < 2e-3
