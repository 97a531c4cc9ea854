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


@pytest.mark.parametrize("tau,H", [(1.0, 8), (0.8, 6)])
def test_free_slip_half_channel_is_half_of_the_no_slip_channel(tau, H):
    """No-slip wall below the first layer, free-slip wall above the last: a
    specular wall is a mirror plane, so the steady profile is the lower half
    of the Poiseuille channel of height 2H, u(z) = g/(2 nu) (z + 1/2)(2H - 1/2 - z),
    which the TRT scheme with half-way bounce-back reproduces exactly."""
    g = 1e-6
    wl = _box((1, 1, H), (1, 1, 0), tau=tau, accel=(g, 0.0, 0.0))
    wl.wall_slip = (0, 0, 0, 0, 0, 1)
    o = oracle.Oracle(wl)
    o.map_particles()
    nu = (tau - 0.5) / 3.0
    z = np.arange(H) + 0.0
    exact = g / (2.0 * nu) * (z + 0.5) * (2 * H - 0.5 - z)
    steps = int(40 * (2 * H) ** 2 / nu) + 2000
    for _ in range(steps):
        o.lbm_step()
    u = o.field(oracle.FIELD_U)[0, :, 0, 0]
    assert np.max(np.abs(u / exact - 1.0)) < 1e-10
    np.testing.assert_allclose(o.field(oracle.FIELD_U)[1:], 0.0, atol=1e-15)


def _momentum(f, c):
    return np.array([f.sum()] + [np.tensordot(c[:, a].astype(float), f, axes=(0, 0)).sum() for a in range(3)])


@pytest.mark.parametrize("slip", [(0, 0, 0, 0, 1, 1), (1, 1, 0, 0, 1, 1)])
def test_free_slip_walls_conserve_tangential_momentum(slip):
    """A free-slip wall reverses only the normal component of a population's
    velocity, so the total mass and the total momentum along every axis that
    has no wall are invariant; at an edge of two free-slip walls a
    population reflects off both.  A uniform flow plus random populations,
    no forcing, no spheres.  With no-slip walls the same momentum decays (the test sees the
    difference)."""
    dims = (8, 6, 10)
    per = tuple(0 if slip[2 * a] else 1 for a in range(3))
    rng = np.random.Generator(np.random.PCG64(17))
    c, w = oracle.lattice()
    cu = (c.astype(float) @ np.array([0.02, -0.015, 0.01]))[:, None, None, None]
    f = w[:, None, None, None] * (1.0 + 3.0 * cu + 0.05 * rng.standard_normal((19, dims[2], dims[1], dims[0])))
    out = {}
    for kind in ("slip", "noslip"):
        wl = _box(dims, per, tau=0.9)
        wl.wall_slip = slip if kind == "slip" else (0,) * 6
        o = oracle.Oracle(wl)
        o.set_field(oracle.FIELD_PDF, f)
        o.map_particles()
        m0 = _momentum(o.field(oracle.FIELD_PDF), c)
        for _ in range(30):
            o.lbm_step()
        out[kind] = (m0, _momentum(o.field(oracle.FIELD_PDF), c))
    m0, m1 = out["slip"]
    free = [1 + a for a in range(3) if per[a]]
    scale = np.abs(f).sum()
    assert abs(m1[0] - m0[0]) < 1e-14 * scale
    for k in free:
        assert abs(m1[k] - m0[k]) < 1e-14 * scale
        assert abs(m0[k]) > 1e-4 * scale  # the random state carries momentum there
    m0n, m1n = out["noslip"]
    assert max(abs(m1n[k] - m0n[k]) for k in free) > 1e-3 * max(abs(m0n[k]) for k in free)


@pytest.mark.parametrize("slip", [(0, 0, 0, 0, 1, 1), (1, 1, 0, 0, 1, 1)])
def test_free_slip_walls_are_mirror_planes(slip):
    """A state that is uniform across the free-slip walls and has no velocity
    normal to them is its own mirror image, so the walls act like periodic
    faces: the run matches the fully periodic run cell by cell.  The flow
    varies along the walls, which checks that a reflected population comes
    from the tangentially displaced cell (and, with two free-slip walls,
    that a population reflected at the edge comes back from the cell
    itself)."""
    dims = (12, 10, 6)
    walls = [a for a in range(3) if slip[2 * a]]
    c, w = oracle.lattice()
    X, Y, Z = np.meshgrid(*[np.arange(n) + 0.5 for n in dims], indexing="ij")
    k = [2.0 * np.pi / n for n in dims]
    u = np.zeros((3,) + X.shape)
    rho = 1.0 + 0.01 * np.cos(k[1] * Y)
    if 0 in walls:  # uniform in x and z, flow along y only
        u[1] = 0.01 * np.sin(k[1] * Y)
    else:
        u[0] = 0.01 * np.sin(k[1] * Y)
        u[1] = 0.008 * np.cos(k[0] * X)
        rho = rho + 0.01 * np.sin(k[0] * X)
    f = _equilibrium(c, w, rho, u).transpose(0, 3, 2, 1)  # (q, z, y, x)
    res = {}
    for kind in ("slip", "periodic"):
        per = tuple(0 if (kind == "slip" and a in walls) else 1 for a in range(3))
        wl = _box(dims, per, tau=0.7)
        wl.wall_slip = slip if kind == "slip" else (0,) * 6
        o = oracle.Oracle(wl)
        o.set_field(oracle.FIELD_PDF, f)
        o.map_particles()
        for _ in range(25):
            o.lbm_step()
        res[kind] = o.field(oracle.FIELD_PDF)
    assert np.max(np.abs(res["slip"] - res["periodic"])) < 1e-15
    # (bounce-back walls give a different flow)
    assert np.max(np.abs(res["periodic"] - f)) > 1e-5
