"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on
the same seeded inputs.  FP64 bar: 1e-12 relative L2; MIXED32 bar: 1e-4
relative L2 on velocity, potential and particle position after 100 steps.
Integer work (the cell-to-sphere mapping) must match exactly."""
import ctypes
import numpy as np
import pytest

import oracle
import paper_1708_08741_gb300 as es
from paper_1708_08741_gb300 import workloads as W

from _pair import Pair, direction_map, rel_l2, to_lib_order, to_oracle_order

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 1e-4
# the quantities every reduced-precision comparison bars: potential (unknown
# cells), velocity (fluid cells), particle displacement, velocity, force and
# torque of the last step
REDUCED_KEYS = ("psi", "u", "disp", "v", "F", "T")


def _assert_reduced(r, bars=None):
    """Every quantity below MIXED_TOL, or below its entry in bars."""
    print("relative L2 against the oracle:", {k: float(r.get(k)) for k in REDUCED_KEYS})
    assert r["owner_equal"]
    for k in REDUCED_KEYS:
        assert r[k] < (bars or {}).get(k, MIXED_TOL), (k, r[k])


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_08741_gb300 import build

    build.build()


def _moving(wl, seed=1, vmax=0.05):
    rng = W.PCG32(seed)
    wl.v = np.array([[rng.uniform_range(-vmax, vmax) for _ in range(3)] for _ in range(wl.n_particles)])
    wl.w = np.array([[rng.uniform_range(-0.01, 0.01) for _ in range(3)] for _ in range(wl.n_particles)])
    return wl


CASES = {
    "single_sphere": lambda: W.single_sphere(),
    "mixed_ragged": lambda: W.mixed_box(),
    "channel64": lambda: _moving(W.channel(n=64, n_spheres=8, radius=5.0, levels=4)),
    "suspension64": lambda: _moving(W.suspension_sample(64, levels=4)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_mapping_and_reconstruction_bit_exact(name):
    wl = CASES[name]()
    p = Pair(wl)
    zero = np.zeros((wl.n_particles, 3))
    for step in range(6):
        p.o.map_particles()
        p.g.map_particles()
        np.testing.assert_array_equal(p.g.field(es.FIELD_OWNER), p.o.owner())
        flags = p.g.field(es.FIELD_FLAGS)
        np.testing.assert_array_equal(flags & 1, (p.o.owner() >= 0).astype(np.uint8))
        # reconstructed PDFs at uncovered cells
        if step > 0:
            fo = p.o.field(oracle.FIELD_PDF)
            fg = to_oracle_order(p.g.field(es.FIELD_PDF))
            fluid = p.o.owner() < 0
            assert np.max(np.abs(fg[:, fluid] - fo[:, fluid])) < 1e-15
        # move the spheres without any fluid update
        p.o.set_forces(zero, zero)
        p.g.set_forces(zero, zero)
        p.o.advance()
        p.g.advance()


@pytest.mark.parametrize("name", sorted(CASES))
def test_potential_solve_and_body_force(name):
    wl = CASES[name]()
    p = Pair(wl)
    p.o.map_particles()
    p.g.map_particles()
    fluid = p.o.owner() < 0
    for k in (0, 1, 2, 3):
        io = p.o.solve(forced_cycles=1 if k else 0)
        ig = p.g.solve(forced_cycles=1 if k else 0)
        assert abs(ig["r0"] - io["r0"]) <= 1e-12 * io["r0"]
        assert rel_l2(p.g.field(es.FIELD_PSI)[fluid], p.o.field(oracle.FIELD_PSI)[fluid]) < FP64_TOL
    # tolerance-driven solve takes the same number of cycles
    io = p.o.solve()
    ig = p.g.solve()
    assert ig["cycles"] == io["cycles"] and ig["r"] < ig["tol"]
    assert rel_l2(p.g.field(es.FIELD_PSI)[fluid], p.o.field(oracle.FIELD_PSI)[fluid]) < FP64_TOL
    p.o.body_force()
    fb_g = p.g.field(es.FIELD_FB)
    fb_o = p.o.field(oracle.FIELD_FB)
    assert rel_l2(fb_g[:, fluid], fb_o[:, fluid]) < FP64_TOL
    assert np.all(fb_g[:, ~fluid] == 0.0)


FUSED_CASES = {
    # 128-wide levels take the fused pass; walls in y and z, 28 rows (the
    # last 12-row tile is ragged), both sphere kinds
    "walls_128x28x32": lambda: W.mixed_box(dims=(128, 28, 32), periodic=(1, 0, 0), levels=3),
    # periodic in all axes, 128^3 and 64^3 levels on the fused pass
    "periodic_128": lambda: W.suspension_sample(128, levels=3),
}


@pytest.mark.parametrize("name", sorted(FUSED_CASES))
def test_fused_smoother(name):
    """The red-black sweep run as one fused out-of-place pass (levels whose
    x extent is a multiple of 128) instead of two in-place passes (one per
    colour): the same V-cycles, so the same iterates as the oracle."""
    wl = FUSED_CASES[name]()
    p = Pair(wl, lib_overrides=dict(smoother=es.ES_SMOOTH_FUSED))
    p.o.map_particles()
    p.g.map_particles()
    fluid = p.o.owner() < 0
    for k in (0, 2):
        io = p.o.solve(forced_cycles=k)
        ig = p.g.solve(forced_cycles=k)
        assert abs(ig["r0"] - io["r0"]) <= 1e-12 * io["r0"]
        assert rel_l2(p.g.field(es.FIELD_PSI)[fluid], p.o.field(oracle.FIELD_PSI)[fluid]) < FP64_TOL


# The solver paths the 512^3 workload takes but small grids do not: levels
# above near_list_cells (default 2^21) smooth their near-boundary cells in
# separate list passes, and grids from fast_update_cells (default 2^21) on
# update the residual after a correction in FP32.  Setting both thresholds to
# one cell forces those paths on 64^3 grids the oracle runs in seconds.
BENCH_PATHS = dict(near_list_cells=1, fast_update_cells=1)
LIST_CASES = {
    "channel64": lambda: _moving(W.channel(n=64, n_spheres=8, radius=5.0, levels=4)),
    "suspension64": lambda: _moving(W.suspension_sample(64, levels=4)),
}


def _profiled_names(g, steps):
    """Kernel records (name, level) -> launches over `steps` coupled steps."""
    g.profile_start()
    for _ in range(steps):
        g.step()
    return {(r["name"], r["level"]): r["launches"] for r in g.profile_stop()}


@pytest.mark.parametrize("name", sorted(LIST_CASES))
def test_list_passes_fp64_forced_cycles(name):
    """FP64 with every level but the coarsest smoothing its near-boundary
    cells from the near-cell list (k_smooth_v's list variant, the list
    shared out to the half-sweep launch's blocks; selected for every level
    above near_list_cells = 1 cell): forced V-cycles against the oracle at
    1e-12, then 10 coupled steps."""
    wl = LIST_CASES[name]()
    p = Pair(wl, lib_overrides=BENCH_PATHS)
    p.o.map_particles()
    p.g.map_particles()
    fluid = p.o.owner() < 0
    for k in (0, 1, 2, 3):
        io = p.o.solve(forced_cycles=1 if k else 0)
        ig = p.g.solve(forced_cycles=1 if k else 0)
        assert abs(ig["r0"] - io["r0"]) <= 1e-12 * io["r0"]
        assert rel_l2(p.g.field(es.FIELD_PSI)[fluid], p.o.field(oracle.FIELD_PSI)[fluid]) < FP64_TOL
    p.o.body_force()
    p.o.lbm_step()
    p.g.lbm_step()
    p.o.forces()
    p.g.forces()
    p.o.advance()
    p.g.advance()
    for _ in range(10):
        info, ginfo, _, _ = p.step()
        assert ginfo["cycles"] == info["cycles"]
    r = p.compare()
    assert r["owner_equal"]
    for k in ("psi", "u", "x", "v", "w"):
        assert r[k] < FP64_TOL, (k, r[k])


@pytest.mark.parametrize("name", sorted(LIST_CASES))
def test_bench_solver_paths_mixed32_after_100_steps(name):
    """MIXED32 with the near-cell list passes on every level and the FP32
    residual update (r - A e after a correction near the tolerance) on: the
    paths of the 512^3 workload, at 64^3, tolerance-driven on both sides,
    against the oracle after 100 steps at 1e-4."""
    wl = LIST_CASES[name]()
    p = Pair(wl, es.ES_MIXED32, lib_overrides=BENCH_PATHS)
    for _ in range(100):
        _, ginfo, _, _ = p.step(forced=False)
        assert ginfo["status"] == es.ES_OK and ginfo["r"] < ginfo["tol"]
    _assert_reduced(p.compare())
    seen = _profiled_names(p.g, 10)
    # solves that start from the carried residual, patched around the spheres
    # and corrected locally around the flipped cells; when a V-cycle still
    # runs, the FP32 update (with psi += e in the same pass) follows it
    assert seen.get(("residual_patch", -1), 0) > 0, "no solve started from a patched residual"
    if seen.get(("smooth_half", 0), 0):
        assert seen.get(("residual_update_correct", -1), 0) > 0, "the FP32 residual update never ran"


@pytest.mark.parametrize("name", sorted(LIST_CASES))
def test_patched_start_and_local_correction(name):
    """A solve that starts from the previous solve's residual -- formed again
    only at the near-boundary cells and around the cells that flipped
    between obstacle and fluid, then lowered by the local correction around
    those cells -- ends at the potential a full start gives (twin run, the
    full start forced by writing psi back unchanged), starts no higher, and
    leaves a carried residual that is the residual of its potential: a
    second solve on the same potential starts from the carried norm, a
    third with the residual formed in full from the same norm."""
    wl = LIST_CASES[name]()
    a = es.Simulation(wl, es.ES_MIXED32, overrides=BENCH_PATHS)
    b = es.Simulation(wl, es.ES_MIXED32, overrides=BENCH_PATHS)
    for _ in range(7):
        a.step()
        b.step()
    # (the twins are in the same state here)
    b.set_field(es.FIELD_PSI, b.field(es.FIELD_PSI))  # (the carried residual is dropped)
    ra, rb = [], []
    for sim, out in ((a, ra), (b, rb)):
        sim.map_particles()
        sim.profile_start()
        out.append(sim.solve())
        out.append({(r["name"], r["level"]) for r in sim.profile_stop()})
    assert ("residual_patch", -1) in ra[1] and ("outer_residual", -1) in rb[1]
    print("start residual: patched and corrected", ra[0]["r0"], "full", rb[0]["r0"], "tol", ra[0]["tol"],
          "cycles", ra[0]["cycles"], rb[0]["cycles"])
    assert ra[0]["r0"] <= rb[0]["r0"] * (1 + 1e-3)
    assert ra[0]["cycles"] <= rb[0]["cycles"]
    pa, pb = a.field(es.FIELD_PSI), b.field(es.FIELD_PSI)
    assert rel_l2(pa, pb) < 1e-5
    again = a.solve()  # nothing changed: the carried residual of the final psi
    a.set_field(es.FIELD_PSI, a.field(es.FIELD_PSI))
    full = a.solve()  # the same psi, residual formed in full
    print("carried", again["r0"], "full", full["r0"], "final", ra[0]["r"])
    # (the final norm comes from the FP32 update, whose rounding, ~1e-6 of the
    # residual before the correction, is ~1 % of a residual at the tolerance;
    # the next start forms the near-boundary cells again in float-float)
    assert again["r0"] == pytest.approx(ra[0]["r"], rel=0.05)
    assert full["r0"] == pytest.approx(again["r0"], rel=0.05)
    a.close()
    b.close()


@pytest.mark.parametrize("precision", [es.ES_MIXED32, es.ES_MIXED16])
@pytest.mark.parametrize("name", ["channel64", "suspension64", "mixed_ragged"])
def test_fused_body_force_equals_the_stored_field(name, precision):
    """The reduced forms evaluate the electric body force inside the
    stream-collide (interior fluid cells, from psi) instead of storing it
    after the solve.  Stepping with that and stepping with the stored field
    (read back, then set) must give the same populations bit for bit, step
    after step, in periodic and walled boxes."""
    sims = [es.Simulation(CASES[name](), precision) for _ in range(2)]
    for _ in range(4):
        for k, g in enumerate(sims):
            g.map_particles()
            g.solve()
            if k == 1:
                g.set_field(es.FIELD_FB, g.field(es.FIELD_FB))
            g.lbm_step()
            g.forces()
            g.advance()
        np.testing.assert_array_equal(sims[0].field(es.FIELD_PDF), sims[1].field(es.FIELD_PDF))
    np.testing.assert_array_equal(sims[0].particles()["x"], sims[1].particles()["x"])
    for g in sims:
        g.close()


@pytest.mark.parametrize("name", sorted(CASES))
def test_lbm_step_forces_and_advance(name):
    wl = CASES[name]()
    p = Pair(wl)
    c, w = oracle.lattice()
    rng = np.random.Generator(np.random.PCG64(5))
    shape = (19,) + tuple(wl.dims[::-1])
    f0 = w[:, None, None, None] * (1.0 + 0.02 * rng.standard_normal(shape))
    fb = 1e-4 * rng.standard_normal((3,) + tuple(wl.dims[::-1]))
    p.o.set_field(oracle.FIELD_PDF, f0)
    p.g.set_field(es.FIELD_PDF, to_lib_order(f0))
    p.o.map_particles()
    p.g.map_particles()
    fluid = p.o.owner() < 0
    fb[:, ~fluid] = 0.0
    p.o.set_field(oracle.FIELD_FB, fb)
    p.g.set_field(es.FIELD_FB, fb)
    p.o.lbm_step()
    p.g.lbm_step()
    fo = p.o.field(oracle.FIELD_PDF)
    fg = to_oracle_order(p.g.field(es.FIELD_PDF))
    assert np.max(np.abs(fg[:, fluid] - fo[:, fluid])) < 1e-15
    assert rel_l2(fg[:, fluid], fo[:, fluid]) < FP64_TOL
    Fo, To = p.o.forces()
    Fg, Tg = p.g.forces()
    if wl.n_particles:
        assert np.max(np.abs(Fg - Fo)) <= FP64_TOL * np.max(np.abs(Fo))
        assert np.max(np.abs(Tg - To)) <= FP64_TOL * max(np.max(np.abs(To)), 1e-300) + 1e-15
    p.o.advance()
    p.g.advance()
    pg, po = p.g.particles(), p.o.particles()
    for k in ("x", "v", "w"):
        np.testing.assert_allclose(pg[k], po[k], rtol=1e-13, atol=1e-16)


def _coupled(wl, steps, precision=es.ES_FP64, overrides=None, forced=True):
    p = Pair(wl, precision, overrides)
    for _ in range(steps):
        info, ginfo, (Fo, To), (Fg, Tg) = p.step(forced=forced)
        if forced:
            assert ginfo["cycles"] == info["cycles"]
    return p, p.compare()


def test_coupled_single_sphere_100_steps_fp64():
    """32^3 periodic box, zeta sphere R = 4, lambda_D = 4, E = 1e-3, 3-level
    V-cycles to 1e-10, 100 steps (the small case the oracle runs in full)."""
    p, r = _coupled(W.single_sphere(), 100)
    assert r["owner_equal"]
    for k in ("psi", "u", "x", "v"):
        assert r[k] < FP64_TOL, (k, r[k])


def test_coupled_mixed_ragged_fp64():
    """Non-cubic 40x24x32 box (ragged thread-block tails), walls in z, both
    sphere kinds, moving and rotating spheres, tau = 0.8."""
    p, r = _coupled(W.mixed_box(), 20)
    assert r["owner_equal"]
    for k in ("psi", "u", "x", "v", "w"):
        assert r[k] < FP64_TOL, (k, r[k])


def test_coupled_channel_fp64():
    """Channel shape (walls in z, charged spheres) at 64^3, 4 levels, with
    moving spheres.  (At rest the flow after 20 steps is ~1e-5 while the
    populations are ~0.05, so FP64 rounding alone differs by ~1e-11 relative
    in u between any two summation orders; moving spheres put u well above
    that floor.)"""
    p, r = _coupled(_moving(W.channel(n=64, n_spheres=8, radius=5.0, levels=4)), 20)
    assert r["owner_equal"]
    for k in ("psi", "u", "x", "v", "w"):
        assert r[k] < FP64_TOL, (k, r[k])


def _electro_osmotic_channel():
    """32^3 channel (walls in z, periodic x and y) with no spheres and
    Dirichlet potentials zeta = 1 and -0.5 on its two walls (the wall
    condition of Sec. 5.5), lambda_D = 3, E = 2e-3 along x: the field acts on
    the walls' double layers and drives an electro-osmotic flow."""
    wl = W.channel(n=32, n_spheres=0, radius=3.0, levels=3, res_rf=1e-10)
    wl.pot_bc = (0, 0, 0, 0, 1, 1)
    wl.pot_val = (0.0, 0.0, 0.0, 0.0, 1.0, -0.5)
    return wl


def test_electro_osmotic_channel_without_spheres_fp64():
    """An empty particle array (the mapping, force and update launches have
    no work) and charged walls: potential and flow within 1e-12 of the
    oracle after 20 steps, the flow (up to 0.018) far above FP64 rounding."""
    p, r = _coupled(_electro_osmotic_channel(), 20)
    assert r["owner_equal"]
    for k in ("psi", "u"):
        assert r[k] < FP64_TOL, (k, r[k])
    assert np.abs(p.g.field(es.FIELD_U)).max() > 1e-2


def test_electro_osmotic_channel_without_spheres_mixed32():
    """The same channel in MIXED32 after 100 steps: potential and flow within
    1e-4 of the FP64 oracle."""
    p, r = _coupled(_electro_osmotic_channel(), 100, precision=es.ES_MIXED32, forced=False)
    print("relative L2 against the oracle:", {k: float(r[k]) for k in ("psi", "u")})
    assert r["owner_equal"]
    for k in ("psi", "u"):
        assert r[k] < MIXED_TOL, (k, r[k])


def test_channel_128_full_size_fp64():
    """The channel configuration at its own size: 128^3, no-slip and
    zero-flux walls at the z faces, periodic x and y, 64 moving spheres of
    radius 6 with charges in [0.5, 1.5], lambda_D = 3, E = 2e-3, 4 levels to
    1e-8.  FP64 against the oracle (its OpenMP build), 5 coupled steps with
    the oracle's cycle counts: 1e-12."""
    p = Pair(_moving(W.channel()), omp=True)
    for _ in range(5):
        info, ginfo, _, _ = p.step()
        assert ginfo["cycles"] == info["cycles"]
    r = p.compare()
    assert r["owner_equal"]
    for k in ("psi", "u", "x", "v", "w", "F", "T"):
        assert r[k] < FP64_TOL, (k, r[k])


def test_channel_128_full_size_mixed32():
    """The same 128^3 channel in MIXED32, each side on its own
    tolerance-driven solver, 20 steps: 1e-4 on every quantity."""
    p = Pair(_moving(W.channel()), es.ES_MIXED32, omp=True)
    for _ in range(20):
        _, ginfo, _, _ = p.step(forced=False)
        assert ginfo["status"] == es.ES_OK and ginfo["r"] < ginfo["tol"]
    _assert_reduced(p.compare())


def _slip(wl, faces):
    wl.wall_slip = faces
    return wl


SLIP_CASES = {
    # walls in z, both free-slip; moving and rotating spheres of both kinds
    "mixed_box_z_free": lambda: _slip(W.mixed_box(), (0, 0, 0, 0, 1, 1)),
    # x walls no-slip, z walls free-slip: edges fall back to bounce-back
    "x_noslip_z_free": lambda: _slip(_moving(W.mixed_box(dims=(40, 24, 32), levels=2, periodic=(0, 1, 0))),
                                     (0, 0, 0, 0, 1, 1)),
    # x and z walls free-slip: populations at the edges reflect off both
    "xz_free": lambda: _slip(_moving(W.mixed_box(dims=(40, 24, 32), levels=2, periodic=(0, 1, 0))),
                             (1, 1, 0, 0, 1, 1)),
}


@pytest.mark.parametrize("name", sorted(SLIP_CASES))
def test_coupled_free_slip_walls_fp64(name):
    """Free-slip walls (specular reflection) in the stream step, coupled
    with moving spheres, against the oracle: FP64 bar."""
    p, r = _coupled(SLIP_CASES[name](), 20)
    assert r["owner_equal"]
    for k in ("psi", "u", "x", "v", "w"):
        assert r[k] < FP64_TOL, (k, r[k])


@pytest.mark.parametrize("precision", [es.ES_MIXED32, es.ES_MIXED16])
def test_free_slip_reduced_precision_after_100_steps(precision):
    wl = _slip(W.channel(n=64, n_spheres=8, radius=5.0, levels=4), (0, 0, 0, 0, 1, 1))
    p, r = _coupled(wl, 100, precision=precision, forced=False)
    _assert_reduced(r, None if precision == es.ES_MIXED32 else MIXED16_BARS)


def _pb(wl, phi_t, sweeps=2, omega=1.5):
    wl.phi_t, wl.levels, wl.coarse_sweeps, wl.omega, wl.max_cycles = phi_t, 1, sweeps, omega, 5000
    return wl


PB_CASES = {
    # zeta = 4 phi_t: far outside the Debye-Hueckel regime
    "sphere_zeta": lambda: _pb(W.single_sphere(n=24, radius=4.0, zeta=2.0), 0.5),
    # walls in z (Dirichlet and zero-flux faces), zeta and charged spheres, moving
    "mixed_walls": lambda: _pb(W.mixed_box(dims=(24, 16, 20)), 0.6, sweeps=1, omega=1.7),
}


@pytest.mark.parametrize("name", sorted(PB_CASES))
def test_coupled_nonlinear_poisson_boltzmann_fp64(name):
    """The nonlinear Poisson-Boltzmann form (SOR-Newton with the stencil
    re-linearised each iteration, sinh charge density in the body force),
    coupled with the LBM and the particles, against the oracle: FP64 bar."""
    p, r = _coupled(PB_CASES[name](), 8)
    assert r["owner_equal"]
    for k in ("psi", "u", "x", "v"):
        assert r[k] < FP64_TOL, (k, r[k])


@pytest.mark.parametrize("maker", [lambda: W.single_sphere(),
                                   lambda: W.channel(n=64, n_spheres=8, radius=5.0, levels=4)])
def test_mixed32_within_1e4_after_100_steps(maker):
    """MIXED32 (FP32 PDFs and multigrid cycles, FP64 defect correction and
    particles) against the FP64 oracle after 100 steps, each side on its own
    tolerance-driven solver."""
    p, r = _coupled(maker(), 100, precision=es.ES_MIXED32, forced=False)
    _assert_reduced(r)


@pytest.mark.parametrize("name", ["single_sphere", "mixed_ragged", "walls_x42"])
def test_mixed32_defect_correction_reaches_fp64_tolerance(name):
    """The MIXED32 outer iteration keeps psi and r = b - A psi in float-float
    (about 48 bits): with FP32 V-cycles it must still reach a relative
    tolerance of 1e-12, five decades below FP32 resolution, and land on the
    oracle's FP64 solution.  (A residual formed in FP32 stalls near 1e-7.)
    Both sides stop at ||r|| < 1e-12 ||r0||; the potential error this leaves
    is bounded by cond(A) * 1e-12, cond(A) <= (12 + kappa^2) / kappa^2 < 200
    here, so the two solutions agree to 1e-9."""
    if name == "walls_x42":  # nx not a multiple of 4: the scalar residual path
        wl = W.mixed_box(dims=(42, 24, 32), levels=2, periodic=(0, 1, 0))
    else:
        wl = CASES[name]()
    over = dict(res_rf=1e-12, max_cycles=200)
    p = Pair(wl, es.ES_MIXED32, over)
    p.o.map_particles()
    p.g.map_particles()
    io = p.o.solve()
    ig = p.g.solve()
    assert ig["status"] == es.ES_OK and ig["r"] < ig["tol"]
    assert abs(ig["r0"] - io["r0"]) <= 1e-6 * io["r0"]
    fluid = p.o.owner() < 0
    assert rel_l2(p.g.field(es.FIELD_PSI)[fluid], p.o.field(oracle.FIELD_PSI)[fluid]) < 1e-9


@pytest.mark.parametrize("maker", [lambda: W.single_sphere(),
                                   lambda: W.channel(n=64, n_spheres=8, radius=5.0, levels=4)])
def test_mg_fp16_within_1e4_after_100_steps(maker):
    """MIXED32 with the finest level's multigrid correction stored as FP16
    (scaled by sqrt(N) / ||r||) against the FP64 oracle after 100 steps."""
    wl = maker()
    p = Pair(wl, es.ES_MIXED32, lib_overrides=dict(mg_storage=es.ES_MG_FP16))
    for _ in range(100):
        _, ginfo, _, _ = p.step(forced=False)
        assert ginfo["status"] == es.ES_OK and ginfo["r"] < ginfo["tol"]
    _assert_reduced(p.compare())


@pytest.mark.parametrize("name", ["single_sphere", "mixed_ragged"])
def test_mg_fp16_defect_correction_reaches_fp64_tolerance(name):
    """The FP16 correction's rounding (unit roundoff 2^-11 of the scaled
    values) only slows the float-float outer iteration: it still reaches
    1e-12 relative and the oracle's FP64 solution, as in the MIXED32 test
    above."""
    wl = CASES[name]()
    over = dict(res_rf=1e-12, max_cycles=300)
    p = Pair(wl, es.ES_MIXED32, over, lib_overrides=dict(mg_storage=es.ES_MG_FP16))
    p.o.map_particles()
    p.g.map_particles()
    p.o.solve()
    ig = p.g.solve()
    assert ig["status"] == es.ES_OK and ig["r"] < ig["tol"]
    fluid = p.o.owner() < 0
    assert rel_l2(p.g.field(es.FIELD_PSI)[fluid], p.o.field(oracle.FIELD_PSI)[fluid]) < 1e-9


@pytest.mark.parametrize("name", ["suspension64", "channel64", "mixed_ragged"])
def test_colour_split_layout_is_bit_identical_to_natural(name):
    """The colour-split storage of the finest level (default in the reduced
    forms when nx % 8 == 0) runs the same arithmetic in the same order as
    the natural layout: 6 coupled MIXED32 steps agree bit for bit."""
    out = []
    for layout in (es.ES_LAYOUT_AUTO, es.ES_LAYOUT_NATURAL):
        g = es.Simulation(CASES[name](), es.ES_MIXED32, overrides=dict(fine_layout=layout))
        cyc = [g.step()["cycles"] for _ in range(6)]
        out.append((cyc, g.field(es.FIELD_PSI), g.field(es.FIELD_U), g.particles()["x"]))
        g.close()
    assert out[0][0] == out[1][0]
    for a, b in zip(out[0][1:], out[1][1:]):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("name", ["suspension64", "channel64", "mixed_ragged"])
def test_bulk_staged_half_sweep_is_bit_identical(name):
    """The finest-level half sweep with its operands staged in shared memory
    by bulk asynchronous copies (sweep_staging = ES_STAGE_BULK) computes the
    same sweep as the register version: 6 coupled MIXED32 steps agree bit
    for bit (walled and periodic boxes, rows of 20 to 32 compact cells)."""
    out = []
    for staging in (es.ES_STAGE_REGISTERS, es.ES_STAGE_BULK):
        g = es.Simulation(CASES[name](), es.ES_MIXED32, overrides=dict(sweep_staging=staging))
        cyc = [g.step()["cycles"] for _ in range(6)]
        out.append((cyc, g.field(es.FIELD_PSI), g.field(es.FIELD_U), g.particles()["x"]))
        g.close()
    assert out[0][0] == out[1][0]
    for a, b in zip(out[0][1:], out[1][1:]):
        np.testing.assert_array_equal(a, b)


def test_mixed32_potential_round_trip():
    """MIXED32 stores psi as a float-float pair: a double written with
    es_set_field comes back to within 2^-47 relative."""
    wl = W.mixed_box()
    g = es.Simulation(wl, es.ES_MIXED32)
    rng = np.random.Generator(np.random.PCG64(11))
    v = rng.standard_normal(wl.n_cells) * np.exp(rng.uniform(-20.0, 20.0, wl.n_cells))
    g.set_field(es.FIELD_PSI, v)
    back = g.field(es.FIELD_PSI).ravel()
    assert np.all(np.abs(back - v) <= 2.0**-47 * np.abs(v))
    idx = np.arange(0, wl.n_cells, 7, dtype=np.int64)[:4096]
    assert np.array_equal(g.gather(es.FIELD_PSI, idx)[0], back[idx])


# MIXED16 keeps each population as an FP16 number (unit roundoff 2^-11) of
# its scaled relative deviation: the stored state is re-rounded every step,
# which leaves a relative error of about 1.3e-4 in the slow velocity field
# (measured, and flat from 100 to 1,000 steps), and the momentum exchange of
# one step sums that rounding over every boundary link.  MIXED16 misses the
# 1e-4 bar on the fluid velocity and on the force and torque of a single
# step; the particles integrate the force noise out (displacement and
# velocity stay within 1e-4), and the potential sees the PDFs only through
# them.  Its bars here are about twice the largest errors measured on these
# cases after 100 steps (u 6.2e-4 in the single-sphere box, F 6.3e-3 there,
# T 2.7e-2 in the free-slip channel; displacement and particle velocity at
# most 8.6e-5).
MIXED16_BARS = {"u": 1.3e-3, "F": 1.3e-2, "T": 6e-2}


@pytest.mark.parametrize("maker", [lambda: W.single_sphere(),
                                   lambda: W.channel(n=64, n_spheres=8, radius=5.0, levels=4)])
def test_mixed16_after_100_steps(maker):
    """FP16 relative-deviation PDF storage (FP32 collision, the MIXED32
    solver) against the FP64 oracle after 100 steps."""
    p, r = _coupled(maker(), 100, precision=es.ES_MIXED16, forced=False)
    _assert_reduced(r, MIXED16_BARS)


@pytest.mark.parametrize("n", [16, 32])
def test_sor_variant(n):
    """The paper's own solver, red-black SOR with omega = 1.7 (Sec. 6.1):
    one level, so a "cycle" is coarse_sweeps SOR sweeps on the defect (the
    same iterates as SOR on psi, the sweeps being affine).  16^3 runs in the
    one-block shared-memory solver, 32^3 in the sweep kernels."""
    wl = W.single_sphere(n=n, radius=4.0 if n == 32 else 3.0, levels=1, res_rf=1e-8)
    over = dict(omega=1.7, coarse_sweeps=10, max_cycles=400)
    p = Pair(wl, overrides=over)
    p.o.map_particles()
    p.g.map_particles()
    fluid = p.o.owner() < 0
    io = p.o.solve(forced_cycles=3)
    ig = p.g.solve(forced_cycles=3)
    assert rel_l2(p.g.field(es.FIELD_PSI)[fluid], p.o.field(oracle.FIELD_PSI)[fluid]) < FP64_TOL
    io = p.o.solve()
    ig = p.g.solve()
    assert ig["cycles"] == io["cycles"] and ig["r"] < ig["tol"]
    assert rel_l2(p.g.field(es.FIELD_PSI)[fluid], p.o.field(oracle.FIELD_PSI)[fluid]) < FP64_TOL


@pytest.mark.parametrize("tau", [6.0, 6.5])
def test_coupled_paper_relaxation_times(tau):
    """The paper's relaxation times (tau = 6 for the validation and scaling
    runs, 6.5 for the micro-channel run; Sec. 6.1), FP64, 20 coupled steps."""
    wl = W.mixed_box()
    wl.tau = tau
    p, r = _coupled(wl, 20)
    assert r["owner_equal"]
    for k in ("psi", "u", "x", "v", "w"):
        assert r[k] < FP64_TOL, (k, r[k])


def test_zero_right_hand_side_is_solved_without_cycles():
    wl = W.single_sphere(n=16, radius=3.0, levels=2, res_rf=1e-8)
    wl.zeta = np.zeros(1)
    g = es.Simulation(wl, es.ES_MIXED32, overrides=dict(max_cycles=3))
    g.map_particles()
    info = g.solve()
    assert info["cycles"] == 0 and info["r0"] == 0.0 and info["status"] == es.ES_OK


def test_overlap_is_reported():
    wl = W.single_sphere(n=32, radius=4.0)
    wl.x = np.array([[10.0, 16.0, 16.0], [16.5, 16.0, 16.0]])
    wl.v = np.zeros((2, 3))
    wl.w = np.zeros((2, 3))
    wl.R = np.array([4.0, 4.0])
    wl.kind = np.array([0, 0], dtype=np.int32)
    wl.zeta = np.array([1.0, 1.0])
    wl.q = np.zeros(2)
    g = es.Simulation(wl)
    g.map_particles()
    with pytest.raises(es.EsError) as e:
        g.solve()
    assert e.value.code == es.ES_EOVERLAP
    # the status is cleared once reported
    g.synchronize()


def test_nonconvergence_and_forced_cycles():
    wl = W.single_sphere(res_rf=1e-12)
    g = es.Simulation(wl, overrides=dict(max_cycles=2))
    g.map_particles()
    r = g.solve(check=False)
    assert r["status"] == es.ES_ENOTCONVERGED and r["cycles"] == 2
    r2 = g.solve(forced_cycles=0)
    assert r2["cycles"] == 0


def test_runs_are_deterministic_and_allocator_independent():
    wl = W.channel(n=64, n_spheres=8, radius=5.0, levels=4)
    out = []
    for torch_memory in (True, False, True):
        g = es.Simulation(wl, es.ES_MIXED32, torch_memory=torch_memory)
        for _ in range(5):
            g.step()
        F, T = g.forces()
        out.append((g.field(es.FIELD_PSI), g.field(es.FIELD_U), F, T, g.particles()["x"]))
        g.close()
    for a, b in zip(out[0], out[1]):
        np.testing.assert_array_equal(a, b)
    for a, b in zip(out[0], out[2]):
        np.testing.assert_array_equal(a, b)


def test_full_size_suspension_sampled():
    """512^3 periodic suspension, 2,880 spheres R = 5, MIXED32, 6 levels: the
    configuration the benchmark times.  Checked on samples the oracle computes
    one by one and on properties that hold at any size."""
    import torch

    wl = W.suspension()
    g = es.Simulation(wl, es.ES_MIXED32)
    for _ in range(3):
        info = g.step()
    assert info["r"] < info["tol"]
    N = wl.n_cells
    nx, ny, nz = wl.dims
    rng = np.random.Generator(np.random.PCG64(9))
    # (1) sampled collisions: gather the pulled populations of fluid cells away
    # from spheres and collide them with the oracle on a 1x1x1 periodic
    # lattice, where streaming maps every population onto itself
    probe = rng.integers(0, N, 4000)
    fl = g.gather(es.FIELD_FLAGS, probe)[0]
    cells = probe[fl == 0][:48]
    c_lib, _ = es.lattice()
    perm = direction_map()
    x, y, z = cells % nx, (cells // nx) % ny, cells // (nx * ny)
    pulled = np.zeros((19, cells.size))
    for q in range(19):
        src = ((x - c_lib[q, 0]) % nx) + nx * (((y - c_lib[q, 1]) % ny) + ny * ((z - c_lib[q, 2]) % nz))
        pulled[q] = g.gather(es.FIELD_PDF_LAST, src)[q]
    fb = g.gather(es.FIELD_FB, cells)
    out = g.gather(es.FIELD_PDF, cells)
    for i in range(cells.size):
        one = W.Workload(name="cell", dims=[1, 1, 1], periodic=(1, 1, 1), tau=wl.tau, kappa=0.0, eps=1.0,
                         E_ext=(0.0, 0.0, 0.0), accel=tuple(fb[:, i]), levels=1, coarse_sweeps=1)
        o = oracle.Oracle(one)
        fin = np.empty(19)
        fin[perm] = pulled[:, i]
        o.set_field(oracle.FIELD_PDF, fin.reshape(19, 1, 1, 1))
        o.map_particles()
        o.lbm_step()
        ref = o.field(oracle.FIELD_PDF).reshape(19)
        got = np.empty(19)
        got[perm] = out[:, i]
        assert np.max(np.abs(got - ref)) < 2e-8
    # (2) discrete Gauss law: kappa^2 eps sum(psi) over fluid cells = sum q
    psi = torch.empty(N, dtype=torch.float64, device="cuda")
    own = torch.empty(N, dtype=torch.int32, device="cuda")
    g.field_device(es.FIELD_PSI, psi)
    g.field_device(es.FIELD_OWNER, own)
    total = (wl.kappa ** 2) * wl.eps * float(psi[own < 0].sum())
    assert abs(total - wl.q.sum()) < 1e-5 * wl.q.sum()
    del psi, own
    # (3) mapping of sampled spheres at their current positions against the
    # cell-in-sphere definition (centre inside, minimum image), exactly
    g.map_particles()
    X = g.particles()["x"]
    for p in rng.choice(wl.n_particles, 24, replace=False):
        lo = np.floor(X[p] - 7.0).astype(int)
        ii, jj, kk = np.meshgrid(*[np.arange(lo[a], lo[a] + 15) for a in range(3)], indexing="ij")
        cells3 = np.stack([ii % nx, jj % ny, kk % nz], -1).reshape(-1, 3)
        d = cells3 + 0.5 - X[p]
        L = np.array([nx, ny, nz], dtype=float)
        d = np.where(d > L / 2, d - L, d)
        d = np.where(d < -L / 2, d + L, d)
        inside = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2] <= wl.R[p] ** 2
        own = g.gather(es.FIELD_OWNER, cells3[:, 0] + nx * (cells3[:, 1] + ny * cells3[:, 2]))[0]
        np.testing.assert_array_equal(own == p, inside)
    g.close()


def test_radius_and_kind_fixed_after_creation():
    """es_set_particles moves spheres but rejects a change of radius or kind
    (the mapping updates flags only near each sphere's surface)."""
    wl = W.mixed_box()
    g = es.Simulation(wl, es.ES_MIXED32)
    for R, kind in ((wl.R * 1.1, wl.kind), (wl.R, 1 - wl.kind)):
        parts = es.pack_particles(wl.x, wl.v, wl.w, R, kind, wl.zeta, wl.q)
        rc = g.lib.es_set_particles(g.h, parts, wl.n_particles)
        assert rc == es.ES_EINVAL and "fixed after creation" in g.lib.es_last_error(g.h).decode()
    g.set_particles(wl.x + 0.25, wl.v, wl.w)
    info = g.step()
    assert info["r"] < info["tol"]
    g.close()


def test_set_particles_is_staged_and_keeps_the_mapped_state():
    """es_set_particles copies the caller's array at the call (it may be
    overwritten at once) and returns without waiting; the state reads back
    exactly, and a round trip of the current state between steps changes no
    bit of the coupled step (the surface charge density of a charged sphere
    and its boundary value are kept until the next mapping)."""
    wl = W.mixed_box()
    n = wl.n_particles
    a = es.Simulation(wl, es.ES_MIXED32)
    b = es.Simulation(wl, es.ES_MIXED32)
    for _ in range(2):
        a.step(forced_cycles=2)
        cur = (es.Particle * n)()
        assert b.lib.es_get_particles(b.h, cur, n) == es.ES_OK
        assert b.lib.es_set_particles(b.h, cur, n) == es.ES_OK
        ctypes.memset(cur, 0, ctypes.sizeof(cur))
        b.step(forced_cycles=2)
    for f in (es.FIELD_PSI, es.FIELD_PDF):
        np.testing.assert_array_equal(a.field(f), b.field(f))
    pa, pb = a.particles(), b.particles()
    for k in ("x", "v", "w"):
        np.testing.assert_array_equal(pa[k], pb[k])

    rng = np.random.default_rng(5)
    x = wl.x + rng.uniform(-0.3, 0.3, wl.x.shape)
    v = rng.normal(0, 1e-3, wl.x.shape)
    w = rng.normal(0, 1e-4, wl.x.shape)
    zeta = wl.zeta * 1.5
    q = wl.q * 0.5
    src = es.pack_particles(x, v, w, wl.R, wl.kind, zeta, q)
    assert b.lib.es_set_particles(b.h, src, n) == es.ES_OK
    ctypes.memset(src, 0, ctypes.sizeof(src))
    out = (es.Particle * n)()
    assert b.lib.es_get_particles(b.h, out, n) == es.ES_OK
    got = {k: np.array([list(getattr(out[i], k)) for i in range(n)]) for k in ("x", "v", "w")}
    np.testing.assert_array_equal(got["x"], x)
    np.testing.assert_array_equal(got["v"], v)
    np.testing.assert_array_equal(got["w"], w)
    np.testing.assert_array_equal([out[i].zeta for i in range(n)], zeta)
    np.testing.assert_array_equal([out[i].q for i in range(n)], q)
    np.testing.assert_array_equal([out[i].kind for i in range(n)], wl.kind)
    np.testing.assert_array_equal([out[i].R for i in range(n)], wl.R)
    a.close()
    b.close()


def test_alu_peak_probe():
    """es_alu_peak measures FMA throughput: positive, FP32 well above FP64
    on GB300 (its FP64 pipe runs at a small fraction of the FP32 rate)."""
    f64 = es.alu_peak(es.ES_FP64)
    f32 = es.alu_peak(es.ES_MIXED32)
    print("FMA peaks GFLOP/s: fp64", f64, "fp32", f32)
    assert f64 > 10.0 and f32 > 4.0 * f64
    rc = es.load().es_alu_peak(es.ES_MIXED16, None)
    assert rc == es.ES_EINVAL
