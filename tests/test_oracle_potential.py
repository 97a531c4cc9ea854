"""Pins of the oracle's Debye-Hueckel solve (Sec. 4.3, 5.3-5.5) and of the EDL
field / body force (Sec. 5.6).  CPU only."""
import numpy as np
import pytest

import oracle
from paper_1708_08741_gb300 import workloads as W


def _wl(dims, periodic, kappa, particles=(), pot_bc=(0,) * 6, pot_val=(0.0,) * 6, levels=1,
        res_rf=1e-14, max_cycles=400, E=(0.0, 0.0, 0.0)):
    wl = W.Workload(name="pot", dims=list(dims), periodic=periodic, tau=1.0, kappa=kappa, eps=1.0,
                    E_ext=E, levels=levels, res_rf=res_rf, max_cycles=max_cycles, pot_bc=pot_bc,
                    pot_val=pot_val, coarse_sweeps=40)
    n = len(particles)
    if n:
        wl.x = np.array([p[0] for p in particles], dtype=float).reshape(n, 3)
        wl.v = np.zeros((n, 3))
        wl.w = np.zeros((n, 3))
        wl.R = np.array([p[1] for p in particles], dtype=float)
        wl.kind = np.array([p[2] for p in particles], dtype=np.int32)
        wl.zeta = np.array([p[3] for p in particles], dtype=float)
        wl.q = np.array([p[4] for p in particles], dtype=float)
    return wl


def _dense_system(dims, periodic, kappa, owner, kinds, zetas, qs, pot_bc, pot_val):
    """Assemble the finite-volume system of Sec. 4.3 directly: for every fluid
    cell, the flux through each face is the central difference of Eq.
    NormalFlux; a face to a Dirichlet cell uses the boundary value linearly
    extrapolated to that cell, a face to a Neumann cell the prescribed flux,
    a zero-flux wall no flux (Sec. 5.4).  Neumann particles spread their
    charge evenly over their faces."""
    nx, ny, nz = dims
    idx = -np.ones(owner.shape, dtype=int)
    cells = [(k, j, i) for k in range(nz) for j in range(ny) for i in range(nx) if owner[k, j, i] < 0]
    for n, c in enumerate(cells):
        idx[c] = n
    faces = {}
    for (k, j, i) in cells:
        for d in range(6):
            ax, s = d // 2, (1 if d % 2 else -1)
            p = [i, j, k]
            p[ax] += s
            if 0 <= p[ax] < dims[ax] or periodic[ax]:
                p[ax] %= dims[ax]
                o = owner[p[2], p[1], p[0]]
                if o >= 0:
                    faces[o] = faces.get(o, 0) + 1
    A = np.zeros((len(cells), len(cells)))
    b = np.zeros(len(cells))
    for n, (k, j, i) in enumerate(cells):
        A[n, n] += kappa ** 2
        for d in range(6):
            ax, s = d // 2, (1 if d % 2 else -1)
            p = [i, j, k]
            p[ax] += s
            if not (0 <= p[ax] < dims[ax]) and not periodic[ax]:
                face = 2 * ax + (1 if s > 0 else 0)
                if pot_bc[face] == 1:  # psi_ghost = 2 v - psi
                    A[n, n] += 2.0
                    b[n] += 2.0 * pot_val[face]
                continue
            p[ax] %= dims[ax]
            o = owner[p[2], p[1], p[0]]
            if o < 0:  # flux (psi_j - psi_i)
                A[n, n] += 1.0
                A[n, idx[p[2], p[1], p[0]]] -= 1.0
            elif kinds[o] == W.KIND_ZETA:
                A[n, n] += 2.0
                b[n] += 2.0 * zetas[o]
            else:
                b[n] += qs[o] / faces[o]
    return A, b, idx, faces


@pytest.mark.parametrize("case", ["periodic_zeta", "walls_charge", "mixed"])
def test_dense_solve_8cubed(case):
    if case == "periodic_zeta":
        wl = _wl((8, 8, 8), (1, 1, 1), 0.4, [((4.0, 4.0, 4.0), 1.6, W.KIND_ZETA, 0.8, 0.0)], levels=2)
    elif case == "walls_charge":
        wl = _wl((8, 8, 8), (1, 0, 0), 0.3, [((3.7, 4.2, 4.1), 1.7, W.KIND_CHARGE, 0.0, 1.3)],
                 pot_bc=(0, 0, 1, 0, 0, 1), pot_val=(0, 0, 0.25, 0, 0, -0.4), levels=3)
    else:
        wl = _wl((8, 8, 8), (0, 1, 1), 0.5, [((2.5, 2.5, 3.0), 1.2, W.KIND_ZETA, -0.6, 0.0),
                                              ((5.6, 5.5, 5.5), 1.5, W.KIND_CHARGE, 0.0, -0.9)],
                 pot_bc=(1, 0, 0, 0, 0, 0), pot_val=(0.3, 0, 0, 0, 0, 0), levels=2)
    o = oracle.Oracle(wl)
    o.map_particles()
    info = o.solve()
    assert info["status"] == 0 and info["r"] < info["tol"]
    owner = o.owner()
    A, b, idx, faces = _dense_system(wl.dims, wl.periodic, wl.kappa, owner, wl.kind, wl.zeta, wl.q,
                                     wl.pot_bc, wl.pot_val)
    nf = o.nfaces()
    for p, n in faces.items():
        assert nf[p] == n
    x = np.linalg.solve(A, b)
    psi = o.field(oracle.FIELD_PSI)
    got = psi[owner < 0]
    ref = x[idx[owner < 0]]
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-12


def test_one_dimensional_discrete_closed_form():
    """Slab periodic in x and y, Dirichlet value zeta at z = 0 and zero flux at
    z = H.  By symmetry the x/y fluxes vanish, and the stencil of Sec. 4.3
    reduces to (2 + kappa^2) psi_k - psi_{k-1} - psi_{k+1} = 0, whose
    solutions are A mu^k + B mu^-k with mu + 1/mu = 2 + kappa^2; the two
    boundary rows fix A and B."""
    H, kappa, zeta = 24, 0.35, 1.7
    wl = _wl((8, 8, H), (1, 1, 0), kappa, pot_bc=(0, 0, 0, 0, 1, 0), pot_val=(0, 0, 0, 0, zeta, 0),
             levels=3)
    o = oracle.Oracle(wl)
    o.map_particles()
    info = o.solve()
    assert info["status"] == 0
    s = 2.0 + kappa ** 2
    mu = (s - np.sqrt(s * s - 4.0)) / 2.0
    # row 0: (s + 1) psi_0 - psi_1 = 2 zeta; row H-1: (s - 1) psi_{H-1} - psi_{H-2} = 0
    M = np.array([[(s + 1.0) - mu, (s + 1.0) - 1.0 / mu],
                  [(s - 1.0) * mu ** (H - 1) - mu ** (H - 2), (s - 1.0) * mu ** (1 - H) - mu ** (2 - H)]])
    A, B = np.linalg.solve(M, np.array([2.0 * zeta, 0.0]))
    k = np.arange(H)
    exact = A * mu ** k + B * mu ** (-k)
    psi = o.field(oracle.FIELD_PSI)
    for j in range(8):
        for i in range(8):
            np.testing.assert_allclose(psi[:, j, i], exact, rtol=1e-12, atol=0)


def _sphere_error(R):
    n = int(8 * R)
    kappa = 1.0 / R
    c = n / 2.0
    wl = _wl((n, n, n), (0, 0, 0), kappa, [((c, c, c), R, W.KIND_ZETA, 1.0, 0.0)], levels=3,
             res_rf=1e-10)
    o = oracle.Oracle(wl)
    o.map_particles()
    o.solve()
    psi = o.field(oracle.FIELD_PSI)
    z, y, x = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5, np.arange(n) + 0.5, indexing="ij")
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    exact = R / r * np.exp(-kappa * (r - R))
    band = (r > R + 1.0) & (r < 3.0 * R)
    return np.sqrt(np.mean((psi[band] - exact[band]) ** 2)) / np.sqrt(np.mean(exact[band] ** 2))


def test_screened_sphere_potential():
    """zeta sphere in a large zero-flux box, kappa R = 1: compare with
    psi(r) = zeta (R/r) exp(-kappa (r - R)) (Eq. PotDistrSphereDH).  The
    staircase surface (Sec. 4.2) is the main error; it shrinks as R grows."""
    e4 = _sphere_error(4.0)
    e8 = _sphere_error(8.0)
    assert e4 < 0.05
    assert e8 < 0.03
    assert e8 < 0.75 * e4


def test_gauss_law_for_surface_charge():
    """Summing the discrete equations over all fluid cells, interior face
    fluxes cancel and zero-flux walls carry none, so kappa^2 eps sum(psi)
    equals the charge imposed at the particle faces: the total charge in the
    EDL balances the particles' charge (Eq. ChrgDensDHA)."""
    q1, q2 = 1.3, -0.45
    wl = _wl((16, 16, 16), (1, 0, 1), 0.4, [((5.2, 6.1, 7.3), 2.6, W.KIND_CHARGE, 0.0, q1),
                                             ((11.0, 10.4, 12.2), 2.2, W.KIND_CHARGE, 0.0, q2)],
             levels=3, res_rf=1e-13)
    o = oracle.Oracle(wl)
    o.map_particles()
    info = o.solve()
    assert info["status"] == 0
    psi = o.field(oracle.FIELD_PSI)
    fluid = o.owner() < 0
    total = wl.kappa ** 2 * wl.eps * psi[fluid].sum()
    assert abs(total - (q1 + q2)) < 1e-9
    # positive charge raises the potential next to the particle, negative lowers it
    assert psi[7, 6, 5 + 3] > 0.0 and psi[12, 10, 11 + 3] < 0.0


def test_multigrid_cycle_contracts_residual():
    """Every V-cycle must cut the residual well below the previous one."""
    wl = W.channel(n=32, n_spheres=4, radius=4.0, levels=3)
    o = oracle.Oracle(wl, dict(max_cycles=1, res_rf=1e-30))
    o.map_particles()
    r_prev = None
    for _ in range(5):
        info = o.solve(forced_cycles=1)
        if r_prev is not None:
            assert info["r"] < 0.3 * r_prev
        r_prev = info["r"]


def test_solver_stops_on_tolerance_and_reports_nonconvergence():
    wl = W.single_sphere(n=16, radius=3.0, levels=2, res_rf=1e-6)
    o = oracle.Oracle(wl)
    o.map_particles()
    info = o.solve()
    assert info["cycles"] > 0 and info["r"] < info["tol"] <= info["r0"] * 1e-6 * (1 + 1e-12)
    again = o.solve()
    assert again["cycles"] == 0  # the check comes before the first cycle
    wl2 = W.single_sphere(n=16, radius=3.0, levels=2, res_rf=1e-12)
    o2 = oracle.Oracle(wl2, dict(max_cycles=1))
    o2.map_particles()
    res = o2.solve(check=False)
    assert res["status"] == oracle.OR_ENOTCONVERGED and res["cycles"] == 1


def test_zero_right_hand_side_is_solved_without_cycles():
    """An uncharged sphere (zeta = 0) and zero-flux walls: b = 0, psi = 0 is
    exact, the first residual is zero and the solve returns at once."""
    wl = W.single_sphere(n=16, radius=3.0, levels=2, res_rf=1e-8)
    wl.zeta = np.zeros(1)
    o = oracle.Oracle(wl, dict(max_cycles=3))
    o.map_particles()
    info = o.solve()
    assert info["status"] == oracle.OR_OK and info["cycles"] == 0 and info["r0"] == 0.0
    assert np.all(o.field(oracle.FIELD_PSI) == 0.0)


def test_gradient_exact_for_linear_potential():
    """Both the D3Q19 stencil (Eq. ElPotGradComp) and the D3Q7 central
    differences with linearly extrapolated Dirichlet values are exact for a
    linear potential; the wall values are the linear function at the faces."""
    a, gx, gy, gz = 0.3, 0.02, -0.05, 0.04
    dims = (6, 6, 10)
    # periodic x/y would break linearity, so use walls with Dirichlet values
    # on the z faces and a linear field only along z; x/y stay periodic.
    wl = _wl(dims, (1, 1, 0), 0.2, pot_bc=(0, 0, 0, 0, 1, 1),
             pot_val=(0, 0, 0, 0, a + gz * 0.0, a + gz * dims[2]), E=(1e-3, 2e-3, 3e-3))
    o = oracle.Oracle(wl)
    o.map_particles()
    z = np.arange(dims[2]) + 0.5
    psi = np.broadcast_to((a + gz * z)[:, None, None], dims[::-1]).copy()
    o.set_field(oracle.FIELD_PSI, psi)
    g = o.gradient()
    np.testing.assert_allclose(g[2], gz, rtol=1e-13)
    np.testing.assert_allclose(g[:2], 0.0, atol=1e-15)
    # body force: f_b = -kappa^2 eps psi (E_ext - grad psi) (Sec. 5.6)
    o.body_force()
    fb = o.field(oracle.FIELD_FB)
    E = np.array(wl.E_ext)
    E_tot = E - np.array([0.0, 0.0, gz])
    for d in range(3):
        np.testing.assert_allclose(fb[d], -wl.kappa ** 2 * psi * E_tot[d], rtol=1e-13, atol=1e-20)
    # one axis at a time with Dirichlet values equal to the linear field on
    # the two faces of that axis, periodic along the other two
    xs = np.arange(8) + 0.5
    for ax in range(3):
        grad = [0.0, 0.0, 0.0]
        grad[ax] = [gx, gy, gz][ax]
        vals = [0.0] * 6
        vals[2 * ax] = a
        vals[2 * ax + 1] = a + grad[ax] * 8
        bc = [0] * 6
        bc[2 * ax] = bc[2 * ax + 1] = 1
        periodic = [1, 1, 1]
        periodic[ax] = 0
        wl3 = _wl((8, 8, 8), tuple(periodic), 0.2, pot_bc=tuple(bc), pot_val=tuple(vals))
        o3 = oracle.Oracle(wl3)
        o3.map_particles()
        Z, Y, X = np.meshgrid(xs, xs, xs, indexing="ij")
        field = a + grad[0] * X + grad[1] * Y + grad[2] * Z
        o3.set_field(oracle.FIELD_PSI, field)
        g3 = o3.gradient()
        for d in range(3):
            np.testing.assert_allclose(g3[d], grad[d], rtol=1e-12, atol=1e-15)


def test_uniform_potential_body_force():
    """psi = const in a periodic box: no EDL field, f_b = -kappa^2 eps psi E."""
    wl = _wl((4, 4, 4), (1, 1, 1), 0.5, E=(1e-3, -2e-3, 5e-4))
    o = oracle.Oracle(wl)
    o.map_particles()
    o.set_field(oracle.FIELD_PSI, np.full((4, 4, 4), 0.7))
    o.body_force()
    fb = o.field(oracle.FIELD_FB)
    for d in range(3):
        np.testing.assert_allclose(fb[d], -0.25 * 0.7 * wl.E_ext[d], rtol=1e-14)


# ---- nonlinear Poisson-Boltzmann form (Eq. SPBE) ---------------------------
# With kappa^2 = 2 z^2 e^2 n / (eps k_B T) and phi_t = k_B T / (z e), Eq. SPBE
# reads -lap psi + kappa^2 phi_t sinh(psi / phi_t) = 0 in the electrolyte; the
# oracle solves it with the paper's SOR sweeps on the stencil re-linearised at
# every iteration (levels == 1).


def _pb(wl, phi_t, sweeps=1, omega=1.0):
    wl.phi_t = phi_t
    wl.levels = 1
    wl.coarse_sweeps = sweeps
    wl.omega = omega
    return wl


def _dense_newton(A, b, kappa, phi_t, iters=60):
    """Newton's method on the dense finite-volume system with the screening
    term replaced: F(x) = (A - kappa^2 I) x + kappa^2 phi_t sinh(x / phi_t) - b."""
    k2 = kappa * kappa
    L = A - k2 * np.eye(len(b))
    x = np.linalg.solve(A, b)
    for _ in range(iters):
        F = L @ x + k2 * phi_t * np.sinh(x / phi_t) - b
        J = L + np.diag(k2 * np.cosh(x / phi_t))
        dx = np.linalg.solve(J, -F)
        x = x + dx
        if np.max(np.abs(dx)) < 1e-15 * max(1.0, np.max(np.abs(x))):
            break
    return x


@pytest.mark.parametrize("case", ["periodic_zeta", "mixed"])
def test_pb_matches_dense_newton_8cubed(case):
    """The oracle's SOR-Newton iteration converges to the solution of the
    nonlinear finite-volume system assembled directly (as in the dense
    Debye-Hueckel test) and solved by Newton's method with dense linear
    algebra.  zeta up to 4 phi_t: far outside the linear regime."""
    if case == "periodic_zeta":
        wl = _wl((8, 8, 8), (1, 1, 1), 0.4, [((4.0, 4.0, 4.0), 1.6, W.KIND_ZETA, 2.0, 0.0)])
        phi_t = 0.5
    else:
        wl = _wl((8, 8, 8), (0, 1, 1), 0.5, [((2.5, 2.5, 3.0), 1.2, W.KIND_ZETA, -1.2, 0.0),
                                              ((5.6, 5.5, 5.5), 1.5, W.KIND_CHARGE, 0.0, -2.5)],
                 pot_bc=(1, 0, 0, 0, 0, 0), pot_val=(0.9, 0, 0, 0, 0, 0))
        phi_t = 0.3
    wl = _pb(wl, phi_t, sweeps=2, omega=1.4)
    wl.max_cycles = 2000
    o = oracle.Oracle(wl)
    o.map_particles()
    info = o.solve()
    assert info["status"] == 0 and info["r"] < info["tol"]
    owner = o.owner()
    A, b, idx, _ = _dense_system(wl.dims, wl.periodic, wl.kappa, owner, wl.kind, wl.zeta, wl.q,
                                 wl.pot_bc, wl.pot_val)
    x = _dense_newton(A, b, wl.kappa, phi_t)
    lin = np.linalg.solve(A, b)
    psi = o.field(oracle.FIELD_PSI)
    got, ref = psi[owner < 0], x[idx[owner < 0]]
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-11
    # (and it is not the Debye-Hueckel solution)
    assert np.max(np.abs(lin[idx[owner < 0]] - ref)) > 1e-2 * np.max(np.abs(ref))


def test_pb_gouy_chapman_profile_and_electroneutrality():
    """Flat Dirichlet wall at z = 0 (zeta = 3 phi_t), zero flux far away: the
    continuum solution is Gouy-Chapman's psi = 4 phi_t artanh(tanh(zeta /
    (4 phi_t)) exp(-kappa d)), d the distance from the wall (cell centres at
    d = k + 1/2).  The finite-volume solution approaches it as kappa h falls:
    the error must drop at least 2.5-fold when kappa h halves.  At convergence
    the double layer's charge, the sum of rho_e over the column (read back
    from f_b = rho_e E_x with a field along the wall), balances the wall
    flux eps (psi_ghost - psi_0) = 2 eps (zeta - psi_0) exactly."""
    phi_t, zeta, E = 0.4, 1.2, 1e-3
    errs = []
    for kappa, H in ((0.2, 80), (0.1, 160)):
        wl = _wl((1, 1, H), (1, 1, 0), kappa, pot_bc=(0, 0, 0, 0, 1, 0),
                 pot_val=(0, 0, 0, 0, zeta, 0), E=(E, 0.0, 0.0), max_cycles=20000)
        wl = _pb(wl, phi_t, sweeps=4, omega=1.9)
        o = oracle.Oracle(wl)
        o.map_particles()
        info = o.solve()
        assert info["status"] == 0 and info["r"] < info["tol"]
        psi = o.field(oracle.FIELD_PSI)[:, 0, 0]
        d = np.arange(H) + 0.5
        gc = 4.0 * phi_t * np.arctanh(np.tanh(zeta / (4.0 * phi_t)) * np.exp(-kappa * d))
        near = d * kappa < 3.0
        errs.append(np.max(np.abs(psi[near] - gc[near])) / zeta)
        o.body_force()
        rho = o.field(oracle.FIELD_FB)[0][:, 0, 0] / E
        assert abs(rho.sum() + 2.0 * (zeta - psi[0])) < 1e-10 * zeta
    assert errs[0] < 2e-2 and errs[1] < 0.4 * errs[0]


def test_pb_tends_to_debye_hueckel_for_large_thermal_voltage():
    """sinh(x) = x + x^3/6 + ...: with phi_t = 1e3 |psi| the nonlinear solve
    lands on the Debye-Hueckel solution to ~1e-7."""
    wl = _wl((8, 8, 8), (1, 1, 1), 0.4, [((4.0, 4.0, 4.0), 1.6, W.KIND_ZETA, 0.8, 0.0)])
    wl.coarse_sweeps = 2
    wl.omega = 1.4
    wl.max_cycles = 2000
    o = oracle.Oracle(wl)
    o.map_particles()
    o.solve()
    lin = o.field(oracle.FIELD_PSI)
    o2 = oracle.Oracle(_pb(wl, 800.0, sweeps=2, omega=1.4))
    o2.map_particles()
    o2.solve()
    nl = o2.field(oracle.FIELD_PSI)
    fluid = o.owner() < 0
    d = np.max(np.abs(nl[fluid] - lin[fluid])) / np.max(np.abs(lin[fluid]))
    assert 1e-12 < d < 1e-6


@pytest.mark.parametrize("case", ["periodic_zeta", "mixed"])
def test_black_residuals_vanish_after_a_gauss_seidel_sweep(case):
    """After a red-black Gauss-Seidel sweep (omega = 1; red, then black) of
    A e = r, every black cell's equation holds for the red values around it,
    which the black half sweep does not change: the black residuals vanish
    and only red ones remain (what lets a restriction after pre-smoothing
    add the red children only).  A is the finite-volume system assembled
    directly (the dense-solve test's assembly), not the oracle's."""
    if case == "periodic_zeta":
        wl = _wl((8, 8, 8), (1, 1, 1), 0.4, [((4.0, 4.0, 4.0), 1.6, W.KIND_ZETA, 0.8, 0.0)])
    else:
        wl = _wl((8, 8, 8), (0, 1, 1), 0.5, [((2.5, 2.5, 3.0), 1.2, W.KIND_ZETA, -0.6, 0.0),
                                              ((5.6, 5.5, 5.5), 1.5, W.KIND_CHARGE, 0.0, -0.9)],
                 pot_bc=(1, 0, 0, 0, 0, 0), pot_val=(0.3, 0, 0, 0, 0, 0))
    o = oracle.Oracle(wl)
    o.map_particles()
    owner = o.owner()
    A, _, idx, _ = _dense_system(wl.dims, wl.periodic, wl.kappa, owner, wl.kind, wl.zeta, wl.q,
                                 wl.pot_bc, wl.pot_val)
    rng = np.random.Generator(np.random.PCG64(5))
    fluid = owner < 0
    r = np.where(fluid, rng.standard_normal(owner.shape), 0.0)
    e = o.smooth(r, np.zeros(owner.shape), 1)
    # residual cell by cell in the dense system's unknown order
    cells = np.argwhere(fluid)  # (k, j, i) in C order, as the dense assembly numbers them
    ev = np.array([e[k, j, i] for k, j, i in cells])
    rv = np.array([r[k, j, i] for k, j, i in cells])
    res = rv - A @ ev
    colour = (cells[:, 0] + cells[:, 1] + cells[:, 2]) % 2
    scale = np.max(np.abs(rv))
    assert np.max(np.abs(res[colour == 1])) < 1e-13 * scale
    assert np.max(np.abs(res[colour == 0])) > 1e-3 * scale
