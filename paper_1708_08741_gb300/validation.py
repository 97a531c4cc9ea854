"""Electrophoretic velocity of a single sphere against Henry's solution.

The paper's validation (Sec. 6, Tab. ValidElectrophoresis) moves one sphere
of fixed zeta potential through a large box under an applied field, takes
the terminal velocity U* from the second half of the run, and compares it
with Henry's velocity for an unbounded electrolyte (Eq. ElPhorVelSphere,
with Ohshima's approximation of Henry's function, Eq. ElPhorMobilitySphere):

    U_EP = 2 eps zeta E / (3 mu) * (1 + 1 / (2 [1 + 2.5 / (kR (1 + 2 exp(-kR)))]^3)).

The confinement is taken out as the paper does: the relative deviation from
Stokes' velocity of the same sphere in the same box, Delta_r U_Stokes, is
subtracted from the electrophoretic deviation Delta_r U = (U* - U_EP) / U_EP.

Two settings.  Periodic box (``validate``): both runs are the
periodic-array setting, with velocities measured relative to the mean fluid
velocity (the Stokes half is described below).  Free-slip box
(``validate_free_slip``, the paper's setting): all six faces are free-slip
walls with zero-flux potential, velocities are absolute (the box holds no
net flow), and the Stokes run drags the same sphere, uncharged, with a
constant external force F_0 = 6 pi mu R U_Henry added to its hydrodynamic
force every step (es_forces, then es_set_forces, then es_advance), so that
Delta_r U_Stokes = U*_Stokes / U_Henry - 1.

In the periodic box:  The electrophoretic run needs no balancing
force: the double layer carries the opposite of the sphere's charge.  The
Stokes run holds an uncharged sphere (zeta = 0, so psi = 0 and no field
force) in place with a very large density and drives the fluid past it with
a uniform body force g.  The mean flow of the whole box approaches its
steady value only on the time N_fluid / (6 pi mu R K), far longer than the
run, but the disturbance around the sphere follows the mean flow within a
few hundred steps, so the drag coefficient K = F / (6 pi mu R U) is read at
every sample from the momentum-exchange force F and the mean fluid velocity
U, and Delta_r U_Stokes = 1 / K - 1 (the velocity the same force would give
relative to Stokes' F / (6 pi mu R)).
Lattice units: dx = dt = rho = eps = 1, mu = (tau - 1/2) / 3.

A third way (``box_extrapolated``) takes the box out with the
electrophoretic sphere itself: periodic runs at several box sizes,
extrapolated to an unbounded box in (R/L)^3, the order in which the
periodic images of a force-free sphere with its screened double layer act
on it.

    python -m paper_1708_08741_gb300.validation [--n 128] [--radius 4] [--kR 0.5] [--walls free-slip]
    python -m paper_1708_08741_gb300.validation --extrapolate 64 96 128 [--kR 0.265 0.5 0.8]
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

import paper_1708_08741_gb300 as es
from paper_1708_08741_gb300 import workloads as W


def henry_velocity(zeta: float, E: float, eps: float, mu: float, kR: float) -> float:
    """Henry's electrophoretic velocity with Ohshima's Henry function."""
    g = 1.0 + 2.5 / (kR * (1.0 + 2.0 * math.exp(-kR)))
    return 2.0 * eps * zeta * E / (3.0 * mu) * (1.0 + 1.0 / (2.0 * g ** 3))


def sphere_charge(zeta: float, R: float, kappa: float, eps: float = 1.0) -> float:
    """q_s = 4 pi R^2 sigma_s with sigma_s = zeta eps (1 + kappa R) / R."""
    return 4.0 * math.pi * R * zeta * eps * (1.0 + kappa * R)


def _box(n, R, tau, kappa, E, zeta, accel, levels, rho_p_ratio=1.195, walls=False):
    wl = W.Workload(name=f"henry_{n}_R{R:g}", dims=[n, n, n], periodic=(0, 0, 0) if walls else (1, 1, 1),
                    tau=tau, kappa=kappa, eps=1.0, E_ext=(E, 0.0, 0.0), accel=accel, levels=levels, res_rf=1e-8,
                    max_cycles=200, rho_p_ratio=rho_p_ratio)
    if walls:
        wl.wall_slip = (1, 1, 1, 1, 1, 1)
    c = np.array([[n / 2.0, n / 2.0, n / 2.0]])
    return W._set_particles(wl, c, np.array([float(R)]), np.array([W.KIND_ZETA]), np.array([zeta]), np.zeros(1))


def _solid_mask(wl):
    """Cells whose centre lies in the sphere (the mapping rule, Sec. 4.2)."""
    n = wl.dims[0]
    c = np.arange(n) + 0.5
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    x0 = wl.x[0]
    return (X - x0[0]) ** 2 + (Y - x0[1]) ** 2 + (Z - x0[2]) ** 2 <= wl.R[0] ** 2


def terminal_velocity(wl, steps: int, sample_every: int = 100, precision: int = es.ES_MIXED32,
                      device: str = "cuda:0", relative: bool = True) -> dict:
    """Runs ``steps`` steps; over the second half of the samples returns the
    mean sphere velocity relative to the mean fluid velocity (U; absolute
    with relative=False), its relative spread (max - min) / mean, and the
    mean of F_x / U_rel with F_x the hydrodynamic force on the sphere (drag
    per unit relative velocity)."""
    sim = es.Simulation(wl, precision, device=device)
    samples, drag = [], []
    try:
        fluid = None
        for s in range(1, steps + 1):
            sim.step()
            if s % sample_every == 0:
                up = sim.particles()["v"][0, 0]
                uf = 0.0
                if relative:
                    fluid = sim.field(es.FIELD_OWNER) < 0
                    uf = sim.field(es.FIELD_U)[0][fluid].mean()
                F, _ = sim.forces()
                samples.append(up - uf)
                drag.append(F[0, 0] / (uf - up) if uf != up else float("nan"))
    finally:
        sim.close()
    h = len(samples) // 2
    tail = np.array(samples[h:])
    mean = float(tail.mean())
    return {"U": mean, "spread": float((tail.max() - tail.min()) / abs(mean)) if mean else float("nan"),
            "drag_per_velocity": float(np.mean(drag[h:])), "samples": len(samples)}


def validate(n: int = 128, R: float = 4.0, kR: float = 0.5, tau: float = 6.0, zeta: float = 1.0,
             E: float = 2.5e-3, steps: int = 12000, levels: int = 5, device: str = "cuda:0") -> dict:
    """One point of the validation: Henry deviation of the electrophoretic
    run, the Stokes deviation of the matching plain-force run, and their
    difference (the corrected deviation of Tab. ValidElectrophoresis)."""
    mu = (tau - 0.5) / 3.0
    kappa = kR / R
    # electrophoresis: the EDL carries about -q, so the net force is ~0; what
    # is left is removed with the mean fluid velocity
    ep = terminal_velocity(_box(n, R, tau, kappa, E, zeta, (0.0, 0.0, 0.0), levels), steps, device=device)
    u_henry = henry_velocity(zeta, E, 1.0, mu, kR)
    # Stokes: fixed uncharged sphere, fluid driven by g with about the
    # electrophoretic speed
    sim_wl = _box(n, R, tau, kappa, 0.0, 0.0, (0.0, 0.0, 0.0), levels, rho_p_ratio=1e12)
    n_fluid = n ** 3 - int(np.count_nonzero(_solid_mask(sim_wl)))
    g = u_henry * 6.0 * math.pi * mu * R / n_fluid
    sim_wl.accel = (g, 0.0, 0.0)
    st = terminal_velocity(sim_wl, steps, device=device)
    K = st["drag_per_velocity"] / (6.0 * math.pi * mu * R)
    d_ep = (ep["U"] - u_henry) / u_henry
    d_st = 1.0 / K - 1.0
    return {"n": n, "R": R, "kR": kR, "tau": tau, "zeta": zeta, "E": E, "steps": steps,
            "U_henry": u_henry, "U_sim": ep["U"], "spread": ep["spread"], "dU": d_ep,
            "K_stokes": K, "dU_stokes": d_st, "dU_corrected": d_ep - d_st}


def dragged_velocity(wl, f0: float, steps: int, sample_every: int = 100, precision: int = es.ES_MIXED32,
                     device: str = "cuda:0") -> dict:
    """The first sphere of ``wl`` (uncharged) moved by the constant force
    (f0, 0, 0) on top of its hydrodynamic force; mean x velocity over the
    second half of the samples, and every sample."""
    sim = es.Simulation(wl, precision, device=device)
    samples = []
    try:
        for s in range(1, steps + 1):
            sim.map_particles()
            sim.solve()
            sim.lbm_step()
            F, T = sim.forces()
            F = F.copy()
            F[0, 0] += f0
            sim.set_forces(F, T)
            sim.advance()
            if s % sample_every == 0:
                samples.append(sim.particles()["v"][0, 0])
    finally:
        sim.close()
    tail = np.array(samples[len(samples) // 2:])
    mean = float(tail.mean())
    return {"U": mean, "spread": float((tail.max() - tail.min()) / abs(mean)) if mean else float("nan"),
            "samples": len(samples), "U_samples": [float(v) for v in samples]}


def box_extrapolated(R: float = 4.0, kR: float = 0.5, sizes=(64, 96, 128), tau: float = 6.0, zeta: float = 1.0,
                     E: float = 2.5e-3, steps: int = 12000, device: str = "cuda:0") -> dict:
    """Henry deviation of the electrophoretic sphere with the box taken out
    by the sphere's own runs instead of a Stokes-drag run: the periodic
    electrophoretic run (velocity relative to the mean fluid velocity) at
    several box sizes L, fitted by least squares to U(L) = U_inf + b (R/L)^3
    -- the far field of an electrophoretic sphere decays like that of a
    dipole, 1/r^3, so its periodic images shift it by O((R/L)^3), where a
    dragged sphere's Stokeslet images shift it by O(R/L) -- and Delta_r U_inf
    = (U_inf - U_EP) / U_EP."""
    mu = (tau - 0.5) / 3.0
    kappa = kR / R
    u_henry = henry_velocity(zeta, E, 1.0, mu, kR)
    runs = []
    for n in sizes:
        levels = 5 if n % 32 == 0 else 4
        r = terminal_velocity(_box(n, R, tau, kappa, E, zeta, (0.0, 0.0, 0.0), levels), steps, device=device)
        runs.append({"n": n, "U": r["U"], "spread": r["spread"], "dU": (r["U"] - u_henry) / u_henry})
    x = np.array([(R / r["n"]) ** 3 for r in runs])
    y = np.array([r["U"] for r in runs])
    A = np.stack([np.ones_like(x), x], 1)
    (u_inf, b), *_ = np.linalg.lstsq(A, y, rcond=None)
    return {"R": R, "kR": kR, "tau": tau, "zeta": zeta, "E": E, "steps": steps, "U_henry": u_henry,
            "boxes": runs, "U_inf": float(u_inf), "b": float(b), "dU_inf": float((u_inf - u_henry) / u_henry)}


def validate_free_slip(n: int = 128, R: float = 4.0, kR: float = 0.5, tau: float = 6.0, zeta: float = 1.0,
                       E: float = 2.5e-3, steps: int = 12000, levels: int = 5, device: str = "cuda:0") -> dict:
    """The validation in a box with free-slip walls on all faces (the
    paper's setting): Henry deviation of the electrophoretic run, the Stokes
    deviation of the same sphere without a double layer (kappa = 0, moved by
    F = q E), and their difference."""
    mu = (tau - 0.5) / 3.0
    ep = terminal_velocity(_box(n, R, tau, kR / R, E, zeta, (0.0, 0.0, 0.0), levels, walls=True), steps,
                           device=device, relative=False)
    u_henry = henry_velocity(zeta, E, 1.0, mu, kR)
    f0 = 6.0 * math.pi * mu * R * u_henry
    st = dragged_velocity(_box(n, R, tau, kR / R, 0.0, 0.0, (0.0, 0.0, 0.0), levels, walls=True), f0, steps,
                          device=device)
    u0 = u_henry
    d_ep = (ep["U"] - u_henry) / u_henry
    d_st = st["U"] / u0 - 1.0
    return {"walls": "free-slip", "n": n, "R": R, "kR": kR, "tau": tau, "zeta": zeta, "E": E, "steps": steps,
            "U_henry": u_henry, "U_sim": ep["U"], "spread": ep["spread"], "dU": d_ep, "U_stokes": st["U"],
            "U0": u0, "dU_stokes": d_st, "dU_corrected": d_ep - d_st}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--radius", type=float, nargs="+", default=[4.0])
    ap.add_argument("--kR", type=float, nargs="+", default=[0.265, 0.5, 0.8])
    ap.add_argument("--steps", type=int, default=12000)
    ap.add_argument("--walls", choices=["periodic", "free-slip"], default="periodic")
    ap.add_argument("--extrapolate", type=int, nargs="+", default=None, metavar="L",
                    help="box sizes of the periodic electrophoretic runs extrapolated to an unbounded box")
    a = ap.parse_args()
    for R in a.radius:
        for kR in a.kR:
            if a.extrapolate:
                res = box_extrapolated(R, kR, sizes=a.extrapolate, steps=a.steps)
            else:
                res = (validate_free_slip if a.walls == "free-slip" else validate)(a.n, R, kR, steps=a.steps)
            print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
