"""Seeded synthetic workloads for the coupled electrophoresis step.

This module is the one piece that the CUDA path and the FP64 oracle both use:
it only draws numbers (sphere centres, radii, charges) and fills in plain
parameter dictionaries.  It holds none of the method's arithmetic: no lattice
Boltzmann, potential, force or unit-conversion formula lives here.

Random numbers come from PCG32 (M. E. O'Neill, "PCG: A Family of Simple Fast
Space-Efficient Statistically Good Algorithms for Random Number Generation",
2014), XSH-RR output on a 64-bit LCG with multiplier 6364136223846793005.

The workloads follow the shapes of the paper's runs (Sec. 6.1 and Sec. 6.5):
charged spheres of a few lattice cells radius in a box that is periodic along
some axes and bounded by no-slip, zero-flux walls along the others, a Debye
length of a few cells and a weak uniform applied field.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence

import numpy as np

# Particle boundary-condition kinds (Sec. 5.5): a prescribed zeta potential is a
# Dirichlet condition, a prescribed surface charge a Neumann condition.
KIND_ZETA = 0
KIND_CHARGE = 1

# Potential boundary kinds of a non-periodic domain face.
POT_ZERO_FLUX = 0
POT_DIRICHLET = 1

_MASK64 = (1 << 64) - 1


class PCG32:
    """PCG32 (XSH-RR 64/32) with a stream selector, as published by O'Neill."""

    MULT = 6364136223846793005

    def __init__(self, seed: int, stream: int = 54) -> None:
        self.state = 0
        self.inc = ((stream << 1) | 1) & _MASK64
        self.next_u32()
        self.state = (self.state + (seed & _MASK64)) & _MASK64
        self.next_u32()

    def next_u32(self) -> int:
        old = self.state
        self.state = (old * self.MULT + self.inc) & _MASK64
        xorshifted = (((old >> 18) ^ old) >> 27) & 0xFFFFFFFF
        rot = old >> 59
        return ((xorshifted >> rot) | (xorshifted << ((-rot) & 31))) & 0xFFFFFFFF

    def uniform(self) -> float:
        """Uniform double in [0, 1) from 53 random bits (two draws)."""
        hi = self.next_u32() >> 5
        lo = self.next_u32() >> 6
        return (hi * 67108864.0 + lo) / 9007199254740992.0

    def uniform_range(self, a: float, b: float) -> float:
        return a + (b - a) * self.uniform()

    def normal(self) -> float:
        """Standard normal deviate by the Box-Muller transform."""
        u1 = self.uniform()
        while u1 <= 0.0:
            u1 = self.uniform()
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


@dataclass
class Workload:
    """A complete, seeded problem description (plain numbers only)."""

    name: str
    dims: Sequence[int]
    periodic: Sequence[int]
    tau: float
    kappa: float
    eps: float
    E_ext: Sequence[float]
    accel: Sequence[float] = (0.0, 0.0, 0.0)
    rho_p_ratio: float = 1.195
    levels: int = 3
    nu1: int = 2
    nu2: int = 2
    coarse_sweeps: int = 32
    omega: float = 1.0
    res_rf: float = 1e-10
    max_cycles: int = 100
    steps: int = 100
    pot_bc: Sequence[int] = (0, 0, 0, 0, 0, 0)
    wall_slip: Sequence[int] = (0, 0, 0, 0, 0, 0)  # per face of a non-periodic axis: 1 = free-slip
    phi_t: float = 0.0  # thermal voltage k_B T / (z e): 0 = Debye-Hueckel, > 0 = nonlinear Poisson-Boltzmann
    pot_val: Sequence[float] = (0.0, 0.0, 0.0, 0.0, 0.0, 0.0)
    # particle arrays
    x: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    v: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    w: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    R: np.ndarray = field(default_factory=lambda: np.zeros(0))
    kind: np.ndarray = field(default_factory=lambda: np.zeros(0, dtype=np.int32))
    zeta: np.ndarray = field(default_factory=lambda: np.zeros(0))
    q: np.ndarray = field(default_factory=lambda: np.zeros(0))

    @property
    def n_particles(self) -> int:
        return int(self.R.shape[0])

    @property
    def n_cells(self) -> int:
        return int(self.dims[0]) * int(self.dims[1]) * int(self.dims[2])

    def describe(self) -> Dict[str, object]:
        return {
            "workload": self.name,
            "dims": list(map(int, self.dims)),
            "periodic": list(map(int, self.periodic)),
            "n_particles": self.n_particles,
            "radius": float(self.R.max()) if self.n_particles else 0.0,
            "kappa": self.kappa,
            "E_ext": list(map(float, self.E_ext)),
            "tau": self.tau,
            "mg_levels": self.levels,
            "res_rf": self.res_rf,
        }


def _set_particles(wl: Workload, centres: np.ndarray, R: np.ndarray, kind: np.ndarray,
                   zeta: np.ndarray, q: np.ndarray) -> Workload:
    n = centres.shape[0]
    wl.x = np.ascontiguousarray(centres, dtype=np.float64).reshape(n, 3)
    wl.v = np.zeros((n, 3))
    wl.w = np.zeros((n, 3))
    wl.R = np.ascontiguousarray(R, dtype=np.float64)
    wl.kind = np.ascontiguousarray(kind, dtype=np.int32)
    wl.zeta = np.ascontiguousarray(zeta, dtype=np.float64)
    wl.q = np.ascontiguousarray(q, dtype=np.float64)
    return wl


def place_spheres(n: int, radius: float, dims: Sequence[int], periodic: Sequence[int],
                  rng: PCG32, gap: Optional[float] = None,
                  wall_clearance: Optional[float] = None,
                  max_tries: int = 2000000) -> np.ndarray:
    """Rejection-sample ``n`` sphere centres of equal ``radius``.

    Centre-to-centre distance (minimum image on periodic axes) is at least
    ``gap`` (default 2R+2) and every centre keeps ``wall_clearance`` (default
    R+1) from a non-periodic face.  A uniform cell list keeps the test O(1).
    """
    gap = 2.0 * radius + 2.0 if gap is None else gap
    clear = radius + 1.0 if wall_clearance is None else wall_clearance
    dims = [int(d) for d in dims]
    lo = [0.0 if periodic[a] else clear for a in range(3)]
    hi = [float(dims[a]) if periodic[a] else dims[a] - clear for a in range(3)]
    for a in range(3):
        if hi[a] <= lo[a]:
            raise ValueError("domain too small for the wall clearance")
    ncell = [max(1, int(dims[a] // gap)) for a in range(3)]
    csize = [dims[a] / ncell[a] for a in range(3)]
    grid: Dict[tuple, List[int]] = {}
    pts: List[List[float]] = []
    tries = 0
    g2 = gap * gap
    while len(pts) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError(f"could only place {len(pts)} of {n} spheres")
        c = [rng.uniform_range(lo[a], hi[a]) for a in range(3)]
        ci = [min(ncell[a] - 1, int(c[a] / csize[a])) for a in range(3)]
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    key = []
                    skip = False
                    for a, d in enumerate((dx, dy, dz)):
                        k = ci[a] + d
                        if periodic[a]:
                            k %= ncell[a]
                        elif k < 0 or k >= ncell[a]:
                            skip = True
                        key.append(k)
                    if skip:
                        continue
                    for j in grid.get(tuple(key), ()):
                        d2 = 0.0
                        for a in range(3):
                            dd = c[a] - pts[j][a]
                            if periodic[a]:
                                dd -= dims[a] * round(dd / dims[a])
                            d2 += dd * dd
                        if d2 < g2:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            grid.setdefault(tuple(ci), []).append(len(pts))
            pts.append(c)
    return np.array(pts, dtype=np.float64).reshape(n, 3)


# ---------------------------------------------------------------------------
# The workloads.  Sizes and parameter ranges follow the paper's setups, scaled
# to lattice units with dx = dt = rho_0 = eps = 1.
# ---------------------------------------------------------------------------

def single_sphere(n: int = 32, radius: float = 4.0, zeta: float = 1.0, debye: float = 4.0,
                  E: float = 1e-3, levels: int = 3, steps: int = 100,
                  res_rf: float = 1e-10, centre: Optional[Sequence[float]] = None,
                  dims: Optional[Sequence[int]] = None) -> Workload:
    """One zeta-potential sphere in a periodic box (32^3, R = 4, lambda_D = 4)."""
    dims = list(dims) if dims is not None else [n, n, n]
    wl = Workload(name=f"single_sphere_{dims[0]}x{dims[1]}x{dims[2]}_R{radius:g}",
                  dims=dims, periodic=(1, 1, 1), tau=1.0, kappa=1.0 / debye, eps=1.0,
                  E_ext=(E, 0.0, 0.0), levels=levels, res_rf=res_rf, steps=steps)
    c = np.array([centre if centre is not None else [d / 2.0 for d in dims]], dtype=np.float64)
    return _set_particles(wl, c, np.array([radius]), np.array([KIND_ZETA]),
                          np.array([zeta]), np.array([0.0]))


def channel(n: int = 128, n_spheres: int = 64, radius: float = 6.0, seed: int = 2,
            debye: float = 3.0, E: float = 2e-3, levels: int = 4, steps: int = 1000,
            res_rf: float = 1e-8, dims: Optional[Sequence[int]] = None) -> Workload:
    """Charged spheres in a channel: walls at the two z faces, periodic x and y.

    Surface charges are drawn uniform in [0.5, 1.5] (Neumann condition)."""
    dims = list(dims) if dims is not None else [n, n, n]
    periodic = (1, 1, 0)
    rng = PCG32(seed)
    centres = place_spheres(n_spheres, radius, dims, periodic, rng)
    q = np.array([rng.uniform_range(0.5, 1.5) for _ in range(n_spheres)])
    wl = Workload(name=f"channel_{dims[0]}x{dims[1]}x{dims[2]}_{n_spheres}xR{radius:g}",
                  dims=dims, periodic=periodic, tau=1.0, kappa=1.0 / debye, eps=1.0,
                  E_ext=(E, 0.0, 0.0), levels=levels, res_rf=res_rf, steps=steps)
    return _set_particles(wl, centres, np.full(n_spheres, radius),
                          np.full(n_spheres, KIND_CHARGE), np.zeros(n_spheres), q)


def suspension(n: int = 512, n_spheres: int = 2880, radius: float = 5.0, seed: int = 3,
               debye: float = 4.0, E: float = 1e-3, levels: int = 6, steps: int = 500,
               res_rf: float = 4e-6, dims: Optional[Sequence[int]] = None) -> Workload:
    """Periodic suspension of charged spheres (the per-GPU weak-scaling shape).

    512^3 cells with 2,880 spheres of radius 5, charges drawn N(1, 0.1^2).
    The residual reduction factor is the one of the paper's weak-scaling
    runs, RES_RF = 4e-6 (Sec. 6.5)."""
    dims = list(dims) if dims is not None else [n, n, n]
    periodic = (1, 1, 1)
    rng = PCG32(seed)
    centres = place_spheres(n_spheres, radius, dims, periodic, rng)
    q = np.array([1.0 + 0.1 * rng.normal() for _ in range(n_spheres)])
    # 8 sweeps solve the coarsest level (h = 2^(levels-1), kappa^2 h^2 >> 1,
    # strongly diagonally dominant) to well below the cycle's contraction
    wl = Workload(name=f"suspension_{dims[0]}x{dims[1]}x{dims[2]}_{n_spheres}xR{radius:g}",
                  dims=dims, periodic=periodic, tau=1.0, kappa=1.0 / debye, eps=1.0,
                  E_ext=(E, 0.0, 0.0), levels=levels, res_rf=res_rf, steps=steps, coarse_sweeps=8)
    return _set_particles(wl, centres, np.full(n_spheres, radius),
                          np.full(n_spheres, KIND_CHARGE), np.zeros(n_spheres), q)


def paper_node(blocks: Sequence[int] = (2, 4, 2), block: int = 144, levels: int = 6) -> Workload:
    """The problem of one node in the paper's scaling runs (Sec. 7): blocks of
    144^3 cells, 2 x 4 x 2 of them a node (288 x 576 x 288 cells), each with
    4^3 spheres of radius 6 spaced 36 cells apart, the first centred at
    (19, 19, 19) (1,024 spheres; their obstacle cells cover 1.955 % of the
    domain, the paper's "about 1.95 %").  Periodic in y; no-slip walls with a
    zero-flux potential on the x and z faces; zeta spheres, the field along
    y, 240 steps to RES_RF 4e-6.  Parameters of the scaling runs (Tab.
    ElectrophorValidSpheres_Parameters): lambda_D = 15.08 cells, tau = 6, and
    in units of zeta = 10 mV and dx = 5 nm the field E_y,Sc = 38.0e6 V/m is
    38.0e6 * 5e-9 / 0.01 = 0.019."""
    dims = [block * b for b in blocks]
    c = [19.0 + 36.0 * np.arange(d // 36) for d in dims]
    Z, Y, X = np.meshgrid(c[2], c[1], c[0], indexing="ij")
    centres = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    n = centres.shape[0]
    wl = Workload(name=f"paper_node_{dims[0]}x{dims[1]}x{dims[2]}_{n}xR6", dims=dims, periodic=(0, 1, 0),
                  tau=6.0, kappa=1.0 / 15.08, eps=1.0, E_ext=(0.0, 0.019, 0.0), levels=levels, res_rf=4e-6,
                  steps=240, coarse_sweeps=8)
    return _set_particles(wl, centres, np.full(n, 6.0), np.full(n, KIND_ZETA), np.ones(n), np.zeros(n))


def suspension_sample(n: int, seed: int = 3, radius: float = 5.0, levels: int = 4) -> Workload:
    """A sub-box of the 512^3 suspension with the same sphere number density."""
    n_spheres = max(1, int(round(2880 * (n / 512.0) ** 3)))
    return suspension(n=n, n_spheres=n_spheres, radius=radius, seed=seed, levels=levels)


def mixed_box(dims: Sequence[int] = (40, 24, 32), seed: int = 11, levels: int = 3,
              n_spheres: int = 4, radius: float = 3.5, periodic: Sequence[int] = (1, 1, 0)) -> Workload:
    """Small mixed test case: walls in z, periodic x/y (by default), zeta and
    charge spheres, random initial velocities, non-cubic extents that leave
    ragged thread-block tails."""
    periodic = tuple(periodic)
    rng = PCG32(seed)
    centres = place_spheres(n_spheres, radius, dims, periodic, rng)
    kind = np.array([KIND_ZETA if i % 2 == 0 else KIND_CHARGE for i in range(n_spheres)])
    zeta = np.array([rng.uniform_range(0.5, 2.0) for _ in range(n_spheres)])
    q = np.array([rng.uniform_range(0.5, 1.5) for _ in range(n_spheres)])
    wl = Workload(name=f"mixed_{dims[0]}x{dims[1]}x{dims[2]}", dims=list(dims), periodic=periodic,
                  tau=0.8, kappa=0.3, eps=1.0, E_ext=(2e-3, 1e-3, -5e-4), levels=levels,
                  res_rf=1e-10, steps=20)
    wl = _set_particles(wl, centres, np.full(n_spheres, radius), kind, zeta, q)
    # seeded initial velocities, large enough that spheres cross cell centres
    wl.v = np.array([[rng.uniform_range(-0.05, 0.05) for _ in range(3)] for _ in range(n_spheres)])
    wl.w = np.array([[rng.uniform_range(-0.01, 0.01) for _ in range(3)] for _ in range(n_spheres)])
    return wl


def random_fields(n_cells: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded uniform numbers in [-scale, scale), e.g. for an initial potential."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.random(n_cells) * 2.0 - 1.0) * scale
