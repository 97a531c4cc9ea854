"""Helpers that drive the CUDA library and the FP64 oracle side by side on the
same seeded inputs.  Test infrastructure only."""
import numpy as np

import oracle
import paper_1708_08741_gb300 as es


def direction_map():
    """perm[q_lib] = q_oracle with equal lattice velocity."""
    c, _ = es.lattice()
    co, _ = oracle.lattice()
    return np.array([[k for k in range(19) if (co[k] == c[q]).all()][0] for q in range(19)])


def to_oracle_order(pdf_lib):
    perm = direction_map()
    out = np.empty_like(pdf_lib)
    out[perm] = pdf_lib
    return out


def to_lib_order(pdf_oracle):
    perm = direction_map()
    return pdf_oracle[perm]


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    d = np.linalg.norm(a - b)
    return d / nb if nb > 0 else d


class Pair:
    """A GPU simulation and an oracle simulation of the same workload."""

    def __init__(self, wl, precision=es.ES_FP64, overrides=None, lib_overrides=None, omp=False):
        self.wl = wl
        # (omp: the oracle's OpenMP build, the same bits on all host cores)
        self.o = oracle.Oracle(wl, overrides, omp=omp)
        self.g = es.Simulation(wl, precision, overrides={**(overrides or {}), **(lib_overrides or {})})
        self.x0 = np.array(wl.x, dtype=np.float64).reshape(-1, 3).copy()
        self.last_forces = None

    def step(self, forced=True):
        self.o.map_particles()
        self.g.map_particles()
        info = self.o.solve()
        ginfo = self.g.solve(forced_cycles=info["cycles"] if forced else -1)
        self.o.body_force()
        self.o.lbm_step()
        self.g.lbm_step()
        Fo, To = self.o.forces()
        Fg, Tg = self.g.forces()
        self.o.advance()
        self.g.advance()
        self.last_forces = ((Fo, To), (Fg, Tg))
        return info, ginfo, (Fo, To), (Fg, Tg)

    def displacement(self, x):
        """x - x0 per sphere, by minimum image on periodic axes (a sphere
        that crossed a periodic face is wrapped back into the box)."""
        d = np.asarray(x, dtype=np.float64) - self.x0
        for a in range(3):
            if self.wl.periodic[a]:
                n = float(self.wl.dims[a])
                d[:, a] -= n * np.round(d[:, a] / n)
        return d

    def compare(self):
        """Relative L2 differences of potential (unknown cells), velocity
        (fluid cells) and particle state, plus owner equality.

        x: the absolute positions; "disp": the displacements since the start
        (x - x0, minimum image), the quantity the forces actually move and
        the one a reduced-precision bar must be set on (absolute coordinates
        of 16 to 60 cells hide errors of a few thousandths of a cell).
        F, T: the force and torque of the last step (Pair.step).  A torque
        that vanishes by symmetry (a centred sphere in an axial field) is
        measured against R times the force instead of its own norm."""
        own_o = self.o.owner()
        own_g = self.g.field(es.FIELD_OWNER)
        fluid = own_o < 0
        res = {"owner_equal": bool((own_o == own_g).all())}
        res["psi"] = rel_l2(self.g.field(es.FIELD_PSI)[fluid], self.o.field(oracle.FIELD_PSI)[fluid])
        ug = self.g.field(es.FIELD_U)
        uo = self.o.field(oracle.FIELD_U)
        res["u"] = rel_l2(ug[:, fluid], uo[:, fluid])
        if self.wl.n_particles:
            pg, po = self.g.particles(), self.o.particles()
            res["x"] = rel_l2(pg["x"], po["x"])
            res["disp"] = rel_l2(self.displacement(pg["x"]), self.displacement(po["x"]))
            res["v"] = rel_l2(pg["v"], po["v"]) if np.linalg.norm(po["v"]) > 0 else 0.0
            res["w"] = np.linalg.norm(pg["w"] - po["w"]) / max(np.linalg.norm(po["w"]), 1e-300)
            if self.last_forces is not None:
                (Fo, To), (Fg, Tg) = self.last_forces
                res["F"] = rel_l2(Fg, Fo)
                arm = float(np.mean(self.wl.R)) * np.linalg.norm(Fo)
                nT = np.linalg.norm(To)
                res["T"] = float(np.linalg.norm(np.asarray(Tg) - np.asarray(To)) /
                                 (nT if nT > 1e-6 * arm else max(arm, 1e-300)))
        return res
