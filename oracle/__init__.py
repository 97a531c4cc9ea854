"""Python handle on the plain FP64 CPU oracle (``es_oracle.c``).

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library and
its Python binding never do, and this package imports nothing from them.

The oracle follows Algorithm 1 of the paper (Sec. 5.7) step by step in double
precision; see ``es_oracle.c`` for the section and equation each function
implements and for the readings taken where the paper is silent or garbled.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "es_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libesoracle.so")

OR_OK = 0
OR_EINVAL = -1
OR_ENOMEM = -2
OR_ENOTCONVERGED = -4
OR_ENAN = -5
OR_EOVERLAP = -6

FIELD_PSI = 0
FIELD_RHO = 1
FIELD_U = 2
FIELD_FB = 3
FIELD_PDF = 4
FIELD_B = 5
FIELD_DIAG = 6
FIELD_PDF_LAST = 7


_LIB_OMP = os.path.join(_HERE, "_build", "libesoracle_omp.so")


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle with gcc -O3 (no FMA contraction, so that decisions
    taken in floating point, such as the cell-in-sphere test, are
    reproducible).  omp: the same source with OpenMP, a separate library used
    only to time the oracle on all host cores (same results bit for bit)."""
    target = _LIB_OMP if omp else _LIB
    os.makedirs(os.path.dirname(target), exist_ok=True)
    if force or not os.path.exists(target) or os.path.getmtime(target) < os.path.getmtime(_SRC):
        tmp = target + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O3", "-std=c99", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fPIC"]
        cmd += ["-fopenmp"] if omp else []
        cmd += ["-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, target)
    return target


class OrParams(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_int * 3),
        ("periodic", ctypes.c_int * 3),
        ("pot_bc", ctypes.c_int * 6),
        ("pot_val", ctypes.c_double * 6),
        ("tau", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("E_ext", ctypes.c_double * 3),
        ("accel", ctypes.c_double * 3),
        ("rho_p_ratio", ctypes.c_double),
        ("levels", ctypes.c_int),
        ("nu1", ctypes.c_int),
        ("nu2", ctypes.c_int),
        ("coarse_sweeps", ctypes.c_int),
        ("omega", ctypes.c_double),
        ("res_rf", ctypes.c_double),
        ("max_cycles", ctypes.c_int),
        ("wall_slip", ctypes.c_int * 6),
        ("phi_t", ctypes.c_double),
    ]


class OrParticle(ctypes.Structure):
    _fields_ = [
        ("x", ctypes.c_double * 3),
        ("v", ctypes.c_double * 3),
        ("w", ctypes.c_double * 3),
        ("R", ctypes.c_double),
        ("kind", ctypes.c_int),
        ("zeta", ctypes.c_double),
        ("q", ctypes.c_double),
    ]


_libs = {}


def lib(omp: bool = False):
    """The oracle library (serial), or its OpenMP build."""
    if omp not in _libs:
        path = build(omp=omp)
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.or_create.argtypes = [ctypes.POINTER(OrParams), ctypes.POINTER(OrParticle), ctypes.c_int,
                                ctypes.POINTER(P)]
        L.or_destroy.argtypes = [P]
        for name in ("or_map", "or_body_force", "or_lbm", "or_advance"):
            getattr(L, name).argtypes = [P]
        L.or_solve.argtypes = [P, ctypes.c_int, dp]
        L.or_forces.argtypes = [P, dp, dp]
        L.or_get_field.argtypes = [P, ctypes.c_int, dp]
        L.or_set_field.argtypes = [P, ctypes.c_int, dp]
        L.or_get_owner.argtypes = [P, ip]
        L.or_get_nfaces.argtypes = [P, ip]
        L.or_get_particles.argtypes = [P, ctypes.POINTER(OrParticle)]
        L.or_set_particles.argtypes = [P, ctypes.POINTER(OrParticle)]
        L.or_lattice.argtypes = [ip, dp]
        L.or_vcycle.argtypes = [P, dp, dp]
        L.or_residual.argtypes = [P, dp]
        L.or_residual.restype = ctypes.c_double
        L.or_smooth.argtypes = [P, dp, dp, ctypes.c_int, dp]
        L.or_gradient.argtypes = [P, dp]
        L.or_set_forces.argtypes = [P, dp, dp]
        L.or_tolerance.argtypes = [P]
        L.or_tolerance.restype = ctypes.c_double
        L.or_num_cells.argtypes = [P]
        L.or_num_cells.restype = ctypes.c_long
        L.or_threads.argtypes = []
        L.or_threads.restype = ctypes.c_int
        L.or_q_from_zeta.argtypes = [ctypes.c_double] * 4
        L.or_q_from_zeta.restype = ctypes.c_double
        _libs[omp] = L
    return _libs[omp]


def threads(omp: bool = False) -> int:
    """Threads the oracle's shared-out loops run on (1 for the serial build)."""
    return int(lib(omp).or_threads())


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def lattice() -> Tuple[np.ndarray, np.ndarray]:
    """The oracle's own D3Q19 velocity (19x3) and weight tables."""
    c = np.zeros(57, dtype=np.int32)
    w = np.zeros(19)
    lib().or_lattice(_iptr(c), _dptr(w))
    return c.reshape(19, 3), w


def q_from_zeta(R: float, zeta: float, kappa: float, eps: float) -> float:
    return lib().or_q_from_zeta(R, zeta, kappa, eps)


class OracleError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"oracle {where} returned {code}")
        self.code = code


class Oracle:
    """One oracle simulation; mirrors the C-ABI call sequence of the library."""

    def __init__(self, wl, params_override: Optional[dict] = None, omp: bool = False):
        self.wl = wl
        self.L = lib(omp)
        P = OrParams()
        d = dict(dims=wl.dims, periodic=wl.periodic, pot_bc=wl.pot_bc, pot_val=wl.pot_val,
                 tau=wl.tau, kappa=wl.kappa, eps=wl.eps, E_ext=wl.E_ext, accel=wl.accel,
                 rho_p_ratio=wl.rho_p_ratio, levels=wl.levels, nu1=wl.nu1, nu2=wl.nu2,
                 coarse_sweeps=wl.coarse_sweeps, omega=wl.omega, res_rf=wl.res_rf,
                 max_cycles=wl.max_cycles, wall_slip=wl.wall_slip, phi_t=wl.phi_t)
        if params_override:
            d.update(params_override)
        for k, v in d.items():
            f = getattr(P, k)
            if isinstance(f, ctypes.Array):
                for i, x in enumerate(v):
                    f[i] = x
            else:
                setattr(P, k, v)
        self.params = P
        self.np = wl.n_particles
        parts = self._pack(wl.x, wl.v, wl.w, wl.R, wl.kind, wl.zeta, wl.q)
        h = ctypes.c_void_p()
        rc = self.L.or_create(ctypes.byref(P), parts, self.np, ctypes.byref(h))
        if rc != OR_OK:
            raise OracleError(rc, "or_create")
        self.h = h
        self.N = int(self.L.or_num_cells(h))
        self.dims = tuple(int(x) for x in wl.dims)

    def _pack(self, x, v, w, R, kind, zeta, q):
        arr = (OrParticle * max(1, len(R)))()
        for i in range(len(R)):
            for a in range(3):
                arr[i].x[a] = x[i][a]
                arr[i].v[a] = v[i][a]
                arr[i].w[a] = w[i][a]
            arr[i].R = R[i]
            arr[i].kind = int(kind[i])
            arr[i].zeta = zeta[i]
            arr[i].q = q[i]
        return arr

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            self.L.or_destroy(h)
            self.h = None

    def _check(self, rc, where):
        if rc != OR_OK:
            raise OracleError(rc, where)

    # --- Algorithm 1 steps ---
    def map_particles(self):
        self._check(self.L.or_map(self.h), "or_map")

    def solve(self, forced_cycles: int = -1, check: bool = True):
        info = np.zeros(4)
        rc = self.L.or_solve(self.h, forced_cycles, _dptr(info))
        if check:
            self._check(rc, "or_solve")
        return {"cycles": int(info[0]), "r0": info[1], "r": info[2], "tol": info[3], "status": rc}

    def body_force(self):
        self._check(self.L.or_body_force(self.h), "or_body_force")

    def lbm_step(self):
        self._check(self.L.or_lbm(self.h), "or_lbm")

    def forces(self):
        F = np.zeros(3 * max(1, self.np))
        T = np.zeros(3 * max(1, self.np))
        self._check(self.L.or_forces(self.h, _dptr(F), _dptr(T)), "or_forces")
        return F[: 3 * self.np].reshape(-1, 3), T[: 3 * self.np].reshape(-1, 3)

    def advance(self):
        self._check(self.L.or_advance(self.h), "or_advance")

    def step(self, forced_cycles: int = -1):
        self.map_particles()
        info = self.solve(forced_cycles)
        self.body_force()
        self.lbm_step()
        F, T = self.forces()
        self.advance()
        return info, F, T

    # --- accessors ---
    def field(self, which: int) -> np.ndarray:
        comps = {FIELD_U: 3, FIELD_FB: 3, FIELD_PDF: 19, FIELD_PDF_LAST: 19}.get(which, 1)
        out = np.zeros(comps * self.N)
        self._check(self.L.or_get_field(self.h, which, _dptr(out)), "or_get_field")
        nx, ny, nz = self.dims
        if comps == 1:
            return out.reshape(nz, ny, nx)
        return out.reshape(comps, nz, ny, nx)

    def set_field(self, which: int, values: np.ndarray):
        v = np.ascontiguousarray(values, dtype=np.float64).ravel()
        self._check(self.L.or_set_field(self.h, which, _dptr(v)), "or_set_field")

    def owner(self) -> np.ndarray:
        out = np.zeros(self.N, dtype=np.int32)
        self.L.or_get_owner(self.h, _iptr(out))
        nx, ny, nz = self.dims
        return out.reshape(nz, ny, nx)

    def nfaces(self) -> np.ndarray:
        out = np.zeros(max(1, self.np), dtype=np.int32)
        self.L.or_get_nfaces(self.h, _iptr(out))
        return out[: self.np]

    def particles(self) -> dict:
        arr = (OrParticle * max(1, self.np))()
        self.L.or_get_particles(self.h, arr)
        return {
            "x": np.array([list(arr[i].x) for i in range(self.np)]).reshape(-1, 3),
            "v": np.array([list(arr[i].v) for i in range(self.np)]).reshape(-1, 3),
            "w": np.array([list(arr[i].w) for i in range(self.np)]).reshape(-1, 3),
        }

    def set_particles(self, x, v, w):
        wl = self.wl
        arr = self._pack(x, v, w, wl.R, wl.kind, wl.zeta, wl.q)
        self.L.or_set_particles(self.h, arr)

    def set_forces(self, F, T):
        F = np.ascontiguousarray(F, dtype=np.float64).ravel()
        T = np.ascontiguousarray(T, dtype=np.float64).ravel()
        self.L.or_set_forces(self.h, _dptr(F), _dptr(T))

    def vcycle(self, rhs: np.ndarray) -> np.ndarray:
        r = np.ascontiguousarray(rhs, dtype=np.float64).ravel()
        e = np.zeros(self.N)
        self.L.or_vcycle(self.h, _dptr(r), _dptr(e))
        return e.reshape(self.dims[::-1])

    def smooth(self, rhs: np.ndarray, e0: np.ndarray, sweeps: int) -> np.ndarray:
        r = np.ascontiguousarray(rhs, dtype=np.float64).ravel()
        e_in = np.ascontiguousarray(e0, dtype=np.float64).ravel()
        e = np.zeros(self.N)
        self.L.or_smooth(self.h, _dptr(r), _dptr(e_in), sweeps, _dptr(e))
        return e.reshape(self.dims[::-1])

    def residual(self) -> Tuple[float, np.ndarray]:
        r = np.zeros(self.N)
        n = self.L.or_residual(self.h, _dptr(r))
        return n, r.reshape(self.dims[::-1])

    def gradient(self) -> np.ndarray:
        g = np.zeros(3 * self.N)
        self.L.or_gradient(self.h, _dptr(g))
        nx, ny, nz = self.dims
        return g.reshape(3, nz, ny, nx)

    def tolerance(self) -> float:
        return self.L.or_tolerance(self.h)
