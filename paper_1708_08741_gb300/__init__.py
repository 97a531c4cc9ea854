"""GB300-native coupled electrophoresis step (Bartuschat & Ruede, arXiv 1708.08741).

This package is a thin ctypes binding of ``libes.so`` (C ABI in
``include/es.h``): the functions here marshal arguments and call the
library, where every step of the time step runs as a CUDA kernel.  PyTorch
supplies the device memory (through the allocator hook of
``es_create_with_allocator``) and the CUDA stream.  There is no CPU
fallback: without the built library every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional, Tuple

import numpy as np

from . import workloads  # noqa: F401  (seeded inputs; no method arithmetic)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libes.so")

ES_OK = 0
ES_EINVAL = -1
ES_ENOMEM = -2
ES_ECUDA = -3
ES_ENOTCONVERGED = -4
ES_ENAN = -5
ES_EOVERLAP = -6
ES_ETIMEOUT = -7

ES_FP64 = 0
ES_MIXED32 = 1
ES_MIXED16 = 2
ES_SMOOTH_TWO_PASS = 0
ES_SMOOTH_FUSED = 1
ES_MG_NATIVE = 0
ES_MG_FP16 = 1
ES_LAYOUT_AUTO = 0
ES_LAYOUT_NATURAL = 1
ES_STAGE_REGISTERS = 0
ES_STAGE_BULK = 1

FIELD_PSI = 0
FIELD_RHO = 1
FIELD_U = 2
FIELD_FB = 3
FIELD_PDF = 4
FIELD_OWNER = 5
FIELD_FLAGS = 6
FIELD_PDF_LAST = 7

# the functions include/es.h declares
EXPORTED = ("es_create", "es_create_with_allocator", "es_destroy", "es_map_particles", "es_potential_solve",
            "es_lbm_step", "es_forces", "es_advance", "es_step", "es_get_field", "es_set_field",
            "es_get_particles", "es_set_particles", "es_set_forces", "es_synchronize", "es_lattice", "es_gather",
            "es_gather_noalloc",
            "es_device_bytes", "es_kernel_launches", "es_last_error", "es_profile_start", "es_profile_stop",
            "es_alu_peak", "es_lbm_step_batch")


class Params(ctypes.Structure):
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
        ("precision", ctypes.c_int),
        ("levels", ctypes.c_int),
        ("nu1", ctypes.c_int),
        ("nu2", ctypes.c_int),
        ("coarse_sweeps", ctypes.c_int),
        ("omega", ctypes.c_double),
        ("res_rf", ctypes.c_double),
        ("max_cycles", ctypes.c_int),
        ("smoother", ctypes.c_int),
        ("mg_storage", ctypes.c_int),
        ("wall_slip", ctypes.c_int * 6),
        ("phi_t", ctypes.c_double),
        ("fine_layout", ctypes.c_int),
        ("near_list_cells", ctypes.c_int),
        ("sweep_staging", ctypes.c_int),
        ("lbm_block", ctypes.c_int * 2),
        ("fast_update_cells", ctypes.c_int),
    ]


class Particle(ctypes.Structure):
    _fields_ = [
        ("x", ctypes.c_double * 3),
        ("v", ctypes.c_double * 3),
        ("w", ctypes.c_double * 3),
        ("R", ctypes.c_double),
        ("kind", ctypes.c_int),
        ("zeta", ctypes.c_double),
        ("q", ctypes.c_double),
    ]


class SolveInfo(ctypes.Structure):
    _fields_ = [
        ("cycles", ctypes.c_int),
        ("r_initial", ctypes.c_double),
        ("r_final", ctypes.c_double),
        ("tol", ctypes.c_double),
    ]


class KernelTime(ctypes.Structure):
    _fields_ = [
        ("name", ctypes.c_char * 32),
        ("level", ctypes.c_int),
        ("launches", ctypes.c_int),
        ("ms", ctypes.c_double),
        ("bytes", ctypes.c_double),
    ]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lib = None


class EsError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where} failed ({code}): {msg}")
        self.code = code


def load():
    """Loads the in-tree libes.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(or python -m paper_1708_08741_gb300.build); there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    L.es_create.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(Particle), ctypes.c_int, P, ctypes.POINTER(P)]
    L.es_create_with_allocator.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(Particle), ctypes.c_int, P,
                                           ALLOC_FN, FREE_FN, P, ctypes.POINTER(P)]
    L.es_destroy.argtypes = [P]
    L.es_map_particles.argtypes = [P]
    L.es_potential_solve.argtypes = [P, ctypes.c_int, ctypes.POINTER(SolveInfo)]
    L.es_lbm_step.argtypes = [P]
    L.es_forces.argtypes = [P, P, P, ctypes.c_int]
    L.es_advance.argtypes = [P]
    L.es_step.argtypes = [P, ctypes.c_int, ctypes.POINTER(SolveInfo)]
    L.es_get_field.argtypes = [P, ctypes.c_int, P, ctypes.c_size_t, ctypes.c_int]
    L.es_set_field.argtypes = [P, ctypes.c_int, P, ctypes.c_size_t, ctypes.c_int]
    L.es_gather.argtypes = [P, ctypes.c_int, P, ctypes.c_int, P]
    L.es_gather_noalloc.argtypes = [P, ctypes.c_int, P, ctypes.c_int, P]
    L.es_get_particles.argtypes = [P, ctypes.POINTER(Particle), ctypes.c_int]
    L.es_set_particles.argtypes = [P, ctypes.POINTER(Particle), ctypes.c_int]
    L.es_set_forces.argtypes = [P, P, P, ctypes.c_int]
    L.es_synchronize.argtypes = [P]
    L.es_lattice.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    L.es_kernel_launches.argtypes = [P]
    L.es_kernel_launches.restype = ctypes.c_uint64
    L.es_device_bytes.argtypes = [ctypes.POINTER(Params), ctypes.c_int]
    L.es_device_bytes.restype = ctypes.c_size_t
    L.es_profile_start.argtypes = [P]
    L.es_profile_stop.argtypes = [P, ctypes.POINTER(KernelTime), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.es_alu_peak.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    L.es_lbm_step_batch.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]
    L.es_last_error.argtypes = [P]
    L.es_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def alu_peak(precision: int = ES_FP64) -> float:
    """Measured FMA throughput of the current device in GFLOP/s (es_alu_peak)."""
    v = ctypes.c_double(0.0)
    rc = load().es_alu_peak(precision, ctypes.byref(v))
    if rc != ES_OK:
        raise EsError(rc, "es_alu_peak", "FMA probe failed")
    return v.value


def lattice() -> Tuple[np.ndarray, np.ndarray]:
    """The library's own D3Q19 velocity (19 x 3) and weight tables."""
    c = (ctypes.c_int * 57)()
    w = (ctypes.c_double * 19)()
    load().es_lattice(c, w)
    return np.array(c[:], dtype=np.int32).reshape(19, 3), np.array(w[:])


def make_params(wl, precision: int = ES_FP64, overrides: Optional[dict] = None) -> Params:
    P = Params()
    d = dict(dims=wl.dims, periodic=wl.periodic, pot_bc=wl.pot_bc, pot_val=wl.pot_val, tau=wl.tau,
             kappa=wl.kappa, eps=wl.eps, E_ext=wl.E_ext, accel=wl.accel, rho_p_ratio=wl.rho_p_ratio,
             precision=precision, levels=wl.levels, nu1=wl.nu1, nu2=wl.nu2, coarse_sweeps=wl.coarse_sweeps,
             omega=wl.omega, res_rf=wl.res_rf, max_cycles=wl.max_cycles, wall_slip=wl.wall_slip,
             phi_t=wl.phi_t)
    if overrides:
        d.update(overrides)
    for k, v in d.items():
        f = getattr(P, k)
        if isinstance(f, ctypes.Array):
            for i, x in enumerate(v):
                f[i] = x
        else:
            setattr(P, k, v)
    return P


def pack_particles(x, v, w, R, kind, zeta, q):
    n = len(R)
    arr = (Particle * max(1, n))()
    for i in range(n):
        for a in range(3):
            arr[i].x[a] = float(x[i][a])
            arr[i].v[a] = float(v[i][a])
            arr[i].w[a] = float(w[i][a])
        arr[i].R = float(R[i])
        arr[i].kind = int(kind[i])
        arr[i].zeta = float(zeta[i])
        arr[i].q = float(q[i])
    return arr


class TorchAllocator:
    """Device memory for a context from PyTorch's caching allocator."""

    def __init__(self, device):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        self.blocks: Dict[int, object] = {}
        self.c_alloc = ALLOC_FN(self._alloc)
        self.c_free = FREE_FN(self._free)

    def _alloc(self, nbytes, user):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
        except RuntimeError:
            return None
        p = t.data_ptr()
        self.blocks[p] = t
        return p

    def _free(self, ptr, user):
        self.blocks.pop(int(ptr) if ptr else 0, None)


class Simulation:
    """One coupled electrophoresis simulation resident on a GPU."""

    _COMPONENTS = {FIELD_U: 3, FIELD_FB: 3, FIELD_PDF: 19, FIELD_PDF_LAST: 19}

    def __init__(self, wl, precision: int = ES_FP64, device: str = "cuda:0", stream=None,
                 overrides: Optional[dict] = None, torch_memory: bool = True):
        import torch

        self.lib = load()
        self.wl = wl
        self.device = torch.device(device)
        self.precision = precision
        self.params = make_params(wl, precision, overrides)
        self.np = wl.n_particles
        self.dims = tuple(int(d) for d in wl.dims)
        self.N = self.dims[0] * self.dims[1] * self.dims[2]
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            parts = pack_particles(wl.x, wl.v, wl.w, wl.R, wl.kind, wl.zeta, wl.q)
            h = ctypes.c_void_p()
            if torch_memory:
                # blocks are taken on the context's stream, so that the
                # caching allocator orders their reuse after its work
                self.allocator = TorchAllocator(self.device)
                with torch.cuda.stream(self.stream):
                    rc = self.lib.es_create_with_allocator(ctypes.byref(self.params), parts, self.np,
                                                           ctypes.c_void_p(self.stream.cuda_stream),
                                                           self.allocator.c_alloc, self.allocator.c_free, None,
                                                           ctypes.byref(h))
            else:
                self.allocator = None
                rc = self.lib.es_create(ctypes.byref(self.params), parts, self.np,
                                        ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if rc != ES_OK:
            raise EsError(rc, "es_create", self.lib.es_last_error(None).decode())
        self.h = h

    # -- errors --
    def _check(self, rc, where):
        if rc != ES_OK:
            raise EsError(rc, where, self.lib.es_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.es_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- Algorithm 1 --
    def map_particles(self):
        self._check(self.lib.es_map_particles(self.h), "es_map_particles")

    def solve(self, forced_cycles: int = -1, check: bool = True) -> dict:
        info = SolveInfo()
        rc = self.lib.es_potential_solve(self.h, forced_cycles, ctypes.byref(info))
        if check:
            self._check(rc, "es_potential_solve")
        return {"cycles": info.cycles, "r0": info.r_initial, "r": info.r_final, "tol": info.tol, "status": rc}

    def lbm_step(self):
        self._check(self.lib.es_lbm_step(self.h), "es_lbm_step")

    def forces(self) -> Tuple[np.ndarray, np.ndarray]:
        F = np.zeros(3 * max(1, self.np))
        T = np.zeros(3 * max(1, self.np))
        self._check(self.lib.es_forces(self.h, F.ctypes.data, T.ctypes.data, 0), "es_forces")
        return F[: 3 * self.np].reshape(-1, 3), T[: 3 * self.np].reshape(-1, 3)

    def forces_device(self, F_ptr: int = 0, T_ptr: int = 0):
        self._check(self.lib.es_forces(self.h, F_ptr or None, T_ptr or None, 1), "es_forces")

    def advance(self):
        self._check(self.lib.es_advance(self.h), "es_advance")

    def step(self, forced_cycles: int = -1) -> dict:
        info = SolveInfo()
        self._check(self.lib.es_step(self.h, forced_cycles, ctypes.byref(info)), "es_step")
        return {"cycles": info.cycles, "r0": info.r_initial, "r": info.r_final, "tol": info.tol}

    def profile_start(self):
        """Start bracketing the grid-sized kernel launches with CUDA events."""
        self._check(self.lib.es_profile_start(self.h), "es_profile_start")

    def profile_stop(self) -> list:
        """Stop profiling; per kernel and level: launches, summed device ms and
        summed algorithmic bytes."""
        cap = 64
        arr = (KernelTime * cap)()
        n = ctypes.c_int(0)
        self._check(self.lib.es_profile_stop(self.h, arr, cap, ctypes.byref(n)), "es_profile_stop")
        return [{"name": arr[i].name.decode(), "level": arr[i].level, "launches": arr[i].launches,
                 "ms": arr[i].ms, "bytes": arr[i].bytes} for i in range(min(n.value, cap))]

    def kernel_launches(self) -> int:
        return int(self.lib.es_kernel_launches(self.h))

    def synchronize(self):
        self._check(self.lib.es_synchronize(self.h), "es_synchronize")

    # -- fields --
    def field(self, which: int) -> np.ndarray:
        nx, ny, nz = self.dims
        if which == FIELD_OWNER:
            out = np.zeros(self.N, dtype=np.int32)
        elif which == FIELD_FLAGS:
            out = np.zeros(self.N, dtype=np.uint8)
        else:
            out = np.zeros(self._COMPONENTS.get(which, 1) * self.N)
        self._check(self.lib.es_get_field(self.h, which, out.ctypes.data, out.nbytes, 0), "es_get_field")
        comps = self._COMPONENTS.get(which, 1)
        return out.reshape(nz, ny, nx) if comps == 1 else out.reshape(comps, nz, ny, nx)

    def field_device(self, which: int, out) -> None:
        """Copies a field into a CUDA tensor (dtype float64 / int32 / uint8)."""
        self._check(self.lib.es_get_field(self.h, which, out.data_ptr(), out.numel() * out.element_size(), 1),
                    "es_get_field")

    def gather(self, which: int, cells: np.ndarray) -> np.ndarray:
        """Field values at the given linear cell indices, shape (components, n)."""
        idx = np.ascontiguousarray(cells, dtype=np.int64).ravel()
        comps = self._COMPONENTS.get(which, 1)
        out = np.zeros(comps * idx.size)
        self._check(self.lib.es_gather(self.h, which, idx.ctypes.data, idx.size, out.ctypes.data), "es_gather")
        return out.reshape(comps, idx.size)

    def set_field(self, which: int, values: np.ndarray):
        v = np.ascontiguousarray(values, dtype=np.float64).ravel()
        self._check(self.lib.es_set_field(self.h, which, v.ctypes.data, v.nbytes, 0), "es_set_field")

    def particles(self) -> dict:
        arr = (Particle * max(1, self.np))()
        self._check(self.lib.es_get_particles(self.h, arr, self.np), "es_get_particles")
        return {k: np.array([list(getattr(arr[i], k)) for i in range(self.np)]).reshape(-1, 3) for k in ("x", "v", "w")}

    def set_particles(self, x, v, w):
        wl = self.wl
        arr = pack_particles(x, v, w, wl.R, wl.kind, wl.zeta, wl.q)
        self._check(self.lib.es_set_particles(self.h, arr, self.np), "es_set_particles")

    def set_forces(self, F, T):
        F = np.ascontiguousarray(F, dtype=np.float64).ravel()
        T = np.ascontiguousarray(T, dtype=np.float64).ravel()
        self._check(self.lib.es_set_forces(self.h, F.ctypes.data, T.ctypes.data, self.np), "es_set_forces")


def lbm_step_batch(sims) -> None:
    """One stream-collide step of every simulation in one launch
    (es_lbm_step_batch); the same result as sim.lbm_step() on each."""
    sims = list(sims)
    arr = (ctypes.c_void_p * len(sims))(*[s.h.value for s in sims])
    rc = load().es_lbm_step_batch(arr, len(sims))
    if rc != ES_OK:
        raise EsError(rc, "es_lbm_step_batch", load().es_last_error(sims[0].h if sims else None).decode())


def device_bytes(wl, precision: int = ES_FP64, overrides: Optional[dict] = None) -> int:
    return int(load().es_device_bytes(ctypes.byref(make_params(wl, precision, overrides)), wl.n_particles))
