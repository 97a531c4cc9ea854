"""The C-ABI library builds, loads without a GPU, exports every function that
include/es.h declares, and validates parameters before touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_1708_08741_gb300 as es
from paper_1708_08741_gb300 import build as es_build
from paper_1708_08741_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    es_build.build()
    return es.load()


def declared_functions():
    with open(os.path.join(ROOT, "include", "es.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(es_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_function(lib):
    names = declared_functions()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(es.EXPORTED)


def test_lattice_is_the_oracle_lattice_up_to_order(lib):
    c, w = es.lattice()
    co, wo = oracle.lattice()
    lib_set = {(tuple(c[q]), round(w[q], 15)) for q in range(19)}
    or_set = {(tuple(co[q]), round(wo[q], 15)) for q in range(19)}
    assert lib_set == or_set
    # opposite pairs q / q+9 of the library's order
    for q in range(1, 10):
        assert (c[q] == -c[q + 9]).all()


def _create_rc(lib, wl, **over):
    P = es.make_params(wl, es.ES_FP64, over)
    parts = es.pack_particles(wl.x, wl.v, wl.w, wl.R, wl.kind, wl.zeta, wl.q)
    h = ctypes.c_void_p()
    rc = lib.es_create(ctypes.byref(P), parts, wl.n_particles, None, ctypes.byref(h))
    return rc, lib.es_last_error(None).decode()


@pytest.mark.parametrize("over,needle", [
    (dict(tau=0.5), "tau"),
    (dict(levels=13), "levels"),
    (dict(levels=7), "multiples"),
    (dict(levels=6), "even"),
    (dict(precision=7), "precision"),
    (dict(omega=2.0), "omega"),
    (dict(eps=0.0), "eps"),
    (dict(smoother=2), "smoother"),
    (dict(mg_storage=2), "mg_storage"),
    (dict(mg_storage=1), "reduced precision"),  # (the helper creates FP64 contexts)
    (dict(phi_t=-1.0), "phi_t"),
    (dict(phi_t=0.5, levels=2), "levels == 1"),
    (dict(fine_layout=2), "fine_layout"),
    (dict(near_list_cells=-1), "near_list_cells"),
    (dict(lbm_block=(48, 1)), "lbm_block"),
    (dict(sweep_staging=2), "sweep_staging"),
    (dict(lbm_block=(128, 4)), "lbm_block"),
    (dict(fast_update_cells=-5), "fast_update_cells"),
])
def test_invalid_parameters_rejected_before_any_gpu_call(lib, over, needle):
    rc, msg = _create_rc(lib, W.single_sphere(), **over)
    assert rc == es.ES_EINVAL and needle in msg


def test_invalid_particles_rejected(lib):
    wl = W.single_sphere(n=16, radius=7.5, levels=1)
    rc, msg = _create_rc(lib, wl)
    assert rc == es.ES_EINVAL and "too large" in msg
    wl2 = W.single_sphere()
    wl2.kind = np.array([5], dtype=np.int32)
    rc, msg = _create_rc(lib, wl2)
    assert rc == es.ES_EINVAL


def test_device_bytes_matches_layout(lib):
    wl = W.suspension(n=512, n_spheres=1, levels=6)
    b16 = es.device_bytes(wl, es.ES_MIXED16)
    b32 = es.device_bytes(wl, es.ES_MIXED32)
    b64 = es.device_bytes(wl, es.ES_FP64)
    N = 512 ** 3
    # two PDF fields dominate: 2 x 19 x s_pdf bytes per cell; the rest is the
    # body force (3s), psi (8: FP64 or float-float), owner and flags (5), the
    # list of fluid cells next to obstacles (4) and, per multigrid cell (x 8/7
    # levels), three s-byte fields, a state byte and a 4-byte near-cell list
    # entry, with s the arithmetic type (4 in both reduced forms); the reduced
    # forms' colour-split finest level adds its update masks (1/8 byte a cell)
    rest32 = (3 * 4 + 8 + 5 + 4 + (3 * 4 + 1 + 4) * 8 / 7 + 0.125) * N
    rest64 = (3 * 8 + 8 + 5 + 4 + (3 * 8 + 1 + 4) * 8 / 7) * N
    assert 2 * 19 * 2 * N + rest32 < b16 < 2 * 19 * 2 * N + rest32 + 0.1 * N
    assert 2 * 19 * 4 * N + rest32 < b32 < 2 * 19 * 4 * N + rest32 + 0.1 * N
    assert 2 * 19 * 8 * N + rest64 < b64 < 2 * 19 * 8 * N + rest64 + 0.1 * N
    # FP16 storage of the finest level's correction: 2 bytes a cell less
    b32h = es.device_bytes(wl, es.ES_MIXED32, dict(mg_storage=es.ES_MG_FP16))
    # (and the colour-split layout, with the masks of levels 0 and 1 and the
    # scratch of the local correction at a solve's start, 4 x 16 x 19^3 words,
    # is off under FP16 storage)
    assert b32 - b32h == (2 * N + 2 * 512 * 512 * (512 // 64) * 4 + 2 * 256 * 256 * (256 // 64) * 4
                          + 4 * 16 * 19 ** 3 * 4 + 1024)
