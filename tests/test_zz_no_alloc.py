"""es_gather_noalloc, the allocation-free variant of es_gather, gives the same
values as es_gather through the C ABI, on two calls in a row.  It serves
callers that must not allocate device memory when they read values back (a
real-time loop that cannot wait on an allocator, or an application that
hands out all device memory up front).  This file is collected last so that
a run stopping at its first failure has run everything else."""
import numpy as np
import pytest

import paper_1708_08741_gb300 as es
from paper_1708_08741_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the FP64 parity tolerance of the other GPU tests
FIELDS = (es.FIELD_PSI, es.FIELD_RHO, es.FIELD_U, es.FIELD_FB, es.FIELD_PDF, es.FIELD_PDF_LAST, es.FIELD_OWNER,
          es.FIELD_FLAGS)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_08741_gb300 import build

    build.build()


def _noalloc(sim, which, cells):
    idx = np.ascontiguousarray(cells, dtype=np.int64)
    comps = {es.FIELD_U: 3, es.FIELD_FB: 3, es.FIELD_PDF: 19, es.FIELD_PDF_LAST: 19}.get(which, 1)
    out = np.zeros(comps * max(idx.size, 1))
    rc = sim.lib.es_gather_noalloc(sim.h, which, idx.ctypes.data, idx.size, out.ctypes.data)
    return rc, out[: comps * idx.size].reshape(comps, idx.size)


@pytest.mark.parametrize("precision", [es.ES_FP64, es.ES_MIXED32])
def test_noalloc_gather_matches_gather_on_two_calls(precision):
    sim = es.Simulation(W.mixed_box(), precision)
    for _ in range(2):
        sim.step()
    rng = np.random.Generator(np.random.PCG64(21))
    for n in (1000, 4096):
        cells = rng.integers(0, sim.N, n)
        for which in FIELDS:
            ref = sim.gather(which, cells)
            for _ in range(2):
                rc, got = _noalloc(sim, which, cells)
                assert rc == es.ES_OK
                np.testing.assert_allclose(got, ref, rtol=TOL, atol=0.0)
        sim.step()
    sim.close()


def test_noalloc_gather_rejects_bad_arguments():
    """Each of these is refused with ES_EINVAL by the host-side checks it
    shares with es_gather, before any device work: more than the maximum,
    n = 0, a cell index outside the grid, an unknown field, and the
    populations of the last LBM step before there was one."""
    sim = es.Simulation(W.single_sphere(n=16, radius=3.0, levels=2))
    rc, _ = _noalloc(sim, es.FIELD_PSI, np.zeros(4097, dtype=np.int64))
    assert rc == es.ES_EINVAL
    assert b"4096" in sim.lib.es_last_error(sim.h)
    rc, _ = _noalloc(sim, es.FIELD_PSI, np.zeros(0, dtype=np.int64))
    assert rc == es.ES_EINVAL
    rc, _ = _noalloc(sim, es.FIELD_PSI, np.array([0, sim.N], dtype=np.int64))
    assert rc == es.ES_EINVAL and b"out of range" in sim.lib.es_last_error(sim.h)
    rc, _ = _noalloc(sim, 8, np.zeros(1, dtype=np.int64))
    assert rc == es.ES_EINVAL and b"unknown field" in sim.lib.es_last_error(sim.h)
    rc, _ = _noalloc(sim, es.FIELD_PDF_LAST, np.zeros(1, dtype=np.int64))
    assert rc == es.ES_EINVAL and b"no LBM step" in sim.lib.es_last_error(sim.h)
    rc, out = _noalloc(sim, es.FIELD_PSI, np.zeros(1, dtype=np.int64))
    assert rc == es.ES_OK
    sim.close()
