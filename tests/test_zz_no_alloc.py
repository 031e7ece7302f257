"""The no-allocation occupancy entry point (ds_occupancy_intensity_noalloc).

It exists for callers that cannot allocate device memory when they need a volume (a host
framework that owns the GPU's memory through its own allocator, a process under a fixed memory
cap, a refinement loop that must not touch the allocator).  It keeps all its scratch in one
static device array, so these tests check that two calls in a row -- the second on a different
model, so stale scratch from the first would show -- agree with the ordinary entry point
ds_request_intensity, that a call on a grid of many zones with ragged edges agrees with the CPU
oracle, and that an oversized request is refused before any work is queued.

This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import synthetic as syn
from _helpers import TOL, qgrid_tuple, rel_err_of_peak

pytestmark = pytest.mark.gpu


def _const_ff_model(cells, nsite, nmodels, seed, sites=None):
    m = syn.small_case(syn.OCC, cells=cells, nsite=nsite, nmodels=nmodels, seed=seed)
    m.ff_kind = np.zeros(nsite, dtype=np.int32)
    m.ff_coef = np.zeros((nsite, 9))
    if sites is not None:
        m.sites = np.array(sites[:nsite], dtype=np.float64)
    return m


def _noalloc(lib, m, mode, out, stream, mean=None):
    import paper_1809_07088_gb300._binding as B
    import torch
    occ = torch.from_numpy(np.ascontiguousarray(m.occ)).cuda()
    lat = (ctypes.c_double * 6)(*m.lattice)
    sites = np.ascontiguousarray(m.sites, dtype=np.float64)
    scat = np.ascontiguousarray(m.scat_len, dtype=np.float64)
    q = B.make_qgrid(*qgrid_tuple(m.qgrid))
    err = ctypes.create_string_buffer(512)
    mean_p = None
    if mean is not None:
        mean = np.ascontiguousarray(mean, dtype=np.float64)
        mean_p = mean.ctypes.data
    st = lib.ds_occupancy_intensity_noalloc(lat, m.nsite, sites.ctypes.data, scat.ctypes.data, *m.cells,
                                            m.nmodels, occ.data_ptr(), mean_p, ctypes.byref(q), mode,
                                            out.data_ptr(), stream, err, len(err))
    return st, err.value.decode(), occ


def test_noalloc_matches_ordinary_entry_point_twice():
    import torch
    import paper_1809_07088_gb300 as ds
    from _helpers import to_library
    torch.cuda.set_device(0)
    ctx = ds.Context(0)
    lib = ctx.lib
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(_const_ff_model((6, 5, 4), 3, 2, 201), ds.DS_DIFFUSE),
             (_const_ff_model((5, 6, 8), 8, 1, 202, sites=syn.PYROCHLORE_SITES), ds.DS_TOTAL)]
    keep = []
    for m, mode in cases:
        want, _ = to_library(ctx, m).intensity(qgrid_tuple(m.qgrid), disorder=ds.DS_OCC, mode=mode,
                                               precision=ds.DS_FP32)
        out = torch.full(m.qgrid.count, float("nan"), dtype=torch.float32, device="cuda")
        st, msg, occ = _noalloc(lib, m, mode, out, stream)
        assert st == 0, msg
        keep.append((out, occ))
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert rel_err_of_peak(got, want) < TOL["fp32"]
    ctx.close()


def test_noalloc_ragged_multizone_grid_against_oracle():
    """A grid spanning 4 x 5 x 6 zones with ragged edges on every side (not a multiple of the
    supercell), DIFFUSE with a caller-given mean and TOTAL, against the oracle's FFT method."""
    import torch
    import paper_1809_07088_gb300 as ds
    from oracle import core
    torch.cuda.set_device(0)
    lib = ds.load()
    stream = torch.cuda.current_stream().cuda_stream
    m = _const_ff_model((5, 6, 4), 5, 2, 204)
    n = m.cells
    m.qgrid = syn.QGrid(h0=tuple(-1.0 - 3.0 / c for c in n), step=tuple(1.0 / c for c in n),
                        count=(3 * n[0] + 7, 4 * n[1] + 1, 5 * n[2] + 3))
    for mode, mean in ((ds.DS_DIFFUSE, np.array([0.3, 0.5, 0.45, 0.6, 0.2])), (ds.DS_TOTAL, None)):
        m.mean_occ = mean
        want = core.occupancy_intensity_fft(m, m.qgrid.g_index(m.cells), mode)
        out = torch.full(m.qgrid.count, float("nan"), dtype=torch.float32, device="cuda")
        st, msg, occ = _noalloc(lib, m, mode, out, stream, mean=mean)
        assert st == 0, msg
        torch.cuda.synchronize()
        assert rel_err_of_peak(out.cpu().numpy(), want) < TOL["fp32"]


def test_noalloc_rejects_oversized_request():
    import torch
    import paper_1809_07088_gb300 as ds
    torch.cuda.set_device(0)
    lib = ds.load()
    m = _const_ff_model((64, 64, 64), 16, 1, 203)
    m.occ = np.zeros((1, 16, 64, 64, 64), dtype=np.uint8)
    out = torch.empty((1, 1, 1), dtype=torch.float32, device="cuda")
    m.qgrid = syn.QGrid((0.0, 0.0, 0.0), (1 / 64,) * 3, (1, 1, 1))
    st, msg, _ = _noalloc(lib, m, 0, out, torch.cuda.current_stream().cuda_stream)
    assert st == ds._binding.DS_ERR_ADMISSION
    assert "bytes of scratch" in msg
