"""Glue shared by the GPU tests: move a synthetic model into the library, and call the oracle."""
import numpy as np

import synthetic as syn


def to_library(ctx, m: syn.Model, with_occ=True, with_spins=True, with_disp=True):
    """Create a library Model from a synthetic one (uploads from host memory)."""
    import paper_1809_07088_gb300 as ds
    lm = ds.Model(ctx, m.lattice, m.sites, m.cells, m.nmodels, scat_len=m.scat_len,
                  ff_kind=m.ff_kind, ff_coef=m.ff_coef)
    if with_occ and m.occ is not None:
        lm.upload_occupancy(np.ascontiguousarray(m.occ), m.mean_occ)
    if with_spins and m.spins is not None:
        lm.upload_spins(np.ascontiguousarray(m.spins))
    if with_disp and m.disp is not None:
        lm.upload_displacements(np.ascontiguousarray(m.disp))
    return lm


def qgrid_tuple(q: syn.QGrid):
    return (q.h0, q.step, q.count)


def rel_err_of_peak(got, want):
    """max |got - want| / max |want| (the tolerance scale of the parity tests)."""
    got = np.asarray(got, dtype=np.float64).reshape(-1)
    want = np.asarray(want, dtype=np.float64).reshape(-1)
    peak = np.max(np.abs(want))
    return float(np.max(np.abs(got - want)) / (peak if peak > 0 else 1.0))


TOL = {"fp64": 1e-10, "fp32": 1e-5}
