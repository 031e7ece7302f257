"""The CUDA library builds for sm_103a, loads, and exports every entry point of include/ds.h
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "ds.h")).read()
    return sorted(set(re.findall(r"^\s*(?:ds_status|const char \*)\s*(ds_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["ds_create", "ds_destroy", "ds_model_create", "ds_model_set_lattice", "ds_model_set_sites",
                 "ds_model_set_supercell", "ds_model_upload_occupancy", "ds_model_upload_spins",
                 "ds_model_upload_displacements", "ds_request_intensity", "ds_submit", "ds_poll", "ds_wait",
                 "ds_backward", "ds_last_error"]:
        assert name in syms


def test_library_exports_every_declared_symbol():
    from paper_1809_07088_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ds_\w+)", out))
    assert set(declared_symbols()) <= exported


def test_binding_signatures_cover_header():
    from paper_1809_07088_gb300 import _binding
    assert set(declared_symbols()) == set(_binding.SIGNATURES)


def test_library_targets_sm103a():
    """The fatbinary carries sm_103a code (checked by the compiler driver listing, not by
    reading the binary)."""
    from paper_1809_07088_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1809_07088_gb300 import _binding
    lib = _binding.load()
    h = ctypes.c_void_p()
    st = lib.ds_create(ctypes.byref(h), 0, 0)
    assert st != 0 and not h.value
    assert lib.ds_version().decode().startswith("paper_1809_07088_gb300")


def test_noalloc_rejects_non_finite_site_data_before_any_gpu_work():
    """The allocation-free entry point checks its host arguments before touching the GPU: a NaN
    coordinate, scattering length or mean occupancy is DS_ERR_ARG with a message (the device
    pointers are never dereferenced, so placeholders are enough)."""
    import numpy as np
    from paper_1809_07088_gb300 import _binding as B
    lib = B.load()
    lat = (ctypes.c_double * 6)(4.0, 4.0, 4.0, 90.0, 90.0, 90.0)
    q = B.make_qgrid((0.0, 0.0, 0.0), (0.25, 0.25, 0.25), (5, 5, 5))
    fake_dev = ctypes.c_void_p(256)
    good = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]])
    for what in ("coord", "scat", "mean"):
        sites, scat, mean = good.copy(), np.ones(2), np.full(2, 0.5)
        if what == "coord":
            sites[1, 2] = np.nan
        elif what == "scat":
            scat[0] = np.inf
        else:
            mean[1] = np.nan
        err = ctypes.create_string_buffer(256)
        st = lib.ds_occupancy_intensity_noalloc(lat, 2, sites.ctypes.data, scat.ctypes.data, 4, 4, 4, 1, fake_dev,
                                                mean.ctypes.data, ctypes.byref(q), 1, fake_dev, None, err, len(err))
        assert st == B.DS_ERR_ARG, what
        assert "site" in err.value.decode()
