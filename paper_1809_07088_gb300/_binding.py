"""ctypes binding of the C boundary declared in include/ds.h.

Argument marshalling only: every step of the calculation runs in the CUDA library.  The
library is built in-tree (paper_1809_07088_gb300/_lib/libds_gb300.so); if it cannot be built
or loaded, importing the functions raises -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import threading

from . import build as _build

DS_OK, DS_ERR_ARG, DS_ERR_STATE, DS_ERR_OOM, DS_ERR_ADMISSION, DS_ERR_TIMEOUT, DS_ERR_CUDA, \
    DS_ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
DS_FF_CONST, DS_FF_GAUSS4, DS_FF_J0 = 0, 1, 2
DS_OCC, DS_SPIN, DS_DISP = 0, 1, 2
DS_TOTAL, DS_DIFFUSE = 0, 1
DS_FP64, DS_FP32 = 0, 1
DS_SMOOTH_NONE, DS_SMOOTH_LANCZOS, DS_SMOOTH_SUBBOX, DS_SMOOTH_SPHERE = 0, 1, 2, 3
DS_TAYLOR_AUTO, DS_TAYLOR_PER_VOXEL, DS_TAYLOR_SUM_FACTORISED = 0, 1, 2

_STATUS = {0: "DS_OK", -1: "DS_ERR_ARG", -2: "DS_ERR_STATE", -3: "DS_ERR_OOM", -4: "DS_ERR_ADMISSION",
           -5: "DS_ERR_TIMEOUT", -6: "DS_ERR_CUDA", -7: "DS_ERR_UNSUPPORTED"}


class ds_qgrid(C.Structure):
    _fields_ = [("h0", C.c_double * 3), ("step", C.c_double * 3), ("count", C.c_int64 * 3)]


class ds_opts(C.Structure):
    _fields_ = [("disorder", C.c_int), ("mode", C.c_int), ("precision", C.c_int),
                ("taylor_order", C.c_int), ("taylor_eps", C.c_double), ("smoothing", C.c_int),
                ("lanczos_m", C.c_int), ("lanczos_mprime", C.c_int), ("subbox_n", C.c_int),
                ("taylor_zonal", C.c_int), ("dw_coupling", C.c_int), ("taylor_kernel", C.c_int)]


class ds_result_info(C.Structure):
    _fields_ = [("taylor_order", C.c_int), ("n_monomials", C.c_int), ("x_max", C.c_double),
                ("trunc_bound", C.c_double), ("nvox", C.c_int64), ("workspace_bytes", C.c_int64),
                ("gpu_ms", C.c_double), ("latency_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


vp, dp, ip, u8p, fp = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_void_p, C.c_void_p
st = C.c_int

# name -> (restype, argtypes); the exported symbol list of include/ds.h
SIGNATURES = {
    "ds_create": (st, [C.POINTER(vp), C.c_int, C.c_size_t]),
    "ds_destroy": (st, [vp]),
    "ds_last_error": (C.c_char_p, [vp]),
    "ds_version": (C.c_char_p, []),
    "ds_model_create": (st, [vp, C.POINTER(vp)]),
    "ds_model_destroy": (st, [vp]),
    "ds_model_set_lattice": (st, [vp] + [C.c_double] * 6),
    "ds_model_set_sites": (st, [vp, C.c_int, vp, vp, vp, vp]),
    "ds_model_set_supercell": (st, [vp, C.c_int, C.c_int, C.c_int, C.c_int]),
    "ds_model_upload_occupancy": (st, [vp, vp, vp, C.c_int, vp]),
    "ds_model_upload_spins": (st, [vp, vp, C.c_int, vp]),
    "ds_model_upload_displacements": (st, [vp, vp, C.c_int, vp]),
    "ds_request_intensity": (st, [vp, C.POINTER(ds_qgrid), C.POINTER(ds_opts), vp, C.c_int, vp,
                                  C.POINTER(ds_result_info)]),
    "ds_request_points": (st, [vp, vp, C.c_int64, C.c_int, C.POINTER(ds_opts), vp, C.c_int, vp,
                               C.POINTER(ds_result_info)]),
    "ds_request_subbox_points": (st, [vp, vp, C.c_int64, vp, C.c_int64, C.c_int, C.POINTER(ds_opts), vp,
                                      C.c_int, vp, C.POINTER(ds_result_info)]),
    "ds_debye_waller": (st, [vp, vp, C.c_int64, C.c_int, C.c_int, C.c_int, vp, C.c_int, vp]),
    "ds_submit": (st, [vp, C.POINTER(ds_qgrid), C.POINTER(ds_opts), vp, C.POINTER(C.c_uint64)]),
    "ds_poll": (st, [vp, C.c_uint64, C.POINTER(ds_result_info)]),
    "ds_wait": (st, [vp, C.c_uint64, C.c_double, C.POINTER(ds_result_info)]),
    "ds_backward": (st, [vp, C.POINTER(ds_qgrid), C.POINTER(ds_opts), vp, vp, C.c_int, vp]),
    "ds_serving_pause": (st, [vp, C.c_int]),
    "ds_profile_enable": (st, [vp, C.c_int]),
    "ds_profile_report": (st, [vp, C.c_char_p, C.c_size_t]),
    "ds_measure_peaks": (st, [C.c_int, C.POINTER(C.c_double)]),
    "ds_occupancy_intensity_noalloc": (st, [C.POINTER(C.c_double), C.c_int, vp, vp, C.c_int, C.c_int, C.c_int,
                                            C.c_int, vp, vp, C.POINTER(ds_qgrid), C.c_int, vp, vp, C.c_char_p,
                                            C.c_size_t]),
}

_lib = None
_lock = threading.Lock()


def load():
    """Load (building first if needed) the CUDA library and declare its signatures."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            lib = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class DSError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (_STATUS.get(status, str(status)), message))
        self.status = status


def check(status, ctx=None):
    if status != DS_OK:
        msg = load().ds_last_error(ctx).decode() if ctx else ""
        raise DSError(status, msg)
    return status


def make_qgrid(h0, step, count) -> ds_qgrid:
    q = ds_qgrid()
    for a in range(3):
        q.h0[a], q.step[a], q.count[a] = float(h0[a]), float(step[a]), int(count[a])
    return q


def make_opts(disorder, mode=DS_DIFFUSE, precision=DS_FP32, taylor_order=-1, taylor_eps=1e-8,
              smoothing=DS_SMOOTH_NONE, lanczos_m=2, lanczos_mprime=2, subbox_n=1,
              taylor_zonal=0, dw_coupling=0, taylor_kernel=0) -> ds_opts:
    o = ds_opts()
    o.disorder, o.mode, o.precision = int(disorder), int(mode), int(precision)
    o.taylor_order, o.taylor_eps = int(taylor_order), float(taylor_eps)
    o.smoothing, o.lanczos_m, o.lanczos_mprime, o.subbox_n = int(smoothing), int(lanczos_m), \
        int(lanczos_mprime), int(subbox_n)
    o.taylor_zonal = int(taylor_zonal)
    o.dw_coupling = int(dw_coupling)
    o.taylor_kernel = int(taylor_kernel)
    return o
