"""GB300-native FFT-based diffuse-scattering calculation (arXiv 1809.07088).

Python front of the C boundary (include/ds.h): a `Context` owns one GPU, a `Model` is an
ensemble of supercells resident in its memory, and `Model.intensity` requests an intensity
volume I(G).  Arrays may be numpy arrays (host) or torch tensors (host or CUDA); CUDA tensors
are used in place on torch's current stream.  All computation happens in the CUDA library.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from ._binding import (DS_DIFFUSE, DS_DISP, DS_FF_CONST, DS_FF_GAUSS4, DS_FF_J0, DS_FP32, DS_FP64,
                       DS_OCC, DS_SMOOTH_LANCZOS, DS_SMOOTH_NONE, DS_SMOOTH_SPHERE, DS_SMOOTH_SUBBOX, DS_SPIN,
                       DS_TAYLOR_AUTO, DS_TAYLOR_PER_VOXEL, DS_TAYLOR_SUM_FACTORISED, DS_TOTAL,
                       DSError, check, ds_result_info, load, make_opts, make_qgrid)

__all__ = ["Context", "Model", "DSError", "load", "make_opts", "make_qgrid", "DS_OCC", "DS_SPIN",
           "DS_DISP", "DS_TAYLOR_AUTO", "DS_TAYLOR_PER_VOXEL", "DS_TAYLOR_SUM_FACTORISED", "DS_TOTAL",
           "DS_DIFFUSE", "DS_FP32", "DS_FP64", "DS_SMOOTH_NONE",
           "DS_SMOOTH_LANCZOS", "DS_SMOOTH_SUBBOX", "DS_SMOOTH_SPHERE", "DS_FF_CONST", "DS_FF_GAUSS4", "DS_FF_J0"]


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """(pointer, is_device) of a C-contiguous numpy array or torch tensor of `dtype`."""
    if _is_torch(x):
        import torch
        want = {np.uint8: torch.uint8, np.float32: torch.float32, np.float64: torch.float64}[dtype]
        if x.dtype != want or not x.is_contiguous():
            raise TypeError("expected a contiguous %s tensor" % want)
        return x.data_ptr(), 1 if x.is_cuda else 0
    a = np.asarray(x)
    if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("expected a C-contiguous %s array" % np.dtype(dtype))
    return a.ctypes.data, 0


def _stream_of(x, stream):
    if stream is not None:
        return stream
    if x is not None and _is_torch(x) and x.is_cuda:
        import torch
        return torch.cuda.current_stream(x.device).cuda_stream
    return None


class Context:
    """One GPU (ds_create).  hbm_budget bounds the scratch of one request (0 = 90% free)."""

    def __init__(self, device: int = 0, hbm_budget: int = 0):
        self.lib = load()
        h = C.c_void_p()
        st = self.lib.ds_create(C.byref(h), int(device), C.c_size_t(int(hbm_budget)))
        if st != 0:
            raise DSError(st, "ds_create(device=%d) failed" % device)
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            self.lib.ds_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, st):
        return check(st, self.h)

    def model(self, lattice, sites, cells, nmodels=1, scat_len=None, ff_kind=None, ff_coef=None):
        return Model(self, lattice, sites, cells, nmodels, scat_len, ff_kind, ff_coef)

    # serving (ds_submit / ds_poll / ds_wait)
    def poll(self, ticket):
        info = ds_result_info()
        st = self.lib.ds_poll(self.h, C.c_uint64(ticket), C.byref(info))
        return st, info

    def pause_serving(self, pause=True):
        self.check(self.lib.ds_serving_pause(self.h, 1 if pause else 0))

    def wait(self, ticket, timeout_s=60.0):
        info = ds_result_info()
        self.check(self.lib.ds_wait(self.h, C.c_uint64(ticket), C.c_double(timeout_s), C.byref(info)))
        return info


class Model:
    """An ensemble of supercells on the context's GPU (ds_model_*)."""

    def __init__(self, ctx: Context, lattice, sites, cells, nmodels=1, scat_len=None, ff_kind=None,
                 ff_coef=None):
        self.ctx, self.lib = ctx, ctx.lib
        h = C.c_void_p()
        ctx.check(self.lib.ds_model_create(ctx.h, C.byref(h)))
        self.h = h
        ctx.check(self.lib.ds_model_set_lattice(h, *[float(x) for x in lattice]))
        s = np.ascontiguousarray(sites, dtype=np.float64).reshape(-1, 3)
        self.nsite = s.shape[0]
        keep = [s]
        b = None if scat_len is None else np.ascontiguousarray(scat_len, dtype=np.float64)
        k = None if ff_kind is None else np.ascontiguousarray(ff_kind, dtype=np.int32)
        c = None if ff_coef is None else np.ascontiguousarray(ff_coef, dtype=np.float64).reshape(-1, 9)
        keep += [b, k, c]
        ptr = lambda a: None if a is None else a.ctypes.data
        ctx.check(self.lib.ds_model_set_sites(h, self.nsite, s.ctypes.data, ptr(b), ptr(k), ptr(c)))
        self.cells = tuple(int(n) for n in cells)
        self.nmodels = int(nmodels)
        ctx.check(self.lib.ds_model_set_supercell(h, *self.cells, self.nmodels))

    def close(self):
        if getattr(self, "h", None) and getattr(self.ctx, "h", None):
            self.lib.ds_model_destroy(self.h)
        self.h = None

    def _shape(self, ncomp):
        s = (self.nmodels, self.nsite) + self.cells
        return s + ((ncomp,) if ncomp else ())

    def upload_occupancy(self, occ, mean_occ=None, stream=None):
        p, dev = _ptr(occ, np.uint8)
        assert tuple(occ.shape) == self._shape(0), (tuple(occ.shape), self._shape(0))
        mean = None if mean_occ is None else np.ascontiguousarray(mean_occ, dtype=np.float64)
        self.ctx.check(self.lib.ds_model_upload_occupancy(self.h, p, None if mean is None else mean.ctypes.data,
                                                          dev, _stream_of(occ, stream)))

    def upload_spins(self, spins, stream=None):
        p, dev = _ptr(spins, np.float32)
        assert tuple(spins.shape) == self._shape(3)
        self.ctx.check(self.lib.ds_model_upload_spins(self.h, p, dev, _stream_of(spins, stream)))

    def upload_displacements(self, disp, stream=None):
        p, dev = _ptr(disp, np.float32)
        assert tuple(disp.shape) == self._shape(3)
        self.ctx.check(self.lib.ds_model_upload_displacements(self.h, p, dev, _stream_of(disp, stream)))

    def intensity(self, qgrid, out=None, stream=None, **opts):
        """I(G) on `qgrid` (h0, step, count) -> (out, info dict).  `out` may be a CUDA tensor
        (filled asynchronously on its stream) or None (a numpy array is returned)."""
        q = make_qgrid(*qgrid)
        o = make_opts(**opts)
        count = tuple(int(c) for c in qgrid[2])
        dt = np.float64 if o.precision == DS_FP64 else np.float32
        if out is None:
            out = np.empty(count, dtype=dt)
        p, dev = _ptr(out, dt)
        info = ds_result_info()
        self.ctx.check(self.lib.ds_request_intensity(self.h, C.byref(q), C.byref(o), p, dev,
                                                     _stream_of(out, stream), C.byref(info)))
        return out, info.as_dict()

    def intensity_points(self, hkl, out=None, stream=None, **opts):
        """I(Q) at arbitrary points hkl [npts, 3] (r.l.u., float64; numpy or torch, host or CUDA)
        by Lanczos resampling of I(G) (ds_request_points); smoothing defaults to Lanczos.
        Returns (out, info dict); `out` may be a preallocated array or tensor of npts values."""
        opts.setdefault("smoothing", DS_SMOOTH_LANCZOS)
        o = make_opts(**opts)
        dt = np.float64 if o.precision == DS_FP64 else np.float32
        if not _is_torch(hkl):
            hkl = np.ascontiguousarray(hkl, dtype=np.float64).reshape(-1, 3)
        ph, hdev = _ptr(hkl, np.float64)
        npts = int(hkl.shape[0]) if len(hkl.shape) == 2 else int(np.prod(hkl.shape)) // 3
        if out is None:
            out = np.empty(npts, dtype=dt)
        po, odev = _ptr(out, dt)
        info = ds_result_info()
        self.ctx.check(self.lib.ds_request_points(self.h, ph, C.c_int64(npts), hdev, C.byref(o), po, odev,
                                                  _stream_of(out, stream), C.byref(info)))
        return out, info.as_dict()

    def subbox_points(self, hkl, origins=None, out=None, stream=None, **opts):
        """Sub-box average at arbitrary points hkl [npts, 3] (ds_request_subbox_points): boxes of
        subbox_n^3 cells at `origins` (int32 [norigin, 4] rows (model, o1, o2, o3), e.g. drawn
        at random) or, with origins=None, at every lattice point of every supercell.
        Returns (out, info dict)."""
        opts.setdefault("smoothing", DS_SMOOTH_SUBBOX)
        o = make_opts(**opts)
        dt = np.float64 if o.precision == DS_FP64 else np.float32
        if not _is_torch(hkl):
            hkl = np.ascontiguousarray(hkl, dtype=np.float64).reshape(-1, 3)
        ph, hdev = _ptr(hkl, np.float64)
        npts = int(hkl.shape[0]) if len(hkl.shape) == 2 else int(np.prod(hkl.shape)) // 3
        porg, norg = None, 0
        if origins is not None:
            origins = np.ascontiguousarray(origins, dtype=np.int32).reshape(-1, 4)
            porg, norg = origins.ctypes.data_as(C.c_void_p), int(origins.shape[0])
        if out is None:
            out = np.empty(npts, dtype=dt)
        po, odev = _ptr(out, dt)
        info = ds_result_info()
        self.ctx.check(self.lib.ds_request_subbox_points(self.h, porg, C.c_int64(norg), ph, C.c_int64(npts), hdev,
                                                         C.byref(o), po, odev, _stream_of(out, stream),
                                                         C.byref(info)))
        return out, info.as_dict()

    def debye_waller(self, hkl, precision=DS_FP64, occupancy_weights=False, out=None, stream=None):
        """T_mu(Q) of the uploaded displacements at points hkl [npts, 3]: [npts, nsite]
        (ds_debye_waller)."""
        dt = np.float64 if precision == DS_FP64 else np.float32
        if not _is_torch(hkl):
            hkl = np.ascontiguousarray(hkl, dtype=np.float64).reshape(-1, 3)
        ph, hdev = _ptr(hkl, np.float64)
        npts = int(hkl.shape[0]) if len(hkl.shape) == 2 else int(np.prod(hkl.shape)) // 3
        if out is None:
            out = np.empty((npts, self.nsite), dtype=dt)
        po, odev = _ptr(out, dt)
        self.ctx.check(self.lib.ds_debye_waller(self.h, ph, C.c_int64(npts), hdev, int(precision),
                                                int(bool(occupancy_weights)), po, odev, _stream_of(out, stream)))
        return out

    def backward(self, qgrid, dL_dI, grad=None, stream=None, **opts):
        """dL/du (displacive) or dL/dM (magnetic) for a given dL/dI on `qgrid`."""
        q = make_qgrid(*qgrid)
        o = make_opts(**opts)
        dt = np.float64 if o.precision == DS_FP64 else np.float32
        if grad is None:
            grad = np.empty(self._shape(3), dtype=dt)
        pg, dev = _ptr(grad, dt)
        pi, dev_i = _ptr(dL_dI, dt)
        if dev != dev_i:
            raise TypeError("dL_dI and grad must both be host or both be device buffers")
        self.ctx.check(self.lib.ds_backward(self.h, C.byref(q), C.byref(o), pi, pg, dev,
                                            _stream_of(grad, stream)))
        return grad

    def submit(self, qgrid, out, **opts):
        """Queue a request (serving); `out` must be a CUDA tensor.  Returns a ticket."""
        q = make_qgrid(*qgrid)
        o = make_opts(**opts)
        dt = np.float64 if o.precision == DS_FP64 else np.float32
        p, dev = _ptr(out, dt)
        if not dev:
            raise TypeError("ds_submit needs a device output buffer")
        t = C.c_uint64()
        self.ctx.check(self.lib.ds_submit(self.h, C.byref(q), C.byref(o), p, C.byref(t)))
        return t.value
