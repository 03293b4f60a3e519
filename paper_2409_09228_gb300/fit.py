"""Thin ctypes binding of libfit (include/fit.h), with the same names.

Argument marshalling only: tensors are passed by data pointer, streams by
handle; every step of the fit runs in the CUDA kernels of libfit.so.  There is
no CPU fallback: if the library is missing or no GPU is present the calls
raise.

Layouts (track index fastest, see fit.h): par (6, ld), cov (21, ld), q (ld,)
int32, chi2 (ld,), hit positions (nlayer, 3, ld), hit covariances
(nlayer, 6, ld), all float32 CUDA tensors on the handle's device.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

from . import build as _build

FIT_MODE_R = 0
FIT_MODE_Z = 1
FIT_OK = 0
FIT_ERR_ARG = -1
FIT_ERR_CUDA = -2
FIT_ERR_TIMEOUT = -3
FIT_ERR_NOMEM = -4
FIT_ST_NO_INTERSECTION = 1
FIT_ST_NOT_CONVERGED = 2
FIT_ST_NONFINITE = 4
FIT_ST_CHARGE_FLIP = 8
FIT_START_CROSSING = 0
FIT_START_LINE = 1
FIT_HOST_CHUNK = 262144
FIT_MAX_LAYERS = 64


class FitError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libfit error {code}: {msg}")
        self.code = code


class fit_config(ctypes.Structure):
    _fields_ = [("B", ctypes.c_float), ("nlayer", ctypes.c_int),
                ("surf", ctypes.POINTER(ctypes.c_float)), ("max_iter", ctypes.c_int),
                ("tol", ctypes.c_float), ("start", ctypes.c_int)]


class fit_tracks_in(ctypes.Structure):
    _fields_ = [("par", ctypes.c_void_p), ("cov", ctypes.c_void_p), ("q", ctypes.c_void_p),
                ("ld", ctypes.c_int64)]


class fit_tracks_out(ctypes.Structure):
    _fields_ = [("par", ctypes.c_void_p), ("cov", ctypes.c_void_p), ("q", ctypes.c_void_p),
                ("chi2", ctypes.c_void_p), ("chi2_layer", ctypes.c_void_p),
                ("status", ctypes.c_void_p), ("ld", ctypes.c_int64)]


class fit_hits(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_void_p), ("cov", ctypes.c_void_p), ("ld", ctypes.c_int64)]


class fit_status(ctypes.Structure):
    _fields_ = [("tracks", ctypes.c_uint64), ("no_intersection", ctypes.c_uint64),
                ("not_converged", ctypes.c_uint64), ("nonfinite", ctypes.c_uint64),
                ("charge_flip", ctypes.c_uint64), ("iterations", ctypes.c_uint64)]


class fit_launch_config(ctypes.Structure):
    _fields_ = [("threads_per_block", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
                ("persistent", ctypes.c_int), ("tracks_per_thread", ctypes.c_int),
                ("layout", ctypes.c_int)]


class fit_plan_info(ctypes.Structure):
    _fields_ = [("config", fit_launch_config), ("tracks", ctypes.c_int64),
                ("items", ctypes.c_int32), ("tuned", ctypes.c_int32), ("best_ms", ctypes.c_float)]


class fit_candidates(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_void_p), ("cov", ctypes.c_void_p), ("ncand", ctypes.c_int32),
                ("ld", ctypes.c_int64)]


class fit_mlp_train_config(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_float),
                ("lr_final", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("seed", ctypes.c_uint64)]


EXPORTS = ("fit_init", "fit_propagate_update", "fit_sync", "fit_destroy", "fit_last_error",
           "fit_propagate_update_noalloc", "fit_plan_create", "fit_plan_run", "fit_plan_tune",
           "fit_plan_get_info", "fit_plan_destroy", "fit_tape_bytes", "fit_adjoint_forward",
           "fit_adjoint_backward", "fit_mlp_create", "fit_mlp_destroy", "fit_mlp_set_params",
           "fit_mlp_get_params", "fit_mlp_prepare", "fit_mlp_forward", "fit_mlp_gradient",
           "fit_mlp_adam_step", "fit_mlp_train", "fit_mlp_attach", "fit_path_lengths",
           "fit_propagate_update_host", "fit_propagate_update_mapped", "fit_propagate_update_f64",
           "fit_propagate_update_layout", "fit_find_tracks", "fit_find_tracks_f64",
           "fit_relayout", "fit_probe_fp32")
FIT_LAYOUT_SOA = 0
FIT_LAYOUT_AOSOA32 = 1
FIT_LAYOUT_TUNE = 2
FIT_MLP_INPUTS = 8
FIT_MLP_HIDDEN = 64
FIT_MLP_PARAMS = 4801
FIT_NOALLOC_MAX_EVENTS = 4096

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libfit.so (building it first if needed); raises if that fails."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libfit.so not found at {path}; run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    L.fit_init.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(fit_config),
                           ctypes.POINTER(fit_config), ctypes.c_int]
    L.fit_init.restype = ctypes.c_int
    L.fit_propagate_update.argtypes = [vp, ctypes.POINTER(fit_tracks_in),
                                       ctypes.POINTER(fit_tracks_out), ctypes.POINTER(fit_hits),
                                       ctypes.c_int, ctypes.POINTER(i64), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int32), vp]
    L.fit_propagate_update.restype = ctypes.c_int
    L.fit_sync.argtypes = [vp, vp, ctypes.c_double, ctypes.POINTER(fit_status)]
    L.fit_sync.restype = ctypes.c_int
    L.fit_destroy.argtypes = [vp]
    L.fit_destroy.restype = None
    L.fit_last_error.argtypes = []
    L.fit_last_error.restype = ctypes.c_char_p
    L.fit_propagate_update_noalloc.argtypes = [
        ctypes.POINTER(fit_config), ctypes.POINTER(fit_config), ctypes.POINTER(fit_tracks_in),
        ctypes.POINTER(fit_tracks_out), ctypes.POINTER(fit_hits), ctypes.c_int,
        ctypes.POINTER(i64), ctypes.c_int, ctypes.POINTER(ctypes.c_int32), vp,
        ctypes.POINTER(fit_status)]
    L.fit_propagate_update_noalloc.restype = ctypes.c_int
    L.fit_plan_create.argtypes = [vp, ctypes.c_int, ctypes.POINTER(i64),
                                  ctypes.POINTER(ctypes.c_int32), ctypes.c_int,
                                  ctypes.POINTER(fit_launch_config), ctypes.POINTER(vp)]
    L.fit_plan_create.restype = ctypes.c_int
    L.fit_plan_run.argtypes = [vp, ctypes.POINTER(fit_tracks_in), ctypes.POINTER(fit_tracks_out),
                               ctypes.POINTER(fit_hits), vp]
    L.fit_plan_run.restype = ctypes.c_int
    L.fit_plan_tune.argtypes = [vp, ctypes.POINTER(fit_tracks_in), ctypes.POINTER(fit_tracks_out),
                                ctypes.POINTER(fit_hits), vp, ctypes.c_char_p]
    L.fit_plan_tune.restype = ctypes.c_int
    L.fit_plan_get_info.argtypes = [vp, ctypes.POINTER(fit_plan_info)]
    L.fit_plan_get_info.restype = ctypes.c_int
    L.fit_plan_destroy.argtypes = [vp]
    L.fit_plan_destroy.restype = None
    L.fit_tape_bytes.argtypes = [ctypes.c_int, i64]
    L.fit_tape_bytes.restype = ctypes.c_size_t
    L.fit_adjoint_forward.argtypes = [vp, ctypes.POINTER(fit_tracks_in),
                                      ctypes.POINTER(fit_tracks_out), ctypes.POINTER(fit_hits),
                                      ctypes.c_int, ctypes.POINTER(i64), ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_int32), vp, vp]
    L.fit_adjoint_forward.restype = ctypes.c_int
    L.fit_adjoint_backward.argtypes = [vp, ctypes.POINTER(fit_hits), ctypes.c_int,
                                       ctypes.POINTER(i64), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int32), vp, vp, vp, vp, vp, vp]
    L.fit_adjoint_backward.restype = ctypes.c_int
    L.fit_find_tracks.argtypes = [vp, ctypes.POINTER(fit_tracks_in), ctypes.POINTER(fit_tracks_out),
                                  ctypes.POINTER(fit_candidates), ctypes.c_float, vp, ctypes.c_int,
                                  ctypes.POINTER(i64), ctypes.c_int, ctypes.POINTER(ctypes.c_int32),
                                  vp]
    L.fit_find_tracks.restype = ctypes.c_int
    L.fit_find_tracks_f64.argtypes = [vp, ctypes.POINTER(fit_tracks_in),
                                      ctypes.POINTER(fit_tracks_out), ctypes.POINTER(fit_candidates),
                                      ctypes.c_double, vp, ctypes.c_int, ctypes.POINTER(i64),
                                      ctypes.c_int, ctypes.POINTER(ctypes.c_int32), vp]
    L.fit_find_tracks_f64.restype = ctypes.c_int
    L.fit_propagate_update_layout.argtypes = L.fit_propagate_update.argtypes[:-1] + [ctypes.c_int, vp]
    L.fit_propagate_update_layout.restype = ctypes.c_int
    L.fit_propagate_update_f64.argtypes = L.fit_propagate_update.argtypes
    L.fit_propagate_update_f64.restype = ctypes.c_int
    L.fit_propagate_update_host.argtypes = L.fit_propagate_update.argtypes
    L.fit_propagate_update_host.restype = ctypes.c_int
    L.fit_propagate_update_mapped.argtypes = L.fit_propagate_update.argtypes
    L.fit_propagate_update_mapped.restype = ctypes.c_int
    i32p = ctypes.POINTER(ctypes.c_int32)
    L.fit_mlp_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_uint64]
    L.fit_mlp_create.restype = ctypes.c_int
    L.fit_mlp_destroy.argtypes = [vp]
    L.fit_mlp_destroy.restype = None
    L.fit_mlp_set_params.argtypes = [vp, vp]
    L.fit_mlp_set_params.restype = ctypes.c_int
    L.fit_mlp_get_params.argtypes = [vp, vp]
    L.fit_mlp_get_params.restype = ctypes.c_int
    L.fit_mlp_prepare.argtypes = [ctypes.c_float, vp, i64, vp, vp, vp, i64, vp, vp, vp]
    L.fit_mlp_prepare.restype = ctypes.c_int
    L.fit_mlp_forward.argtypes = [vp, vp, i64, vp, vp]
    L.fit_mlp_forward.restype = ctypes.c_int
    L.fit_mlp_gradient.argtypes = [vp, vp, vp, i64, vp, vp, vp]
    L.fit_mlp_gradient.restype = ctypes.c_int
    L.fit_mlp_adam_step.argtypes = [vp, vp, ctypes.c_float, vp]
    L.fit_mlp_adam_step.restype = ctypes.c_int
    L.fit_mlp_train.argtypes = [vp, vp, vp, i64, ctypes.POINTER(fit_mlp_train_config), vp, vp]
    L.fit_mlp_train.restype = ctypes.c_int
    L.fit_mlp_attach.argtypes = [vp, vp, vp]
    L.fit_mlp_attach.restype = ctypes.c_int
    L.fit_path_lengths.argtypes = [vp, vp, i64, vp, vp, i64, vp, i32p, ctypes.c_int, vp]
    L.fit_path_lengths.restype = ctypes.c_int
    L.fit_probe_fp32.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp,
                                 ctypes.POINTER(ctypes.c_double)]
    L.fit_probe_fp32.restype = ctypes.c_int
    L.fit_relayout.argtypes = [vp, i64, ctypes.c_int, vp, i64, ctypes.c_int, ctypes.c_int, i64, vp]
    L.fit_relayout.restype = ctypes.c_int
    _lib = L
    return L


def _check(code: int):
    if code != FIT_OK:
        raise FitError(code, load().fit_last_error().decode())


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return getattr(stream, "cuda_stream", stream) or None


@dataclass
class Geometry:
    """One mode's surfaces: radii (p2r) or z positions (p2z) in cm, field in T."""
    B: float
    surf: Sequence[float]
    max_iter: int = 10
    tol: float = 1e-6
    start: int = FIT_START_CROSSING  # or FIT_START_LINE: the straight-line start


def _config(g: Optional[Geometry]):
    if g is None:
        return None, None
    arr = (ctypes.c_float * len(g.surf))(*[float(s) for s in g.surf])
    return fit_config(float(g.B), len(g.surf), arr, int(g.max_iter), float(g.tol),
                      int(g.start)), arr


def fit_init(geom_r: Optional[Geometry], geom_z: Optional[Geometry], device: int = 0) -> int:
    L = load()
    h = ctypes.c_void_p()
    cr, _keep_r = _config(geom_r)
    cz, _keep_z = _config(geom_z)
    _check(L.fit_init(ctypes.byref(h), ctypes.byref(cr) if cr else None,
                      ctypes.byref(cz) if cz else None, int(device)))
    return h.value


def fit_propagate_update(h: int, par_in, cov_in, q_in, hpos, hcov, ntrk: Sequence[int],
                         mode: Sequence[int], par_out=None, cov_out=None, q_out=None, chi2=None,
                         chi2_layer=None, status=None, stream=None) -> None:
    """The fused fit on device tensors; outputs default to the inputs (in place)."""
    L = load()
    par_out = par_in if par_out is None else par_out
    cov_out = cov_in if cov_out is None else cov_out
    q_out = q_in if q_out is None else q_out
    nlayer = hpos.shape[0]
    tin = fit_tracks_in(_ptr(par_in), _ptr(cov_in), _ptr(q_in), par_in.shape[-1])
    tout = fit_tracks_out(_ptr(par_out), _ptr(cov_out), _ptr(q_out), _ptr(chi2),
                          _ptr(chi2_layer), _ptr(status), par_out.shape[-1])
    hits = fit_hits(_ptr(hpos), _ptr(hcov), hpos.shape[-1])
    nt = np.ascontiguousarray(ntrk, dtype=np.int64)
    md = np.ascontiguousarray(mode, dtype=np.int32)
    _check(L.fit_propagate_update(
        ctypes.c_void_p(h), ctypes.byref(tin), ctypes.byref(tout), ctypes.byref(hits), len(nt),
        nt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), nlayer,
        md.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _stream_handle(stream)))


def fit_propagate_update_layout(h: int, par_in, cov_in, q_in, hpos, hcov, ntrk: Sequence[int],
                                mode: Sequence[int], layout: int, ld: int, par_out, cov_out, q_out,
                                chi2, chi2_layer=None, status=None, stream=None) -> None:
    """The fused fit on arrays in `layout` (see fit.h); ld = track slots (for
    FIT_LAYOUT_AOSOA32 a multiple of 32).  Tensors are passed by pointer."""
    L = load()
    tin = fit_tracks_in(_ptr(par_in), _ptr(cov_in), _ptr(q_in), ld)
    tout = fit_tracks_out(_ptr(par_out), _ptr(cov_out), _ptr(q_out), _ptr(chi2),
                          _ptr(chi2_layer), _ptr(status), ld)
    hits = fit_hits(_ptr(hpos), _ptr(hcov), ld)
    nt = np.ascontiguousarray(ntrk, dtype=np.int64)
    md = np.ascontiguousarray(mode, dtype=np.int32)
    nlayer = hpos.numel() // (3 * ld)
    _check(L.fit_propagate_update_layout(
        ctypes.c_void_p(h), ctypes.byref(tin), ctypes.byref(tout), ctypes.byref(hits), len(nt),
        nt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), nlayer,
        md.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(layout), _stream_handle(stream)))


def fit_propagate_update_f64(h: int, par_in, cov_in, q_in, hpos, hcov, ntrk: Sequence[int],
                             mode: Sequence[int], par_out, cov_out, q_out, chi2,
                             chi2_layer=None, status=None, stream=None) -> None:
    """The FP64 variant of the fused fit on float64 CUDA tensors (same layouts)."""
    import torch
    for t in (par_in, cov_in, hpos, hcov, par_out, cov_out, chi2):
        if t.dtype != torch.float64:
            raise ValueError("fit_propagate_update_f64 takes float64 tensors")
    L = load()
    tin = fit_tracks_in(_ptr(par_in), _ptr(cov_in), _ptr(q_in), par_in.shape[-1])
    tout = fit_tracks_out(_ptr(par_out), _ptr(cov_out), _ptr(q_out), _ptr(chi2),
                          _ptr(chi2_layer), _ptr(status), par_out.shape[-1])
    hits = fit_hits(_ptr(hpos), _ptr(hcov), hpos.shape[-1])
    nt = np.ascontiguousarray(ntrk, dtype=np.int64)
    md = np.ascontiguousarray(mode, dtype=np.int32)
    _check(L.fit_propagate_update_f64(
        ctypes.c_void_p(h), ctypes.byref(tin), ctypes.byref(tout), ctypes.byref(hits), len(nt),
        nt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), hpos.shape[0],
        md.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _stream_handle(stream)))


def fit_find_tracks(h: int, par_in, cov_in, q_in, cpos, ccov, ntrk: Sequence[int],
                    mode: Sequence[int], chi2_gate: float, chosen, par_out, cov_out, q_out, chi2,
                    chi2_layer=None, status=None, stream=None) -> None:
    """Track finding on CUDA tensors: cpos (nlayer, ncand, 3, ld), ccov
    (nlayer, ncand, 6, ld), chosen (nlayer, ld) int8; float32 tensors call the
    FP32 kernels, float64 tensors the FP64 ones."""
    import torch
    f64 = par_in.dtype == torch.float64
    L = load()
    tin = fit_tracks_in(_ptr(par_in), _ptr(cov_in), _ptr(q_in), par_in.shape[-1])
    tout = fit_tracks_out(_ptr(par_out), _ptr(cov_out), _ptr(q_out), _ptr(chi2),
                          _ptr(chi2_layer), _ptr(status), par_out.shape[-1])
    cand = fit_candidates(_ptr(cpos), _ptr(ccov), cpos.shape[1], cpos.shape[-1])
    nt = np.ascontiguousarray(ntrk, dtype=np.int64)
    md = np.ascontiguousarray(mode, dtype=np.int32)
    fn = L.fit_find_tracks_f64 if f64 else L.fit_find_tracks
    _check(fn(ctypes.c_void_p(h), ctypes.byref(tin), ctypes.byref(tout), ctypes.byref(cand),
              float(chi2_gate), _ptr(chosen), len(nt),
              nt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cpos.shape[0],
              md.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _stream_handle(stream)))


def fit_find_tracks_f64(h: int, par_in, cov_in, q_in, cpos, ccov, ntrk, mode, chi2_gate, chosen,
                        par_out, cov_out, q_out, chi2, chi2_layer=None, status=None,
                        stream=None) -> None:
    """fit_find_tracks on float64 tensors (the FP64 kernels)."""
    import torch
    if par_in.dtype != torch.float64:
        raise ValueError("fit_find_tracks_f64 takes float64 tensors")
    fit_find_tracks(h, par_in, cov_in, q_in, cpos, ccov, ntrk, mode, chi2_gate, chosen, par_out,
                    cov_out, q_out, chi2, chi2_layer, status, stream)


def _hptr(a) -> Optional[int]:
    """Address of a host array: a (pinned) torch CPU tensor or a numpy array."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if a.is_cuda:
            raise ValueError("the host entry points take host arrays")
        return a.data_ptr()
    return np.asarray(a).ctypes.data


def fit_propagate_update_host(h: int, par_in, cov_in, q_in, hpos, hcov, ntrk: Sequence[int],
                              mode: Sequence[int], par_out=None, cov_out=None, q_out=None,
                              chi2=None, chi2_layer=None, status=None, stream=None) -> None:
    """The fused fit on HOST arrays (page-locked torch tensors for overlap, or
    numpy arrays), copied through the library's device staging in chunks; the
    arrays must stay alive until the stream passes the call (fit_sync)."""
    L = load()
    par_out = par_in if par_out is None else par_out
    cov_out = cov_in if cov_out is None else cov_out
    q_out = q_in if q_out is None else q_out
    tin = fit_tracks_in(_hptr(par_in), _hptr(cov_in), _hptr(q_in), par_in.shape[-1])
    tout = fit_tracks_out(_hptr(par_out), _hptr(cov_out), _hptr(q_out), _hptr(chi2),
                          _hptr(chi2_layer), _hptr(status), par_out.shape[-1])
    hits = fit_hits(_hptr(hpos), _hptr(hcov), hpos.shape[-1])
    nt = np.ascontiguousarray(ntrk, dtype=np.int64)
    md = np.ascontiguousarray(mode, dtype=np.int32)
    _check(L.fit_propagate_update_host(
        ctypes.c_void_p(h), ctypes.byref(tin), ctypes.byref(tout), ctypes.byref(hits), len(nt),
        nt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), hpos.shape[0],
        md.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _stream_handle(stream)))


def fit_propagate_update_mapped(h: int, par_in, cov_in, q_in, hpos, hcov, ntrk: Sequence[int],
                                mode: Sequence[int], par_out=None, cov_out=None, q_out=None,
                                chi2=None, chi2_layer=None, status=None, stream=None) -> None:
    """The fused fit reading and writing page-locked HOST tensors in place
    (zero-copy over the host link); the tensors must stay alive, and the
    outputs unread, until the stream passes the call (fit_sync)."""
    L = load()
    par_out = par_in if par_out is None else par_out
    cov_out = cov_in if cov_out is None else cov_out
    q_out = q_in if q_out is None else q_out
    tin = fit_tracks_in(_hptr(par_in), _hptr(cov_in), _hptr(q_in), par_in.shape[-1])
    tout = fit_tracks_out(_hptr(par_out), _hptr(cov_out), _hptr(q_out), _hptr(chi2),
                          _hptr(chi2_layer), _hptr(status), par_out.shape[-1])
    hits = fit_hits(_hptr(hpos), _hptr(hcov), hpos.shape[-1])
    nt = np.ascontiguousarray(ntrk, dtype=np.int64)
    md = np.ascontiguousarray(mode, dtype=np.int32)
    _check(L.fit_propagate_update_mapped(
        ctypes.c_void_p(h), ctypes.byref(tin), ctypes.byref(tout), ctypes.byref(hits), len(nt),
        nt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), hpos.shape[0],
        md.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _stream_handle(stream)))


def fit_propagate_update_noalloc(geom_r: Optional[Geometry], geom_z: Optional[Geometry], par_in,
                                 cov_in, q_in, hpos, hcov, ntrk: Sequence[int],
                                 mode: Sequence[int], par_out=None, cov_out=None, q_out=None,
                                 chi2=None, chi2_layer=None, status=None, stream=None,
                                 per_event: bool = True):
    """The fused fit without a handle and without any allocation by the library.

    For callers that must not allocate device memory while they run (see
    fit.h).  Returns a list with one counter dict per event when per_event is
    true (the call then waits for its work), else None.
    """
    L = load()
    par_out = par_in if par_out is None else par_out
    cov_out = cov_in if cov_out is None else cov_out
    q_out = q_in if q_out is None else q_out
    cr, _keep_r = _config(geom_r)
    cz, _keep_z = _config(geom_z)
    tin = fit_tracks_in(_ptr(par_in), _ptr(cov_in), _ptr(q_in), par_in.shape[-1])
    tout = fit_tracks_out(_ptr(par_out), _ptr(cov_out), _ptr(q_out), _ptr(chi2),
                          _ptr(chi2_layer), _ptr(status), par_out.shape[-1])
    hits = fit_hits(_ptr(hpos), _ptr(hcov), hpos.shape[-1])
    nt = np.ascontiguousarray(ntrk, dtype=np.int64)
    md = np.ascontiguousarray(mode, dtype=np.int32)
    st = (fit_status * max(1, len(nt)))() if per_event else None
    _check(L.fit_propagate_update_noalloc(
        ctypes.byref(cr) if cr else None, ctypes.byref(cz) if cz else None, ctypes.byref(tin),
        ctypes.byref(tout), ctypes.byref(hits), len(nt),
        nt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), hpos.shape[0],
        md.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _stream_handle(stream), st))
    if not per_event:
        return None
    return [{k: int(getattr(st[e], k)) for k, _ in fit_status._fields_} for e in range(len(nt))]


def _buffers(par_in, cov_in, q_in, hpos, hcov, par_out, cov_out, q_out, chi2, chi2_layer, status):
    par_out = par_in if par_out is None else par_out
    cov_out = cov_in if cov_out is None else cov_out
    q_out = q_in if q_out is None else q_out
    tin = fit_tracks_in(_ptr(par_in), _ptr(cov_in), _ptr(q_in), par_in.shape[-1])
    tout = fit_tracks_out(_ptr(par_out), _ptr(cov_out), _ptr(q_out), _ptr(chi2),
                          _ptr(chi2_layer), _ptr(status), par_out.shape[-1])
    return tin, tout, fit_hits(_ptr(hpos), _ptr(hcov), hpos.shape[-1])


def fit_plan_create(h: int, ntrk: Sequence[int], mode: Sequence[int], nlayer: int,
                    threads_per_block: int = 128, blocks_per_sm: int = 0,
                    persistent: bool = True, tracks_per_thread: int = 2,
                    layout: int = FIT_LAYOUT_SOA) -> int:
    """A plan for the batched persistent form (see fit.h)."""
    nt = np.ascontiguousarray(ntrk, dtype=np.int64)
    md = np.ascontiguousarray(mode, dtype=np.int32)
    cfg = fit_launch_config(threads_per_block, blocks_per_sm, int(persistent),
                            int(tracks_per_thread), int(layout))
    p = ctypes.c_void_p()
    _check(load().fit_plan_create(ctypes.c_void_p(h), len(nt),
                                  nt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                  md.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), nlayer,
                                  ctypes.byref(cfg), ctypes.byref(p)))
    return p.value


def fit_plan_run(plan: int, par_in, cov_in, q_in, hpos, hcov, par_out=None, cov_out=None,
                 q_out=None, chi2=None, chi2_layer=None, status=None, stream=None) -> None:
    tin, tout, hits = _buffers(par_in, cov_in, q_in, hpos, hcov, par_out, cov_out, q_out, chi2,
                               chi2_layer, status)
    _check(load().fit_plan_run(ctypes.c_void_p(plan), ctypes.byref(tin), ctypes.byref(tout),
                               ctypes.byref(hits), _stream_handle(stream)))


def fit_plan_tune(plan: int, par_in, cov_in, q_in, hpos, hcov, par_out, cov_out, q_out, chi2,
                  chi2_layer=None, status=None, stream=None, cache_path: Optional[str] = None) -> dict:
    tin, tout, hits = _buffers(par_in, cov_in, q_in, hpos, hcov, par_out, cov_out, q_out, chi2,
                               chi2_layer, status)
    _check(load().fit_plan_tune(ctypes.c_void_p(plan), ctypes.byref(tin), ctypes.byref(tout),
                                ctypes.byref(hits), _stream_handle(stream),
                                cache_path.encode() if cache_path else None))
    return fit_plan_get_info(plan)


def fit_plan_get_info(plan: int) -> dict:
    info = fit_plan_info()
    _check(load().fit_plan_get_info(ctypes.c_void_p(plan), ctypes.byref(info)))
    c = info.config
    return {"threads_per_block": c.threads_per_block, "blocks_per_sm": c.blocks_per_sm,
            "persistent": bool(c.persistent), "tracks_per_thread": c.tracks_per_thread,
            "layout": c.layout,
            "tracks": info.tracks, "items": info.items,
            "tuned": info.tuned, "best_ms": info.best_ms}


def fit_relayout(src, src_layout: int, dst, dst_layout: int, n: Optional[int] = None,
                 stream=None) -> None:
    """Copies the (rows, ld) device array src into dst, converting between
    FIT_LAYOUT_SOA and FIT_LAYOUT_AOSOA32 (4-byte elements; rows = all
    leading dimensions of src but the last; n tracks, default all)."""
    rows = int(np.prod(src.shape[:-1]))
    n = src.shape[-1] if n is None else n
    _check(load().fit_relayout(ctypes.c_void_p(src.data_ptr()), src.shape[-1], int(src_layout),
                               ctypes.c_void_p(dst.data_ptr()), dst.shape[-1], int(dst_layout),
                               rows, int(n), _stream_handle(stream)))


def fit_plan_destroy(plan: int) -> None:
    if plan:
        load().fit_plan_destroy(ctypes.c_void_p(plan))


def fit_tape_bytes(nlayer: int, ld: int) -> int:
    return int(load().fit_tape_bytes(nlayer, ld))


def _events(ntrk, mode):
    nt = np.ascontiguousarray(ntrk, dtype=np.int64)
    md = np.ascontiguousarray(mode, dtype=np.int32)
    return (len(nt), nt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            md.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), nt, md)


def fit_adjoint_forward(h: int, par_in, cov_in, q_in, hpos, hcov, ntrk, mode, tape, par_out,
                        cov_out, q_out, chi2, chi2_layer=None, status=None, stream=None) -> None:
    """The fused fit that also records the per-layer checkpoints in `tape`."""
    tin, tout, hits = _buffers(par_in, cov_in, q_in, hpos, hcov, par_out, cov_out, q_out, chi2,
                               chi2_layer, status)
    nevt, pn, pm, _k1, _k2 = _events(ntrk, mode)
    _check(load().fit_adjoint_forward(ctypes.c_void_p(h), ctypes.byref(tin), ctypes.byref(tout),
                                      ctypes.byref(hits), nevt, pn, hpos.shape[0], pm,
                                      _ptr(tape), _stream_handle(stream)))


def fit_adjoint_backward(h: int, hpos, hcov, ntrk, mode, tape, grad_chi2, grad_hpos, grad_par0,
                         grad_cov0=None, stream=None) -> None:
    """Reverse sweep: gradients of grad_chi2-weighted summed chi2 (see fit.h)."""
    hits = fit_hits(_ptr(hpos), _ptr(hcov), hpos.shape[-1])
    nevt, pn, pm, _k1, _k2 = _events(ntrk, mode)
    _check(load().fit_adjoint_backward(ctypes.c_void_p(h), ctypes.byref(hits), nevt, pn,
                                       hpos.shape[0], pm, _ptr(tape), _ptr(grad_chi2),
                                       _ptr(grad_hpos), _ptr(grad_par0), _ptr(grad_cov0),
                                       _stream_handle(stream)))


def _chi2_function():
    import torch

    class Chi2(torch.autograd.Function):
        """chi2 per track of the fused fit, differentiable in the hit positions
        and the initial parameters and covariance (hand-written adjoint)."""

        @staticmethod
        def forward(ctx, hpos, par0, cov0, q, hcov, fitter, ntrk, mode):
            ld, nlayer = hpos.shape[-1], hpos.shape[0]
            tape = torch.empty(fit_tape_bytes(nlayer, ld) // 4, dtype=torch.float32,
                               device=hpos.device)
            out = fitter.outputs(int(np.sum(ntrk)), ld=ld)
            fit_adjoint_forward(fitter.h, par0, cov0, q, hpos, hcov, ntrk, mode, tape,
                                out["par"], out["cov"], out["q"], out["chi2"],
                                status=out["status"])
            ctx.save_for_backward(hpos, hcov, tape)
            ctx.fitter, ctx.ntrk, ctx.mode = fitter, list(ntrk), list(mode)
            ctx.mark_non_differentiable(out["par"], out["cov"])
            return out["chi2"], out["par"], out["cov"]

        @staticmethod
        def backward(ctx, grad_chi2, _gpar, _gcov):
            hpos, hcov, tape = ctx.saved_tensors
            ld = hpos.shape[-1]
            g_hpos = torch.empty_like(hpos)
            g_par0 = torch.empty((6, ld), dtype=torch.float32, device=hpos.device)
            g_cov0 = torch.empty((21, ld), dtype=torch.float32, device=hpos.device)
            fit_adjoint_backward(ctx.fitter.h, hpos, hcov, ctx.ntrk, ctx.mode, tape,
                                 grad_chi2.contiguous(), g_hpos, g_par0, g_cov0)
            return g_hpos, g_par0, g_cov0, None, None, None, None, None

    return Chi2


_CHI2 = None


def chi2(fitter: "Fitter", hpos, par0, cov0, q, hcov, ntrk, mode):
    """(chi2 per track, fitted par, fitted cov) with autograd through chi2 to
    hpos, par0 and cov0."""
    global _CHI2
    if _CHI2 is None:
        _CHI2 = _chi2_function()
    return _CHI2.apply(hpos, par0, cov0, q, hcov, fitter, ntrk, mode)


# ---- learned path-length seed (p2r) -------------------------------------------------


def fit_mlp_create(device: int = 0, seed: int = 1) -> int:
    m = ctypes.c_void_p()
    _check(load().fit_mlp_create(ctypes.byref(m), int(device), int(seed)))
    return m.value


def fit_mlp_destroy(m: int) -> None:
    if m:
        load().fit_mlp_destroy(ctypes.c_void_p(m))


def fit_mlp_set_params(m: int, params) -> None:
    """params: FIT_MLP_PARAMS floats (host), W1, b1, W2, b2, W3, b3."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.shape != (FIT_MLP_PARAMS,):
        raise ValueError(f"expected {FIT_MLP_PARAMS} parameters, got {p.shape}")
    _check(load().fit_mlp_set_params(ctypes.c_void_p(m), p.ctypes.data))


def fit_mlp_get_params(m: int) -> np.ndarray:
    p = np.empty(FIT_MLP_PARAMS, np.float32)
    _check(load().fit_mlp_get_params(ctypes.c_void_p(m), p.ctypes.data))
    return p


def fit_mlp_prepare(B: float, par, q, R, x, h_exact=None, target=None, n: Optional[int] = None,
                    stream=None) -> None:
    """Network inputs x (n, 8) (and targets from h_exact) of states par (6, ld)."""
    n = R.shape[0] if n is None else n
    _check(load().fit_mlp_prepare(float(B), _ptr(par), par.shape[-1], _ptr(q), _ptr(R),
                                  _ptr(h_exact), n, _ptr(x), _ptr(target), _stream_handle(stream)))


def fit_mlp_forward(m: int, x, y, stream=None) -> None:
    _check(load().fit_mlp_forward(ctypes.c_void_p(m), _ptr(x), x.shape[0], _ptr(y),
                                  _stream_handle(stream)))


def fit_mlp_gradient(m: int, x, target, grad, loss, stream=None) -> None:
    _check(load().fit_mlp_gradient(ctypes.c_void_p(m), _ptr(x), _ptr(target), x.shape[0],
                                   _ptr(grad), _ptr(loss), _stream_handle(stream)))


def fit_mlp_adam_step(m: int, grad, lr: float, stream=None) -> None:
    _check(load().fit_mlp_adam_step(ctypes.c_void_p(m), _ptr(grad), float(lr),
                                    _stream_handle(stream)))


def fit_mlp_train(m: int, x, target, epochs: int, batch: int = 4096, lr: float = 2e-3,
                  lr_final: float = 1e-5, beta1: float = 0.9, beta2: float = 0.999,
                  eps: float = 1e-8, seed: int = 1, stream=None) -> np.ndarray:
    """Adam on the mean squared error; returns the mean loss of each epoch."""
    cfg = fit_mlp_train_config(int(epochs), int(batch), float(lr), float(lr_final), float(beta1),
                               float(beta2), float(eps), int(seed))
    curve = np.zeros(int(epochs), np.float32)
    _check(load().fit_mlp_train(ctypes.c_void_p(m), _ptr(x), _ptr(target), x.shape[0],
                                ctypes.byref(cfg), curve.ctypes.data, _stream_handle(stream)))
    return curve


def fit_mlp_attach(h: int, m: Optional[int], stream=None) -> None:
    _check(load().fit_mlp_attach(ctypes.c_void_p(h), ctypes.c_void_p(m) if m else None,
                                 _stream_handle(stream)))


def fit_path_lengths(h: int, par, q, R, h_out, iters_out=None, seeded: bool = False,
                     n: Optional[int] = None, stream=None) -> None:
    n = R.shape[0] if n is None else n
    it = None if iters_out is None else ctypes.cast(_ptr(iters_out), ctypes.POINTER(ctypes.c_int32))
    _check(load().fit_path_lengths(ctypes.c_void_p(h), _ptr(par), par.shape[-1], _ptr(q), _ptr(R),
                                   n, _ptr(h_out), it, int(bool(seeded)), _stream_handle(stream)))


def fit_sync(h: int, stream=None, timeout_s: float = 0.0) -> dict:
    st = fit_status()
    _check(load().fit_sync(ctypes.c_void_p(h), _stream_handle(stream), float(timeout_s),
                           ctypes.byref(st)))
    return {k: int(getattr(st, k)) for k, _ in fit_status._fields_}


def fit_destroy(h: int) -> None:
    if h:
        load().fit_destroy(ctypes.c_void_p(h))


def fit_last_error() -> str:
    return load().fit_last_error().decode()


FIT_PROBE_THREADS = 256


def fit_probe_fp32(packed: bool, blocks: int, iters: int, out, stream=None) -> float:
    """Queues the FP32 throughput probe (include/fit_probe.h) on `stream`;
    `out` holds at least blocks x FIT_PROBE_THREADS floats.  Returns the
    launch's FP32 flops (FMA = 2)."""
    if out.numel() < blocks * FIT_PROBE_THREADS:
        raise FitError(FIT_ERR_ARG, "fit_probe_fp32: out is too small")
    flops = ctypes.c_double()
    _check(load().fit_probe_fp32(int(bool(packed)), int(blocks), int(iters),
                                 ctypes.c_void_p(out.data_ptr()), _stream_handle(stream),
                                 ctypes.byref(flops)))
    return float(flops.value)


class Fitter:
    """Owns a handle; allocates output tensors; calls fit_propagate_update."""

    def __init__(self, geom_r: Optional[Geometry], geom_z: Optional[Geometry], device: int = 0):
        self.device = device
        self.h = fit_init(geom_r, geom_z, device)
        self.nlayer = len((geom_r or geom_z).surf)

    def close(self):
        if self.h:
            fit_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def outputs(self, n: int, ld: Optional[int] = None, layers: bool = False):
        import torch
        ld = ld or (n + 3) // 4 * 4
        dev = torch.device("cuda", self.device)
        out = {"par": torch.empty((6, ld), device=dev), "cov": torch.empty((21, ld), device=dev),
               "q": torch.empty((ld,), dtype=torch.int32, device=dev),
               "chi2": torch.empty((ld,), device=dev),
               "status": torch.empty((ld,), dtype=torch.uint8, device=dev)}
        out["chi2_layer"] = torch.empty((self.nlayer, ld), device=dev) if layers else None
        return out

    def run(self, par, cov, q, hpos, hcov, ntrk, mode, out=None, layers=False, stream=None):
        n = int(np.sum(ntrk))
        out = out or self.outputs(n, ld=par.shape[-1], layers=layers)
        fit_propagate_update(self.h, par, cov, q, hpos, hcov, ntrk, mode, par_out=out["par"],
                             cov_out=out["cov"], q_out=out["q"], chi2=out["chi2"],
                             chi2_layer=out["chi2_layer"], status=out["status"], stream=stream)
        return out

    def sync(self, stream=None, timeout_s: float = 0.0) -> dict:
        return fit_sync(self.h, stream, timeout_s)
