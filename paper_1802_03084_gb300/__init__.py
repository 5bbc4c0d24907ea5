"""Python binding of the realfast GB300 engine (C ABI in include/realfast_gb300.h).

The functions here carry the C names and only marshal arguments: every step
of the search runs in the CUDA kernels of ``librealfast_gb300.so``.  There is
no CPU fallback: if the library is missing, :func:`lib` raises.

Device buffers and streams may be PyTorch tensors and streams; host inputs
may be numpy arrays or (pinned) CPU tensors.
"""

from __future__ import annotations

import ctypes
import os
import re
from typing import Optional, Sequence

import numpy as np

from .build import lib_path

__all__ = [
    "RfError", "RfPlanDesc", "RfCandidate", "RfImageStat", "RfPlanInfo",
    "lib", "make_desc", "rf_plan_create", "rf_plan_destroy", "rf_search_segment",
    "rf_search_segment_stats", "rf_render_images", "rf_plan_set_form", "rf_plan_get_info",
    "rf_plan_delays", "rf_plan_cells", "rf_count_images", "rf_last_error", "rf_version",
    "rf_plan_set_profiling", "rf_plan_get_profile", "RfKernelProfile", "rf_image_stats_noalloc", "rf_plan_set_tuning", "rf_plan_get_tuning", "rf_plan_autotune",
    "RfTuneReport", "Server", "RfServerDesc", "RfRequestInfo", "rf_plan_estimate_bytes",
    "Stream", "RfStreamInfo", "RfCandidateFeatures", "FEATURES_DTYPE", "rf_candidate_products",
    "RfPeriodicCandidate", "PERIODIC_DTYPE", "rf_periodicity_search", "rf_selftest_bounded_wait",
    "Plan", "CANDIDATE_DTYPE", "STAT_DTYPE", "declared_symbols",
    "RF_STORE_FP16", "RF_EDGE_PARTIAL", "RF_MEAN_SUBTRACT", "RF_NOISE_CLIPPED", "RF_TUNE_WIDE_INDEX", "RF_TUNE_FUSED", "RF_TUNE_RING", "RF_TUNE_OVERLAP", "RF_STREAM_KEEP_STATS", "RF_HOST_ONLY", "RF_FORM_BATCHED", "RF_FORM_PLAIN",
]

RF_OK = 0
RF_ERR_INVALID_ARG = 1
RF_ERR_NO_MEMORY = 2
RF_ERR_CUDA = 3
RF_ERR_SHAPE = 4
RF_ERR_CAPACITY = 5
RF_ERR_TIMEOUT = 6
RF_ERR_BUSY = 7
RF_ERR_NO_DEVICE = 8
STATUS_NAMES = {0: "RF_OK", 1: "RF_ERR_INVALID_ARG", 2: "RF_ERR_NO_MEMORY", 3: "RF_ERR_CUDA",
                4: "RF_ERR_SHAPE", 5: "RF_ERR_CAPACITY", 6: "RF_ERR_TIMEOUT", 7: "RF_ERR_BUSY",
                8: "RF_ERR_NO_DEVICE"}

RF_STORE_FP16 = 0x1
RF_EDGE_PARTIAL = 0x2
RF_MEAN_SUBTRACT = 0x4
RF_NOISE_CLIPPED = 0x8
RF_STREAM_KEEP_STATS = 0x1
RF_HOST_ONLY = 0x100
RF_FORM_BATCHED = 0
RF_FORM_PLAIN = 1
RF_NOALLOC_MAX_NPIX = 1024
RF_TUNE_WAVE_IMAGES = 1
RF_TUNE_GRAPHS = 2
RF_TUNE_WIDE_INDEX = 3
RF_TUNE_FUSED = 4
RF_TUNE_RING = 5
RF_TUNE_OVERLAP = 6

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "realfast_gb300.h")


class RfError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.message = message


class RfPlanDesc(ctypes.Structure):
    _fields_ = [
        ("nant", ctypes.c_int32), ("ant_uvw_m", ctypes.POINTER(ctypes.c_double)),
        ("nchan", ctypes.c_int32), ("freq_hz", ctypes.POINTER(ctypes.c_double)),
        ("npol", ctypes.c_int32), ("inttime_s", ctypes.c_double),
        ("npix", ctypes.c_int32), ("cell_rad", ctypes.c_double),
        ("ndm", ctypes.c_int32), ("dm_list", ctypes.POINTER(ctypes.c_double)),
        ("ndt", ctypes.c_int32), ("dt_list", ctypes.POINTER(ctypes.c_int32)),
        ("threshold_sigma", ctypes.c_double), ("flags", ctypes.c_uint32),
        ("max_nint", ctypes.c_int32), ("device", ctypes.c_int32),
    ]


class RfCandidate(ctypes.Structure):
    _fields_ = [("dm_idx", ctypes.c_int32), ("dt_idx", ctypes.c_int32), ("t_idx", ctypes.c_int32),
                ("x", ctypes.c_int32), ("y", ctypes.c_int32), ("snr", ctypes.c_float),
                ("peak", ctypes.c_float), ("sigma", ctypes.c_float), ("dm", ctypes.c_double),
                ("l_rad", ctypes.c_double), ("m_rad", ctypes.c_double)]


class RfImageStat(ctypes.Structure):
    _fields_ = [("dm_idx", ctypes.c_int32), ("dt_idx", ctypes.c_int32), ("t_idx", ctypes.c_int32),
                ("x", ctypes.c_int32), ("y", ctypes.c_int32), ("peak", ctypes.c_float),
                ("sigma", ctypes.c_float), ("snr", ctypes.c_float), ("mean", ctypes.c_double),
                ("weight", ctypes.c_double)]


class RfPlanInfo(ctypes.Structure):
    _fields_ = [("nbl", ctypes.c_int32), ("nchan", ctypes.c_int32), ("npix", ctypes.c_int32),
                ("ndm", ctypes.c_int32), ("ndt", ctypes.c_int32), ("iu_max", ctypes.c_int32),
                ("iv_max", ctypes.c_int32), ("n_offgrid", ctypes.c_int32), ("n_cells", ctypes.c_int32),
                ("n_entries", ctypes.c_int32), ("max_delay", ctypes.c_int32),
                ("images_per_group", ctypes.c_int32), ("device_bytes", ctypes.c_uint64)]


class RfTuneReport(ctypes.Structure):
    _fields_ = [("best_wave_images", ctypes.c_int32), ("best_graphs", ctypes.c_int32), ("ntried", ctypes.c_int32),
                ("tried_wave_images", ctypes.c_int32 * 16), ("tried_graphs", ctypes.c_int32 * 16),
                ("tried_ms", ctypes.c_float * 16), ("best_fused", ctypes.c_int32), ("best_ring", ctypes.c_int32),
                ("tried_fused", ctypes.c_int32 * 16), ("tried_ring", ctypes.c_int32 * 16),
                ("best_overlap", ctypes.c_int32), ("tried_overlap", ctypes.c_int32 * 16)]


class RfServerDesc(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("slots", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_uint64),
                ("wave_images", ctypes.c_int64)]


class RfRequestInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("done", ctypes.c_int32), ("submit_s", ctypes.c_double),
                ("start_s", ctypes.c_double), ("done_s", ctypes.c_double), ("n_images", ctypes.c_int64),
                ("n_candidates", ctypes.c_uint64), ("plan_reused", ctypes.c_int32)]


class RfCandidateFeatures(ctypes.Structure):
    _fields_ = [("dm_idx", ctypes.c_int32), ("dt_idx", ctypes.c_int32), ("t_idx", ctypes.c_int32),
                ("x", ctypes.c_int32), ("y", ctypes.c_int32), ("nchan_used", ctypes.c_int32),
                ("image_mean", ctypes.c_double), ("image_sigma", ctypes.c_double),
                ("image_skew", ctypes.c_double), ("image_kurtosis", ctypes.c_double),
                ("spec_mean", ctypes.c_double), ("spec_std", ctypes.c_double),
                ("spec_skew", ctypes.c_double), ("spec_kurtosis", ctypes.c_double),
                ("peak_from_spectrum", ctypes.c_double)]


class RfPeriodicCandidate(ctypes.Structure):
    _fields_ = [("dm_idx", ctypes.c_int32), ("k", ctypes.c_int32), ("x", ctypes.c_int32), ("y", ctypes.c_int32),
                ("snr", ctypes.c_float), ("amplitude", ctypes.c_float), ("sigma", ctypes.c_float),
                ("pad", ctypes.c_float), ("dm", ctypes.c_double), ("freq_hz", ctypes.c_double),
                ("l_rad", ctypes.c_double), ("m_rad", ctypes.c_double)]


class RfStreamInfo(ctypes.Structure):
    _fields_ = [("stride", ctypes.c_int32), ("overlap", ctypes.c_int32), ("segment_nint", ctypes.c_int32),
                ("fill", ctypes.c_int32), ("pushed", ctypes.c_int64), ("segments", ctypes.c_int64),
                ("pending_candidates", ctypes.c_uint64), ("pending_stats", ctypes.c_uint64)]


class RfKernelProfile(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


def _np_dtype(struct) -> np.dtype:
    m = {ctypes.c_int32: "i4", ctypes.c_float: "f4", ctypes.c_double: "f8", ctypes.c_uint64: "u8"}
    names = [f[0] for f in struct._fields_]
    fmts = [m[f[1]] for f in struct._fields_]
    offs = [getattr(struct, n).offset for n in names]
    return np.dtype({"names": names, "formats": fmts, "offsets": offs, "itemsize": ctypes.sizeof(struct)})


CANDIDATE_DTYPE = _np_dtype(RfCandidate)
STAT_DTYPE = _np_dtype(RfImageStat)
FEATURES_DTYPE = _np_dtype(RfCandidateFeatures)
PERIODIC_DTYPE = _np_dtype(RfPeriodicCandidate)

_LIB = None


def lib() -> ctypes.CDLL:
    """Load the engine library (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1802_03084_gb300.build.build()")
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    S = ctypes.c_size_t
    sig = {
        "rf_plan_create": ([ctypes.POINTER(RfPlanDesc), ctypes.POINTER(P)], ctypes.c_int),
        "rf_plan_destroy": ([P], ctypes.c_int),
        "rf_last_error": ([], ctypes.c_char_p),
        "rf_version": ([], ctypes.c_char_p),
        "rf_search_segment": ([P, P, ctypes.c_int32, P, P, S, ctypes.POINTER(S)], ctypes.c_int),
        "rf_search_segment_stats": ([P, P, ctypes.c_int32, P, P, S, ctypes.POINTER(S), P, S, ctypes.POINTER(S)],
                                    ctypes.c_int),
        "rf_render_images": ([P, P, ctypes.c_int32, P, P, ctypes.c_int32, P], ctypes.c_int),
        "rf_plan_set_form": ([P, ctypes.c_int32], ctypes.c_int),
        "rf_plan_get_info": ([P, ctypes.POINTER(RfPlanInfo)], ctypes.c_int),
        "rf_plan_delays": ([P, P], ctypes.c_int),
        "rf_plan_cells": ([P, P, P, P], ctypes.c_int),
        "rf_count_images": ([P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "rf_plan_set_profiling": ([P, ctypes.c_int32], ctypes.c_int),
        "rf_plan_set_tuning": ([P, ctypes.c_int32, ctypes.c_int64], ctypes.c_int),
        "rf_plan_get_tuning": ([P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "rf_image_stats_noalloc": ([P, ctypes.c_int32, ctypes.c_double, P, P], ctypes.c_int),
        "rf_plan_autotune": ([P, P, ctypes.c_int32, P, ctypes.POINTER(RfTuneReport)], ctypes.c_int),
        "rf_plan_estimate_bytes": ([ctypes.POINTER(RfPlanDesc), ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64)],
                                   ctypes.c_int),
        "rf_server_create": ([ctypes.POINTER(RfServerDesc), ctypes.POINTER(P)], ctypes.c_int),
        "rf_server_submit": ([P, ctypes.POINTER(RfPlanDesc), P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)],
                             ctypes.c_int),
        "rf_server_wait": ([P, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(RfRequestInfo)], ctypes.c_int),
        "rf_server_results": ([P, ctypes.c_int64, P, S, ctypes.POINTER(S)], ctypes.c_int),
        "rf_server_destroy": ([P], ctypes.c_int),
        "rf_plan_get_profile": ([P, P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "rf_periodicity_search": ([P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_double, P, P, S, ctypes.POINTER(S), P, S, ctypes.POINTER(S)], ctypes.c_int),
        "rf_selftest_bounded_wait": ([ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "rf_candidate_products": ([P, P, ctypes.c_int32, P, P, ctypes.c_int32, P, P, P], ctypes.c_int),
        "rf_stream_create": ([P, ctypes.c_int32, ctypes.c_uint32, ctypes.POINTER(P)], ctypes.c_int),
        "rf_stream_push": ([P, P, ctypes.c_int32, P, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "rf_stream_flush": ([P, P, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "rf_stream_pop": ([P, P, S, ctypes.POINTER(S)], ctypes.c_int),
        "rf_stream_pop_stats": ([P, P, S, ctypes.POINTER(S)], ctypes.c_int),
        "rf_stream_get_info": ([P, ctypes.POINTER(RfStreamInfo)], ctypes.c_int),
        "rf_stream_destroy": ([P], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _LIB = L
    return L


def declared_symbols() -> list:
    """Function names declared in include/realfast_gb300.h."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rf_[a-z0-9_]+)\s*\(", text)))


def _check(status: int):
    if status != RF_OK:
        raise RfError(status, rf_last_error())


def rf_last_error() -> str:
    return lib().rf_last_error().decode()


def rf_version() -> str:
    return lib().rf_version().decode()


def make_desc(ant_uvw, freq_hz, inttime_s, npix, cell_rad, dm_list, dt_list, threshold,
              npol=2, flags=0, max_nint=1, device=0) -> RfPlanDesc:
    """Build an RfPlanDesc; the numpy arrays it points to are kept on it."""
    ant = np.ascontiguousarray(ant_uvw, dtype=np.float64)
    fr = np.ascontiguousarray(freq_hz, dtype=np.float64)
    dm = np.ascontiguousarray(dm_list, dtype=np.float64)
    dt = np.ascontiguousarray(dt_list, dtype=np.int32)
    D = ctypes.POINTER(ctypes.c_double)
    d = RfPlanDesc(nant=ant.shape[0], ant_uvw_m=ant.ctypes.data_as(D), nchan=fr.shape[0],
                   freq_hz=fr.ctypes.data_as(D), npol=npol, inttime_s=inttime_s, npix=npix,
                   cell_rad=cell_rad, ndm=dm.shape[0], dm_list=dm.ctypes.data_as(D), ndt=dt.shape[0],
                   dt_list=dt.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), threshold_sigma=threshold,
                   flags=flags, max_nint=max_nint, device=device)
    d._keep = (ant, fr, dm, dt)
    return d


def rf_plan_create(desc: RfPlanDesc) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().rf_plan_create(ctypes.byref(desc), ctypes.byref(h)))
    return h


def rf_plan_destroy(plan) -> None:
    _check(lib().rf_plan_destroy(plan))


def _ptr(x) -> int:
    """Data pointer of a torch tensor or numpy array (must be C contiguous)."""
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    a = np.asarray(x)
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C contiguous")
    return a.ctypes.data


def _stream(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def rf_search_segment(plan, vis, nint: int, stream=None, cap: Optional[int] = None) -> np.ndarray:
    """Search one segment; returns a structured array (CANDIDATE_DTYPE)."""
    L = lib()
    if cap is None:
        n = ctypes.c_int64()
        _check(L.rf_count_images(plan, nint, ctypes.byref(n)))
        cap = max(int(n.value), 1)
    out = np.zeros(cap, dtype=CANDIDATE_DTYPE)
    n_out = ctypes.c_size_t()
    _check(L.rf_search_segment(plan, _ptr(vis), nint, _stream(stream), out.ctypes.data, cap, ctypes.byref(n_out)))
    return out[:n_out.value]


def rf_search_segment_stats(plan, vis, nint: int, stream=None):
    """Search and also return the statistics of every searched image."""
    L = lib()
    n = ctypes.c_int64()
    _check(L.rf_count_images(plan, nint, ctypes.byref(n)))
    cap = max(int(n.value), 1)
    out = np.zeros(cap, dtype=CANDIDATE_DTYPE)
    st = np.zeros(cap, dtype=STAT_DTYPE)
    n_out = ctypes.c_size_t()
    n_st = ctypes.c_size_t()
    _check(L.rf_search_segment_stats(plan, _ptr(vis), nint, _stream(stream), out.ctypes.data, cap,
                                     ctypes.byref(n_out), st.ctypes.data, cap, ctypes.byref(n_st)))
    return out[:n_out.value], st[:n_st.value]


def rf_render_images(plan, vis, nint: int, trials: Sequence, npix: int, stream=None) -> np.ndarray:
    """Full dirty images of the listed (dm_idx, dt_idx, t_idx) trials, [n, N, N] float32."""
    tr = np.ascontiguousarray(np.asarray(trials, dtype=np.int32).reshape(-1, 3))
    out = np.zeros((tr.shape[0], npix, npix), dtype=np.float32)
    _check(lib().rf_render_images(plan, _ptr(vis), nint, _stream(stream), tr.ctypes.data, tr.shape[0],
                                  out.ctypes.data))
    return out


def rf_candidate_products(plan, vis, nint: int, cands, npix: int, nchan: int, spectra=True, images=True,
                          stream=None):
    """Features [n] (FEATURES_DTYPE) and, if asked, spectra [n, nchan] complex64
    and images [n, N, N] float32 of the given candidates (CANDIDATE_DTYPE)."""
    c = np.ascontiguousarray(cands, dtype=CANDIDATE_DTYPE)
    n = c.shape[0]
    feats = np.zeros(max(n, 1), dtype=FEATURES_DTYPE)
    sp = np.zeros((max(n, 1), nchan), dtype=np.complex64) if spectra else None
    im = np.zeros((max(n, 1), npix, npix), dtype=np.float32) if images else None
    _check(lib().rf_candidate_products(plan, _ptr(vis), nint, _stream(stream), c.ctypes.data, n,
                                       feats.ctypes.data, sp.ctypes.data if spectra else None,
                                       im.ctypes.data if images else None))
    return feats[:n], (sp[:n] if spectra else None), (im[:n] if images else None)


def rf_periodicity_search(plan, vis, nint: int, L: int, kmin: int, kmax: int, threshold: float, ndm: int,
                          with_stats=False, stream=None):
    """Periodicity search: candidates (PERIODIC_DTYPE) and, with_stats, every
    searched (DM, k) in (dm_idx, k) order."""
    cap = max(ndm * (kmax - kmin + 1), 1)
    out = np.zeros(cap, dtype=PERIODIC_DTYPE)
    st = np.zeros(cap if with_stats else 1, dtype=PERIODIC_DTYPE)
    n_out = ctypes.c_size_t()
    n_st = ctypes.c_size_t()
    _check(lib().rf_periodicity_search(plan, _ptr(vis), nint, L, kmin, kmax, threshold, _stream(stream),
                                       out.ctypes.data, cap, ctypes.byref(n_out),
                                       st.ctypes.data if with_stats else None, cap if with_stats else 0,
                                       ctypes.byref(n_st)))
    if with_stats:
        return out[:n_out.value], st[:n_st.value]
    return out[:n_out.value]


def rf_selftest_bounded_wait(device: int = 0, polls: int = 1000) -> int:
    """1 if the device-side bounded wait gave up as it must (see the header)."""
    g = ctypes.c_int32()
    _check(lib().rf_selftest_bounded_wait(device, polls, ctypes.byref(g)))
    return int(g.value)


def rf_plan_set_form(plan, form: int) -> None:
    _check(lib().rf_plan_set_form(plan, form))


def rf_plan_get_info(plan) -> RfPlanInfo:
    info = RfPlanInfo()
    _check(lib().rf_plan_get_info(plan, ctypes.byref(info)))
    return info


def rf_plan_delays(plan) -> np.ndarray:
    info = rf_plan_get_info(plan)
    out = np.zeros((info.ndm, info.nchan), dtype=np.int32)
    _check(lib().rf_plan_delays(plan, out.ctypes.data))
    return out


def rf_plan_cells(plan):
    info = rf_plan_get_info(plan)
    iu = np.zeros((info.nbl, info.nchan), dtype=np.int32)
    iv = np.zeros_like(iu)
    on = np.zeros((info.nbl, info.nchan), dtype=np.uint8)
    _check(lib().rf_plan_cells(plan, iu.ctypes.data, iv.ctypes.data, on.ctypes.data))
    return iu, iv, on.astype(bool)


def rf_count_images(plan, nint: int) -> int:
    n = ctypes.c_int64()
    _check(lib().rf_count_images(plan, nint, ctypes.byref(n)))
    return int(n.value)


def rf_plan_set_profiling(plan, enable: bool) -> None:
    _check(lib().rf_plan_set_profiling(plan, 1 if enable else 0))


def rf_plan_get_profile(plan) -> dict:
    """{kernel name: (launches, total_ms)} accumulated since profiling was enabled."""
    arr = (RfKernelProfile * 16)()
    n = ctypes.c_int32()
    _check(lib().rf_plan_get_profile(plan, arr, 16, ctypes.byref(n)))
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(min(n.value, 16))}


def rf_plan_set_tuning(plan, key: int, value: int) -> None:
    _check(lib().rf_plan_set_tuning(plan, key, value))


def rf_plan_get_tuning(plan, key: int) -> int:
    v = ctypes.c_int64()
    _check(lib().rf_plan_get_tuning(plan, key, ctypes.byref(v)))
    return int(v.value)


def rf_plan_autotune(plan, vis, nint: int, stream=None) -> dict:
    """Time the tuning ladder on this segment, apply the fastest, return what was tried."""
    rep = RfTuneReport()
    _check(lib().rf_plan_autotune(plan, _ptr(vis), nint, _stream(stream), ctypes.byref(rep)))
    return {"wave_images": rep.best_wave_images, "graphs": rep.best_graphs, "fused": rep.best_fused,
            "ring": rep.best_ring, "overlap": rep.best_overlap,
            "tried": [(rep.tried_wave_images[i], rep.tried_graphs[i], rep.tried_fused[i], rep.tried_ring[i],
                       rep.tried_overlap[i], float(rep.tried_ms[i])) for i in range(rep.ntried)]}


def rf_image_stats_noalloc(half_plane, npix: int, weight: float, stat, stream=None) -> None:
    """Image one device half plane into the device rf_image_stat `stat` (no allocation)."""
    _check(lib().rf_image_stats_noalloc(_ptr(half_plane), npix, weight, _stream(stream), _ptr(stat)))


def rf_plan_estimate_bytes(desc: RfPlanDesc, wave_images: int = 0) -> int:
    b = ctypes.c_uint64()
    _check(lib().rf_plan_estimate_bytes(ctypes.byref(desc), wave_images, ctypes.byref(b)))
    return int(b.value)


class Stream:
    """Continuous search of a run of integrations in segments that overlap by
    the plan's longest sweep (rf_stream_* in the C ABI).  t_idx of every
    output counts from the start of the run."""

    def __init__(self, plan, stride: int, keep_stats: bool = False):
        self.plan = plan
        self.handle = ctypes.c_void_p()
        flags = RF_STREAM_KEEP_STATS if keep_stats else 0
        _check(lib().rf_stream_create(plan.handle, stride, flags, ctypes.byref(self.handle)))

    def push(self, vis, nint=None, stream=None) -> int:
        """Append integrations (host or device); returns the segments searched."""
        n = ctypes.c_int32()
        nint = len(vis) if nint is None else nint
        _check(lib().rf_stream_push(self.handle, _ptr(vis), nint, _stream(stream), ctypes.byref(n)))
        return int(n.value)

    def flush(self, stream=None) -> int:
        n = ctypes.c_int32()
        _check(lib().rf_stream_flush(self.handle, _stream(stream), ctypes.byref(n)))
        return int(n.value)

    def info(self) -> dict:
        i = RfStreamInfo()
        _check(lib().rf_stream_get_info(self.handle, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in RfStreamInfo._fields_}

    def pop(self) -> np.ndarray:
        cap = max(int(self.info()["pending_candidates"]), 1)
        out = np.zeros(cap, dtype=CANDIDATE_DTYPE)
        n = ctypes.c_size_t()
        _check(lib().rf_stream_pop(self.handle, out.ctypes.data, cap, ctypes.byref(n)))
        return out[:n.value]

    def pop_stats(self) -> np.ndarray:
        cap = max(int(self.info()["pending_stats"]), 1)
        out = np.zeros(cap, dtype=STAT_DTYPE)
        n = ctypes.c_size_t()
        _check(lib().rf_stream_pop_stats(self.handle, out.ctypes.data, cap, ctypes.byref(n)))
        return out[:n.value]

    def close(self):
        if self.handle:
            _check(lib().rf_stream_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Server:
    """Serving runtime: resident plans, admission by HBM budget, `slots`
    segments in flight on their own streams (rf_server_* in the C ABI)."""

    def __init__(self, device=0, slots=2, hbm_budget_bytes=64 << 30, wave_images=0):
        self.desc = RfServerDesc(device=device, slots=slots, hbm_budget_bytes=hbm_budget_bytes,
                                 wave_images=wave_images)
        self.handle = ctypes.c_void_p()
        _check(lib().rf_server_create(ctypes.byref(self.desc), ctypes.byref(self.handle)))
        self._keep = {}

    def submit(self, desc: RfPlanDesc, vis, nint: int) -> int:
        """Queue a segment; `vis` (and `desc`'s arrays) are kept alive until results() is called."""
        t = ctypes.c_int64()
        _check(lib().rf_server_submit(self.handle, ctypes.byref(desc), _ptr(vis), nint, ctypes.byref(t)))
        self._keep[t.value] = (desc, vis)
        return int(t.value)

    def wait(self, ticket: int, timeout_ms: int = -1) -> dict:
        info = RfRequestInfo()
        st = lib().rf_server_wait(self.handle, ticket, timeout_ms, ctypes.byref(info))
        if st not in (RF_OK, RF_ERR_TIMEOUT):
            raise RfError(st, rf_last_error())
        return {f: getattr(info, f) for f, _ in RfRequestInfo._fields_}

    def results(self, ticket: int) -> np.ndarray:
        info = self.wait(ticket)
        cap = max(int(info["n_candidates"]), 1)
        out = np.zeros(cap, dtype=CANDIDATE_DTYPE)
        n = ctypes.c_size_t()
        _check(lib().rf_server_results(self.handle, ticket, out.ctypes.data, cap, ctypes.byref(n)))
        self._keep.pop(ticket, None)
        return out[:n.value]

    def close(self):
        if self.handle:
            _check(lib().rf_server_destroy(self.handle))
            self.handle = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Plan:
    """Owning wrapper around an rf_plan handle."""

    def __init__(self, ant_uvw, freq_hz, inttime_s, npix, cell_rad, dm_list, dt_list, threshold,
                 npol=2, flags=0, max_nint=1, device=0):
        self.desc = make_desc(ant_uvw, freq_hz, inttime_s, npix, cell_rad, dm_list, dt_list, threshold,
                              npol=npol, flags=flags, max_nint=max_nint, device=device)
        self.npix = npix
        self.handle = rf_plan_create(self.desc)

    @classmethod
    def from_spec(cls, spec, ant_uvw, freq_hz, flags=None, max_nint=None, device=0):
        """Plan for a ``synth.SegmentSpec``-like object (edge/store fields select flags)."""
        if flags is None:
            flags = 0
            if getattr(spec, "edge", "full") == "partial":
                flags |= RF_EDGE_PARTIAL
            if getattr(spec, "store", "fp32") == "fp16":
                flags |= RF_STORE_FP16
            if getattr(spec, "mean_subtract", False):
                flags |= RF_MEAN_SUBTRACT
            if getattr(spec, "noise_clipped", False):
                flags |= RF_NOISE_CLIPPED
        return cls(ant_uvw, freq_hz, spec.inttime_s, spec.npix, spec.cell_rad, spec.dm_list, spec.dt_list,
                   spec.threshold, npol=spec.npol, flags=flags, max_nint=max_nint or spec.nint, device=device)

    def search(self, vis, nint=None, stream=None):
        return rf_search_segment(self.handle, vis, nint if nint is not None else len(vis), stream)

    def search_stats(self, vis, nint=None, stream=None):
        return rf_search_segment_stats(self.handle, vis, nint if nint is not None else len(vis), stream)

    def render(self, vis, trials, nint=None, stream=None):
        return rf_render_images(self.handle, vis, nint if nint is not None else len(vis), trials, self.npix, stream)

    def periodicity_search(self, vis, L, kmin, kmax, threshold, nint=None, with_stats=False, stream=None):
        """Fourier transform over time and image each fluctuation frequency."""
        nint = nint if nint is not None else len(vis)
        return rf_periodicity_search(self.handle, vis, nint, L, kmin, kmax, threshold, self.desc.ndm, with_stats,
                                     stream)

    def candidate_products(self, vis, cands, nint=None, spectra=True, images=True, stream=None):
        """Features (and spectra, images) of candidates of this segment."""
        nint = nint if nint is not None else len(vis)
        return rf_candidate_products(self.handle, vis, nint, cands, self.npix, self.desc.nchan, spectra, images,
                                     stream)

    def candidate_tiers(self, vis, cands, stats_sigma=6.0, plot_sigma=7.0, nint=None, stream=None):
        """Sec. 3.3 tiers: features for candidates with snr >= stats_sigma,
        spectra and images as well for those with snr >= plot_sigma.
        Returns (features, plot_index, spectra, images); plot_index indexes
        the features array."""
        c = np.asarray(cands, dtype=CANDIDATE_DTYPE)
        c = c[c["snr"] >= stats_sigma]
        if len(c) == 0:
            return np.zeros(0, FEATURES_DTYPE), np.zeros(0, np.int64), None, None
        feats, _, _ = self.candidate_products(vis, c, nint, spectra=False, images=False, stream=stream)
        idx = np.nonzero(c["snr"] >= plot_sigma)[0]
        sp = im = None
        if len(idx):
            _, sp, im = self.candidate_products(vis, c[idx], nint, stream=stream)
        return feats, idx, sp, im

    def info(self) -> RfPlanInfo:
        return rf_plan_get_info(self.handle)

    def delays(self):
        return rf_plan_delays(self.handle)

    def cells(self):
        return rf_plan_cells(self.handle)

    def count_images(self, nint: int) -> int:
        return rf_count_images(self.handle, nint)

    def set_form(self, form: int):
        rf_plan_set_form(self.handle, form)

    def set_profiling(self, enable: bool = True):
        rf_plan_set_profiling(self.handle, enable)

    def profile(self) -> dict:
        return rf_plan_get_profile(self.handle)

    def set_wave_images(self, n: int):
        rf_plan_set_tuning(self.handle, RF_TUNE_WAVE_IMAGES, n)

    def wave_images(self) -> int:
        return rf_plan_get_tuning(self.handle, RF_TUNE_WAVE_IMAGES)

    def set_graphs(self, enable: bool):
        rf_plan_set_tuning(self.handle, RF_TUNE_GRAPHS, 1 if enable else 0)

    def set_wide_index(self, enable: bool):
        """Gridding with 64-bit sample offsets even where 32-bit ones fit."""
        rf_plan_set_tuning(self.handle, RF_TUNE_WIDE_INDEX, 1 if enable else 0)

    def set_fused(self, enable: bool):
        """The fused column + row pass (npix 1024 .. 4096) on or off."""
        rf_plan_set_tuning(self.handle, RF_TUNE_FUSED, 1 if enable else 0)

    def set_ring(self, slots: int):
        """Chunk slots of the fused pass's L2-resident ring (2 .. 8)."""
        rf_plan_set_tuning(self.handle, RF_TUNE_RING, slots)

    def set_overlap(self, enable: bool):
        """Overlapped waves: one wave's column pass beside the previous wave's row pass."""
        rf_plan_set_tuning(self.handle, RF_TUNE_OVERLAP, 1 if enable else 0)

    def autotune(self, vis, nint=None, stream=None, cache_path=None, key_extra=""):
        """Apply a cached tuning for this shape, or run the autotuner and cache it.

        The cache is a JSON file mapping a shape key (image size, channels,
        baselines, trials, segment length, flags, device name) to the chosen
        wave size and graph mode.
        """
        import json
        n = nint if nint is not None else len(vis)
        info = self.info()
        try:
            import torch
            dev = torch.cuda.get_device_name(self.desc.device)
        except Exception:
            dev = "cuda"
        key = f"{info.npix}/{info.nchan}/{info.nbl}/{info.ndm}/{info.ndt}/{n}/{self.desc.flags}/{dev}{key_extra}"
        cache = {}
        if cache_path and os.path.exists(cache_path):
            try:
                with open(cache_path) as f:
                    cache = json.load(f)
            except (OSError, ValueError):
                cache = {}
        if key in cache and "overlap" in cache[key]:
            rf_plan_set_tuning(self.handle, RF_TUNE_WAVE_IMAGES, int(cache[key]["wave_images"]))
            rf_plan_set_tuning(self.handle, RF_TUNE_GRAPHS, int(cache[key]["graphs"]))
            rf_plan_set_tuning(self.handle, RF_TUNE_FUSED, int(cache[key]["fused"]))
            rf_plan_set_tuning(self.handle, RF_TUNE_RING, int(cache[key]["ring"]))
            rf_plan_set_tuning(self.handle, RF_TUNE_OVERLAP, int(cache[key]["overlap"]))
            return dict(cache[key], cached=True)
        res = rf_plan_autotune(self.handle, vis, n, stream)
        if cache_path:
            cache[key] = {"wave_images": res["wave_images"], "graphs": res["graphs"], "fused": res["fused"],
                          "ring": res["ring"], "overlap": res["overlap"]}
            os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1)
        return dict(res, cached=False)

    def close(self):
        if self.handle:
            rf_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
