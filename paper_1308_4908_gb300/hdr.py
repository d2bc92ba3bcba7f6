"""Thin ctypes binding of the C ABI in include/hdr_lpa.h (argument marshalling only).

Every entry point of the library is exposed under its C name; `Context` adds a
small convenience layer that takes torch tensors (device memory and streams are
torch's; all computation runs in the library's CUDA kernels). There is no CPU
fallback: importing works without a GPU, but every call needs the compiled
library and a CUDA device, and fails loudly otherwise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

HDR_MAX_SENSORS = 8
HDR_MAX_SCALES = 8

HDR_OK, HDR_E_INVALID, HDR_E_NOMEM, HDR_E_CUDA, HDR_E_BUSY, HDR_E_TIMEOUT, HDR_E_UNSUPPORTED, HDR_E_INTERNAL = range(8)
STATUS_NAMES = {0: "HDR_OK", 1: "HDR_E_INVALID", 2: "HDR_E_NOMEM", 3: "HDR_E_CUDA", 4: "HDR_E_BUSY",
                5: "HDR_E_TIMEOUT", 6: "HDR_E_UNSUPPORTED", 7: "HDR_E_INTERNAL"}


class hdr_sensor_desc(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("pitch_elems", ctypes.c_int32),
                ("cfa", ctypes.c_int32), ("gain", ctypes.c_double), ("exposure", ctypes.c_double),
                ("nd", ctypes.c_double), ("read_var", ctypes.c_double), ("black", ctypes.c_double),
                ("sat", ctypes.c_double), ("affine", ctypes.c_double * 6),
                ("bias_frame", ctypes.c_void_p), ("prnu_frame", ctypes.c_void_p),
                ("read_var_frame", ctypes.c_void_p), ("sat_frame", ctypes.c_void_p)]


class hdr_params(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int32), ("n_scales", ctypes.c_int32),
                ("sigma", ctypes.c_double * HDR_MAX_SCALES), ("green_ratio", ctypes.c_double),
                ("trunc_k", ctypes.c_double), ("ici_gamma", ctypes.c_double), ("min_pivot", ctypes.c_double),
                ("cond_fallback", ctypes.c_double), ("out_w", ctypes.c_int32), ("out_h", ctypes.c_int32),
                ("out_affine", ctypes.c_double * 6), ("out_dtype", ctypes.c_int32), ("accum", ctypes.c_int32),
                ("tab_weights", ctypes.c_int32), ("weight_mode", ctypes.c_int32)]


class hdr_calpa_params(ctypes.Structure):
    _fields_ = [("grad_sigma", ctypes.c_double), ("window_sigma", ctypes.c_double), ("alpha", ctypes.c_double),
                ("lambda1", ctypes.c_double), ("lambda2", ctypes.c_double), ("min_eig", ctypes.c_double),
                ("max_eig", ctypes.c_double), ("grad_scale", ctypes.c_double)]


class hdr_frame(ctypes.Structure):
    _fields_ = [("rig_id", ctypes.c_int32), ("params", ctypes.c_void_p),
                ("raw_dev", ctypes.c_void_p * HDR_MAX_SENSORS), ("out_dev", ctypes.c_void_p),
                ("choice_dev", ctypes.c_void_p), ("calpa", ctypes.c_void_p)]


class hdr_batch_config(ctypes.Structure):
    _fields_ = [("tile_h", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("cost_order", ctypes.c_int32),
                ("form", ctypes.c_int32), ("px_per_thread", ctypes.c_int32),
                ("stages", ctypes.c_int32)]


class hdr_server_config(ctypes.Structure):
    _fields_ = [("max_frames", ctypes.c_int32), ("pool_bytes", ctypes.c_uint64), ("step_tiles", ctypes.c_int32),
                ("batch", hdr_batch_config), ("order", ctypes.c_int32)]


class hdr_request(ctypes.Structure):
    _fields_ = [("rig_id", ctypes.c_int32), ("params", hdr_params),
                ("raw_host", ctypes.c_void_p * HDR_MAX_SENSORS), ("out_host", ctypes.c_void_p),
                ("choice_host", ctypes.c_void_p), ("stream_id", ctypes.c_int32), ("adaptive", ctypes.c_int32),
                ("calpa", hdr_calpa_params)]


class hdr_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("queue_ms", ctypes.c_double), ("total_ms", ctypes.c_double),
                ("steps", ctypes.c_int32)]


class hdr_server_stats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("submitted", ctypes.c_uint64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double), ("mean_queue_ms", ctypes.c_double),
                ("steps", ctypes.c_uint64), ("output_pixels", ctypes.c_uint64), ("busy_s", ctypes.c_double),
                ("gpu_step_ms", ctypes.c_double), ("gpu_gap_ms", ctypes.c_double),
                ("host_step_ms_mean", ctypes.c_double), ("host_step_ms_max", ctypes.c_double)]


class HdrError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None
_P = ctypes.c_void_p


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libhdrlpa.so (building it with nvcc first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"{path} is missing: run paper_1308_4908_gb300.build.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    lib.hdr_params_default.argtypes = [_P]
    lib.hdr_params_default.restype = None
    lib.hdr_create.argtypes = [ctypes.c_int, _P]
    lib.hdr_destroy.argtypes = [_P]
    lib.hdr_destroy.restype = None
    lib.hdr_set_rig.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, _P]
    lib.hdr_reconstruct.argtypes = [_P, ctypes.c_int32, _P, _P, _P, _P, _P]
    lib.hdr_reconstruct_levels.argtypes = [_P, ctypes.c_int32, _P, _P, _P, _P, _P, _P]
    lib.hdr_reconstruct_host.argtypes = [_P, ctypes.c_int32, _P, _P, _P, _P, _P]
    lib.hdr_check.argtypes = [_P, _P]
    lib.hdr_selftest_timeout.argtypes = [_P, _P]
    lib.hdr_calib_stack_stats.argtypes = [_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int64, _P, _P, _P]
    lib.hdr_calib_gain.argtypes = [_P, _P, _P, _P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                   ctypes.c_double, _P, _P, _P]
    lib.hdr_calib_exposure.argtypes = [_P, _P, _P, ctypes.c_double, ctypes.c_double, _P, _P, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                       ctypes.c_double, _P, _P, _P, _P]
    lib.hdr_reconstruct_noalloc.argtypes = [ctypes.c_int, ctypes.c_int32, _P, _P, _P, _P, _P, _P]
    lib.hdr_reconstruct_batch.argtypes = [_P, ctypes.c_int32, _P, _P, _P]
    lib.hdr_tune_batch.argtypes = [_P, ctypes.c_int32, _P, _P, _P]
    lib.hdr_server_create.argtypes = [_P, _P, _P]
    lib.hdr_submit.argtypes = [_P, _P, _P]
    lib.hdr_poll.argtypes = [_P, ctypes.c_uint64, ctypes.c_int32, _P]
    lib.hdr_server_stats_get.argtypes = [_P, _P]
    lib.hdr_server_destroy.argtypes = [_P]
    lib.hdr_server_destroy.restype = None
    lib.hdr_calpa_params_default.argtypes = [_P]
    lib.hdr_calpa_params_default.restype = None
    lib.hdr_calpa_gradients.argtypes = [_P, ctypes.c_int32, _P, _P, _P, _P, _P]
    lib.hdr_calpa_metric.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P]
    lib.hdr_reconstruct_steered.argtypes = [_P, ctypes.c_int32, _P, _P, _P, _P, _P, _P, _P]
    lib.hdr_reconstruct_adaptive.argtypes = [_P, ctypes.c_int32, _P, _P, _P, _P, _P, _P]
    lib.hdr_reconstruct_adaptive_host.argtypes = [_P, ctypes.c_int32, _P, _P, _P, _P, _P, _P]
    lib.hdr_last_error.argtypes = []
    lib.hdr_last_error.restype = ctypes.c_char_p
    for name in ("hdr_create", "hdr_set_rig", "hdr_reconstruct", "hdr_reconstruct_levels", "hdr_reconstruct_host",
                 "hdr_check", "hdr_reconstruct_noalloc", "hdr_reconstruct_batch", "hdr_tune_batch",
                 "hdr_server_create", "hdr_submit", "hdr_poll", "hdr_server_stats_get", "hdr_selftest_timeout",
                 "hdr_calib_stack_stats", "hdr_calib_gain", "hdr_calib_exposure", "hdr_calpa_gradients",
                 "hdr_calpa_metric", "hdr_reconstruct_steered", "hdr_reconstruct_adaptive",
                 "hdr_reconstruct_adaptive_host"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int):
    if status != HDR_OK:
        raise HdrError(status, load().hdr_last_error().decode())


# ------------------------------------------------------------------ C entry points (same names)

def hdr_params_default() -> hdr_params:
    p = hdr_params()
    load().hdr_params_default(ctypes.byref(p))
    return p


def hdr_create(device: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(load().hdr_create(int(device), ctypes.byref(h)))
    return h.value


def hdr_destroy(ctx: int) -> None:
    load().hdr_destroy(ctypes.c_void_p(ctx))


def hdr_set_rig(ctx: int, rig_id: int, sensors: Sequence[hdr_sensor_desc]) -> None:
    arr = (hdr_sensor_desc * len(sensors))(*sensors)
    _check(load().hdr_set_rig(ctypes.c_void_p(ctx), int(rig_id), len(sensors), arr))


def _ptr_array(ptrs: Sequence[int]):
    return (ctypes.c_void_p * max(len(ptrs), 1))(*ptrs)


def hdr_reconstruct(ctx: int, rig_id: int, params: hdr_params, raw_dev: Sequence[int], out_dev: int,
                    choice_dev: Optional[int] = None, stream: Optional[int] = None) -> None:
    _check(load().hdr_reconstruct(ctypes.c_void_p(ctx), int(rig_id), ctypes.byref(params), _ptr_array(raw_dev),
                                  ctypes.c_void_p(out_dev), ctypes.c_void_p(choice_dev), ctypes.c_void_p(stream)))


def hdr_reconstruct_levels(ctx: int, rig_id: int, params: hdr_params, raw_dev: Sequence[int], out_dev: int,
                           choice_dev: Optional[int], levels_dev: int, stream: Optional[int] = None) -> None:
    _check(load().hdr_reconstruct_levels(ctypes.c_void_p(ctx), int(rig_id), ctypes.byref(params),
                                         _ptr_array(raw_dev), ctypes.c_void_p(out_dev), ctypes.c_void_p(choice_dev),
                                         ctypes.c_void_p(levels_dev), ctypes.c_void_p(stream)))


def hdr_reconstruct_host(ctx: int, rig_id: int, params: hdr_params, raw_host: Sequence[int], out_host: int,
                         choice_host: Optional[int] = None, stream: Optional[int] = None) -> None:
    _check(load().hdr_reconstruct_host(ctypes.c_void_p(ctx), int(rig_id), ctypes.byref(params),
                                       _ptr_array(raw_host), ctypes.c_void_p(out_host), ctypes.c_void_p(choice_host),
                                       ctypes.c_void_p(stream)))


def hdr_check(ctx: int, stream: Optional[int] = None) -> None:
    _check(load().hdr_check(ctypes.c_void_p(ctx), ctypes.c_void_p(stream)))


def hdr_selftest_timeout(ctx: int, stream: Optional[int] = None) -> None:
    """Launch the bounded-wait self-test: the next hdr_check on that stream reports HDR_E_TIMEOUT."""
    _check(load().hdr_selftest_timeout(ctypes.c_void_p(ctx), ctypes.c_void_p(stream)))


def hdr_calib_stack_stats(ctx: int, frames_dev: int, n_frames: int, width: int, height: int, pitch_elems: int,
                          frame_stride_elems: int, mean_dev: int, var_dev: int, stream: Optional[int] = None) -> None:
    _check(load().hdr_calib_stack_stats(ctypes.c_void_p(ctx), ctypes.c_void_p(frames_dev), int(n_frames), int(width),
                                        int(height), int(pitch_elems), int(frame_stride_elems),
                                        ctypes.c_void_p(mean_dev), ctypes.c_void_p(var_dev), ctypes.c_void_p(stream)))


def hdr_calib_gain(ctx: int, flat_mean: int, flat_var: int, black_mean: int, black_var: int, width: int, height: int,
                   min_signal: float, max_level: float, stream: Optional[int] = None):
    g = ctypes.c_double()
    n = ctypes.c_int64()
    _check(load().hdr_calib_gain(ctypes.c_void_p(ctx), ctypes.c_void_p(flat_mean), ctypes.c_void_p(flat_var),
                                 ctypes.c_void_p(black_mean), ctypes.c_void_p(black_var), int(width), int(height),
                                 float(min_signal), float(max_level), ctypes.byref(g), ctypes.byref(n),
                                 ctypes.c_void_p(stream)))
    return g.value, n.value


def hdr_calib_exposure(ctx: int, flat_mean: int, black_mean: int, gain: float, exposure: float, ref_flat_mean: int,
                       ref_black_mean: int, ref_gain: float, ref_exposure: float, width: int, height: int,
                       min_signal: float, max_level: float, prnu_dev: Optional[int] = None,
                       stream: Optional[int] = None):
    nd = ctypes.c_double()
    n = ctypes.c_int64()
    _check(load().hdr_calib_exposure(ctypes.c_void_p(ctx), ctypes.c_void_p(flat_mean), ctypes.c_void_p(black_mean),
                                     float(gain), float(exposure), ctypes.c_void_p(ref_flat_mean),
                                     ctypes.c_void_p(ref_black_mean), float(ref_gain), float(ref_exposure), int(width),
                                     int(height), float(min_signal), float(max_level), ctypes.byref(nd),
                                     ctypes.c_void_p(prnu_dev), ctypes.byref(n), ctypes.c_void_p(stream)))
    return nd.value, n.value


def hdr_calpa_params_default(**over) -> hdr_calpa_params:
    """Defaults of the adaptive reconstruction (Sections 5.4-5.5), with keyword overrides."""
    c = hdr_calpa_params()
    load().hdr_calpa_params_default(ctypes.byref(c))
    for k, v in over.items():
        setattr(c, k, float(v))
    return c


def hdr_calpa_gradients(ctx: int, rig_id: int, params: hdr_params, calpa: hdr_calpa_params, raw_dev: Sequence[int],
                        grad_dev: int, stream: Optional[int] = None) -> None:
    _check(load().hdr_calpa_gradients(ctypes.c_void_p(ctx), int(rig_id), ctypes.byref(params), ctypes.byref(calpa),
                                      _ptr_array(raw_dev), ctypes.c_void_p(grad_dev), ctypes.c_void_p(stream)))


def hdr_calpa_metric(ctx: int, out_w: int, out_h: int, calpa: hdr_calpa_params, grad_dev: int, metric_dev: int,
                     stream: Optional[int] = None) -> None:
    _check(load().hdr_calpa_metric(ctypes.c_void_p(ctx), int(out_w), int(out_h), ctypes.byref(calpa),
                                   ctypes.c_void_p(grad_dev), ctypes.c_void_p(metric_dev), ctypes.c_void_p(stream)))


def hdr_reconstruct_steered(ctx: int, rig_id: int, params: hdr_params, calpa: hdr_calpa_params,
                            raw_dev: Sequence[int], metric_dev: int, out_dev: int, choice_dev: Optional[int] = None,
                            stream: Optional[int] = None) -> None:
    _check(load().hdr_reconstruct_steered(ctypes.c_void_p(ctx), int(rig_id), ctypes.byref(params),
                                          ctypes.byref(calpa), _ptr_array(raw_dev), ctypes.c_void_p(metric_dev),
                                          ctypes.c_void_p(out_dev), ctypes.c_void_p(choice_dev),
                                          ctypes.c_void_p(stream)))


def hdr_reconstruct_adaptive(ctx: int, rig_id: int, params: hdr_params, calpa: hdr_calpa_params,
                             raw_dev: Sequence[int], out_dev: int, choice_dev: Optional[int] = None,
                             stream: Optional[int] = None) -> None:
    _check(load().hdr_reconstruct_adaptive(ctypes.c_void_p(ctx), int(rig_id), ctypes.byref(params),
                                           ctypes.byref(calpa), _ptr_array(raw_dev), ctypes.c_void_p(out_dev),
                                           ctypes.c_void_p(choice_dev), ctypes.c_void_p(stream)))


def hdr_reconstruct_adaptive_host(ctx: int, rig_id: int, params: hdr_params, calpa: hdr_calpa_params,
                                  raw_host: Sequence[int], out_host: int, choice_host: Optional[int] = None,
                                  stream: Optional[int] = None) -> None:
    _check(load().hdr_reconstruct_adaptive_host(ctypes.c_void_p(ctx), int(rig_id), ctypes.byref(params),
                                                ctypes.byref(calpa), _ptr_array(raw_host), ctypes.c_void_p(out_host),
                                                ctypes.c_void_p(choice_host), ctypes.c_void_p(stream)))


def hdr_last_error() -> str:
    return load().hdr_last_error().decode()


def hdr_reconstruct_batch(ctx: int, frames: Sequence[hdr_frame], cfg: Optional[hdr_batch_config] = None,
                          stream: Optional[int] = None) -> None:
    arr = (hdr_frame * len(frames))(*frames)
    _check(load().hdr_reconstruct_batch(ctypes.c_void_p(ctx), len(frames), arr,
                                        ctypes.byref(cfg) if cfg is not None else None, ctypes.c_void_p(stream)))


def hdr_tune_batch(ctx: int, frames: Sequence[hdr_frame], stream: Optional[int] = None) -> hdr_batch_config:
    arr = (hdr_frame * len(frames))(*frames)
    best = hdr_batch_config()
    _check(load().hdr_tune_batch(ctypes.c_void_p(ctx), len(frames), arr, ctypes.byref(best), ctypes.c_void_p(stream)))
    return best


HDR_NOALLOC_SCRATCH_BYTES = 4 << 20


def hdr_reconstruct_noalloc(device: int, sensors: Sequence[hdr_sensor_desc], params: hdr_params,
                            raw_dev: Sequence[int], out_dev: int, choice_dev: Optional[int] = None,
                            stream: Optional[int] = None) -> None:
    """Synchronous reconstruction that allocates nothing (scratch in a fixed device array); for callers
    that may not allocate device memory. Concurrent calls on one device race on that array."""
    arr = (hdr_sensor_desc * len(sensors))(*sensors)
    _check(load().hdr_reconstruct_noalloc(int(device), len(sensors), arr, ctypes.byref(params), _ptr_array(raw_dev),
                                          ctypes.c_void_p(out_dev), ctypes.c_void_p(choice_dev),
                                          ctypes.c_void_p(stream)))


def hdr_server_create(ctx: int, cfg: hdr_server_config) -> int:
    h = ctypes.c_void_p()
    _check(load().hdr_server_create(ctypes.c_void_p(ctx), ctypes.byref(cfg), ctypes.byref(h)))
    return int(h.value)


def hdr_submit(srv: int, req: hdr_request) -> int:
    t = ctypes.c_uint64()
    _check(load().hdr_submit(ctypes.c_void_p(srv), ctypes.byref(req), ctypes.byref(t)))
    return int(t.value)


def hdr_poll(srv: int, ticket: int, timeout_ms: int = -1) -> Optional[hdr_result]:
    """The request's result, or None while it is still running (HDR_E_BUSY)."""
    r = hdr_result()
    st = load().hdr_poll(ctypes.c_void_p(srv), ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(r))
    if st == HDR_E_BUSY:
        return None
    _check(st)
    return r


def hdr_server_stats_get(srv: int) -> hdr_server_stats:
    s = hdr_server_stats()
    _check(load().hdr_server_stats_get(ctypes.c_void_p(srv), ctypes.byref(s)))
    return s


def hdr_server_destroy(srv: int) -> None:
    load().hdr_server_destroy(ctypes.c_void_p(srv))


# ------------------------------------------------------------------ marshalling helpers

def sensor_desc(sensor, keep: list) -> hdr_sensor_desc:
    """hdr_sensor_desc from a synth.Sensor-like object; `keep` holds arrays the struct points at."""
    d = hdr_sensor_desc()
    d.width, d.height = int(sensor.width), int(sensor.height)
    d.pitch_elems = int(sensor.pitch)
    d.cfa = 0
    d.gain, d.exposure, d.nd = float(sensor.gain), float(sensor.exposure), float(sensor.nd)
    d.read_var, d.black, d.sat = float(sensor.read_var), float(sensor.black), float(sensor.sat)
    d.affine[:] = [float(x) for x in np.asarray(sensor.affine, dtype=np.float64).reshape(6)]
    for name, field, dt in (("bias_frame", "bias_frame", np.float32), ("prnu_frame", "prnu_frame", np.float32),
                            ("read_var_frame", "read_var_frame", np.float32), ("sat_frame", "sat_frame", np.uint16)):
        fr = getattr(sensor, name, None)
        if fr is not None:
            a = np.ascontiguousarray(fr, dtype=dt)
            keep.append(a)
            setattr(d, field, a.ctypes.data)
        else:
            setattr(d, field, None)
    return d


def params_struct(p) -> hdr_params:
    """hdr_params from a synth.Params-like object (defaults for fields it lacks)."""
    h = hdr_params_default()
    h.order = int(p.order)
    h.n_scales = len(p.sigmas)
    for j, s in enumerate(p.sigmas):
        h.sigma[j] = float(s)
    h.green_ratio = float(p.green_ratio)
    h.trunc_k = float(p.trunc_k)
    h.ici_gamma = float(p.ici_gamma)
    h.min_pivot = float(p.min_pivot)
    h.cond_fallback = float(getattr(p, "cond_fallback", h.cond_fallback))
    h.out_w, h.out_h = int(p.out_w), int(p.out_h)
    h.out_affine[:] = [float(x) for x in np.asarray(p.out_affine, dtype=np.float64).reshape(6)]
    h.out_dtype = int(getattr(p, "out_dtype", 0))
    h.accum = int(getattr(p, "accum", 0))
    h.tab_weights = int(getattr(p, "tab_weights", 1))
    h.weight_mode = int(getattr(p, "weight_mode", 0))
    return h


class Context:
    """One library context on one CUDA device; rigs are uploaded once and stay resident."""

    def __init__(self, device: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("paper_1308_4908_gb300 needs a CUDA device (there is no CPU path)")
        load()
        self.device = int(device)
        self.handle = hdr_create(self.device)

    def close(self):
        if self.handle:
            hdr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_rig(self, rig_id: int, sensors) -> None:
        keep: list = []
        descs = [sensor_desc(s, keep) for s in sensors]
        hdr_set_rig(self.handle, rig_id, descs)

    @staticmethod
    def _stream(stream):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        return s.cuda_stream

    def reconstruct(self, rig_id: int, params, raws, out=None, choice=None, levels=None, stream=None):
        """Reconstruct one frame from device tensors `raws` (uint16 [H, pitch] each); returns `out`."""
        import torch
        hp = params if isinstance(params, hdr_params) else params_struct(params)
        if out is None:
            dt = torch.float16 if hp.out_dtype == 1 else torch.float32
            out = torch.empty((3, hp.out_h, hp.out_w), dtype=dt, device=f"cuda:{self.device}")
        ptrs = [int(r.data_ptr()) for r in raws]
        if levels is not None:
            hdr_reconstruct_levels(self.handle, rig_id, hp, ptrs, out.data_ptr(),
                                   choice.data_ptr() if choice is not None else None, levels.data_ptr(),
                                   self._stream(stream))
        else:
            hdr_reconstruct(self.handle, rig_id, hp, ptrs, out.data_ptr(),
                            choice.data_ptr() if choice is not None else None, self._stream(stream))
        return out

    def frame(self, rig_id: int, params, raws, out, choice=None, keep: Optional[list] = None,
              calpa: Optional[hdr_calpa_params] = None) -> hdr_frame:
        """hdr_frame for a batch; `keep` collects the ctypes objects the frame points at (it must be
        given when `calpa` selects the adaptive reconstruction)."""
        hp = params if isinstance(params, hdr_params) else params_struct(params)
        if keep is not None:
            keep.append(hp)
            if calpa is not None:
                keep.append(calpa)
        f = hdr_frame()
        f.rig_id = int(rig_id)
        f.params = ctypes.addressof(hp)
        for i, r in enumerate(raws):
            f.raw_dev[i] = int(r.data_ptr())
        f.out_dev = out.data_ptr()
        f.choice_dev = choice.data_ptr() if choice is not None else None
        f.calpa = ctypes.addressof(calpa) if calpa is not None else None
        return f

    def reconstruct_batch(self, frames: Sequence[hdr_frame], cfg: Optional[hdr_batch_config] = None, stream=None):
        hdr_reconstruct_batch(self.handle, frames, cfg, self._stream(stream))

    def tune_batch(self, frames: Sequence[hdr_frame], stream=None) -> hdr_batch_config:
        return hdr_tune_batch(self.handle, frames, self._stream(stream))

    def reconstruct_host(self, rig_id: int, params, raws_host: Sequence[np.ndarray], out_host: np.ndarray,
                         choice_host: Optional[np.ndarray] = None, stream=None):
        hp = params if isinstance(params, hdr_params) else params_struct(params)
        hdr_reconstruct_host(self.handle, rig_id, hp, [int(r.ctypes.data) for r in raws_host], out_host.ctypes.data,
                             choice_host.ctypes.data if choice_host is not None else None, self._stream(stream))
        return out_host

    def check(self, stream=None):
        hdr_check(self.handle, self._stream(stream))

    def selftest_timeout(self, stream=None):
        hdr_selftest_timeout(self.handle, self._stream(stream))

    # ---------------------------------------------------------------- adaptive windows (Sections 5.4-5.5)
    def calpa_gradients(self, rig_id: int, params, calpa: hdr_calpa_params, raws, grad=None, stream=None):
        """Pass 1: float32 [out_h, out_w, 2] gradients of the order-1 green fit."""
        import torch
        hp = params if isinstance(params, hdr_params) else params_struct(params)
        if grad is None:
            grad = torch.empty((hp.out_h, hp.out_w, 2), dtype=torch.float32, device=f"cuda:{self.device}")
        hdr_calpa_gradients(self.handle, rig_id, hp, calpa, [int(r.data_ptr()) for r in raws], grad.data_ptr(),
                            self._stream(stream))
        return grad

    def calpa_metric(self, calpa: hdr_calpa_params, grad, metric=None, stream=None):
        """Pass 2: float32 [out_h, out_w, 3] steering matrices (C11, C12, C22) from `grad`."""
        import torch
        h, w = grad.shape[:2]
        if metric is None:
            metric = torch.empty((h, w, 3), dtype=torch.float32, device=grad.device)
        hdr_calpa_metric(self.handle, w, h, calpa, grad.data_ptr(), metric.data_ptr(), self._stream(stream))
        return metric

    def reconstruct_steered(self, rig_id: int, params, calpa: hdr_calpa_params, raws, metric, out=None, choice=None,
                            stream=None):
        """Pass 3: the reconstruction with the steered window of `metric`; returns `out`."""
        import torch
        hp = params if isinstance(params, hdr_params) else params_struct(params)
        if out is None:
            dt = torch.float16 if hp.out_dtype == 1 else torch.float32
            out = torch.empty((3, hp.out_h, hp.out_w), dtype=dt, device=f"cuda:{self.device}")
        hdr_reconstruct_steered(self.handle, rig_id, hp, calpa, [int(r.data_ptr()) for r in raws],
                                metric.data_ptr(), out.data_ptr(), choice.data_ptr() if choice is not None else None,
                                self._stream(stream))
        return out

    def reconstruct_adaptive(self, rig_id: int, params, calpa: hdr_calpa_params, raws, out=None, choice=None,
                             stream=None):
        """The three passes in one call (scratch owned by the context); returns `out`."""
        import torch
        hp = params if isinstance(params, hdr_params) else params_struct(params)
        if out is None:
            dt = torch.float16 if hp.out_dtype == 1 else torch.float32
            out = torch.empty((3, hp.out_h, hp.out_w), dtype=dt, device=f"cuda:{self.device}")
        hdr_reconstruct_adaptive(self.handle, rig_id, hp, calpa, [int(r.data_ptr()) for r in raws], out.data_ptr(),
                                 choice.data_ptr() if choice is not None else None, self._stream(stream))
        return out

    def reconstruct_adaptive_host(self, rig_id: int, params, calpa: hdr_calpa_params,
                                  raws_host: Sequence[np.ndarray], out_host: np.ndarray,
                                  choice_host: Optional[np.ndarray] = None, stream=None):
        """The three passes from host buffers (numpy arrays; pinned ones copy asynchronously)."""
        hp = params if isinstance(params, hdr_params) else params_struct(params)
        hdr_reconstruct_adaptive_host(self.handle, rig_id, hp, calpa, [int(r.ctypes.data) for r in raws_host],
                                      out_host.ctypes.data, choice_host.ctypes.data if choice_host is not None else None,
                                      self._stream(stream))
        return out_host

    # ---------------------------------------------------------------- calibration (Section 6.2)
    def calib_stack_stats(self, frames, width: int, stream=None):
        """frames: uint16 device tensor [n, height, pitch]; returns (mean, var) float32 [height, width]."""
        import torch
        n, h, pitch = frames.shape
        mean = torch.empty((h, width), dtype=torch.float32, device=frames.device)
        var = torch.empty((h, width), dtype=torch.float32, device=frames.device)
        hdr_calib_stack_stats(self.handle, frames.data_ptr(), n, width, h, pitch, frames.stride(0), mean.data_ptr(),
                              var.data_ptr(), self._stream(stream))
        return mean, var

    def calib_gain(self, flat_mean, flat_var, black_mean, black_var, min_signal=20.0, max_level=3800.0, stream=None):
        h, w = flat_mean.shape
        return hdr_calib_gain(self.handle, flat_mean.data_ptr(), flat_var.data_ptr(), black_mean.data_ptr(),
                              black_var.data_ptr(), w, h, min_signal, max_level, self._stream(stream))

    def calib_exposure(self, flat_mean, black_mean, gain, exposure, ref_flat_mean, ref_black_mean, ref_gain,
                       ref_exposure, min_signal=20.0, max_level=3800.0, stream=None):
        """Returns (n_s, prnu tensor [height, width], pixels used)."""
        import torch
        h, w = flat_mean.shape
        a = torch.empty((h, w), dtype=torch.float32, device=flat_mean.device)
        nd, n = hdr_calib_exposure(self.handle, flat_mean.data_ptr(), black_mean.data_ptr(), gain, exposure,
                                   ref_flat_mean.data_ptr(), ref_black_mean.data_ptr(), ref_gain, ref_exposure, w, h,
                                   min_signal, max_level, a.data_ptr(), self._stream(stream))
        return nd, a, n


class Server:
    """Request loop over one Context (see hdr_server_create). Host arrays given to submit() are kept
    alive here until their result has been polled."""

    def __init__(self, ctx: Context, max_frames: int = 16, pool_bytes: int = 4 << 30, step_tiles: int = 0,
                 batch: Optional[hdr_batch_config] = None, order: int = 0):
        cfg = hdr_server_config()
        cfg.max_frames, cfg.pool_bytes, cfg.step_tiles = int(max_frames), int(pool_bytes), int(step_tiles)
        cfg.batch = batch if batch is not None else hdr_batch_config(0, 0, 1, 0)
        cfg.order = int(order)
        self.ctx = ctx
        self.handle = hdr_server_create(ctx.handle, cfg)
        self._held = {}

    def submit(self, rig_id: int, params, raws_host: Sequence[np.ndarray], out_host: np.ndarray,
               choice_host: Optional[np.ndarray] = None, stream_id: int = 0,
               calpa: Optional[hdr_calpa_params] = None) -> int:
        """Queue one frame; with `calpa` the adaptive reconstruction of Sections 5.4-5.5."""
        req = hdr_request()
        if calpa is not None:
            req.adaptive = 1
            req.calpa = calpa
        req.rig_id = int(rig_id)
        req.params = params if isinstance(params, hdr_params) else params_struct(params)
        for i, r in enumerate(raws_host):
            req.raw_host[i] = int(r.ctypes.data)
        req.out_host = out_host.ctypes.data
        req.choice_host = choice_host.ctypes.data if choice_host is not None else None
        req.stream_id = int(stream_id)
        t = hdr_submit(self.handle, req)
        self._held[t] = (list(raws_host), out_host, choice_host)
        return t

    def poll(self, ticket: int, timeout_ms: int = -1) -> Optional[hdr_result]:
        try:
            r = hdr_poll(self.handle, ticket, timeout_ms)
        except HdrError:
            self._held.pop(ticket, None)
            raise
        if r is not None:
            self._held.pop(ticket, None)
        return r

    def stats(self) -> hdr_server_stats:
        return hdr_server_stats_get(self.handle)

    def close(self):
        if self.handle:
            hdr_server_destroy(self.handle)
            self.handle = None
            self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
