"""ctypes binding of libcombgpu.so: argument marshalling only.

Every function here has the name of the C entry point it calls (see
include/combgpu.h) and does no arithmetic of the method: device buffers are
passed as raw pointers (a torch CUDA tensor or an integer address), host
arrays as numpy arrays.  Loading fails loudly when the CUDA library is not
built; there is no fallback of any kind.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

CG_OK = 0
CG_ERR_ARG = 1
STATUS_NAMES = {0: "CG_OK", 1: "CG_ERR_ARG", 2: "CG_ERR_CUDA", 3: "CG_ERR_NOMEM",
                4: "CG_ERR_TOOTH_RANGE", 5: "CG_ERR_OVERFLOW", 6: "CG_ERR_TIMEOUT",
                7: "CG_ERR_DEVICE_CHECK", 8: "CG_ERR_UNSUPPORTED", 9: "CG_ERR_STATE"}
FIT_CONVERGED, FIT_MAX_ITER, FIT_SINGULAR, FIT_NONFINITE, FIT_INIT_FLAT = 0, 1, 2, 3, 0x10
FIT_FALLBACK = 0x20
STAGE_READOUT, STAGE_INIT, STAGE_MLP, STAGE_FIT, STAGE_FALLBACK, STAGE_FUSED = 0, 1, 2, 3, 4, 5
N_STAGES = 8
STAGE_NAMES = {0: "readout", 1: "init", 2: "mlp", 3: "fit", 4: "fallback", 5: "fused", 6: "median"}
READOUT_FFT, READOUT_GEMM_SPLIT, READOUT_FOLD_GEMM = 0, 1, 2
FFT_AUTO, FFT_FULL, FFT_COSET = 0, 1, 2
INIT_MOMENT, INIT_MLP, INIT_MEDIAN = 0, 1, 2
PATH_AUTO, PATH_FUSED, PATH_SPLIT, PATH_PIPELINE = 0, 1, 2, 3
MODEL_LORENTZ, MODEL_FANO = 0, 1


class CgError(RuntimeError):
    """A library call returned a status other than CG_OK."""

    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {detail}")


class cg_opts(ctypes.Structure):
    _fields_ = [("readout", ctypes.c_int), ("fft", ctypes.c_int), ("init", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("tol", ctypes.c_double),
                ("lambda0", ctypes.c_double), ("lanes_per_frame", ctypes.c_int),
                ("path", ctypes.c_int), ("chunk_frames", ctypes.c_int),
                ("sample_bits", ctypes.c_int), ("solve_f64", ctypes.c_int),
                ("polish_iter", ctypes.c_int), ("model", ctypes.c_int),
                ("reserved", ctypes.c_int * 3), ("fano_q", ctypes.c_double),
                ("fano_gamma", ctypes.c_double), ("fano_A", ctypes.c_double),
                ("fano_B", ctypes.c_double), ("fano_box", ctypes.c_double)]


class cg_plan_info(ctypes.Structure):
    _fields_ = [("frame_len", ctypes.c_int), ("n_teeth", ctypes.c_int),
                ("fft_kind", ctypes.c_int), ("coset_modulus", ctypes.c_int),
                ("coset_residue", ctypes.c_int), ("fft_len", ctypes.c_int),
                ("n_radices", ctypes.c_int), ("radices", ctypes.c_int * 8),
                ("frames_per_cta", ctypes.c_int), ("lanes_per_frame", ctypes.c_int),
                ("n_collisions", ctypes.c_int), ("path", ctypes.c_int)]


class cg_result(ctypes.Structure):
    _fields_ = [("seq", ctypes.c_uint64), ("t_arrival", ctypes.c_double), ("t_done", ctypes.c_double),
                ("params", ctypes.c_float * 4), ("rss", ctypes.c_float), ("iters", ctypes.c_int16),
                ("status", ctypes.c_int16)]


RESULT_DTYPE = np.dtype([("seq", np.uint64), ("t_arrival", np.float64), ("t_done", np.float64),
                         ("params", np.float32, 4), ("rss", np.float32), ("iters", np.int16),
                         ("status", np.int16)], align=True)


class cg_stream_stats_t(ctypes.Structure):
    _fields_ = [("frames_pushed", ctypes.c_int64), ("frames_dropped", ctypes.c_int64),
                ("frames_done", ctypes.c_int64), ("frames_polled", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("latency_p50_s", ctypes.c_double),
                ("latency_p99_s", ctypes.c_double), ("latency_max_s", ctypes.c_double),
                ("input_bytes_per_s", ctypes.c_double), ("admitted", ctypes.c_int),
                ("window_index", ctypes.c_int64), ("window_frames", ctypes.c_int64)]


INJECT_THROTTLE_S, INJECT_HOLD, INJECT_FAIL_LAUNCH = 1, 2, 3

_P = ctypes.c_void_p
_SIGS = {
    "cg_opts_default": (None, [ctypes.POINTER(cg_opts)]),
    "cg_plan": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_double, ctypes.c_int, ctypes.c_int,
                               _P, _P, _P, ctypes.POINTER(cg_opts)]),
    "cg_plan_destroy": (None, [_P]),
    "cg_plan_describe": (ctypes.c_int, [_P, ctypes.POINTER(cg_plan_info), _P]),
    "cg_set_reference": (ctypes.c_int, [_P, _P]),
    "cg_process": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P, _P, _P, _P, _P, _P]),
    "cg_process_i8": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P, _P, _P, _P, _P, _P]),
    "cg_readout": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P, _P]),
    "cg_readout_i8": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P, _P]),
    "cg_fit": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P, _P, _P, _P, _P]),
    "cg_psd_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_P)]),
    "cg_psd_destroy": (None, [_P]),
    "cg_psd_welch": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int64, ctypes.c_double, _P,
                                    ctypes.POINTER(ctypes.c_int64), _P]),
    "cg_resonance_fit": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, ctypes.c_double, _P, _P]),
    "cg_reference_accumulate": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P]),
    "cg_reference_accumulate_noalloc": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P]),
    "cg_check_device": (ctypes.c_int, [_P]),
    "cg_timing_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "cg_fp32_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), _P]),
    "cg_timing_collect": (ctypes.c_int, [_P, _P, _P]),
    "cg_mlp_param_count": (ctypes.c_int64, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "cg_mlp_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_uint64]),
    "cg_mlp_destroy": (None, [_P]),
    "cg_mlp_get_params": (ctypes.c_int, [_P, _P, ctypes.c_int64]),
    "cg_mlp_set_params": (ctypes.c_int, [_P, _P, ctypes.c_int64]),
    "cg_mlp_forward": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P]),
    "cg_mlp_backward": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P, _P, _P]),
    "cg_mlp_adam": (ctypes.c_int, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                   _P]),
    "cg_mlp_train_epoch": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P, ctypes.c_int, ctypes.c_float,
                                          _P, _P]),
    "cg_mlp_set_norm": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "cg_mlp_save": (ctypes.c_int, [_P, _P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "cg_mlp_load": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "cg_mlp_infer": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P]),
    "cg_clock": (ctypes.c_double, []),
    "cg_server_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_size_t]),
    "cg_server_destroy": (ctypes.c_int, [_P]),
    "cg_server_inject": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double]),
    "cg_stream_create": (ctypes.c_int, [ctypes.POINTER(_P), _P, _P, ctypes.c_size_t, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_int64]),
    "cg_stream_push": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double]),
    "cg_stream_poll": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                      ctypes.c_double]),
    "cg_stream_flush": (ctypes.c_int, [_P, ctypes.c_double]),
    "cg_stream_stats": (ctypes.c_int, [_P, ctypes.POINTER(cg_stream_stats_t)]),
    "cg_stream_window": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                        _P, _P]),
    "cg_stream_destroy": (ctypes.c_int, [_P]),
    "cg_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "cg_last_error": (ctypes.c_char_p, []),
    "cg_version": (ctypes.c_int, []),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libcombgpu.so (building it first when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise ImportError(f"libcombgpu.so is not built ({_build.LIB}); run "
                              "paper_2307_12988_gb300.build.build() with nvcc available")
        lib = ctypes.CDLL(_build.LIB)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


def _ptr(x) -> int | None:
    """Device or host address of a torch tensor / numpy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:   # torch absent: legacy default stream
            return None
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(st: int, where: str):
    if st != CG_OK:
        detail = load().cg_last_error().decode(errors="replace")
        raise CgError(st, where, detail)


def cg_opts_default(**overrides) -> cg_opts:
    o = cg_opts()
    load().cg_opts_default(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def cg_plan(sample_rate: float, frame_len: int, tooth_freqs, tooth_x=None, ref_spectrum=None,
            opts: cg_opts | None = None) -> int:
    f = np.ascontiguousarray(tooth_freqs, dtype=np.float64)
    x = None if tooth_x is None else np.ascontiguousarray(tooth_x, dtype=np.float64)
    r = None if ref_spectrum is None else np.ascontiguousarray(ref_spectrum, dtype=np.float64)
    if x is not None and x.size != f.size or r is not None and r.size != f.size:
        raise ValueError("tooth_x / ref_spectrum must have one value per tooth")
    h = _P()
    st = load().cg_plan(ctypes.byref(h), float(sample_rate), int(frame_len), int(f.size),
                        _ptr(f), _ptr(x), _ptr(r), ctypes.byref(opts) if opts else None)
    _check(st, "cg_plan")
    return h.value


def cg_plan_destroy(plan: int) -> None:
    if plan:
        load().cg_plan_destroy(plan)


def cg_plan_describe(plan: int) -> dict:
    info = cg_plan_info()
    probe = cg_plan_info()
    _check(load().cg_plan_describe(plan, ctypes.byref(probe), None), "cg_plan_describe")
    bins = np.empty(probe.n_teeth, dtype=np.int32)
    _check(load().cg_plan_describe(plan, ctypes.byref(info), _ptr(bins)), "cg_plan_describe")
    d = {name: getattr(info, name) for name, _ in cg_plan_info._fields_}
    d["radices"] = list(info.radices)[:info.n_radices]
    d["bins"] = bins
    return d


def cg_set_reference(plan: int, ref_spectrum) -> None:
    r = np.ascontiguousarray(ref_spectrum, dtype=np.float64)
    _check(load().cg_set_reference(plan, _ptr(r)), "cg_set_reference")


def cg_process(plan: int, frames, n_frames: int, amps, y, params, rss, iters, status,
               stream=None) -> None:
    _check(load().cg_process(plan, _ptr(frames), int(n_frames), _ptr(amps), _ptr(y),
                             _ptr(params), _ptr(rss), _ptr(iters), _ptr(status),
                             _stream(stream)), "cg_process")


def cg_process_i8(plan: int, frames, n_frames: int, amps, y, params, rss, iters, status,
                  stream=None) -> None:
    _check(load().cg_process_i8(plan, _ptr(frames), int(n_frames), _ptr(amps), _ptr(y),
                                _ptr(params), _ptr(rss), _ptr(iters), _ptr(status),
                                _stream(stream)), "cg_process_i8")


def cg_readout_i8(plan: int, frames, n_frames: int, amps, y, stream=None) -> None:
    _check(load().cg_readout_i8(plan, _ptr(frames), int(n_frames), _ptr(amps), _ptr(y),
                                _stream(stream)), "cg_readout_i8")


def cg_readout(plan: int, frames, n_frames: int, amps, y, stream=None) -> None:
    _check(load().cg_readout(plan, _ptr(frames), int(n_frames), _ptr(amps), _ptr(y),
                             _stream(stream)), "cg_readout")


def cg_psd_create(seg_len: int) -> int:
    h = _P()
    _check(load().cg_psd_create(int(seg_len), ctypes.byref(h)), "cg_psd_create")
    return h.value


def cg_psd_destroy(h: int) -> None:
    load().cg_psd_destroy(h)


def cg_psd_welch(h: int, x, n: int, stride: int, fs: float, psd_out, stream=None) -> int:
    k = ctypes.c_int64(0)
    _check(load().cg_psd_welch(h, _ptr(x), int(n), int(stride), float(fs), _ptr(psd_out), ctypes.byref(k),
                               _stream(stream)), "cg_psd_welch")
    return int(k.value)


def cg_resonance_fit(psd, n_bins: int, df: float, f_lo: float, f_hi: float, max_iter: int, tol: float, out,
                     stream=None) -> None:
    _check(load().cg_resonance_fit(_ptr(psd), int(n_bins), float(df), float(f_lo), float(f_hi), int(max_iter),
                                   float(tol), _ptr(out), _stream(stream)), "cg_resonance_fit")


def cg_fit(plan: int, y, n: int, p0, params, rss, iters, status, stream=None) -> None:
    _check(load().cg_fit(plan, _ptr(y), int(n), _ptr(p0), _ptr(params), _ptr(rss),
                         _ptr(iters), _ptr(status), _stream(stream)), "cg_fit")


def cg_reference_accumulate(plan: int, frames, n: int, stream=None) -> np.ndarray:
    ref = None
    info = cg_plan_describe(plan)
    ref = np.empty(info["n_teeth"], dtype=np.float64)
    _check(load().cg_reference_accumulate(plan, _ptr(frames), int(n), _ptr(ref),
                                          _stream(stream)), "cg_reference_accumulate")
    return ref


def cg_reference_accumulate_noalloc(plan: int, frames, n: int, ref_dev, stream=None) -> None:
    """Reference average into the caller's device buffer ``ref_dev`` (float64
    [n_teeth]) without any allocation by the library (see the C header).

    ``frames`` (int16, at least n * frame_len elements) and ``ref_dev``
    (float64, contiguous, at least n_teeth elements) must be CUDA tensors on
    one device; anything else raises CgError before the call."""
    info = cg_plan_describe(plan)
    need_frames = int(n) * info["frame_len"]

    def _bad(what):
        raise CgError(CG_ERR_ARG, "cg_reference_accumulate_noalloc", what)

    for name, t, dtype, count in (("frames", frames, "torch.int16", need_frames),
                                  ("ref_dev", ref_dev, "torch.float64", info["n_teeth"])):
        if not (hasattr(t, "is_cuda") and t.is_cuda):
            _bad(f"{name} must be a CUDA tensor")
        if str(t.dtype) != dtype:
            _bad(f"{name} must be {dtype}, not {t.dtype}")
        if not t.is_contiguous():
            _bad(f"{name} must be contiguous")
        if t.numel() < count:
            _bad(f"{name} holds {t.numel()} elements, needs {count}")
    if frames.device != ref_dev.device:
        _bad("frames and ref_dev are on different devices")
    _check(load().cg_reference_accumulate_noalloc(plan, _ptr(frames), int(n), _ptr(ref_dev),
                                                  _stream(stream)),
           "cg_reference_accumulate_noalloc")


def cg_check_device(plan: int) -> None:
    """Synchronise and raise CgError if a kernel recorded a device-side error."""
    _check(load().cg_check_device(plan), "cg_check_device")


def cg_fp32_peak(packed: bool, reps: int = 20, stream=None) -> float:
    """Measured FP32 FMA throughput of the current device in TFLOP/s."""
    out = ctypes.c_double(0.0)
    _check(load().cg_fp32_peak(1 if packed else 0, int(reps), ctypes.byref(out), _stream(stream)),
           "cg_fp32_peak")
    return float(out.value)


def cg_timing_enable(plan: int, enable: bool) -> None:
    _check(load().cg_timing_enable(plan, 1 if enable else 0), "cg_timing_enable")


def cg_timing_collect(plan: int) -> dict:
    """{stage name: (total ms, launches)} since the last collect."""
    ms = np.zeros(N_STAGES, dtype=np.float64)
    cnt = np.zeros(N_STAGES, dtype=np.int64)
    _check(load().cg_timing_collect(plan, _ptr(ms), _ptr(cnt)), "cg_timing_collect")
    return {STAGE_NAMES[i]: (float(ms[i]), int(cnt[i])) for i in STAGE_NAMES if cnt[i] > 0}


def cg_mlp_param_count(n_in: int, n_hidden: int, n_out: int) -> int:
    return int(load().cg_mlp_param_count(int(n_in), int(n_hidden), int(n_out)))


def cg_mlp_create(n_in: int, n_hidden: int, n_out: int, max_batch: int, seed: int) -> int:
    h = _P()
    _check(load().cg_mlp_create(ctypes.byref(h), int(n_in), int(n_hidden), int(n_out), int(max_batch),
                                int(seed) & 0xFFFFFFFFFFFFFFFF), "cg_mlp_create")
    return h.value


def cg_mlp_destroy(mlp: int) -> None:
    if mlp:
        load().cg_mlp_destroy(mlp)


def cg_mlp_get_params(mlp: int, count: int) -> np.ndarray:
    out = np.empty(int(count), dtype=np.float32)
    _check(load().cg_mlp_get_params(mlp, _ptr(out), int(count)), "cg_mlp_get_params")
    return out


def cg_mlp_set_params(mlp: int, params) -> None:
    a = np.ascontiguousarray(params, dtype=np.float32)
    _check(load().cg_mlp_set_params(mlp, _ptr(a), int(a.size)), "cg_mlp_set_params")


def cg_mlp_forward(mlp: int, x, n: int, out, stream=None) -> None:
    _check(load().cg_mlp_forward(mlp, _ptr(x), int(n), _ptr(out), _stream(stream)), "cg_mlp_forward")


def cg_mlp_backward(mlp: int, x, t, n: int, loss=None, grad=None, stream=None) -> None:
    _check(load().cg_mlp_backward(mlp, _ptr(x), _ptr(t), int(n), _ptr(loss), _ptr(grad), _stream(stream)),
           "cg_mlp_backward")


def cg_mlp_adam(mlp: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
                stream=None) -> None:
    _check(load().cg_mlp_adam(mlp, float(lr), float(beta1), float(beta2), float(eps), _stream(stream)),
           "cg_mlp_adam")


def cg_mlp_train_epoch(mlp: int, x, t, n: int, perm, batch: int, lr: float, losses=None,
                       stream=None) -> None:
    _check(load().cg_mlp_train_epoch(mlp, _ptr(x), _ptr(t), int(n), _ptr(perm), int(batch), float(lr),
                                     _ptr(losses), _stream(stream)), "cg_mlp_train_epoch")


def cg_mlp_set_norm(mlp: int, in_mean, in_scale, out_mean, out_scale) -> None:
    arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (in_mean, in_scale, out_mean, out_scale)]
    _check(load().cg_mlp_set_norm(mlp, *[_ptr(a) for a in arrs]), "cg_mlp_set_norm")


def cg_mlp_save(mlp: int) -> bytes:
    size = ctypes.c_size_t(0)
    _check(load().cg_mlp_save(mlp, None, 0, ctypes.byref(size)), "cg_mlp_save")
    buf = ctypes.create_string_buffer(size.value)
    _check(load().cg_mlp_save(mlp, buf, size.value, ctypes.byref(size)), "cg_mlp_save")
    return buf.raw[:size.value]


def cg_mlp_load(plan: int, blob: bytes) -> None:
    buf = ctypes.create_string_buffer(bytes(blob), len(blob))
    _check(load().cg_mlp_load(plan, buf, len(blob)), "cg_mlp_load")


def cg_mlp_infer(plan: int, y, n: int, p0, stream=None) -> None:
    _check(load().cg_mlp_infer(plan, _ptr(y), int(n), _ptr(p0), _stream(stream)), "cg_mlp_infer")


def cg_clock() -> float:
    return float(load().cg_clock())


def cg_server_create(device_budget_bytes: int) -> int:
    h = _P()
    _check(load().cg_server_create(ctypes.byref(h), int(device_budget_bytes)), "cg_server_create")
    return h.value


def cg_server_destroy(server: int) -> None:
    if server:
        _check(load().cg_server_destroy(server), "cg_server_destroy")


def cg_server_inject(server: int, what: int, value: float) -> None:
    _check(load().cg_server_inject(server, int(what), float(value)), "cg_server_inject")


def cg_stream_create(server: int, plan: int, ring_bytes: int, batch_frames: int, max_delay_s: float,
                     avg_window: int) -> int:
    h = _P()
    _check(load().cg_stream_create(ctypes.byref(h), server, plan, int(ring_bytes), int(batch_frames),
                                   float(max_delay_s), int(avg_window)), "cg_stream_create")
    return h.value


def cg_stream_push(stream: int, frames_host, n: int, first_seq: int, t_arrival: float = -1.0) -> int:
    """Returns the status code (CG_OK or CG_ERR_OVERFLOW) instead of raising on overflow."""
    st = load().cg_stream_push(stream, _ptr(frames_host), int(n), int(first_seq), float(t_arrival))
    if st not in (CG_OK, 5):
        _check(st, "cg_stream_push")
    return st


def cg_stream_poll(stream: int, recs: np.ndarray, amps_host=None, timeout_s: float = 0.0) -> tuple[int, int]:
    """Fill recs (RESULT_DTYPE array); returns (count, status) with status CG_OK or
    CG_ERR_TIMEOUT (other errors raise)."""
    n = ctypes.c_int64(0)
    st = load().cg_stream_poll(stream, _ptr(recs), _ptr(amps_host), int(recs.shape[0]), ctypes.byref(n),
                               float(timeout_s))
    if st not in (CG_OK, 6):
        _check(st, "cg_stream_poll")
    return int(n.value), st


def cg_stream_flush(stream: int, timeout_s: float) -> int:
    st = load().cg_stream_flush(stream, float(timeout_s))
    if st not in (CG_OK, 6):
        _check(st, "cg_stream_flush")
    return st


def cg_stream_stats(stream: int) -> dict:
    o = cg_stream_stats_t()
    _check(load().cg_stream_stats(stream, ctypes.byref(o)), "cg_stream_stats")
    return {name: getattr(o, name) for name, _ in cg_stream_stats_t._fields_}


def cg_stream_window(stream: int, n_teeth: int) -> dict:
    idx, cnt = ctypes.c_int64(0), ctypes.c_int64(0)
    y = np.full(n_teeth, np.nan)
    p = np.full(4, np.nan)
    _check(load().cg_stream_window(stream, ctypes.byref(idx), ctypes.byref(cnt), _ptr(y), _ptr(p)),
           "cg_stream_window")
    return {"index": idx.value, "count": cnt.value, "mean_y": y, "mean_params": p}


def cg_stream_destroy(stream: int) -> None:
    if stream:
        _check(load().cg_stream_destroy(stream), "cg_stream_destroy")


def cg_status_string(status: int) -> str:
    return load().cg_status_string(int(status)).decode()


def cg_last_error() -> str:
    return load().cg_last_error().decode(errors="replace")


def cg_version() -> int:
    return load().cg_version()
