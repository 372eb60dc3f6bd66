"""GB300-native comb-spectrum readout and Lorentzian fit (arXiv 2307.12988).

The compute path is libcombgpu.so (hand-written CUDA for sm_103a behind a C
ABI, include/combgpu.h).  This package only marshals arguments: ``_binding``
exposes the C entry points under their own names, and ``Plan`` below is a
convenience wrapper that allocates output tensors with PyTorch (device memory
and streams only) and calls them.
"""
from __future__ import annotations

import numpy as np

from . import _binding
from ._binding import (CgError, cg_check_device, cg_fit, cg_opts_default, cg_plan, cg_plan_describe,
                       cg_plan_destroy, cg_process, cg_process_i8, cg_readout, cg_readout_i8,
                       cg_reference_accumulate,
                       cg_set_reference, cg_status_string, cg_version, load)
from ._binding import (cg_mlp_adam, cg_mlp_backward, cg_mlp_create, cg_mlp_destroy, cg_mlp_forward,
                       cg_mlp_get_params, cg_mlp_infer, cg_mlp_load, cg_mlp_param_count, cg_mlp_save,
                       cg_mlp_set_norm, cg_mlp_set_params, cg_mlp_train_epoch, cg_timing_collect,
                       cg_timing_enable)
from ._binding import cg_psd_create, cg_psd_destroy, cg_psd_welch, cg_resonance_fit
from ._binding import cg_fp32_peak
from ._binding import (RESULT_DTYPE, INJECT_FAIL_LAUNCH, INJECT_HOLD, INJECT_THROTTLE_S, cg_clock,
                       cg_server_create, cg_server_destroy, cg_server_inject, cg_stream_create,
                       cg_stream_destroy, cg_stream_flush, cg_stream_poll, cg_stream_push,
                       cg_stream_stats, cg_stream_window)
from ._binding import (FFT_AUTO, FFT_COSET, FFT_FULL, FIT_CONVERGED, FIT_FALLBACK, FIT_INIT_FLAT,
                       FIT_MAX_ITER, FIT_NONFINITE, FIT_SINGULAR, INIT_MEDIAN, INIT_MLP, INIT_MOMENT,
                       READOUT_FFT, READOUT_GEMM_SPLIT, READOUT_FOLD_GEMM, PATH_AUTO, PATH_FUSED, PATH_SPLIT,
                       PATH_PIPELINE, MODEL_LORENTZ, MODEL_FANO)

__all__ = ["Plan", "Mlp", "Psd", "Server", "Stream", "CgError", "load", "cg_plan", "cg_plan_destroy", "cg_plan_describe",
           "cg_process", "cg_readout", "cg_fit", "cg_reference_accumulate",
           "cg_set_reference", "cg_opts_default", "cg_status_string", "cg_version"]


class Plan:
    """A geometry plan on the current CUDA device.

    Parameters follow ``cg_plan``: sample rate (Hz), frame length N, signed
    tooth RF frequencies (Hz), optional fit abscissa and reference spectrum;
    keyword options are fields of ``cg_opts``."""

    def __init__(self, sample_rate, frame_len, tooth_freqs, tooth_x=None, ref=None, **opts):
        self._opts = cg_opts_default(**opts)
        self.handle = cg_plan(sample_rate, frame_len, tooth_freqs, tooth_x, ref, self._opts)
        info = cg_plan_describe(self.handle)
        self.info = info
        self.N = info["frame_len"]
        self.T = info["n_teeth"]
        self.bins = info["bins"]

    def close(self):
        if getattr(self, "handle", None):
            cg_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_reference(self, ref):
        cg_set_reference(self.handle, ref)

    def _outputs(self, n, device, want_y=True, want_amps=True):
        import torch
        out = {}
        if want_amps:
            out["amps"] = torch.empty((n, self.T), dtype=torch.float32, device=device)
        out["y"] = torch.empty((n, self.T), dtype=torch.float32, device=device) if want_y else None
        out["params"] = torch.empty((n, 4), dtype=torch.float32, device=device)
        out["rss"] = torch.empty(n, dtype=torch.float32, device=device)
        out["iters"] = torch.empty(n, dtype=torch.int16, device=device)
        out["status"] = torch.empty(n, dtype=torch.int16, device=device)
        return out

    def process(self, frames, want_y=True, stream=None):
        """Whole path on int16 (or int8) frames [n, N] resident on the device."""
        n = frames.shape[0]
        if frames.dim() != 2 or frames.shape[1] != self.N:
            raise ValueError(f"frames must be [n, {self.N}]")
        o = self._outputs(n, frames.device, want_y)
        import torch
        fn = cg_process_i8 if frames.dtype == torch.int8 else cg_process
        fn(self.handle, frames, n, o["amps"], o["y"], o["params"], o["rss"], o["iters"], o["status"], stream)
        return o

    def readout(self, frames, want_y=True, stream=None):
        import torch
        n = frames.shape[0]
        amps = torch.empty((n, self.T), dtype=torch.float32, device=frames.device)
        y = torch.empty_like(amps) if want_y else None
        fn = cg_readout_i8 if frames.dtype == torch.int8 else cg_readout
        fn(self.handle, frames, n, amps, y, stream)
        return amps, y

    def fit(self, y, p0=None, stream=None):
        n = y.shape[0]
        o = self._outputs(n, y.device, want_y=False, want_amps=False)
        cg_fit(self.handle, y, n, p0, o["params"], o["rss"], o["iters"], o["status"], stream)
        return o

    def reference_accumulate(self, frames, stream=None) -> np.ndarray:
        return cg_reference_accumulate(self.handle, frames, frames.shape[0], stream)

    def mlp_load(self, blob: bytes):
        """Attach a learned initial guess (a ``cg_mlp_save`` blob)."""
        cg_mlp_load(self.handle, blob)

    def mlp_infer(self, y, stream=None):
        """Learned initial guess p0 [n, 4] for normalised spectra y [n, T]."""
        import torch
        p0 = torch.empty((y.shape[0], 4), dtype=torch.float32, device=y.device)
        cg_mlp_infer(self.handle, y, y.shape[0], p0, stream)
        return p0

    def timing(self, enable: bool = True):
        cg_timing_enable(self.handle, enable)

    def timing_collect(self) -> dict:
        return cg_timing_collect(self.handle)


class Psd:
    """Welch PSD of a device series and the mechanical-resonance fit
    (``cg_psd_*``, ``cg_resonance_fit``)."""

    def __init__(self, seg_len=32768):
        self.seg_len = int(seg_len)
        self.handle = cg_psd_create(self.seg_len)

    def close(self):
        if getattr(self, "handle", None):
            cg_psd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def welch(self, x, fs, stride=1, n=None):
        """One-sided density of x[::stride] (device float tensor) as a device
        float64 tensor [seg_len/2 + 1], and the number of segments."""
        import torch
        n = (x.numel() + stride - 1) // stride if n is None else n
        out = torch.empty(self.seg_len // 2 + 1, dtype=torch.float64, device=x.device)
        k = cg_psd_welch(self.handle, x, n, stride, fs, out)
        return out, k

    @staticmethod
    def resonance(psd, df, f_lo, f_hi, max_iter=200, tol=1e-12):
        """(f0, Q, A, B, their standard errors, chi^2, steps, status, bins)
        fitted to the device PSD tensor, as a host numpy array."""
        import torch
        out = torch.empty(12, dtype=torch.float64, device=psd.device)
        cg_resonance_fit(psd, psd.numel(), df, f_lo, f_hi, max_iter, tol, out)
        return out.cpu().numpy()


class Mlp:
    """Network of the learned initial guess, trained on the device by the
    library's kernels (``cg_mlp_*``).  Inputs and targets are standardised
    by the caller; ``set_norm`` stores the standardisation with the blob."""

    def __init__(self, n_in, n_hidden=256, n_out=4, max_batch=4096, seed=0):
        self.n_in, self.n_hidden, self.n_out, self.max_batch = n_in, n_hidden, n_out, max_batch
        self.n_params = cg_mlp_param_count(n_in, n_hidden, n_out)
        self.handle = cg_mlp_create(n_in, n_hidden, n_out, max_batch, seed)

    def close(self):
        if getattr(self, "handle", None):
            cg_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        return cg_mlp_get_params(self.handle, self.n_params)

    def set_params(self, theta):
        cg_mlp_set_params(self.handle, theta)

    def forward(self, x, stream=None):
        import torch
        out = torch.empty((x.shape[0], self.n_out), dtype=torch.float32, device=x.device)
        cg_mlp_forward(self.handle, x, x.shape[0], out, stream)
        return out

    def backward(self, x, t, stream=None):
        """(loss tensor [1], gradient tensor [n_params]) of one batch."""
        import torch
        loss = torch.empty(1, dtype=torch.float32, device=x.device)
        grad = torch.empty(self.n_params, dtype=torch.float32, device=x.device)
        cg_mlp_backward(self.handle, x, t, x.shape[0], loss, grad, stream)
        return loss, grad

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        cg_mlp_adam(self.handle, lr, beta1, beta2, eps, stream)

    def train_epoch(self, x, t, perm, batch, lr, stream=None):
        import torch
        nb = (x.shape[0] + batch - 1) // batch
        losses = torch.empty(nb, dtype=torch.float32, device=x.device)
        cg_mlp_train_epoch(self.handle, x, t, x.shape[0], perm, batch, lr, losses, stream)
        return losses

    def set_norm(self, in_mean, in_scale, out_mean, out_scale):
        cg_mlp_set_norm(self.handle, in_mean, in_scale, out_mean, out_scale)

    def save(self) -> bytes:
        return cg_mlp_save(self.handle)


class Server:
    """Streaming scheduler on the current device (``cg_server_*``)."""

    def __init__(self, device_budget_bytes: int):
        self.handle = cg_server_create(device_budget_bytes)

    def inject(self, what: int, value: float):
        cg_server_inject(self.handle, what, value)

    def close(self):
        if getattr(self, "handle", None):
            cg_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Stream:
    """One instrument stream on a Server (``cg_stream_*``); the plan must
    outlive it.  Frames are pushed from host numpy arrays."""

    def __init__(self, server: Server, plan: Plan, ring_bytes: int, batch_frames: int,
                 max_delay_s: float = 1e-3, avg_window: int = 10_000):
        self.plan = plan
        self.T = plan.T
        self.handle = cg_stream_create(server.handle, plan.handle, ring_bytes, batch_frames,
                                       max_delay_s, avg_window)

    def push(self, frames: np.ndarray, first_seq: int, t_arrival: float = -1.0) -> int:
        f = np.ascontiguousarray(frames, dtype=np.int16)
        return cg_stream_push(self.handle, f, f.shape[0], first_seq, t_arrival)

    def poll(self, cap: int = 65536, timeout_s: float = 0.0, want_amps: bool = False):
        """(results array of RESULT_DTYPE, amps [k, T] or None, status)."""
        recs = np.empty(cap, dtype=RESULT_DTYPE)
        amps = np.empty((cap, self.T), dtype=np.float32) if want_amps else None
        k, st = cg_stream_poll(self.handle, recs, amps, timeout_s)
        return recs[:k], (amps[:k] if want_amps else None), st

    def flush(self, timeout_s: float = 30.0) -> int:
        return cg_stream_flush(self.handle, timeout_s)

    def stats(self) -> dict:
        return cg_stream_stats(self.handle)

    def window(self) -> dict:
        return cg_stream_window(self.handle, self.T)

    def close(self):
        if getattr(self, "handle", None):
            cg_stream_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
