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
                       cg_plan_destroy, cg_process, cg_readout, cg_reference_accumulate,
                       cg_set_reference, cg_status_string, cg_version, load)
from ._binding import (FFT_AUTO, FFT_COSET, FFT_FULL, FIT_CONVERGED, FIT_INIT_FLAT,
                       FIT_MAX_ITER, FIT_NONFINITE, FIT_SINGULAR, INIT_MLP, INIT_MOMENT,
                       READOUT_FFT, READOUT_GEMM_SPLIT, PATH_AUTO, PATH_FUSED, PATH_SPLIT,
                       PATH_PIPELINE)

__all__ = ["Plan", "CgError", "load", "cg_plan", "cg_plan_destroy", "cg_plan_describe",
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
        """Whole path on int16 frames [n, N] resident on the device."""
        n = frames.shape[0]
        if frames.dim() != 2 or frames.shape[1] != self.N:
            raise ValueError(f"frames must be [n, {self.N}]")
        o = self._outputs(n, frames.device, want_y)
        cg_process(self.handle, frames, n, o["amps"], o["y"], o["params"], o["rss"],
                   o["iters"], o["status"], stream)
        return o

    def readout(self, frames, want_y=True, stream=None):
        import torch
        n = frames.shape[0]
        amps = torch.empty((n, self.T), dtype=torch.float32, device=frames.device)
        y = torch.empty_like(amps) if want_y else None
        cg_readout(self.handle, frames, n, amps, y, stream)
        return amps, y

    def fit(self, y, p0=None, stream=None):
        n = y.shape[0]
        o = self._outputs(n, y.device, want_y=False, want_amps=False)
        cg_fit(self.handle, y, n, p0, o["params"], o["rss"], o["iters"], o["status"], stream)
        return o

    def reference_accumulate(self, frames, stream=None) -> np.ndarray:
        return cg_reference_accumulate(self.handle, frames, frames.shape[0], stream)
