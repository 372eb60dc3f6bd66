"""The C ABI library loads without a GPU and exports every declared symbol;
host-side argument checks answer before any CUDA call (CPU only)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import paper_2307_12988_gb300 as cg
from paper_2307_12988_gb300 import _binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(cg_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = cg.load()
    declared = _declared_functions()
    assert declared, "no declarations found"
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding marshals every one of them
    assert set(declared) <= set(_binding.exported_symbols()) | {"cg_opts_default"}


def test_status_strings_and_version():
    assert cg.cg_version() == 100
    assert cg.cg_status_string(0) == "ok"
    assert "argument" in cg.cg_status_string(1)
    assert cg.cg_status_string(99) == "unknown status"


def test_defaults():
    o = cg.cg_opts_default()
    assert (o.max_iter, o.tol, o.lambda0, o.path) == (20, 1e-6, 1e-3, 0)


@pytest.mark.parametrize("kw,err", [
    (dict(frame_len=7), "frame_len"),
    (dict(frame_len=20000), "frame_len"),
    (dict(tooth_freqs=np.array([1e6, 2e6, 3e6])), "n_teeth"),
    (dict(sample_rate=-1.0), "sample_rate"),
    (dict(ref=np.array([1.0, 1.0, 0.0, 1.0, 1.0])), "ref_spectrum"),
    (dict(tooth_freqs=np.array([1e6, np.nan, 3e6, 4e6, 5e6])), "tooth_freqs"),
    (dict(opts=dict(lanes_per_frame=5)), "lanes_per_frame"),
    (dict(opts=dict(lanes_per_frame=3)), "lanes_per_frame"),
    (dict(opts=dict(max_iter=-1)), "max_iter"),
])
def test_plan_argument_errors_before_cuda(kw, err):
    args = dict(sample_rate=1e9, frame_len=1000,
                tooth_freqs=np.array([11e6, 21e6, 31e6, 41e6, 51e6]), ref=None, opts={})
    args.update(kw)
    opts = cg.cg_opts_default(**args.pop("opts"))
    with pytest.raises(cg.CgError) as ei:
        cg.cg_plan(args["sample_rate"], args["frame_len"], args["tooth_freqs"], None,
                   args["ref"], opts)
    assert ei.value.status == 1
    assert err in str(ei.value)


def test_null_arguments_rejected():
    lib = cg.load()
    assert lib.cg_plan(None, 1e9, 1000, 5, None, None, None, None) == 1
    assert lib.cg_process(None, None, 0, None, None, None, None, None, None, None) == 1
    assert lib.cg_fit(None, None, 1, None, None, None, None, None, None) == 1
    assert lib.cg_plan_describe(None, None, None) == 1


def test_new_entry_points_reject_bad_arguments_before_cuda():
    """Argument checks of the learned-guess, streaming and timing entry points
    answer without touching the device."""
    import ctypes
    lib = cg.load()
    h = ctypes.c_void_p()
    # network shapes and batch limits
    assert lib.cg_mlp_create(ctypes.byref(h), 0, 256, 4, 16, 1) == 1
    assert lib.cg_mlp_create(ctypes.byref(h), 221, 2000, 4, 16, 1) == 1
    assert lib.cg_mlp_create(ctypes.byref(h), 221, 256, 0, 16, 1) == 1
    assert lib.cg_mlp_create(ctypes.byref(h), 221, 256, 4, 0, 1) == 1
    assert lib.cg_mlp_create(None, 221, 256, 4, 16, 1) == 1
    assert cg.cg_mlp_param_count(221, 256, 4) == 256 * 221 + 256 + 256 * 256 + 256 + 4 * 256 + 4
    assert cg.cg_mlp_param_count(0, 256, 4) == 0
    assert lib.cg_mlp_forward(None, None, 1, None, None) == 1
    assert lib.cg_mlp_backward(None, None, None, 1, None, None, None) == 1
    assert lib.cg_mlp_adam(None, ctypes.c_float(1e-3), ctypes.c_float(0.9), ctypes.c_float(0.999),
                           ctypes.c_float(1e-8), None) == 1
    assert lib.cg_mlp_load(None, None, 0) == 1
    assert lib.cg_mlp_infer(None, None, 1, None, None) == 1
    size = ctypes.c_size_t()
    assert lib.cg_mlp_save(None, None, 0, ctypes.byref(size)) == 1
    # streaming
    assert lib.cg_server_create(ctypes.byref(h), 0) == 1
    assert lib.cg_server_create(None, 1 << 20) == 1
    assert lib.cg_server_inject(None, 1, 0.0) == 1
    assert lib.cg_stream_create(ctypes.byref(h), None, None, 1 << 20, 16, 1e-3, 100) == 1
    assert lib.cg_stream_push(None, None, 1, 0, -1.0) == 1
    n = ctypes.c_int64()
    assert lib.cg_stream_poll(None, None, None, 1, ctypes.byref(n), 0.0) == 1
    assert lib.cg_stream_flush(None, 0.0) == 1
    assert lib.cg_stream_destroy(None) == 0          # NULL is ignored
    assert lib.cg_server_destroy(None) == 0
    # timing
    assert lib.cg_timing_enable(None, 1) == 1
    assert lib.cg_timing_collect(None, None, None) == 1
    assert cg.cg_clock() > 0


@pytest.mark.parametrize("kw", [dict(init=7), dict(polish_iter=-1)])
def test_plan_rejects_bad_learned_options(kw):
    opts = cg.cg_opts_default(**kw)
    with pytest.raises(cg.CgError) as ei:
        cg.cg_plan(1e9, 1000, np.array([11e6, 21e6, 31e6, 41e6, 51e6]), None, None, opts)
    assert ei.value.status == 1


def test_fano_defaults_and_layout():
    o = cg.cg_opts_default()
    assert (o.model, o.fano_box, o.fano_q, o.fano_gamma) == (cg.MODEL_LORENTZ, 0.1, 0.0, 0.0)
    # the ctypes mirror has the C layout: five doubles after the int block
    assert ctypes.sizeof(_binding.cg_opts) == 112
    assert _binding.cg_opts.fano_q.offset == 72


@pytest.mark.parametrize("kw,status,err", [
    (dict(model=7), 1, "model"),
    (dict(model=1, fano_gamma=0.0, fano_A=0.7), 1, "fano_gamma"),
    (dict(model=1, fano_gamma=4e7, fano_A=0.0), 1, "fano_A"),
    (dict(model=1, fano_gamma=4e7, fano_A=0.7, fano_box=1.5), 1, "fano_box"),
    (dict(model=1, fano_gamma=4e7, fano_A=0.7, fano_B=float("nan")), 1, "fano_A"),
    (dict(model=1, fano_gamma=4e7, fano_A=0.7, init=1), 8, "Fano"),
])
def test_plan_rejects_bad_fano_options(kw, status, err):
    opts = cg.cg_opts_default(**kw)
    with pytest.raises(cg.CgError) as ei:
        cg.cg_plan(1e9, 1000, np.array([11e6, 21e6, 31e6, 41e6, 51e6]), None, None, opts)
    assert ei.value.status == status
    assert err in str(ei.value)


def test_psd_entry_points_reject_bad_arguments_before_cuda():
    lib = cg.load()
    h = ctypes.c_void_p()
    for bad in (0, 1000, 2048, 65536, 32769):
        assert lib.cg_psd_create(bad, ctypes.byref(h)) == 1
    assert lib.cg_psd_create(32768, None) == 1
    k = ctypes.c_int64(0)
    assert lib.cg_psd_welch(None, None, 100000, 1, 1e6, None, ctypes.byref(k), None) == 1
    assert lib.cg_resonance_fit(None, 100, 30.0, 1e3, 2e3, 100, 1e-12, None, None) == 1
    lib.cg_psd_destroy(None)                                           # NULL is ignored
