"""8-bit input path (GPU): the paper's digitiser format, int8 samples at
2.2 GS/s in 2200-sample frames, through cg_process_i8 / cg_readout_i8.

The oracle reads the same samples widened to int16 (exact); amplitudes must
meet |dy| <= 1e-5 and converged centres 1e-4 of the linewidth; the int8 path
must equal the int16 path on the widened samples bit for bit; any byte
alignment, ragged and empty batches; geometries and readouts without an int8
kernel are refused.
"""
import numpy as np
import pytest

import synth
from tests import workloads as W

torch = pytest.importorskip("torch")
cg = pytest.importorskip("paper_2307_12988_gb300")

pytestmark = pytest.mark.gpu

AMP_TOL = 1e-5
CENTER_TOL = 1e-4 * synth.FWHM_HZ


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def w():
    return W.workload("paper8")


def _plan(w, **opts):
    return cg.Plan(*W.plan_args(w), **opts)


def _amp_err(amps, w, a=0, b=None):
    return np.max(np.abs(amps - w["oracle"]["amps"][a:b]) / w["ref"][None, :])


def test_int8_frames_are_int8_and_coset(w):
    assert w["frames"].dtype == np.int8
    with _plan(w) as p:
        assert p.info["fft_kind"] == cg.FFT_COSET and p.info["fft_len"] == 220


def test_int8_readout_parity(dev, w):
    fr = torch.from_numpy(w["frames"]).to(dev)
    with _plan(w) as p:
        amps, y = p.readout(fr)
        cg.cg_check_device(p.handle)
        amps, y = amps.cpu().numpy(), y.cpu().numpy()
    err = _amp_err(amps, w)
    print(f"\n[int8 readout] max rel-to-ref {err:.3e}")
    assert err <= AMP_TOL
    assert np.max(np.abs(y - w["oracle"]["y"])) <= AMP_TOL


def test_int8_equals_widened_int16_bit_for_bit(dev, w):
    fr8 = torch.from_numpy(w["frames"]).to(dev)
    fr16 = fr8.to(torch.int16)
    with _plan(w) as p:
        o8 = p.process(fr8)
        o16 = p.process(fr16)
        torch.cuda.synchronize()
    for k in ("amps", "y", "params", "rss", "iters", "status"):
        assert torch.equal(o8[k], o16[k]), k


def test_int8_any_alignment_ragged_and_empty(dev, w):
    fr = torch.from_numpy(w["frames"]).to(dev)
    flat = fr.reshape(-1)
    N = w["frames"].shape[1]
    with _plan(w) as p:
        for a, b in [(1, 130), (3, 4), (0, 257), (5, 1500)]:
            amps, _ = p.readout(fr[a:b], want_y=False)
            cg.cg_check_device(p.handle)
            assert _amp_err(amps.cpu().numpy(), w, a, b) <= AMP_TOL, (a, b)
        # frames starting 1..3 bytes past a 4-byte boundary
        for shift in (1, 2, 3):
            buf = torch.zeros(shift + 40 * N, dtype=torch.int8, device=dev)
            buf[shift:] = flat[: 40 * N]
            view = buf[shift:].view(40, N)
            amps, _ = p.readout(view, want_y=False)
            cg.cg_check_device(p.handle)
            assert _amp_err(amps.cpu().numpy(), w, 0, 40) <= AMP_TOL, shift
        amps, _ = p.readout(fr[:0])
        assert amps.shape == (0, w["ref"].size)


def test_int8_process_parity(dev, w):
    fr = torch.from_numpy(w["frames"]).to(dev)
    with _plan(w) as p:
        assert p.info["path"] == cg.PATH_PIPELINE
        o = {k: v.cpu().numpy() for k, v in p.process(fr).items() if v is not None}
        cg.cg_check_device(p.handle)
    ok = W.judge_fit(o["params"], o["status"], w["oracle"], w["converged"], CENTER_TOL, "int8")
    conv = w["converged"]["params"]
    dc = np.abs(o["params"][ok, 0] - conv[ok, 0])
    print(f"\n[int8 + fit] centre err max {dc.max():.1f} Hz, mean iters {o['iters'].mean():.2f}")
    assert dc.max() <= CENTER_TOL


def test_int8_unsupported_cases_are_refused(dev, w):
    fr8 = torch.zeros((4, 1100), dtype=torch.int8, device=dev)
    with _plan(W.workload("paper_rate")) as p:      # N = 1100: no int8 kernel
        with pytest.raises(cg.CgError, match="CG_ERR_UNSUPPORTED"):
            p.process(fr8)
    fr = torch.from_numpy(w["frames"][:4]).to(dev)
    with _plan(w, readout=cg.READOUT_GEMM_SPLIT) as p:
        with pytest.raises(cg.CgError, match="CG_ERR_UNSUPPORTED"):
            p.readout(fr)
