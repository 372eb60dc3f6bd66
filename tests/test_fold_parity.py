"""Folded DFT-at-teeth readout on the tensor cores against the FP64 oracle
(GPU).

Each frame is folded to L = N / 10 complex values on the CUDA cores, then the
L-point DFT at the teeth runs as a split-precision product (FP16 hi + lo of
the folded values and of the twiddles, three products, FP32 accumulation) on
the tensor cores.  Amplitudes must meet the readout tolerance (|dy| <= 1e-5),
the fit that follows the centre tolerance (1e-4 of the linewidth); ragged
tiles, misaligned and empty inputs and full-range int16 samples are covered.
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


def _plan(w, **opts):
    return cg.Plan(*W.plan_args(w), readout=cg.READOUT_FOLD_GEMM, **opts)


def _errs(amps, y, w, lo=0, hi=None):
    o = w["oracle"]
    rel = np.abs(amps - o["amps"][lo:hi]) / w["ref"][None, :]
    dy = np.abs(y - o["y"][lo:hi]) if y is not None else np.zeros(1)
    return rel.max(), dy.max()


@pytest.mark.parametrize("name", ["tiny", "paper_rate", "tiny_peak"])
def test_fold_readout_parity(dev, name):
    w = W.workload(name)
    fr = torch.from_numpy(w["frames"]).to(dev)
    with _plan(w) as p:
        amps, y = p.readout(fr)
        cg.cg_check_device(p.handle)
        amps, y = amps.cpu().numpy(), y.cpu().numpy()
    rel, dy = _errs(amps, y, w)
    print(f"\n[fold {name}] max|dy| {dy:.3e} max rel-to-ref {rel:.3e}")
    assert rel <= AMP_TOL
    assert dy <= AMP_TOL


def test_fold_ragged_misaligned_and_empty(dev):
    w = W.workload("paper_rate")
    fr = torch.from_numpy(w["frames"]).to(dev)
    with _plan(w) as p:
        # 4-byte aligned slices with ragged last tiles; a 2-byte aligned slice
        # (read out by the general transform); a single frame
        for a, b in [(2, 131), (0, 129), (4, 1500), (1, 130), (7, 8), (0, 1)]:
            amps, y = p.readout(fr[a:b])
            cg.cg_check_device(p.handle)
            rel, dy = _errs(amps.cpu().numpy(), y.cpu().numpy(), w, a, b)
            assert rel <= AMP_TOL and dy <= AMP_TOL, (a, b, rel, dy)
        amps, y = p.readout(fr[:0])
        assert amps.shape == (0, w["ref"].size)


def test_fold_full_range_int16(dev):
    # 12-bit samples times 16 span the int16 range; the readout is linear,
    # so the amplitudes scale by exactly 16
    w = W.workload("paper_rate")
    fr16 = (w["frames"][:600].astype(np.int32) * 16).astype(np.int16)
    with _plan(w) as p:
        amps, _ = p.readout(torch.from_numpy(fr16).to(dev), want_y=False)
        cg.cg_check_device(p.handle)
        amps = amps.cpu().numpy() / 16.0
    rel, _ = _errs(amps, None, w, 0, 600)
    assert rel <= AMP_TOL


@pytest.mark.parametrize("name", ["tiny", "paper_rate"])
def test_fold_process_parity(dev, name):
    w = W.workload(name)
    fr = torch.from_numpy(w["frames"]).to(dev)
    with _plan(w) as p:
        assert p.info["path"] == cg.PATH_PIPELINE
        out = p.process(fr)
        cg.cg_check_device(p.handle)
        o = {k: v.cpu().numpy() for k, v in out.items() if v is not None}
    ok = W.judge_fit(o["params"], o["status"], w["oracle"], w["converged"], CENTER_TOL, f"fold {name}")
    conv = w["converged"]["params"]
    dc = np.abs(o["params"][ok, 0] - conv[ok, 0])
    print(f"\n[fold + fit {name}] centre err max {dc.max():.1f} Hz, mean iters {o['iters'].mean():.2f}")
    assert dc.max() <= CENTER_TOL


def test_fold_results_independent_of_requesting_y(dev):
    w = W.workload("paper_rate")
    fr = torch.from_numpy(w["frames"]).to(dev)
    with _plan(w) as p:
        a1, _ = p.readout(fr)
        a2, _ = p.readout(fr, want_y=False)
        torch.cuda.synchronize()
        assert torch.equal(a1, a2)


def test_fold_unsupported_geometries_are_refused(dev):
    for name in ("wide", "serve4096"):     # 221 teeth; N = 4096 is no radix-10 coset
        w = W.workload(name)
        with pytest.raises(cg.CgError, match="CG_ERR_UNSUPPORTED"):
            _plan(w)
