"""Split-precision tensor-core readout (DFT-at-teeth GEMM) against the FP64
oracle (GPU).

The readout is Re/Im of X at the tooth bins as a product of the FP16 samples
with FP16 hi + lo twiddles, accumulated in FP32 on the tensor cores; its
amplitudes must meet the readout tolerance (|dy| <= 1e-5) and the fit that
follows (FP64 4x4 solve) the centre tolerance (1e-4 of the linewidth).  The
measured error statistics are printed for the error table."""
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


def _plan(w, bits):
    return cg.Plan(*W.plan_args(w), readout=cg.READOUT_GEMM_SPLIT, sample_bits=bits)


@pytest.mark.parametrize("name", ["tiny", "wide", "paper_rate", "serve4096"])
@pytest.mark.parametrize("bits", [12, 16])
def test_gemm_readout_parity(dev, name, bits):
    w = W.workload(name)
    fr = torch.from_numpy(w["frames"]).to(dev)
    with _plan(w, bits) as p:
        amps, y = p.readout(fr)
        cg.cg_check_device(p.handle)
        amps, y = amps.cpu().numpy(), y.cpu().numpy()
    dy = np.abs(y - w["oracle"]["y"])
    rel = np.abs(amps - w["oracle"]["amps"]) / w["ref"][None, :]
    print(f"\n[gemm {name} bits={bits}] max|dy| {dy.max():.3e} rms {np.sqrt((dy**2).mean()):.3e} "
          f"max rel-to-ref {rel.max():.3e}")
    assert rel.max() <= AMP_TOL
    assert dy.max() <= AMP_TOL


def test_gemm_ragged_and_misaligned(dev):
    w = W.workload("wide")
    fr = torch.from_numpy(w["frames"]).to(dev)
    with _plan(w, 12) as p:
        for a, b in [(1, 130), (3, 4), (0, 257)]:
            amps, _ = p.readout(fr[a:b], want_y=False)
            cg.cg_check_device(p.handle)
            err = np.max(np.abs(amps.cpu().numpy() - w["oracle"]["amps"][a:b]) / w["ref"])
            assert err <= AMP_TOL, (a, b, err)


@pytest.mark.parametrize("name", ["tiny", "wide"])
def test_gemm_process_parity(dev, name):
    w = W.workload(name)
    fr = torch.from_numpy(w["frames"]).to(dev)
    with _plan(w, 12) as p:
        assert p.info["path"] == cg.PATH_PIPELINE
        out = p.process(fr)
        cg.cg_check_device(p.handle)
        o = {k: v.cpu().numpy() for k, v in out.items() if v is not None}
    ok = W.judge_fit(o["params"], o["status"], w["oracle"], w["converged"], CENTER_TOL, f"gemm {name}")
    conv = w["converged"]["params"]
    dc = np.abs(o["params"][ok, 0] - conv[ok, 0])
    print(f"\n[gemm+fp64 fit {name}] centre err max {dc.max():.1f} Hz, mean iters {o['iters'].mean():.2f}")
    assert dc.max() <= CENTER_TOL
