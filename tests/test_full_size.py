"""Parity at the full workload sizes, in the launch configuration the
benchmark times (GPU).

Each case builds the benchmark's seeded workload on the device (10^6
paper-rate frames; 4 x 10^5 wide frames for the split-precision GEMM readout;
10^6 learned-guess frames; 10^6 8-bit 2200-sample frames), runs one ``cg_process`` call over all of it with
the benchmark's outputs (amplitudes, no y), then checks sampled frames one by
one against the FP64 oracle (tooth amplitudes within 1e-5 of the reference,
converged centres within 1e-4 of the linewidth, statuses equal to the
oracle's capped run) and properties that hold at any size (finite
parameters, iteration bound).  The sample covers the first and last frames,
both sides of 128-frame tile edges, random frames and every frame the GPU
did not report converged.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from tests import workloads as W

torch = pytest.importorskip("torch")
cg = pytest.importorskip("paper_2307_12988_gb300")

pytestmark = pytest.mark.gpu

AMP_TOL = 1e-5
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MLP_BLOB = os.path.join(ROOT, "paper_2307_12988_gb300", "data", "mlp_wide_t221.cgmlp")

# name: (geometry, frames, generator keywords, plan options) -- the benchmark's
# workloads and seeds (stream seed BASE_SEED + 2, learned parameters + 600)
CASES = {
    "paper_rate_fft": (synth.PAPER_RATE, 1_000_000, dict(snr_db=30.0, center_amp_hz=20e6), {}),
    "paper_rate_fold": (synth.PAPER_RATE, 1_000_000, dict(snr_db=30.0, center_amp_hz=20e6),
                        dict(readout=cg.READOUT_FOLD_GEMM)),
    "wide_gemm": (synth.WIDE, 400_000, dict(snr_db=30.0, center_amp_hz=20e6),
                  dict(readout=cg.READOUT_GEMM_SPLIT, sample_bits=12)),
    "learned_mlp": (synth.WIDE, 1_000_000, "learned", dict(init=cg.INIT_MLP)),
    "paper8_int8": (synth.PAPER_8BIT, 1_000_000, dict(snr_db=30.0, center_amp_hz=20e6, bits=8), {}),
}


def _sample(n, rng):
    edges = np.arange(128, n, 128 * 997)
    idx = np.concatenate([np.arange(64), np.arange(n - 64, n), edges - 1, edges,
                          rng.integers(0, n, 128)])
    return np.unique(idx[(idx >= 0) & (idx < n)])


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.mark.parametrize("case", list(CASES))
def test_full_size_sampled_parity(dev, case):
    g, n, kw, opts = CASES[case]
    stream = synth.make_stream(g, synth.BASE_SEED + 2)
    fwhm = None
    if kw == "learned":
        lp = synth.learned_params(n, seed=synth.BASE_SEED + 600)
        kw = dict(centers=lp["c"], fwhm_hz=lp["fwhm"], snr_db=lp["snr_db"])
        fwhm = lp["fwhm"]
        noise = dict(snr_db=30.0)
    else:
        noise = {k: v for k, v in kw.items() if k in ("snr_db", "sigma", "bits")}
    frames = synth.frames(stream, n, device=dev, **kw)["frames"]
    ref_frames = synth.frames(stream, 2000, cavity=False, noise_stream=1, **noise)["frames"]
    bins = oracle.tooth_bins(g.sample_rate, g.frame_len, g.tooth_freqs)
    ref = oracle.reference(ref_frames, bins)
    T = g.n_teeth
    with cg.Plan(g.sample_rate, g.frame_len, g.tooth_freqs, g.tooth_x, ref, **opts) as p:
        if opts.get("init") == cg.INIT_MLP:
            with open(MLP_BLOB, "rb") as f:
                p.mlp_load(f.read())
        amps = torch.empty((n, T), dtype=torch.float32, device=dev)
        params = torch.empty((n, 4), dtype=torch.float32, device=dev)
        rss = torch.empty(n, dtype=torch.float32, device=dev)
        iters = torch.empty(n, dtype=torch.int16, device=dev)
        status = torch.empty(n, dtype=torch.int16, device=dev)
        process = cg.cg_process_i8 if frames.dtype == torch.int8 else cg.cg_process
        process(p.handle, frames, n, amps, None, params, rss, iters, status, None)
        torch.cuda.synchronize()
        cg.cg_check_device(p.handle)
        max_iter = 20
    # properties of every frame
    st = status.cpu().numpy()
    pr = params.cpu().numpy()
    it = iters.cpu().numpy()
    conv = (st & 3) == 0
    assert np.all(np.isfinite(pr[conv]))
    # (the learned path reports its polish steps plus the fallback's)
    assert it.max() <= max_iter + (2 if opts.get("init") == cg.INIT_MLP else 0)
    # sampled frames against the oracle; every frame the GPU did not report
    # converged joins the sample, so that no frame goes unjudged
    idx = np.union1d(_sample(n, np.random.default_rng(11)), np.flatnonzero(~conv))
    assert idx.size <= 4096, np.unique(st, return_counts=True)
    fr_host = frames[torch.from_numpy(idx).to(dev)].cpu().numpy()
    o = oracle.process(fr_host, bins, ref, g.tooth_x)
    a = amps[torch.from_numpy(idx).to(dev)].cpu().numpy()
    err = np.max(np.abs(a - o["amps"]) / ref[None, :])
    full = oracle.fit_batch(o["y"], g.tooth_x, converged=True)
    if fwhm is None:
        # status of each sampled frame as the oracle's capped run, centres
        # against the converged optimum (unconverged: the capped result)
        W.judge_fit(pr[idx], st[idx], o, full, 1e-4 * synth.FWHM_HZ, case)
    ok = conv[idx] & (full["status"] == 0)
    tol = 1e-4 * (fwhm[idx][ok] if fwhm is not None else synth.FWHM_HZ)
    dc = np.abs(pr[idx][ok, 0] - full["params"][ok, 0])
    print(f"\n[{case}] {idx.size} sampled frames: amp err {err:.2e}, centre err max {dc.max():.1f} Hz "
          f"(ratio to tol {np.max(dc / tol):.3f}), converged {conv.mean():.5f}")
    assert err <= AMP_TOL
    if fwhm is None:
        assert np.all(dc <= tol)
    else:
        # the learned path's bar: as often within 1e-4 of each frame's linewidth
        # as the held-out gain test asks (99.9 %), on this smaller sample 99 %
        assert np.mean(dc <= tol) >= 0.99
