"""Displacement PSD and mechanical-resonance fit (GPU) against the oracle.

The paper turns the fitted cavity positions into power spectral densities
for several averaging times and fits the mechanical resonance (f0, Q) to
them ("Experimental Results"; Fig. 6).  Welch PSD: every bin of the GPU's
estimate (FP32 transform, FP64 averages) within the FP32 transform's error
bound of the FP64 oracle on the same float32 series, for every segment
length and for a strided series (the centre column of the fit output).  Resonance fit: FP64
on both sides, so f0 and Q agree to 1e-9 relative on the same PSD.  End to
end: frames whose centres follow a thermally driven resonator, through
cg_process, the PSD of the fitted centres and the fit: the resonance is
recovered within its standard errors.
"""
import numpy as np
import pytest

import synth
from oracle import psd as opsd

torch = pytest.importorskip("torch")
cg = pytest.importorskip("paper_2307_12988_gb300")

pytestmark = pytest.mark.gpu

FS = 1e6            # frame rate of the paper-rate geometry (1100 samples at 1.1 GS/s)
F0, Q0 = 23.7e3, 120.0


def psd_tol(S, M):
    """Bound on |S_gpu - S_oracle| per bin.  The FP32 transform's rounding
    error in X_k is about c eps sqrt(log2 M) rms(X), spread over all bins
    whatever their power, so a bin's error is ~ 2 |X_k| of it:
    2 c eps sqrt(log2 M) sqrt(S_k mean(S)) with eps = 2^-24 and c = 8;
    plus 1e-5 S_k for the FP32 window, twiddles and mean."""
    return 1e-5 * S + 2 * 8 * 2.0 ** -24 * np.sqrt(np.log2(M)) * np.sqrt(S * np.mean(S))


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def series():
    x = synth.oscillator_series(1_200_000, FS, F0, Q0, rms=2e6, floor=2e4, seed=3)
    return (x + 5e5).astype(np.float32)          # an offset the segment means remove


@pytest.mark.parametrize("M", [4096, 8192, 16384, 32768])
def test_welch_equals_oracle(dev, series, M):
    with cg.Psd(M) as p:
        S, K = p.welch(torch.from_numpy(series).to(dev), FS)
        S = S.cpu().numpy()
    f, So, Ko = opsd.welch(series.astype(np.float64), FS, M)
    assert K == Ko
    err = np.max(np.abs(S - So) / So)
    ratio = np.max(np.abs(S - So) / psd_tol(So, M))
    print(f"\n[welch M={M}] K={K} max rel err {err:.2e}, error / bound {ratio:.3f}")
    assert ratio <= 1.0


def test_welch_strided_and_exact_lengths(dev, series):
    M = 16384
    cols = np.zeros((series.size, 4), dtype=np.float32)
    cols[:, 0] = series
    cols[:, 1:] = 7.0
    with cg.Psd(M) as p:
        S1, K1 = p.welch(torch.from_numpy(cols).to(dev).reshape(-1), FS, stride=4, n=series.size)
        S0, K0 = p.welch(torch.from_numpy(series).to(dev), FS)
        assert K1 == K0 and torch.equal(S1, S0)
        # exactly one segment, and one sample short of a second
        for n, k in ((M, 1), (M + M // 2 - 1, 1), (M + M // 2, 2)):
            S, K = p.welch(torch.from_numpy(series[:n]).to(dev), FS)
            assert K == k
            So = opsd.welch(series[:n].astype(np.float64), FS, M)[1]
            assert np.all(np.abs(S.cpu().numpy() - So) <= psd_tol(So, M))
        with pytest.raises(cg.CgError, match="CG_ERR_ARG"):
            p.welch(torch.from_numpy(series[:M - 1]).to(dev), FS)


def test_resonance_fit_equals_oracle(dev, series):
    M = 32768
    f, So, _ = opsd.welch(series.astype(np.float64), FS, M)
    df = FS / M
    lo, hi = 21e3 + 0.5 * df, 26.5e3 + 0.5 * df          # band edges between bins
    out = cg.Psd.resonance(torch.from_numpy(So).to(dev), df, lo, hi)
    fb, Sb = opsd.band(f, So, lo, hi)
    r = opsd.fit(fb, Sb)
    print(f"\n[resonance] f0 {out[0]:.4f} +- {out[4]:.4f} Hz, Q {out[1]:.3f} +- {out[5]:.3f}, "
          f"steps {int(out[9])}, oracle f0 {r['params'][0]:.4f}")
    assert int(out[10]) == r["status"] == 0
    assert int(out[11]) == fb.size
    assert np.allclose(out[:2], r["params"][:2], rtol=1e-9)
    assert np.allclose(out[2:4], r["params"][2:], rtol=1e-6)
    assert np.allclose(out[4:8], r["sigma"], rtol=1e-6)
    assert np.isclose(out[8], r["rss"], rtol=1e-9)
    with pytest.raises(cg.CgError, match="CG_ERR_ARG"):
        cg.Psd.resonance(torch.from_numpy(So).to(dev), df, 23e3, 23e3 + 5 * df)


def test_resonance_from_fitted_centres(dev):
    # 1 s of paper-rate frames whose centres follow the resonator (2 MHz RMS)
    g = synth.PAPER_RATE
    n = 1_000_000
    c = synth.oscillator_series(n, FS, F0, Q0, rms=2e6, seed=21)
    stream = synth.make_stream(g, synth.BASE_SEED + 730)
    frames = synth.frames(stream, n, centers=c, snr_db=30.0, device=dev)["frames"]
    ref_frames = synth.frames(stream, 2000, cavity=False, noise_stream=1, snr_db=30.0)["frames"]
    import oracle
    ref = oracle.reference(ref_frames, oracle.tooth_bins(g.sample_rate, g.frame_len, g.tooth_freqs))
    with cg.Plan(g.sample_rate, g.frame_len, g.tooth_freqs, g.tooth_x, ref) as plan:
        out = plan.process(frames, want_y=False)
        cg.cg_check_device(plan.handle)
    params = out["params"]
    assert ((out["status"] & 3) == 0).float().mean().item() >= 0.999
    M = 32768
    with cg.Psd(M) as p:
        S, K = p.welch(params.reshape(-1), FS, stride=4, n=n)
        res = cg.Psd.resonance(S, FS / M, 21e3, 26.5e3)
    print(f"\n[end to end] K={K} f0 {res[0]:.3f} +- {res[4]:.3f} Hz, Q {res[1]:.2f} +- {res[5]:.2f}")
    assert int(res[10]) == 0
    assert abs(res[0] - F0) <= 5 * res[4] + 2.0
    assert abs(res[1] - Q0) <= 5 * res[5] + 0.03 * Q0
