"""The paper's median-filter initial centre (GPU) against the oracle.

The frames of one call form a time x tooth image; a 7x7 median filter with
mirrored edges and the lowest filtered value of each row give the initial
centre ("Data Capture and Processing", initial-value paragraph).  The tooth
index chosen is index work, so it must equal the oracle's bit for bit on the
same float32 spectra (cg_fit with max_iter = 0 returns the guess): noisy
Fano and Lorentzian workloads, random images full of ties, images smaller
than the footprint, ragged row counts across the kernel's 32-row blocks.
Through cg_process the fit from that guess must meet the usual bars
(converged centres within 1e-4 of the linewidth), independent of
chunk_frames, for both lineshapes.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import workloads as W

torch = pytest.importorskip("torch")
cg = pytest.importorskip("paper_2307_12988_gb300")

pytestmark = pytest.mark.gpu

CENTER_TOL = 1e-4 * synth.FWHM_HZ
GAMMA = synth.FWHM_HZ / 2.0


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _fano_opts(q):
    return dict(model=cg.MODEL_FANO, fano_q=q, fano_gamma=GAMMA, fano_A=0.7, fano_B=0.3, fano_box=0.1)


def _guess_index(dev, g, y32, shift=0.0, **opts):
    """Tooth index of the GPU's median-filter centre for the rows of y32."""
    n = y32.shape[0]
    with cg.Plan(g.sample_rate, g.frame_len, g.tooth_freqs, g.tooth_x, None, init=cg.INIT_MEDIAN,
                 max_iter=0, **opts) as p:
        y = torch.from_numpy(y32).to(dev)
        params = torch.empty((n, 4), dtype=torch.float32, device=dev)
        status = torch.empty(n, dtype=torch.int16, device=dev)
        cg.cg_fit(p.handle, y, n, None, params, None, None, status, None)
        torch.cuda.synchronize()
        cg.cg_check_device(p.handle)
    c = params[:, 0].cpu().numpy().astype(np.float64)
    dx = g.tooth_x[1] - g.tooth_x[0]
    return np.rint((c - shift - g.tooth_x[0]) / dx).astype(np.int64)


def _fano_y(q, n, seed_off=710):
    g = synth.PAPER_RATE
    stream = synth.make_stream(g, synth.BASE_SEED + seed_off)
    fr = synth.frames(stream, n, snr_db=30.0, center_amp_hz=20e6, shape="fano", fano_q=q)
    rf = synth.frames(stream, 1000, cavity=False, noise_stream=1, snr_db=30.0)
    bins = oracle.tooth_bins(g.sample_rate, g.frame_len, g.tooth_freqs)
    ref = oracle.reference(rf["frames"], bins)
    return fr["frames"], ref, oracle.process(fr["frames"], bins, ref, g.tooth_x)["y"]


@pytest.mark.parametrize("q", [0.0, 0.3])
def test_guess_index_equals_oracle_on_fano_spectra(dev, q):
    g = synth.PAPER_RATE
    _, _, y = _fano_y(q, 3000)
    y32 = y.astype(np.float32)
    want = oracle.median_init(y32, g.tooth_x)["kmin"]
    got = _guess_index(dev, g, y32, shift=q * GAMMA, **_fano_opts(q))
    assert np.array_equal(got, want)
    got_l = _guess_index(dev, g, y32)                      # the Lorentzian plan, same centre
    assert np.array_equal(got_l, want)


@pytest.mark.parametrize("geom,n", [(synth.PAPER_RATE, 1), (synth.PAPER_RATE, 2), (synth.PAPER_RATE, 3),
                                    (synth.TINY, 7), (synth.TINY, 33), (synth.PAPER_RATE, 257),
                                    (synth.WIDE, 300), (synth.SERVE_4096, 65)])
def test_guess_index_equals_oracle_with_ties(dev, geom, n):
    rng = np.random.default_rng(n + geom.n_teeth)
    T = geom.n_teeth
    # integer-valued images: many equal medians, the first tooth must win
    y32 = rng.integers(0, 6, (n, T)).astype(np.float32)
    want = oracle.median_init(y32, geom.tooth_x)["kmin"]
    assert np.array_equal(_guess_index(dev, geom, y32), want)
    # a smooth dip with noise, and a constant image (every window ties)
    c = rng.uniform(-0.3, 0.3, n) * (geom.tooth_x[-1] - geom.tooth_x[0])
    d = geom.tooth_x[None, :] - c[:, None]
    y32 = (1.0 - 0.7 * GAMMA ** 2 / (d * d + GAMMA ** 2) + 0.02 * rng.standard_normal((n, T))).astype(np.float32)
    assert np.array_equal(_guess_index(dev, geom, y32), oracle.median_init(y32, geom.tooth_x)["kmin"])
    y32 = np.full((n, T), 0.5, dtype=np.float32)
    assert np.all(_guess_index(dev, geom, y32) == 0)


def _fano_capped(y, g, q):
    """The oracle's capped Fano run from the median-filter centre (the GPU's
    starting point): scale and offset start at their averages."""
    c0 = oracle.median_init(y.astype(np.float32), g.tooth_x, shift=q * GAMMA)["c0"]
    p0 = np.stack([c0, np.full_like(c0, 0.7), np.full_like(c0, 0.3)], axis=1)
    return oracle.fano_fit_batch(y, g.tooth_x, q, GAMMA, 0.7, 0.3, box=0.1, p0=p0)


def _lorentz_capped(y, g):
    """The oracle's capped Lorentzian run from the median-filter centre with
    the moment guess's width, scale and offset."""
    p0 = oracle.fit_batch(y, g.tooth_x, max_iter=0)["init"]
    p0[:, 0] = oracle.median_init(y.astype(np.float32), g.tooth_x)["c0"]
    return oracle.fit_batch(y, g.tooth_x, p0=p0)


def _process(dev, g, frames, ref, **opts):
    with cg.Plan(g.sample_rate, g.frame_len, g.tooth_freqs, g.tooth_x, ref, init=cg.INIT_MEDIAN, **opts) as p:
        assert p.info["path"] == cg.PATH_PIPELINE
        out = p.process(torch.from_numpy(frames).to(dev))
        cg.cg_check_device(p.handle)
        return {k: v.cpu().numpy() for k, v in out.items() if v is not None}


def test_fano_fit_from_the_median_guess(dev):
    g = synth.PAPER_RATE
    q = 0.3
    frames, ref, y = _fano_y(q, 3000)
    o = _process(dev, g, frames, ref, **_fano_opts(q))
    rf = oracle.fano_fit_batch(y, g.tooth_x, q, GAMMA, 0.7, 0.3, box=0.1, converged=True)
    ok = W.judge_fit(o["params"], o["status"], _fano_capped(y, g, q), rf, CENTER_TOL, "median + fano")
    dc = np.abs(o["params"][ok, 0] - rf["params"][ok, 0])
    print(f"\n[median + fano] centre err max {dc.max():.1f} Hz, mean iters {o['iters'].mean():.2f}")
    assert np.all(dc <= CENTER_TOL)
    # chunking does not change the image
    o2 = _process(dev, g, frames, ref, chunk_frames=512, **_fano_opts(q))
    for k in ("params", "status", "iters"):
        assert np.array_equal(o[k], o2[k]), k


def test_lorentzian_fit_from_the_median_guess(dev):
    g = synth.PAPER_RATE
    stream = synth.make_stream(g, synth.BASE_SEED + 720)
    frames = synth.frames(stream, 3000, snr_db=30.0, center_amp_hz=20e6)["frames"]
    rf = synth.frames(stream, 1000, cavity=False, noise_stream=1, snr_db=30.0)["frames"]
    bins = oracle.tooth_bins(g.sample_rate, g.frame_len, g.tooth_freqs)
    ref = oracle.reference(rf, bins)
    y = oracle.process(frames, bins, ref, g.tooth_x)["y"]
    o = _process(dev, g, frames, ref)
    full = oracle.fit_batch(y, g.tooth_x, converged=True)
    ok = W.judge_fit(o["params"], o["status"], _lorentz_capped(y, g), full, CENTER_TOL, "median + lorentz")
    dc = np.abs(o["params"][ok, 0] - full["params"][ok, 0])
    print(f"\n[median + lorentz] centre err max {dc.max():.1f} Hz, mean iters {o['iters'].mean():.2f}")
    assert np.all(dc <= CENTER_TOL)


def test_the_papers_configuration_on_8bit_frames(dev):
    # 8-bit samples at 2.2 GS/s in 2200-sample frames, the median-filter
    # centre and the boxed Fano fit: the paper's whole processing chain
    g = synth.PAPER_8BIT
    q = 0.3
    stream = synth.make_stream(g, synth.BASE_SEED + 740)
    frames = synth.frames(stream, 2000, snr_db=30.0, center_amp_hz=20e6, shape="fano", fano_q=q, bits=8)["frames"]
    rf = synth.frames(stream, 1000, cavity=False, noise_stream=1, snr_db=30.0, bits=8)["frames"]
    bins = oracle.tooth_bins(g.sample_rate, g.frame_len, g.tooth_freqs)
    ref = oracle.reference(rf, bins)
    y = oracle.readout(frames, bins, ref)[1]
    assert frames.dtype == np.int8
    o = _process(dev, g, frames, ref, **_fano_opts(q))
    rf_ = oracle.fano_fit_batch(y, g.tooth_x, q, GAMMA, 0.7, 0.3, box=0.1, converged=True)
    ok = W.judge_fit(o["params"], o["status"], _fano_capped(y, g, q), rf_, CENTER_TOL, "8-bit median + fano")
    dc = np.abs(o["params"][ok, 0] - rf_["params"][ok, 0])
    print(f"\n[8-bit + median + fano] centre err max {dc.max():.1f} Hz, mean iters {o['iters'].mean():.2f}")
    assert np.all(dc <= CENTER_TOL)
