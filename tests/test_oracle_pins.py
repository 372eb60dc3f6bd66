"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each test ties one oracle function to a closed form, an invariant, brute
force, or an independent library routine, chosen so that a plausible slip
(dropped term, wrong sign or index, transposed operand) fails at least one:

* DFT at the teeth ("Data Capture and Processing": per-row transform read at
  the tooth bins): pure tone gives a N/2, X_0 = sum x, X_{N/2} = alternating
  sum, Parseval, numpy's rfft (real and imaginary parts, so the sign of the
  exponent is pinned too).
* readout and reference, through ``oracle.readout`` / ``oracle.reference``
  themselves: integer-valued tones at N/4 and N/6 give a N/2 and a N
  (magnitude, not power) at teeth listed out of bin order, y divides by the
  reference of the same tooth, the reference is the mean (not the sum) of
  the frames' magnitudes (not the magnitude of their mean).
* normalisation: noise-free unquantised frames divided by a cavity-free
  reference give the lineshape exactly.
* Lorentzian model and Jacobian: values at x = c and |x-c| = g; central
  finite differences.
* LM (fit paragraph: Levenberg-Marquardt, 20 iterations, tolerance 1e-6):
  noise-free recovery to 1e-12, shift / scale / mirror invariants, a
  brute-force variable-projection grid, and MINPACK's LM (scipy).
* moment initial guess: a hand-computed example (tests/golden).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tone(N, b, a=1.0, phi=0.3):
    n = np.arange(N)
    return a * np.cos(2 * np.pi * b * n / N + phi)


@pytest.mark.parametrize("N,b", [(1000, 51), (1100, 541), (2500, 1), (4096, 1944), (64, 31)])
def test_pure_tone_gives_half_N(N, b):
    a = 37.25
    re, im = oracle.dft_bins(_tone(N, b, a), [b, b + 1, max(b - 3, 0)])
    mag = np.hypot(re, im)[0]
    assert abs(mag[0] - a * N / 2) <= 1e-12 * a * N
    assert mag[1] <= 1e-9 * a * N and mag[2] <= 1e-9 * a * N


def test_dc_and_nyquist_bins_exact():
    rng = np.random.default_rng(1)
    N = 1100
    x = rng.integers(-2048, 2048, N).astype(np.int16)
    re, im = oracle.dft_bins(x, [0, N // 2])
    assert re[0, 0] == float(x.astype(np.int64).sum())
    alt = float((x.astype(np.int64) * (-1) ** np.arange(N)).sum())
    assert re[0, 1] == alt
    assert abs(im[0, 0]) == 0.0
    assert abs(im[0, 1]) <= 1e-12 * np.abs(x).sum()


@pytest.mark.parametrize("N", [16, 30, 44, 100])
def test_parseval(N):
    rng = np.random.default_rng(N)
    x = rng.integers(-2048, 2048, (3, N)).astype(np.int16)
    re, im = oracle.dft_bins(x, np.arange(N))
    lhs = (x.astype(np.float64) ** 2).sum(axis=1)
    rhs = (re ** 2 + im ** 2).sum(axis=1) / N
    np.testing.assert_allclose(rhs, lhs, rtol=1e-12)


@pytest.mark.parametrize("N", [1000, 1100, 2500, 4096])
def test_against_numpy_rfft(N):
    rng = np.random.default_rng(N + 7)
    x = rng.integers(-2048, 2048, (4, N)).astype(np.int16)
    bins = np.array([0, 1, 9, 11, 51, N // 3, N // 2 - 1, N // 2])
    re, im = oracle.dft_bins(x, bins)
    ref = np.fft.rfft(x.astype(np.float64), axis=1)[:, bins]
    scale = np.abs(x).sum(axis=1, keepdims=True)
    assert np.max(np.abs(re - ref.real) / scale) < 1e-13
    assert np.max(np.abs(im - ref.imag) / scale) < 1e-13


def test_tooth_bins_on_grid_and_alias():
    for g in (synth.TINY, synth.PAPER_RATE, synth.WIDE):
        bins = oracle.tooth_bins(g.sample_rate, g.frame_len, g.tooth_freqs)
        np.testing.assert_array_equal(bins, np.abs(51 + 10 * g.k))
    g = synth.SERVE_4096
    bins = oracle.tooth_bins(g.sample_rate, g.frame_len, g.tooth_freqs)
    # 1051 MHz at 2.0 GS/s aliases to 949 MHz, the bin of the -949 MHz tooth
    assert bins[-1] == 1944 and bins[0] == 1944
    assert bins[g.k.tolist().index(0)] == round(51e6 * 4096 / 2e9)


def _c4(N, a, sine=False):
    """a cos(pi n / 2) (or a sin): the integer sequence a, 0, -a, 0 -- a tone
    at bin N/4 whose samples are exact int16 values."""
    n = np.arange(N)
    return a * (np.array([0, 1, 0, -1]) if sine else np.array([1, 0, -1, 0]))[n % 4]


def _c6(N, a):
    """2a cos(pi n / 3): the integer sequence 2a, a, -a, -2a, -a, a (bin N/6)."""
    return a * np.array([2, 1, -1, -2, -1, 1])[np.arange(N) % 6]


@pytest.mark.parametrize("N", [1200, 2400])
def test_readout_exact_tones_by_tooth(N):
    # teeth listed out of bin order; two tones of different amplitude
    a1, a2 = 300, 200
    x = (_c4(N, a1) + _c6(N, a2)).astype(np.int16)
    bins = np.array([N // 6, N // 4, 0, N // 3], dtype=np.int32)
    ref = np.array([2.0, 5.0, 1.0, 3.0])
    amps, y = oracle.readout(x[None], bins, ref)
    exp = np.array([a2 * N, a1 * N / 2, 0.0, 0.0])   # |2 a cos| -> a N, |a cos| -> a N / 2
    np.testing.assert_allclose(amps[0], exp, rtol=1e-13, atol=1e-9 * a1 * N)
    np.testing.assert_allclose(y[0], exp / ref, rtol=1e-13, atol=1e-9 * a1 * N)
    # without ref no y; the FP64 entry reads the same integer samples alike
    amps2, y2 = oracle.readout(x[None], bins)
    assert y2 is None
    np.testing.assert_array_equal(amps2, amps)
    amps3, y3 = oracle.readout(x[None].astype(np.float64), bins, ref)
    np.testing.assert_array_equal(amps3, amps)
    np.testing.assert_array_equal(y3, y)
    with pytest.raises(ValueError):
        oracle.readout(x[None], bins, ref[:3])


def test_readout_rows_independent():
    # frame i of a batch reads the same as frame i alone
    N = 1200
    rng = np.random.default_rng(5)
    x = rng.integers(-2048, 2048, (5, N)).astype(np.int16)
    bins = np.array([7, 300, 200, 1, 600], dtype=np.int32)
    ref = rng.uniform(0.5, 2.0, bins.size)
    amps, y = oracle.readout(x, bins, ref)
    for i in range(5):
        a1, y1 = oracle.readout(x[i], bins, ref)
        np.testing.assert_array_equal(a1[0], amps[i])
        np.testing.assert_array_equal(y1[0], y[i])
    re, im = oracle.dft_bins(x, bins)
    np.testing.assert_allclose(amps, np.hypot(re, im), rtol=1e-15)


def test_reference_is_mean_of_magnitudes():
    N = 1200
    amps_in = [100, -300, 500]                  # a negative amplitude has magnitude |a|
    rows = [_c4(N, amps_in[0]), _c4(N, amps_in[1], sine=True), _c4(N, amps_in[2])]
    x = np.stack(rows).astype(np.int16)
    bins = np.array([N // 4, N // 6], dtype=np.int32)
    ref = oracle.reference(x, bins)
    # mean of |a_i| N / 2 (a sum would be 3x; the magnitude of the mean spectrum
    # |(100 + 500)/3 + i 300/3| N / 2 differs as well)
    assert abs(ref[0] - np.mean(np.abs(amps_in)) * N / 2) <= 1e-12 * 500 * N
    assert abs(ref[1]) <= 1e-9 * 500 * N
    # one frame: the reference is that frame's readout
    one = oracle.reference(x[:1], bins)
    np.testing.assert_array_equal(one, oracle.readout(x[:1], bins)[0][0])
    with pytest.raises(ValueError):
        oracle.reference(x[:0], bins)


def test_normalisation_noise_free_gives_lineshape():
    g = synth.PAPER_RATE
    N, fs = g.frame_len, g.sample_rate
    n = np.arange(N)
    rng = np.random.default_rng(3)
    env = rng.uniform(0.9, 1.1, g.n_teeth)
    ph = rng.uniform(0, 2 * np.pi, g.n_teeth)
    c, gam = 12.5e6, 40e6
    L = 1 - 0.7 * gam ** 2 / ((g.tooth_x - c) ** 2 + gam ** 2)
    basis = np.cos(2 * np.pi * np.outer(g.tooth_freqs, n) / fs + ph[:, None])
    cav = (env * L) @ basis
    refr = env @ basis
    bins = oracle.tooth_bins(fs, N, g.tooth_freqs)
    re1, im1 = oracle.dft_bins(cav[None], bins)
    re0, im0 = oracle.dft_bins(refr[None], bins)
    y = np.hypot(re1, im1)[0] / np.hypot(re0, im0)[0]
    np.testing.assert_allclose(y, L, rtol=0, atol=1e-12)
    # the same through the oracle's own readout and reference: three
    # cavity-free frames whose phases differ (equal magnitudes, so the mean
    # of magnitudes is each frame's), then the normalised cavity frame
    refs = np.stack([env @ np.cos(2 * np.pi * np.outer(g.tooth_freqs, n) / fs + ph[:, None] + s)
                     for s in (0.0, 0.7, 2.1)])
    ref = oracle.reference(refs, bins)
    np.testing.assert_allclose(ref, np.hypot(re0, im0)[0], rtol=1e-12)
    amps, y2 = oracle.readout(cav[None], bins, ref)
    np.testing.assert_allclose(y2[0], L, rtol=0, atol=1e-12)
    np.testing.assert_allclose(amps[0], np.hypot(re1, im1)[0], rtol=1e-13)


def test_model_closed_forms():
    p = np.array([3.0, 2.0, -0.7, 1.25])
    m = oracle.model([3.0, 5.0, 1.0, 1e9], p)
    np.testing.assert_allclose(m, [1.25 - 0.7, 1.25 - 0.35, 1.25 - 0.35, 1.25], atol=1e-15)


@pytest.mark.parametrize("p", [[3.0, 2.0, -0.7, 1.25], [-40.0, 35.0, 0.9, 0.1]])
def test_jacobian_finite_differences(p):
    x = np.linspace(-100, 100, 41)
    J = oracle.jacobian(x, p)
    for j in range(4):
        h = 1e-6 * max(1.0, abs(p[j]))
        pp, pm = np.array(p, float), np.array(p, float)
        pp[j] += h
        pm[j] -= h
        fd = (oracle.model(x, pp) - oracle.model(x, pm)) / (2 * h)
        np.testing.assert_allclose(J[:, j], fd, rtol=1e-6, atol=1e-9)


TRUE_PARAMS = [
    ([0.0, 40.0, -0.7, 1.0], "dip at centre"),
    ([17.3, 40.0, -0.7, 1.0], "dip off centre"),
    ([-63.1, 31.0, 1.0, 0.0], "literal peak"),
    ([5.2e6, 4.0e7, -0.7, 1.0], "Hz units"),
]


@pytest.mark.parametrize("p_true,label", TRUE_PARAMS)
def test_lm_noise_free_recovery(p_true, label):
    scale = 1e6 if abs(p_true[1]) > 1e3 else 1.0
    x = np.arange(-49, 50) * 10.0 * scale
    y = oracle.model(x, p_true)
    p0, flag = oracle.moment_init(y, x)
    assert flag == 0
    p, rss, it, st = oracle.lm_fit(y, x, p0, max_iter=oracle.CONVERGED_MAX_ITER,
                                   tol=oracle.CONVERGED_TOL)
    assert st == oracle.CONVERGED, (label, st, it)
    tol = np.array([1e-12 * scale * 100, 1e-12 * scale * 100, 1e-12, 1e-12])
    assert np.all(np.abs(p - np.array(p_true)) <= tol), (label, p - np.array(p_true))


def _noisy(p_true, x, sigma, seed):
    rng = np.random.default_rng(seed)
    return oracle.model(x, p_true) + sigma * rng.standard_normal(x.size)


def _conv_fit(y, x):
    p0, _ = oracle.moment_init(y, x)
    return oracle.lm_fit(y, x, p0, max_iter=oracle.CONVERGED_MAX_ITER, tol=oracle.CONVERGED_TOL)


def test_lm_shift_scale_mirror_invariants():
    x = np.arange(-49, 50) * 10.0
    y = _noisy([11.0, 40.0, -0.7, 1.0], x, 0.01, 11)
    p, *_ = _conv_fit(y, x)
    # shift: x -> x + delta moves c by delta, nothing else
    ps, *_ = _conv_fit(y, x + 123.0)
    np.testing.assert_allclose(ps - p, [123.0, 0, 0, 0], atol=1e-7)
    # scale: y -> s y scales A and B
    pk, *_ = _conv_fit(2.5 * y, x)
    np.testing.assert_allclose(pk, [p[0], p[1], 2.5 * p[2], 2.5 * p[3]], rtol=1e-8, atol=1e-8)
    # mirror-symmetric data about x = 0 gives c = 0
    ym = 0.5 * (y + y[::-1])
    pm, *_ = _conv_fit(ym, x)
    assert abs(pm[0]) < 1e-9


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_lm_matches_bruteforce_grid_and_minpack(seed):
    opt = pytest.importorskip("scipy.optimize")
    x = np.arange(-5, 6) * 10.0                       # T = 11 teeth
    p_true = [4.0 * seed - 6.0, 22.0, -0.6, 1.0]
    y = _noisy(p_true, x, 0.02, seed)
    cgrid = np.linspace(-40, 40, 801)
    ggrid = np.linspace(5, 60, 551)
    pg, chi2g = oracle.grid_fit(y, x, cgrid, ggrid)
    p, rss, it, st = _conv_fit(y, x)
    assert st == oracle.CONVERGED
    # the LM optimum is at least as good as the best grid point, and close to it
    assert rss <= chi2g * (1 + 1e-12)
    assert abs(p[0] - pg[0]) <= 0.1 + 1e-9 and abs(p[1] - pg[1]) <= 0.1 + 1e-9
    # MINPACK's LM from the grid point lands on the same optimum
    res = opt.least_squares(lambda q: oracle.model(x, q) - y, pg, method="lm",
                            xtol=1e-15, ftol=1e-15, gtol=1e-15)
    q = res.x.copy()
    q[1] = abs(q[1])
    np.testing.assert_allclose(p, q, rtol=1e-7, atol=1e-9)


def test_moment_init_hand_example():
    with open(os.path.join(GOLDEN, "moment_init_example.json")) as f:
        ex = json.load(f)
    p0, flag = oracle.moment_init(ex["y"], ex["x"])
    assert flag == 0
    np.testing.assert_allclose(p0, ex["p0"], rtol=1e-12, atol=1e-14)


def test_lm_flat_and_nonfinite_status():
    x = np.arange(-10, 11) * 10.0
    out = oracle.fit_batch(np.ones((1, x.size)), x)
    assert out["status"][0] == (oracle.SINGULAR | oracle.INIT_FLAT)
    y = np.ones(x.size)
    y[3] = np.nan
    out = oracle.fit_batch(y[None], x)
    assert out["status"][0] & 0xF == oracle.NONFINITE


def test_lm_iteration_cap_and_typical_count():
    """Capped fits stop at max_iter; with a moment start the tiny workload
    typically converges in a handful of iterations (the paper reports ~4)."""
    g = synth.TINY
    s = synth.make_stream(g, synth.BASE_SEED + 1)
    fr = synth.frames(s, 200, sigma=0.01 * synth.FULL_SCALE)
    rf = synth.frames(s, 200, cavity=False, sigma=0.01 * synth.FULL_SCALE, noise_stream=1)
    bins = oracle.tooth_bins(g.sample_rate, g.frame_len, g.tooth_freqs)
    ref = oracle.reference(rf["frames"], bins)
    out = oracle.process(fr["frames"], bins, ref, g.tooth_x)
    assert np.all(out["status"] == oracle.CONVERGED)
    assert 2.0 <= out["iters"].mean() <= 8.0
    capped = oracle.fit_batch(out["y"], g.tooth_x, max_iter=1)
    assert np.all(capped["iters"] == 1)
    conv = oracle.fit_batch(out["y"], g.tooth_x, converged=True)
    fwhm = synth.FWHM_HZ
    assert np.max(np.abs(conv["params"][:, 0] - out["params"][:, 0])) < 1e-4 * fwhm


def test_cavity_linewidth_closed_form():
    """FWHM = c / (2 L F) for the paper's cavity (finesse 9200, length 203 um)."""
    with open(os.path.join(GOLDEN, "cavity_linewidth.json")) as f:
        ex = json.load(f)
    fwhm = 299792458.0 / (2 * ex["length_m"] * ex["finesse"])
    assert abs(fwhm - ex["fwhm_hz"]) < 0.01e6
    assert abs(fwhm - synth.FWHM_HZ) / fwhm < 0.01
