"""Pins of the oracle's displacement PSD and resonance fit (CPU).

The paper estimates the power spectral density of the fitted cavity
positions for several averaging times and fits the mechanical resonance
(f0, Q) ("Experimental Results"; Fig. 6).  Pins: SciPy's Welch estimate with
the same settings; Parseval's theorem; the Hann-window peak of a bin-centred
sinusoid; the model's closed forms and its Jacobian by central differences;
noise-free recovery; MINPACK's LM on the same log residuals; the fit of an
AR(2) oscillator's spectrum recovers its resonance.
"""
import numpy as np
import pytest

from oracle import psd

signal = pytest.importorskip("scipy.signal")
optimize = pytest.importorskip("scipy.optimize")


@pytest.mark.parametrize("M,n", [(256, 256), (1024, 5000), (4096, 40000)])
def test_welch_equals_scipy(M, n):
    x = np.random.default_rng(M).standard_normal(n) * 3.0 + 7.0
    f, S, K = psd.welch(x, 1e6, M)
    fs_, Ss = signal.welch(x, fs=1e6, window="hann", nperseg=M, noverlap=M // 2, detrend="constant",
                           scaling="density", return_onesided=True)
    assert K == (n - M) // (M // 2) + 1
    assert np.allclose(f, fs_, rtol=0, atol=1e-9)
    assert np.allclose(S, Ss, rtol=1e-12, atol=0)


def test_parseval_one_segment():
    # with a rectangular view: sum_k c_k |X_k|^2 / M = sum_n (w_n x_n)^2
    M = 512
    x = np.random.default_rng(1).standard_normal(M)
    f, S, K = psd.welch(x, 2.0, M)
    w = psd.hann(M)
    xw = (x - x.mean()) * w
    assert np.isclose(np.sum(S) * (2.0 / M) * np.sum(w * w), np.sum(xw ** 2), rtol=1e-12)


def test_sinusoid_peak():
    # a sinusoid of amplitude a on bin b: |X_b| = a M / 4 under the Hann window
    M, b, a, fs = 1024, 37, 2.5, 1e6
    n = np.arange(4 * M)
    x = a * np.cos(2 * np.pi * b * n / M)
    f, S, K = psd.welch(x, fs, M)
    w = psd.hann(M)
    assert np.isclose(S[b], 2 * (a * M / 4) ** 2 / (fs * np.sum(w * w)), rtol=1e-9)


def test_model_closed_forms_and_jacobian():
    p = np.array([23.7e3, 120.0, 3.0, 0.5])
    assert np.isclose(psd.model([0.0], p)[0], p[2] + p[3], rtol=1e-14)
    assert np.isclose(psd.model([p[0]], p)[0], p[2] * p[1] ** 2 + p[3], rtol=1e-14)
    f = np.linspace(22e3, 25.5e3, 57)
    J = psd.jacobian(f, p)
    steps = np.array([1e-3, 1e-4, 1e-6, 1e-6])
    for i in range(4):
        dp = np.zeros(4)
        dp[i] = steps[i]
        num = (psd.model(f, p + dp) - psd.model(f, p - dp)) / (2 * steps[i])
        assert np.max(np.abs(num - J[:, i])) <= 1e-6 * np.max(np.abs(J[:, i])), i


def test_noise_free_recovery():
    p = np.array([23.7e3, 114.4, 2.0e-3, 4.0e-6])
    f = np.arange(22000.0, 25500.0, 30.0)
    r = psd.fit(f, psd.model(f, p))
    assert r["status"] == 0
    assert np.allclose(r["params"], p, rtol=1e-8)


def test_agrees_with_minpack_on_noisy_spectrum():
    rng = np.random.default_rng(5)
    p = np.array([23.7e3, 120.0, 1.0, 0.02])
    f = np.arange(21000.0, 26500.0, 30.5)
    S = psd.model(f, p) * rng.gamma(50.0, 1.0 / 50.0, f.size)       # a 50-segment Welch estimate's spread
    r = psd.fit(f, S)

    def res(q):
        return np.log(S) - np.log(psd.model(f, q))
    ls = optimize.least_squares(res, psd.init(f, S), method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15)
    assert r["status"] == 0
    # the same optimum: equal objective; f0 and Q to 1e-7; scale and floor,
    # nearly degenerate inside a narrow band, to 1e-5
    assert np.isclose(r["rss"], 2 * ls.cost, rtol=1e-10)
    assert np.allclose(r["params"][:2], ls.x[:2], rtol=1e-7)
    assert np.allclose(r["params"][2:], ls.x[2:], rtol=1e-5)
    assert abs(r["params"][0] - p[0]) < 5 * r["sigma"][0]
    assert abs(r["params"][1] - p[1]) < 5 * r["sigma"][1]


def test_ar2_oscillator_resonance_is_recovered():
    # x_n = 2 r cos(w_d) x_{n-1} - r^2 x_{n-2} + e_n: a sampled damped
    # oscillator; its resonance lies at f0 with Q = pi f0 / (fs (-ln r))
    fs, f0, Q = 1e6, 23.7e3, 120.0
    rng = np.random.default_rng(8)
    n = 2_000_000
    r = np.exp(-np.pi * f0 / (Q * fs))
    wd = 2 * np.pi * f0 / fs * np.sqrt(1 - 1 / (4 * Q * Q))
    a1, a2 = 2 * r * np.cos(wd), -r * r
    e = rng.standard_normal(n)
    x = np.empty(n)
    x[0] = x[1] = 0.0
    for i in range(2, n):                 # plain loop: the recurrence is the definition
        x[i] = a1 * x[i - 1] + a2 * x[i - 2] + e[i]
    x += 3.0 * rng.standard_normal(n)     # white measurement floor
    f, S, K = psd.welch(x, fs, 32768)
    fb, Sb = psd.band(f, S, 21e3, 26.5e3)
    fit = psd.fit(fb, Sb)
    assert fit["status"] == 0
    assert abs(fit["params"][0] - f0) < 4 * fit["sigma"][0] + 5.0
    assert abs(fit["params"][1] - Q) < 4 * fit["sigma"][1] + 3.0
