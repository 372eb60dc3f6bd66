"""Property tests of the FP64 oracle over random geometries (CPU, hypothesis).

Frame lengths are products of the radices 2, 3, 5 and 11 (the transform
lengths of the paper's comb geometries and their neighbours), tooth sets are
random distinct bins, parameters random within the fit's domain.  Each
property holds for every draw:

* the direct-sum DFT at any bins equals numpy's rfft ("Data Capture and
  Processing": per-row transform read at the tooth bins);
* a tone at any bin reads a N/2 through ``oracle.readout``, divided by the
  reference of its own tooth;
* noise-free Lorentzian spectra on any tooth set are recovered by the
  converged LM to 1e-8 (fit paragraph: Levenberg-Marquardt on each
  normalised spectrum), and shifting the abscissa shifts the centre alone.
"""
import numpy as np
import pytest

import oracle

try:
    from hypothesis import given, settings, strategies as st
except ImportError:   # (not installed everywhere: the tests are skipped, not the module)
    given = settings = None

pytestmark = pytest.mark.skipif(given is None, reason="hypothesis is not installed")

if given is None:
    def _no_hypothesis(*args, **kwargs):
        return lambda fn: fn

    class _NoStrategies:
        def __getattr__(self, name):
            return lambda *args, **kwargs: _NoStrategies()

        def filter(self, *args, **kwargs):
            return self

    given = settings = _no_hypothesis
    st = _NoStrategies()


def _length(e2, e3, e5, e11):
    return (2 ** e2) * (3 ** e3) * (5 ** e5) * (11 ** e11)


lengths = st.builds(_length, st.integers(2, 6), st.integers(0, 2), st.integers(0, 2), st.integers(0, 1)).filter(
    lambda n: 16 <= n <= 4400)


@settings(max_examples=40, deadline=None)
@given(N=lengths, seed=st.integers(0, 2 ** 31 - 1))
def test_dft_at_bins_equals_rfft(N, seed):
    rng = np.random.default_rng(seed)
    x = rng.integers(-32768, 32768, (2, N)).astype(np.int16)
    bins = rng.choice(N // 2 + 1, size=min(12, N // 2 + 1), replace=False)
    re, im = oracle.dft_bins(x, bins)
    ref = np.fft.rfft(x.astype(np.float64), axis=1)[:, bins]
    scale = np.abs(x.astype(np.float64)).sum(axis=1, keepdims=True)
    assert np.max(np.abs(re - ref.real) / scale) < 1e-13
    assert np.max(np.abs(im - ref.imag) / scale) < 1e-13


@settings(max_examples=40, deadline=None)
@given(N=lengths, seed=st.integers(0, 2 ** 31 - 1))
def test_tone_reads_half_N_times_amplitude(N, seed):
    rng = np.random.default_rng(seed)
    T = int(rng.integers(1, min(8, N // 2 - 1) + 1))
    bins = rng.choice(np.arange(1, N // 2), size=T, replace=False)
    amp = rng.uniform(0.5, 100.0, T)
    phase = rng.uniform(0, 2 * np.pi, T)
    n = np.arange(N)
    frame = (amp[:, None] * np.cos(2 * np.pi * np.outer(bins, n) / N + phase[:, None])).sum(axis=0)
    ref = rng.uniform(0.5, 2.0, T)
    amps, y = oracle.readout(frame[None], bins, ref)
    np.testing.assert_allclose(amps[0], amp * N / 2, rtol=1e-10)
    np.testing.assert_allclose(y[0], amp * N / 2 / ref, rtol=1e-10)


@settings(max_examples=30, deadline=None)
@given(seed=st.integers(0, 2 ** 31 - 1), T=st.integers(11, 120))
def test_noise_free_lorentzian_recovered_on_any_tooth_set(seed, T):
    rng = np.random.default_rng(seed)
    # a random, increasing tooth abscissa (irregular spacing)
    x = np.cumsum(rng.uniform(0.5, 1.5, T)) * 10e6
    x -= x.mean()
    span = x[-1] - x[0]
    p = np.array([rng.uniform(-0.25, 0.25) * span, rng.uniform(0.04, 0.2) * span,
                  rng.choice([-1.0, 1.0]) * rng.uniform(0.2, 0.9), rng.uniform(0.5, 1.5)])
    y = oracle.model(x, p)
    fit = oracle.fit_batch(y[None], x, converged=True)
    assert fit["status"][0] == oracle.CONVERGED
    got = fit["params"][0]
    assert abs(got[0] - p[0]) <= 1e-8 * span
    assert abs(abs(got[1]) - p[1]) <= 1e-8 * span
    np.testing.assert_allclose(got[2:], p[2:], rtol=0, atol=1e-8)
    # a shifted abscissa moves the centre by the shift and nothing else
    d = rng.uniform(-1, 1) * span
    fit2 = oracle.fit_batch(y[None], x + d, converged=True)["params"][0]
    assert abs(fit2[0] - (got[0] + d)) <= 1e-8 * span
    assert abs(abs(fit2[1]) - abs(got[1])) <= 1e-8 * span
    np.testing.assert_allclose(fit2[2:], got[2:], rtol=0, atol=1e-8)
