"""The seeded input generators (CPU): the lineshapes, the 8-bit frames and
the resonator series the Fano, 8-bit and PSD workloads are built from."""
import numpy as np
import pytest

import oracle
import synth
from oracle import psd as opsd


def test_fano_lineshape_reduces_to_the_dip_and_has_its_minimum_at_c_minus_q_gamma():
    x = np.arange(-49, 50) * 10e6
    c = np.array([3e6, -12e6])
    dip = synth.lineshape(x, c, 80e6, 0.7, "dip")
    assert np.allclose(synth.lineshape(x, c, 80e6, 0.7, "fano", fano_q=0.0), dip, rtol=0, atol=1e-15)
    # (1 - d) + d (q + e)^2 / (1 + e^2) is 1 - d at e = -q: the minimum
    q, g = 0.3, 40e6
    xm = np.array([c[0] - q * g])
    assert np.isclose(synth.lineshape(xm, c[:1], 80e6, 0.7, "fano", fano_q=q)[0, 0], 0.3, rtol=0, atol=1e-15)
    fine = np.linspace(-200e6, 200e6, 400001)
    prof = synth.lineshape(fine, c[:1], 80e6, 0.7, "fano", fano_q=q)[0]
    assert abs(fine[np.argmin(prof)] - (c[0] - q * g)) <= 1e3
    # and it matches the oracle's Fano model with A = d, B = 1 - d
    m = oracle.fano_model(x, q, g, [c[0], 0.7, 0.3])
    assert np.allclose(synth.lineshape(x, c[:1], 80e6, 0.7, "fano", fano_q=q)[0], m, rtol=0, atol=1e-14)


def test_eight_bit_frames():
    g = synth.PAPER_8BIT
    fr = synth.frames(synth.make_stream(g, 5), 8, snr_db=30.0, bits=8)["frames"]
    assert fr.dtype == np.int8 and fr.shape == (8, g.frame_len)
    # a quarter of full scale RMS before noise, so the samples use the range
    assert 20 < np.std(fr.astype(np.float64)) < 50


@pytest.mark.parametrize("f0,Q", [(23.7e3, 120.0), (40e3, 60.0)])
def test_oscillator_series_rms_and_resonance(f0, Q):
    x = synth.oscillator_series(1 << 20, 1e6, f0, Q, rms=2.5, seed=4)
    assert np.isclose(np.std(x), 2.5, rtol=1e-12)
    f, S, _ = opsd.welch(x, 1e6, 16384)
    assert abs(f[np.argmax(S)] - f0) <= 2 * f[1]
    # half-power width ~ f0 / Q
    band = (f > f0 - 10 * f0 / Q) & (f < f0 + 10 * f0 / Q)
    fit = opsd.fit(f[band], S[band])
    assert fit["status"] == 0
    assert abs(fit["params"][0] - f0) < 5 * fit["sigma"][0] + 5.0
    assert abs(fit["params"][1] / Q - 1.0) < 0.1


def test_generators_are_seeded():
    a = synth.oscillator_series(4096, 1e6, 23.7e3, 120.0, rms=1.0, floor=0.1, seed=9)
    b = synth.oscillator_series(4096, 1e6, 23.7e3, 120.0, rms=1.0, floor=0.1, seed=9)
    assert np.array_equal(a, b)
    g = synth.TINY
    f1 = synth.frames(synth.make_stream(g, 3), 5, sigma=10.0, shape="fano", fano_q=0.2)["frames"]
    f2 = synth.frames(synth.make_stream(g, 3), 5, sigma=10.0, shape="fano", fano_q=0.2)["frames"]
    assert np.array_equal(f1, f2)
