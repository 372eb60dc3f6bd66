"""Pins of the oracle's median-filter initial centre (CPU).

The paper takes the batch of spectra as a time x tooth image, applies a 2-D
median filter with a 7x7 footprint and uses the lowest value of each
filtered row as the initial centre ("Data Capture and Processing",
initial-value paragraph).  Pins: the filter equals SciPy's median filter
with mirrored ("reflect") edges, also for images smaller than the footprint;
brute force with numpy's median over explicitly mirrored indices; the
closed form of the row minimum for a noise-free symmetric dip (a plateau of
five equal medians from k0 - 2 to k0 + 2, first tooth taken); isolated
outliers far from the dip leave the result unchanged; the Fano shift.
"""
import numpy as np
import pytest

import oracle

ndimage = pytest.importorskip("scipy.ndimage")


@pytest.mark.parametrize("shape", [(1, 5), (2, 7), (3, 9), (6, 5), (13, 21), (40, 99), (7, 221)])
def test_filter_equals_scipy_reflect(shape):
    rng = np.random.default_rng(shape[0] * 1000 + shape[1])
    y = rng.random(shape).astype(np.float32).astype(np.float64)
    got = oracle.median_filter7(y)
    want = ndimage.median_filter(y, size=7, mode="reflect")
    assert np.array_equal(got, want)


def _mirror(i, n):
    j = i % (2 * n)
    return j if j < n else 2 * n - 1 - j


def test_filter_brute_force_with_ties():
    rng = np.random.default_rng(9)
    y = rng.integers(0, 4, (9, 12)).astype(np.float64)        # many equal values
    got = oracle.median_filter7(y)
    n, T = y.shape
    for i in range(n):
        for k in range(T):
            win = [y[_mirror(i + a, n), _mirror(k + b, T)] for a in range(-3, 4) for b in range(-3, 4)]
            assert got[i, k] == np.median(win)


@pytest.mark.parametrize("k0", [10, 37, 49, 80])
def test_symmetric_dip_gives_the_plateau_start(k0):
    # a dip symmetric about tooth k0, constant in time: the 7-wide running
    # median equals y(k0 +- 2) at k0 - 2 .. k0 + 2 and is larger elsewhere
    x = np.arange(99) * 10e6
    g = 40e6
    row = 1.0 - 0.7 * g * g / ((x - x[k0]) ** 2 + g * g)
    y = np.tile(row, (12, 1))
    r = oracle.median_init(y, x)
    assert np.all(r["kmin"] == k0 - 2)
    f = r["filtered"][0]
    assert np.all(f[k0 - 2:k0 + 3] == row[k0 + 2])
    assert f[k0 - 3] > row[k0 + 2] and f[k0 + 3] > row[k0 + 2]


def test_isolated_outliers_do_not_move_the_minimum():
    rng = np.random.default_rng(4)
    x = np.arange(99) * 10e6
    g = 40e6
    n = 60
    c = 10e6 * np.sin(np.arange(n) / 9.0) + 300e6
    y = 1.0 - 0.7 * g * g / ((x[None, :] - c[:, None]) ** 2 + g * g) + 0.01 * rng.standard_normal((n, 99))
    clean = oracle.median_init(y, x)["kmin"]
    spiked = y.copy()
    for i in range(n):                                     # one deep outlier per row, far from the dip
        k = rng.choice(np.r_[0:15, 60:99])
        spiked[i, k] = -5.0
    assert np.array_equal(oracle.median_init(spiked, x)["kmin"], clean)
    # without the filter the raw row minimum lands on the outliers
    assert np.mean(np.argmin(spiked, axis=1) != clean) > 0.9


def test_shift_and_output_abscissa():
    x = np.arange(21) * 10e6 - 100e6
    y = np.random.default_rng(2).random((5, 21))
    r0 = oracle.median_init(y, x)
    r1 = oracle.median_init(y, x, shift=12e6)
    assert np.array_equal(r0["kmin"], r1["kmin"])
    assert np.array_equal(r0["c0"], x[r0["kmin"]])
    assert np.allclose(r1["c0"], x[r0["kmin"]] + 12e6, rtol=0, atol=1e-6)
