"""The GPU path on random geometries, against the FP64 oracle (GPU).

A fixed seeded set of geometries (frame lengths from the radices 2, 3, 5 and
11, 21 to 100 teeth on random distinct bins in random order, irregular tooth
abscissae, random dip centres, dips 4 to 10 tooth spacings wide as the
paper's cavity is about 8): synthetic 12-bit frames are read
out and fit by ``cg_process`` and compared frame by frame with the oracle's
readout (|dy| <= 1e-5) and fits (every frame's status as the oracle's run
with the same iteration cap, converged centres within 1e-4 of the dip's
FWHM of the oracle's converged optimum, or chi^2 within the LM tolerance
of the optimum's where chi^2 is too flat for the stopping rule to place the
centre that closely).  Both sides run up to 100 LM
steps: on irregular tooth sets with the dip off centre the moment guess can
start a linewidth away, and at the paper's cap of 20 the cap rather than
the arithmetic would decide many frames' status.  The geometries exercise the general
transform, whichever LM kernel the plan picks and the readout's mapping of
teeth to bins in any order.
"""
import numpy as np
import pytest

import oracle
from tests import workloads as W

torch = pytest.importorskip("torch")
cg = pytest.importorskip("paper_2307_12988_gb300")

pytestmark = pytest.mark.gpu

AMP_TOL = 1e-5


def _geometry(rng):
    """Frame length, bins, abscissa and lineshape of one random geometry."""
    e = [int(rng.integers(2, 7)), int(rng.integers(0, 3)), int(rng.integers(0, 3)), int(rng.integers(0, 2))]
    N = 2 ** e[0] * 3 ** e[1] * 5 ** e[2] * 11 ** e[3]
    while N < 200 or N > 4400:
        e = [int(rng.integers(2, 7)), int(rng.integers(0, 3)), int(rng.integers(0, 3)), int(rng.integers(0, 2))]
        N = 2 ** e[0] * 3 ** e[1] * 5 ** e[2] * 11 ** e[3]
    T = int(rng.integers(21, min(100, N // 2 - 2)))
    bins = rng.choice(np.arange(2, N // 2 - 1), size=T, replace=False)
    x = np.cumsum(rng.uniform(0.6, 1.4, T)) * 10e6
    x -= x.mean()
    span = x[-1] - x[0]
    c = rng.uniform(-0.2, 0.2) * span
    # a dip 4 to 10 tooth spacings wide (the paper's cavity spans about 8)
    g = rng.uniform(2.0, 5.0) * span / (T - 1)
    return N, bins, x, c, g


def _frames(rng, N, bins, x, c, g, n, cavity=True):
    T = bins.size
    env = rng.uniform(0.9, 1.1, T)
    ph = rng.uniform(0, 2 * np.pi, T)
    L = 1 - 0.7 * g ** 2 / ((x - c) ** 2 + g ** 2) if cavity else np.ones(T)
    E = 512 * np.sqrt(2.0 / T)
    nn = np.arange(N)
    basis = np.cos(2 * np.pi * np.outer(bins, nn) / N + ph[:, None])
    clean = (E * env * L) @ basis
    noisy = clean[None, :] + rng.normal(0, 20.0, (n, N))
    return np.clip(np.rint(noisy), -2048, 2047).astype(np.int16)


@pytest.mark.parametrize("seed", range(8))
def test_random_geometry_parity(seed):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(20260000 + seed)
    N, bins, x, c, g = _geometry(rng)
    fs = 1.0e9
    freqs = bins * fs / N                       # teeth exactly on their bins
    frames = _frames(np.random.default_rng(seed), N, bins, x, c, g, 150)
    ref_frames = _frames(np.random.default_rng(seed + 100), N, bins, x, c, g, 200, cavity=False)
    ref = oracle.reference(ref_frames, bins)
    o = oracle.process(frames, bins, ref, x, max_iter=100)
    conv = oracle.fit_batch(o["y"], x, converged=True)
    with cg.Plan(fs, N, freqs, x, ref, max_iter=100) as p:
        np.testing.assert_array_equal(p.bins, bins)
        out = p.process(torch.from_numpy(frames).to(dev))
        cg.cg_check_device(p.handle)
        got = {k: v.cpu().numpy() for k, v in out.items() if v is not None}
    assert np.max(np.abs(got["amps"] - o["amps"]) / ref[None, :]) <= AMP_TOL, (seed, N)
    assert np.max(np.abs(got["y"] - o["y"])) <= AMP_TOL
    # (a frame neither side fits within the cap may end as max_iter on one
    # and singular on the other: both are failures, compared as one class)
    ok = W.judge_fit(got["params"], got["status"], o, conv, 1e-4 * 2 * g, f"seed {seed} N {N} T {bins.size}",
                     failures_alike=True, y=o["y"], x=x)
    assert ok.mean() >= 0.99
