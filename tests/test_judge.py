"""The frame-by-frame fit judgement of the parity tests (CPU).

``tests.workloads.judge_fit`` decides every GPU parity verdict, so its
readings are checked here on constructed cases: a status that differs from
the oracle's capped run fails; a converged centre beyond the tolerance
fails; with ``failures_alike``, a cap-or-singular frame passes either way, a
frame the oracle leaves at the cap passes only if the GPU converged to the
oracle's optimum, a frame neither side can fit passes only if the GPU
centre left the tooth span, and a converged centre off the optimum passes
only if its FP64 chi^2 is within the LM tolerance of the optimum's.
"""
import numpy as np
import pytest

import oracle
from tests import workloads as W

X = np.linspace(-50e6, 50e6, 41)
P_OPT = np.array([1.0e6, 8.0e6, -0.7, 1.0])


def _case(n=3):
    y = np.stack([oracle.model(X, P_OPT) for _ in range(n)])
    y = y + np.random.default_rng(0).normal(0, 1e-3, y.shape)
    conv = oracle.fit_batch(y, X, converged=True)
    capped = {"status": conv["status"].copy(), "params": conv["params"].copy()}
    return y, capped, conv


def test_equal_runs_pass_and_a_status_change_fails():
    y, capped, conv = _case()
    params = conv["params"].astype(np.float32)
    status = conv["status"].copy()
    W.judge_fit(params, status, capped, conv, 1e3)
    status[1] = 1
    with pytest.raises(AssertionError):
        W.judge_fit(params, status, capped, conv, 1e3)


def test_a_converged_centre_beyond_the_tolerance_fails():
    y, capped, conv = _case()
    params = conv["params"].copy()
    params[2, 0] += 2e3
    with pytest.raises(AssertionError):
        W.judge_fit(params, conv["status"], capped, conv, 1e3)


def test_cap_and_singular_are_one_class_only_when_asked():
    y, capped, conv = _case()
    capped["status"][0] = 1
    status = conv["status"].copy()
    status[0] = 2
    with pytest.raises(AssertionError):
        W.judge_fit(conv["params"], status, capped, conv, 1e3)
    W.judge_fit(conv["params"], status, capped, conv, 1e3, failures_alike=True)


def test_converged_past_the_cap_needs_the_optimum():
    y, capped, conv = _case()
    capped["status"][1] = 1                          # the oracle stopped at its cap
    params = conv["params"].copy()
    W.judge_fit(params, conv["status"], capped, conv, 1e3, failures_alike=True)
    params[1, 0] += 5e3                             # ... and the GPU converged elsewhere
    with pytest.raises(AssertionError):
        W.judge_fit(params, conv["status"], capped, conv, 1e3, failures_alike=True)


def test_a_lost_dip_passes_only_outside_the_tooth_span():
    y, capped, conv = _case()
    capped["status"][2] = 1
    conv = {k: v.copy() for k, v in conv.items()}
    conv["status"][2] = 1                            # not even the long run fits it
    params = conv["params"].copy()
    params[2, 0] = 3.0 * X.max()
    W.judge_fit(params, np.zeros(3, np.int16), capped, conv, 1e3, failures_alike=True, y=y, x=X)
    params[2, 0] = 0.5 * X.max()
    with pytest.raises(AssertionError):
        W.judge_fit(params, np.zeros(3, np.int16), capped, conv, 1e3, failures_alike=True, y=y, x=X)


def test_an_off_optimum_centre_passes_only_on_flat_chi2():
    y, capped, conv = _case()
    params = conv["params"].copy()
    tol = 1.0
    # 2 Hz off on a 16 MHz-wide dip: past a 1 Hz tolerance, chi^2 unchanged to 1e-7
    params[0, 0] += 2.0
    r_opt = y[0] - oracle.model(X, conv["params"][0])
    r_off = y[0] - oracle.model(X, params[0])
    assert (r_off @ r_off) <= (r_opt @ r_opt) * (1 + 1e-7)
    W.judge_fit(params, conv["status"], capped, conv, tol, failures_alike=True, y=y, x=X)
    # without the spectra the rule does not apply
    with pytest.raises(AssertionError):
        W.judge_fit(params, conv["status"], capped, conv, tol, failures_alike=True)
    # far off: chi^2 rises well beyond the tolerance and the frame fails
    params[0, 0] += 2e6
    with pytest.raises(AssertionError):
        W.judge_fit(params, conv["status"], capped, conv, tol, failures_alike=True, y=y, x=X)
