"""Pins of the oracle's Fano lineshape and box-constrained LM (CPU).

The paper fits a 5-parameter Fano profile with only the centre free, the
scale and offset held to about +-10 % of pre-computed averages and the
asymmetry and width fixed ("Data Capture and Processing", fit paragraph).
Pins: the q = 0 profile equals the independently coded Lorentzian dip;
the Jacobian equals central differences; noise-free data are recovered;
parameters past the box end on its edge; the LM optimum is no worse than a
brute-force grid; the "lowest value" initial guess lands on the minimum.
"""
import numpy as np
import pytest

import oracle

X = np.arange(-49, 50) * 10e6          # the paper-rate tooth abscissa (Hz)
GAMMA = 40e6


@pytest.mark.parametrize("c", [0.0, 3.3e6, -17e6])
def test_q0_profile_is_the_lorentzian_dip(c):
    A, B = 0.7, 0.3
    m = oracle.fano_model(X, 0.0, GAMMA, [c, A, B])
    # B + A eps^2/(1+eps^2) = (A + B) - A gamma^2 / ((x-c)^2 + gamma^2)
    lor = oracle.model(X, [c, GAMMA, -A, A + B])
    assert np.max(np.abs(m - lor)) <= 1e-14


@pytest.mark.parametrize("q", [0.0, 0.3, -0.8])
def test_fano_jacobian_matches_central_differences(q):
    p = np.array([4.1e6, 0.72, 0.31])
    J = oracle.fano_jacobian(X, q, GAMMA, p)
    steps = np.array([1e2, 1e-7, 1e-7])
    for i in range(3):
        dp = np.zeros(3)
        dp[i] = steps[i]
        num = (oracle.fano_model(X, q, GAMMA, p + dp) - oracle.fano_model(X, q, GAMMA, p - dp)) / (2 * steps[i])
        scale = np.max(np.abs(J[:, i]))
        assert np.max(np.abs(num - J[:, i])) <= 1e-6 * scale, i


@pytest.mark.parametrize("q,c", [(0.0, 5.5e6), (0.3, -12.25e6), (-0.5, 31e6)])
def test_noise_free_recovery(q, c):
    A, B = 0.69, 0.305
    y = oracle.fano_model(X, q, GAMMA, [c, A, B])
    r = oracle.fano_fit_batch(y, X, q, GAMMA, 0.7, 0.3, box=0.1, converged=True)
    assert r["status"][0] == 0
    assert abs(r["params"][0, 0] - c) <= 1e-9 * GAMMA
    assert abs(r["params"][0, 1] - A) <= 1e-10
    assert abs(r["params"][0, 2] - B) <= 1e-10


def test_parameters_past_the_box_end_on_its_edge():
    q, c = 0.3, 7e6
    y = oracle.fano_model(X, q, GAMMA, [c, 0.7 * 1.3, 0.3])      # scale 30 % above its average
    r = oracle.fano_fit_batch(y, X, q, GAMMA, 0.7, 0.3, box=0.1, converged=True)
    assert r["params"][0, 1] == pytest.approx(0.7 * 1.1, abs=0.0, rel=1e-15)
    lo, hi = 0.3 * 0.9, 0.3 * 1.1
    assert lo <= r["params"][0, 2] <= hi
    # with a box wide enough the same data are recovered exactly
    r2 = oracle.fano_fit_batch(y, X, q, GAMMA, 0.7, 0.3, box=0.5, converged=True)
    assert abs(r2["params"][0, 0] - c) <= 1e-9 * GAMMA
    assert abs(r2["params"][0, 1] - 0.91) <= 1e-10


def test_lm_optimum_is_no_worse_than_brute_force():
    rng = np.random.default_rng(3)
    q, c = 0.3, 2.5e6
    x = X[35:64]                                                  # tiny: 29 teeth
    y = oracle.fano_model(x, q, GAMMA, [c, 0.71, 0.295]) + 0.003 * rng.standard_normal(x.size)
    r = oracle.fano_fit_batch(y, x, q, GAMMA, 0.7, 0.3, box=0.1, converged=True)
    p = r["params"][0]
    cg = p[0] + np.linspace(-2e5, 2e5, 41)
    Ag = np.clip(p[1] + np.linspace(-2e-3, 2e-3, 21), 0.63, 0.77)
    Bg = np.clip(p[2] + np.linspace(-2e-3, 2e-3, 21), 0.27, 0.33)
    pg, chi2g = oracle.fano_grid_fit(y, x, q, GAMMA, cg, Ag, Bg)
    assert r["rss"][0] <= chi2g * (1 + 1e-12)
    assert abs(pg[0] - p[0]) <= 1e4 and abs(pg[1] - p[1]) <= 2e-4 and abs(pg[2] - p[2]) <= 2e-4


def test_lowest_value_initial_guess():
    q = 0.25
    c = X[60] + q * GAMMA                 # the profile's minimum (eps = -q) on tooth 60
    y = oracle.fano_model(X, q, GAMMA, [c, 0.7, 0.3])
    p0 = oracle.fano_init(y, X, q, GAMMA, 0.7, 0.3)
    assert p0[0] == pytest.approx(c, abs=1e-6)
    assert (p0[1], p0[2]) == (0.7, 0.3)


def _kkt(y, x, q, p, lo, hi):
    """Normalised gradient J^T (y - m) / sqrt(diag(J^T J) chi2) at p, and which
    of A, B sit on a bound."""
    r = y - oracle.fano_model(x, q, GAMMA, p)
    J = oracle.fano_jacobian(x, q, GAMMA, p)
    g = J.T @ r / np.sqrt(np.sum(J * J, axis=0) * np.sum(r * r))
    at_lo = np.array([False, p[1] <= lo[0], p[2] <= lo[1]])
    at_hi = np.array([False, p[1] >= hi[0], p[2] >= hi[1]])
    return g, at_lo, at_hi


@pytest.mark.parametrize("fa,fb", [(1.0, 1.0), (1.3, 1.0), (1.0, 0.8), (0.8, 1.25), (1.25, 1.25)])
def test_box_constrained_optimum_satisfies_kkt(fa, fb):
    # Karush-Kuhn-Tucker conditions of min chi^2 over the box: zero gradient
    # in the free coordinates, gradient pointing out of the box on a bound
    rng = np.random.default_rng(5)
    q = 0.3
    y = oracle.fano_model(X, q, GAMMA, [3.1e6, 0.7 * fa, 0.3 * fb]) + 0.004 * rng.standard_normal(X.size)
    r = oracle.fano_fit_batch(y, X, q, GAMMA, 0.7, 0.3, box=0.1, converged=True)
    p = r["params"][0]
    g, at_lo, at_hi = _kkt(y, X, q, p, (0.63, 0.27), (0.77, 0.33))
    free = ~(at_lo | at_hi)
    assert np.all(np.abs(g[free]) <= 1e-7), g
    assert np.all(g[at_lo] <= 0.0) and np.all(g[at_hi] >= 0.0), (g, at_lo, at_hi)
    # data inside the box leave it free; data outside put a bound in play
    assert bool(np.any(at_lo | at_hi)) == ((fa, fb) != (1.0, 1.0))


@pytest.mark.parametrize("fa,fb", [(1.3, 1.0), (1.0, 0.8), (0.8, 1.25), (1.25, 1.25)])
def test_active_bounds_converge_within_the_papers_iterations(fa, fb):
    # holding a bound parameter out of the step keeps the centre's step
    # consistent; the fit settles within the paper's 20 iterations at tol 1e-6
    rng = np.random.default_rng(6)
    q = -0.5
    y = oracle.fano_model(X, q, GAMMA, [-8e6, 0.7 * fa, 0.3 * fb]) + 0.004 * rng.standard_normal(X.size)
    r20 = oracle.fano_fit_batch(y, X, q, GAMMA, 0.7, 0.3, box=0.1, max_iter=20, tol=1e-6)
    rc = oracle.fano_fit_batch(y, X, q, GAMMA, 0.7, 0.3, box=0.1, converged=True)
    assert r20["status"][0] == 0 and r20["iters"][0] <= 20
    assert abs(r20["params"][0, 0] - rc["params"][0, 0]) <= 1e-4 * 2 * GAMMA
