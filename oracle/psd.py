"""FP64 reference of the displacement PSD and the mechanical-resonance fit
(TEST INFRASTRUCTURE ONLY).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
module; the library never imports it.

The paper turns the series of fitted cavity positions into a power spectral
density for several averaging times and fits the accelerometer's mechanical
resonance to it, reporting the frequency f0 and the quality factor Q
("Experimental Results"; Fig. 6).  Readings of what it leaves open:

* PSD: Welch's method -- segments of M samples (M a power of two) advanced by
  M/2, the segment mean removed, a periodic Hann window
  w_n = 1/2 - 1/2 cos(2 pi n / M), |rfft|^2 averaged over the K complete
  segments, one-sided density S_k = c_k mean|X_k|^2 / (fs sum w^2) with
  c_k = 2 except at k = 0 and k = M/2 (c = 1); bin k at f_k = k fs / M.
* Resonance model: a damped harmonic oscillator driven by white force noise
  over a white floor,
      S(f) = A f0^4 / ((f0^2 - f^2)^2 + (f f0 / Q)^2) + B,
  so that S(0) = A + B and S(f0) = A Q^2 + B.
* Fit: Levenberg-Marquardt (as or_lm_fit: solve (H + lambda diag H) d = J^T r,
  lambda0 1e-3, /10 on a lower chi^2, *10 otherwise) on the residuals
  ln S_k - ln S(f_k) over the bins of a band [f_lo, f_hi]: the log makes each
  bin's relative error count alike (a Welch estimate's relative error is the
  same at every bin).  Initial values from the band: f0 at the largest bin,
  B the smallest bin, Q = f0 / (width at half the peak above B), A from the
  peak height.  Standard errors: sqrt(diag(H^-1) chi^2 / (n - 4)).

Pinned by: SciPy's Welch estimate with the same settings, Parseval's
theorem, the closed-form peak of a sinusoid; the model's closed-form values
and its Jacobian by central differences; noise-free recovery; MINPACK's LM
(scipy.optimize.least_squares) on the same residuals.
"""
from __future__ import annotations

import numpy as np


def hann(M: int) -> np.ndarray:
    """Periodic Hann window of M samples."""
    n = np.arange(M)
    return 0.5 - 0.5 * np.cos(2.0 * np.pi * n / M)


def welch(x, fs: float, M: int):
    """One-sided Welch PSD of x: returns (f [M/2+1], S [M/2+1], K segments)."""
    x = np.asarray(x, dtype=np.float64)
    hop = M // 2
    K = 0 if x.size < M else (x.size - M) // hop + 1
    if K == 0:
        raise ValueError("series shorter than one segment")
    w = hann(M)
    acc = np.zeros(M // 2 + 1)
    for s in range(K):
        seg = x[s * hop:s * hop + M]
        X = np.fft.rfft((seg - seg.mean()) * w)
        acc += X.real ** 2 + X.imag ** 2
    c = np.full(M // 2 + 1, 2.0)
    c[0] = 1.0
    c[-1] = 1.0
    S = c * acc / K / (fs * np.sum(w * w))
    return np.arange(M // 2 + 1) * fs / M, S, K


def model(f, p) -> np.ndarray:
    f0, Q, A, B = p
    f = np.asarray(f, dtype=np.float64)
    D = (f0 * f0 - f * f) ** 2 + (f * f0 / Q) ** 2
    return A * f0 ** 4 / D + B


def jacobian(f, p) -> np.ndarray:
    """d model / d (f0, Q, A, B), shape [n, 4]."""
    f0, Q, A, B = p
    f = np.asarray(f, dtype=np.float64)
    u = f0 * f0 - f * f
    D = u * u + (f * f0 / Q) ** 2
    g = f0 ** 4 / D
    dD_df0 = 4.0 * f0 * u + 2.0 * f * f * f0 / (Q * Q)
    dD_dQ = -2.0 * (f * f0) ** 2 / Q ** 3
    J = np.empty((f.size, 4))
    J[:, 0] = A * (4.0 * f0 ** 3 / D - f0 ** 4 * dD_df0 / (D * D))
    J[:, 1] = -A * f0 ** 4 * dD_dQ / (D * D)
    J[:, 2] = g
    J[:, 3] = 1.0
    return J


def init(f, S) -> np.ndarray:
    """Initial (f0, Q, A, B) from the band's bins (see the module notes)."""
    f = np.asarray(f, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    kp = int(np.argmax(S))
    B = float(np.min(S))
    h = S[kp] - B
    half = B + 0.5 * h
    # half-height crossings on either side, linearly interpolated
    lo = kp
    while lo > 0 and S[lo - 1] > half:
        lo -= 1
    hi = kp
    while hi < S.size - 1 and S[hi + 1] > half:
        hi += 1
    fl = f[lo] if lo == 0 else f[lo - 1] + (half - S[lo - 1]) / (S[lo] - S[lo - 1]) * (f[lo] - f[lo - 1])
    fh = f[hi] if hi == S.size - 1 else f[hi] + (S[hi] - half) / (S[hi] - S[hi + 1]) * (f[hi + 1] - f[hi])
    width = max(fh - fl, f[1] - f[0])
    f0 = f[kp]
    Q = f0 / width
    return np.array([f0, Q, h / (Q * Q), B])


def _solve(H, lam, g):
    d = np.sqrt(np.diag(H))
    if not np.all(d > 0) or not np.all(np.isfinite(d)):
        return None
    Ms = H / np.outer(d, d)
    Ms[np.diag_indices(4)] = 1.0 + lam
    try:
        L = np.linalg.cholesky(Ms)
    except np.linalg.LinAlgError:
        return None
    z = np.linalg.solve(L, g / d)
    return np.linalg.solve(L.T, z) / d


def fit(f, S, p0=None, max_iter=200, tol=1e-12, lambda0=1e-3) -> dict:
    """LM fit of ln S by ln model over the given bins.  Returns dict(params,
    sigma, rss, iters, status) with status 0 converged, 1 iteration limit,
    2 singular, 3 non-finite."""
    f = np.asarray(f, dtype=np.float64)
    y = np.log(np.asarray(S, dtype=np.float64))
    p = init(f, S) if p0 is None else np.asarray(p0, dtype=np.float64).copy()

    def evaluate(q):
        m = model(f, q)
        if not np.all(m > 0):
            return np.inf, None, None
        r = y - np.log(m)
        J = jacobian(f, q) / m[:, None]
        return float(r @ r), J.T @ J, J.T @ r

    lam = lambda0
    chi2, H, g = evaluate(p)
    it, st = 0, 1
    if not np.isfinite(chi2):
        st = 3
    else:
        while it < max_iter:
            it += 1
            d = _solve(H, lam, g)
            if d is None:
                st = 2
                break
            pt = p + d
            c2, Ht, gt = evaluate(pt)
            if not np.isfinite(c2):
                lam *= 10.0
                continue
            if abs(c2 - chi2) <= tol * chi2:
                if c2 <= chi2:
                    p, chi2 = pt, c2
                st = 0
                break
            if c2 < chi2:
                p, chi2, H, g = pt, c2, Ht, gt
                lam *= 0.1
            else:
                lam *= 10.0
    _, H, _ = evaluate(p)
    sigma = np.full(4, np.nan)
    if H is not None and f.size > 4:
        try:
            sigma = np.sqrt(np.diag(np.linalg.inv(H)) * chi2 / (f.size - 4))
        except np.linalg.LinAlgError:
            pass
    return dict(params=p, sigma=sigma, rss=chi2, iters=it, status=st)


def band(f, S, f_lo, f_hi):
    """The bins with f_lo <= f_k <= f_hi."""
    f = np.asarray(f)
    sel = (f >= f_lo) & (f <= f_hi)
    return f[sel], np.asarray(S)[sel]
