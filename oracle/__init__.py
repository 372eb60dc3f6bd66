"""FP64 CPU oracle for the comb-spectrum readout and Lorentzian LM fit.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline leg may use this package; the library never does.  It
shares no code with the CUDA path.  The arithmetic lives in ``cg_oracle.c``
(plain C, FP64, OpenMP over frames only); this module compiles it with gcc
on first use and marshals numpy arrays through ctypes.

Each function follows arXiv 2307.12988, "Data Capture and Processing":
cast, per-frame Fourier transform read at the comb-tooth bins, division by
the averaged reference spectrum, and a Levenberg-Marquardt fit of each
normalised spectrum (at most 20 iterations, tolerance 1e-6).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cg_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libcg_oracle.so")
_lock = threading.Lock()
_lib = None

CONVERGED, MAX_ITER, SINGULAR, NONFINITE = 0, 1, 2, 3
INIT_FLAT = 0x10

# settings of the fully converged reference fit that parity is judged against
CONVERGED_MAX_ITER = 1000
CONVERGED_TOL = 1e-15


def build(force: bool = False) -> str:
    """Compile cg_oracle.c into libcg_oracle.so beside it (gcc, -O2, OpenMP)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.c_void_p
    i32, i64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "or_tooth_bins": (i32, [f64, i32, i32, P, P]),
        "or_dft_bins": (i32, [P, i64, i32, i32, P, P, P]),
        "or_dft_bins_f64": (i32, [P, i64, i32, i32, P, P, P]),
        "or_readout": (i32, [P, i64, i32, i32, P, P, P, P]),
        "or_reference": (i32, [P, i64, i32, i32, P, P]),
        "or_readout_f64": (i32, [P, i64, i32, i32, P, P, P, P]),
        "or_reference_f64": (i32, [P, i64, i32, i32, P, P]),
        "or_model": (None, [P, i32, P, P]),
        "or_jacobian": (None, [P, i32, P, P]),
        "or_moment_init": (i32, [P, P, i32, P]),
        "or_lm_fit": (None, [P, P, i32, P, i32, f64, f64, P, P, P, P]),
        "or_fit_batch": (None, [P, i64, P, i32, P, i32, f64, f64, P, P, P, P, P]),
        "or_process": (i32, [P, i64, i32, i32, P, P, P, i32, f64, f64, P, P, P, P, P, P]),
        "or_grid_fit": (None, [P, P, i32, P, i32, P, i32, P, P]),
        "or_fano_model": (None, [P, i32, f64, f64, P, P]),
        "or_fano_jacobian": (None, [P, i32, f64, f64, P, P]),
        "or_fano_init": (None, [P, P, i32, f64, f64, f64, f64, P]),
        "or_fano_fit_batch": (None, [P, i64, P, i32, f64, f64, f64, f64, f64, P, i32, f64, f64,
                                     P, P, P, P, P]),
        "or_fano_grid_fit": (None, [P, P, i32, f64, f64, P, i32, P, i32, P, i32, P, P]),
        "or_median_filter7": (None, [P, i64, i32, P]),
        "or_median_init": (i32, [P, i64, i32, P, f64, P, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def tooth_bins(sample_rate: float, frame_len: int, tooth_freqs) -> np.ndarray:
    """Bin of each tooth: floor(|f| N / fs + 1/2), reduced mod N, folded to [0, N/2]."""
    f = _f64(tooth_freqs)
    out = np.empty(f.size, dtype=np.int32)
    rc = _load().or_tooth_bins(float(sample_rate), int(frame_len), f.size, _p(f), _p(out))
    if rc != 0:
        raise ValueError("bad geometry")
    return out


def dft_bins(frames, bins) -> tuple[np.ndarray, np.ndarray]:
    """Direct-sum DFT sum_n x_n exp(-2 pi i b n / N) of each row at the given bins.

    ``frames`` is int16 [n, N] (cast to FP64) or float64 [n, N]."""
    x = np.asarray(frames)
    if x.ndim == 1:
        x = x[None, :]
    n, N = x.shape
    b = np.ascontiguousarray(bins, dtype=np.int32)
    re = np.empty((n, b.size))
    im = np.empty((n, b.size))
    if x.dtype == np.int16:
        x = np.ascontiguousarray(x)
        rc = _load().or_dft_bins(_p(x), n, N, b.size, _p(b), _p(re), _p(im))
    else:
        x = _f64(x)
        rc = _load().or_dft_bins_f64(_p(x), n, N, b.size, _p(b), _p(re), _p(im))
    if rc != 0:
        raise MemoryError
    return re, im


def _frames(frames):
    """Integer samples (int8, int16) as int16; floating point as FP64
    (noise-free, unquantised input)."""
    x = np.asarray(frames)
    if x.ndim == 1:
        x = x[None, :]
    if np.issubdtype(x.dtype, np.integer):
        if x.dtype.itemsize > 2:
            raise TypeError("samples wider than 16 bits")
        return np.ascontiguousarray(x, dtype=np.int16), True
    return _f64(x), False


def readout(frames, bins, ref=None) -> tuple[np.ndarray, np.ndarray | None]:
    """Tooth amplitudes |X_{b_k}| and, with ``ref``, normalised y_k = amps_k / ref_k.

    ``frames`` is int16 [n, N] (the digitised samples) or float [n, N]
    (noise-free, unquantised input, read in FP64); ``ref`` is indexed by tooth."""
    x, is16 = _frames(frames)
    n, N = x.shape
    b = np.ascontiguousarray(bins, dtype=np.int32)
    T = b.size
    amps = np.empty((n, T))
    y = None
    r = None
    if ref is not None:
        r = _f64(ref)
        if r.size != T:
            raise ValueError("ref must hold one value per tooth")
        y = np.empty((n, T))
    fn = _load().or_readout if is16 else _load().or_readout_f64
    rc = fn(_p(x), n, N, T, _p(b), _p(r), _p(amps), _p(y))
    if rc != 0:
        raise MemoryError
    return amps, y


def reference(frames, bins) -> np.ndarray:
    """Averaged reference spectrum: mean over cavity-free frames of |X_{b_k}|
    (int16 frames, or float frames read in FP64)."""
    x, is16 = _frames(frames)
    n, N = x.shape
    b = np.ascontiguousarray(bins, dtype=np.int32)
    out = np.empty(b.size)
    fn = _load().or_reference if is16 else _load().or_reference_f64
    if fn(_p(x), n, N, b.size, _p(b), _p(out)) != 0:
        raise ValueError("no reference frames")
    return out


def model(x, p) -> np.ndarray:
    """m(x) = B + A g^2 / ((x-c)^2 + g^2) with p = (c, g, A, B)."""
    xa = _f64(x)
    pa = _f64(p)
    out = np.empty(xa.size)
    _load().or_model(_p(xa), xa.size, _p(pa), _p(out))
    return out


def jacobian(x, p) -> np.ndarray:
    """d m / d (c, g, A, B) at each abscissa, shape [T, 4]."""
    xa = _f64(x)
    pa = _f64(p)
    out = np.empty((xa.size, 4))
    _load().or_jacobian(_p(xa), xa.size, _p(pa), _p(out))
    return out


def moment_init(y, x) -> tuple[np.ndarray, int]:
    """Moment initial guess (c0, g0, A0, B0) and the INIT_FLAT flag (0 or 0x10)."""
    ya, xa = _f64(y), _f64(x)
    out = np.empty(4)
    flag = _load().or_moment_init(_p(ya), _p(xa), xa.size, _p(out))
    return out, int(flag)


def lm_fit(y, x, p0, max_iter=20, tol=1e-6, lambda0=1e-3):
    """One Levenberg-Marquardt fit; returns (p, rss, iters, status)."""
    ya, xa, pa = _f64(y), _f64(x), _f64(p0)
    p = np.empty(4)
    rss = ctypes.c_double()
    it = ctypes.c_int()
    st = ctypes.c_int()
    _load().or_lm_fit(_p(ya), _p(xa), xa.size, _p(pa), int(max_iter), float(tol),
                      float(lambda0), _p(p), ctypes.byref(rss), ctypes.byref(it),
                      ctypes.byref(st))
    return p, rss.value, it.value, st.value


def fit_batch(y, x, p0=None, max_iter=20, tol=1e-6, lambda0=1e-3, converged=False):
    """Fit each row of y[n, T]; ``converged`` runs the fully converged reference fit.

    Returns dict(init, params, rss, iters, status)."""
    ya = _f64(y)
    if ya.ndim == 1:
        ya = ya[None, :]
    n, T = ya.shape
    xa = _f64(x)
    if converged:
        max_iter, tol = CONVERGED_MAX_ITER, CONVERGED_TOL
    pa = None if p0 is None else _f64(p0).reshape(n, 4)
    init = np.empty((n, 4))
    params = np.empty((n, 4))
    rss = np.empty(n)
    iters = np.empty(n, dtype=np.int32)
    status = np.empty(n, dtype=np.int32)
    _load().or_fit_batch(_p(ya), n, _p(xa), T, _p(pa), int(max_iter), float(tol),
                         float(lambda0), _p(init), _p(params), _p(rss), _p(iters),
                         _p(status))
    return dict(init=init, params=params, rss=rss, iters=iters, status=status)


def process(frames, bins, ref, x, max_iter=20, tol=1e-6, lambda0=1e-3):
    """Whole path on int16 frames[n, N]: amps, y, params, rss, iters, status."""
    fr = np.ascontiguousarray(frames, dtype=np.int16)
    n, N = fr.shape
    b = np.ascontiguousarray(bins, dtype=np.int32)
    T = b.size
    r, xa = _f64(ref), _f64(x)
    amps = np.empty((n, T))
    y = np.empty((n, T))
    params = np.empty((n, 4))
    rss = np.empty(n)
    iters = np.empty(n, dtype=np.int32)
    status = np.empty(n, dtype=np.int32)
    rc = _load().or_process(_p(fr), n, N, T, _p(b), _p(r), _p(xa), int(max_iter),
                            float(tol), float(lambda0), _p(amps), _p(y), _p(params),
                            _p(rss), _p(iters), _p(status))
    if rc != 0:
        raise MemoryError
    return dict(amps=amps, y=y, params=params, rss=rss, iters=iters, status=status)


def grid_fit(y, x, cgrid, ggrid):
    """Brute-force variable projection: best (c, g) on the grid with (A, B) solved
    by linear least squares; returns (p, chi2)."""
    ya, xa = _f64(y), _f64(x)
    cg, gg = _f64(cgrid), _f64(ggrid)
    p = np.empty(4)
    chi2 = ctypes.c_double()
    _load().or_grid_fit(_p(ya), _p(xa), xa.size, _p(cg), cg.size, _p(gg), gg.size,
                        _p(p), ctypes.byref(chi2))
    return p, chi2.value


# ---------------------------------------------------------------------------
# The paper's Fano lineshape with box-constrained scale and offset
# ---------------------------------------------------------------------------
def fano_model(x, q, gamma, p) -> np.ndarray:
    """m(x) = B + A (q + e)^2 / (1 + e^2), e = (x - c) / gamma, p = (c, A, B)."""
    xa, pa = _f64(x), _f64(p)
    out = np.empty(xa.size)
    _load().or_fano_model(_p(xa), xa.size, float(q), float(gamma), _p(pa), _p(out))
    return out


def fano_jacobian(x, q, gamma, p) -> np.ndarray:
    """d m / d (c, A, B) at each abscissa, shape [T, 3]."""
    xa, pa = _f64(x), _f64(p)
    out = np.empty((xa.size, 3))
    _load().or_fano_jacobian(_p(xa), xa.size, float(q), float(gamma), _p(pa), _p(out))
    return out


def fano_init(y, x, q, gamma, A_bar, B_bar) -> np.ndarray:
    ya, xa = _f64(y), _f64(x)
    out = np.empty(3)
    _load().or_fano_init(_p(ya), _p(xa), xa.size, float(q), float(gamma), float(A_bar), float(B_bar), _p(out))
    return out


def fano_fit_batch(y, x, q, gamma, A_bar, B_bar, box=0.1, p0=None, max_iter=20, tol=1e-6, lambda0=1e-3,
                   converged=False):
    """Box-constrained LM fit of each row of y[n, T] with the Fano model:
    c free, A in A_bar (1 +- box), B in B_bar (1 +- box), q and gamma fixed.
    Returns dict(init, params [n, 3] = (c, A, B), rss, iters, status)."""
    ya = _f64(y)
    if ya.ndim == 1:
        ya = ya[None, :]
    n, T = ya.shape
    xa = _f64(x)
    if converged:
        max_iter, tol = CONVERGED_MAX_ITER, CONVERGED_TOL
    pa = None if p0 is None else _f64(p0).reshape(n, 3)
    init = np.empty((n, 3))
    params = np.empty((n, 3))
    rss = np.empty(n)
    iters = np.empty(n, dtype=np.int32)
    status = np.empty(n, dtype=np.int32)
    _load().or_fano_fit_batch(_p(ya), n, _p(xa), T, float(q), float(gamma), float(A_bar), float(B_bar),
                              float(box), _p(pa), int(max_iter), float(tol), float(lambda0), _p(init),
                              _p(params), _p(rss), _p(iters), _p(status))
    return dict(init=init, params=params, rss=rss, iters=iters, status=status)


def fano_grid_fit(y, x, q, gamma, cgrid, Agrid, Bgrid):
    """Brute force: least chi^2 over the (c, A, B) grid; returns (p, chi2)."""
    ya, xa = _f64(y), _f64(x)
    cg_, ag, bg = _f64(cgrid), _f64(Agrid), _f64(Bgrid)
    p = np.empty(3)
    chi2 = ctypes.c_double()
    _load().or_fano_grid_fit(_p(ya), _p(xa), xa.size, float(q), float(gamma), _p(cg_), cg_.size, _p(ag), ag.size,
                             _p(bg), bg.size, _p(p), ctypes.byref(chi2))
    return p, chi2.value


# ---------------------------------------------------------------------------
# The paper's initial centre: 7x7 median filter of the time x tooth image
# ---------------------------------------------------------------------------
def median_filter7(y) -> np.ndarray:
    """7x7 median filter of the image y[n, T] (rows = frames in time order),
    mirrored edges (index -1 -> 0, n -> n - 1)."""
    ya = _f64(y)
    n, T = ya.shape
    out = np.empty((n, T))
    _load().or_median_filter7(_p(ya), n, T, _p(out))
    return out


def median_init(y, x, shift=0.0) -> dict:
    """Initial centres of the rows of y[n, T]: x at the lowest value of each
    median-filtered row (first tooth on ties) plus shift.  Returns dict(c0,
    kmin, filtered)."""
    ya = _f64(y)
    n, T = ya.shape
    xa = _f64(x)
    c0 = np.empty(n)
    kmin = np.empty(n, dtype=np.int32)
    filt = np.empty((n, T))
    if _load().or_median_init(_p(ya), n, T, _p(xa), float(shift), _p(c0), _p(kmin), _p(filt)) != 0:
        raise MemoryError
    return dict(c0=c0, kmin=kmin, filtered=filt)
