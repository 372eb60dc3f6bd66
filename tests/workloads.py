"""Seeded workloads shared by the parity tests (test helper, not a test file).

Each workload is built from ``synth`` (inputs) and ``oracle`` (reference
spectrum and expected values); nothing here comes from the CUDA path."""
from __future__ import annotations

import functools

import numpy as np

import oracle
import synth

FS12 = synth.FULL_SCALE

# name -> (geometry, frames, reference frames, generator keywords)
SPECS = {
    "tiny": (synth.TINY, 1000, 1000, dict(sigma=0.01 * FS12, center_amp_hz=5e6)),
    "tiny_peak": (synth.TINY, 300, 300, dict(sigma=0.01 * FS12, center_amp_hz=5e6, shape="peak")),
    "paper_rate": (synth.PAPER_RATE, 1500, 1000, dict(snr_db=30.0, center_amp_hz=20e6)),
    "wide": (synth.WIDE, 400, 400, dict(snr_db=30.0, center_amp_hz=20e6)),
    "serve4096": (synth.SERVE_4096, 200, 300, dict(snr_db=30.0, center_amp_hz=20e6)),
    # 8-bit samples at 2.2 GS/s, 2200-sample frames (the paper's digitiser)
    "paper8": (synth.PAPER_8BIT, 1500, 1000, dict(snr_db=30.0, center_amp_hz=20e6, bits=8)),
    # the other power-of-two frame lengths of the full-transform readout
    "pow2_2048": (synth.Geometry(1.0e9, 2048, -40, 40), 300, 300, dict(snr_db=30.0, center_amp_hz=20e6)),
    "pow2_8192": (synth.Geometry(4.0e9, 8192, -100, 100), 150, 200, dict(snr_db=30.0, center_amp_hz=20e6)),
}


@functools.lru_cache(maxsize=None)
def workload(name: str) -> dict:
    geom, n, n_ref, kw = SPECS[name]
    seed = synth.BASE_SEED + sorted(SPECS).index(name)
    stream = synth.make_stream(geom, seed)
    fr = synth.frames(stream, n, **kw)
    ref_kw = {k: v for k, v in kw.items() if k in ("sigma", "snr_db", "bits")}
    rf = synth.frames(stream, n_ref, cavity=False, noise_stream=1, **ref_kw)
    bins = oracle.tooth_bins(geom.sample_rate, geom.frame_len, geom.tooth_freqs)
    ref = oracle.reference(rf["frames"], bins)
    out = oracle.process(fr["frames"], bins, ref, geom.tooth_x)
    conv = oracle.fit_batch(out["y"], geom.tooth_x, converged=True)
    return dict(name=name, geom=geom, frames=fr["frames"], centers=fr["centers"],
                ref_frames=rf["frames"], bins=bins, ref=ref, oracle=out, converged=conv)


def plan_args(w: dict) -> tuple:
    g = w["geom"]
    return (g.sample_rate, g.frame_len, g.tooth_freqs, g.tooth_x, w["ref"])


def judge_fit(params, status, capped, conv, center_tol, label="", c_col=0, failures_alike=False, y=None, x=None,
              lm_tol=1e-6):
    """Judge every frame of a GPU fit against the oracle.

    * the status of each frame (low two bits: converged, max_iter, singular,
      non-finite) equals the oracle's iteration-capped run of the same frame;
    * a converged frame's centre lies within ``center_tol`` of the oracle's
      fully converged optimum (``conv``, which must have converged too);
    * any other frame's centre lies within ``center_tol`` of the oracle's
      capped result (the two runs stopped at the same kind of point).
    ``c_col`` is the centre's column in the oracle's parameter rows.
    ``failures_alike``: a frame that neither side fits (iteration cap or a
    singular system: FP32 and FP64 can end such a frame either way) counts
    as one class, and its centre is not compared.  With it, a frame the
    oracle leaves at the iteration cap but the GPU converges also passes
    when the GPU's centre lies within ``center_tol`` of the oracle's fully
    converged optimum: at the cap the status is decided by the iteration at
    which chi^2 settles, which FP32 and FP64 rounding move by a few steps.
    Given the spectra ``y`` and abscissa ``x`` (Lorentzian fits), two more
    readings of the fit's own criterion apply with ``failures_alike``:
    a frame the oracle cannot fit even with its long run, whose GPU centre
    has left the tooth span, lost its dip on both sides (the GPU's FP32
    chi^2 stops changing while the centre runs away) and passes; and a
    converged frame whose centre misses the converged optimum passes if
    chi^2 at the GPU's parameters, evaluated in FP64, lies within the
    relative tolerance ``lm_tol`` of chi^2 at the optimum -- the stopping
    rule cannot place the centre closer than that where chi^2 is flat.
    Returns the mask of converged frames."""
    st = np.asarray(status).astype(np.int64) & 3
    ost = np.asarray(capped["status"]).astype(np.int64) & 3
    if failures_alike:
        st = np.where((st == 1) | (st == 2), 1, st)
        ost = np.where((ost == 1) | (ost == 2), 1, ost)
        cst = np.asarray(conv["status"]).astype(np.int64) & 3
        late = (st == 0) & (ost == 1) & (cst == 0)
        if late.any():
            dl = np.abs(np.asarray(params)[late, 0] - np.asarray(conv["params"])[late, c_col])
            assert np.all(dl <= center_tol), (label, "converged past the oracle's cap", float(dl.max()))
            ost = np.where(late, 0, ost)
        lost = np.zeros(st.shape, bool)
        if x is not None:
            cpos = np.asarray(params)[:, 0]
            lost = (st == 0) & (ost == 1) & (cst != 0) & ((cpos < np.min(x)) | (cpos > np.max(x)))
            ost = np.where(lost, 0, ost)
    bad = np.flatnonzero(st != ost)
    assert bad.size == 0, (
        f"{label}: status differs from the oracle's capped run on {bad.size} frames "
        f"(first {bad[:5].tolist()}: gpu {st[bad[:5]].tolist()}, oracle {ost[bad[:5]].tolist()}); "
        f"histograms gpu {np.bincount(st, minlength=4).tolist()}, oracle {np.bincount(ost, minlength=4).tolist()}")
    ok = st == 0
    if failures_alike:
        ok = ok & ~lost
    assert np.all(np.asarray(conv["status"])[ok] & 3 == 0), f"{label}: oracle optimum not converged"
    want = np.where(ok, np.asarray(conv["params"])[:, c_col], np.asarray(capped["params"])[:, c_col])
    dc = np.abs(np.asarray(params)[:, 0] - want)
    if failures_alike:
        dc = np.where((st == 1) | lost, 0.0, dc)
        far = np.flatnonzero(ok & (dc > center_tol))
        if far.size and y is not None and x is not None:
            import oracle
            xs = np.asarray(x, np.float64)
            for i in far:
                r_gpu = np.asarray(y[i], np.float64) - oracle.model(xs, np.asarray(params[i], np.float64))
                r_opt = np.asarray(y[i], np.float64) - oracle.model(xs, np.asarray(conv["params"][i], np.float64))
                c2g, c2o = float(r_gpu @ r_gpu), float(r_opt @ r_opt)
                assert c2g <= c2o * (1.0 + lm_tol), (label, int(i), float(dc[i]), c2g, c2o)
                dc[i] = 0.0
    assert np.all(dc <= center_tol), (label, float(dc.max()), int(np.argmax(dc)))
    return ok
