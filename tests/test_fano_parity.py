"""Fano lineshape fit (GPU) against the FP64 oracle.

The paper fits each spectrum with a Fano profile whose centre is free, whose
scale and offset stay within about +-10 % of pre-computed averages and whose
asymmetry and width are fixed ("Data Capture and Processing").  Frames are
synthesised with that profile (per-frame depth spread, 30 dB SNR) at the
paper-rate geometry; the oracle reads them out in FP64 and runs its
box-constrained LM to convergence.  Bars: converged centres within 1e-4 of
the linewidth; scale and offset within 1e-4 (their box edges reached on the
same frames); the q = 0 case; a scale pushed past the box; ragged, empty
and single-frame batches; lane counts; the FP64 solve and the tensor-core
readout; cg_fit on given spectra; refused
options.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import workloads as W

torch = pytest.importorskip("torch")
cg = pytest.importorskip("paper_2307_12988_gb300")

pytestmark = pytest.mark.gpu

G = synth.PAPER_RATE
GAMMA = synth.FWHM_HZ / 2.0
CENTER_TOL = 1e-4 * synth.FWHM_HZ
AB_TOL = 1e-4
A_BAR, B_BAR = 0.7, 0.3
N_FRAMES = 3000


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _workload(q, depth_scale=1.0, n=N_FRAMES, seed_off=700):
    """Fano frames with per-frame depth 0.7 (1 + 0.03 N(0, 1)) x depth_scale."""
    stream = synth.make_stream(G, synth.BASE_SEED + seed_off)
    rng = np.random.default_rng(synth.BASE_SEED + seed_off)
    depth = A_BAR * depth_scale * (1.0 + 0.03 * rng.standard_normal(n))
    fr = synth.frames(stream, n, snr_db=30.0, center_amp_hz=20e6, shape="fano", fano_q=q, depth=depth)
    rf = synth.frames(stream, 1000, cavity=False, noise_stream=1, snr_db=30.0)
    bins = oracle.tooth_bins(G.sample_rate, G.frame_len, G.tooth_freqs)
    ref = oracle.reference(rf["frames"], bins)
    o = oracle.process(fr["frames"], bins, ref, G.tooth_x)
    return dict(frames=fr["frames"], ref=ref, y=o["y"], q=q)


_CACHE = {}


def _w(q, depth_scale=1.0):
    key = (q, depth_scale)
    if key not in _CACHE:
        _CACHE[key] = _workload(q, depth_scale)
    return _CACHE[key]


def _plan(w, box=0.1, **opts):
    return cg.Plan(G.sample_rate, G.frame_len, G.tooth_freqs, G.tooth_x, w["ref"], model=cg.MODEL_FANO,
                   fano_q=w["q"], fano_gamma=GAMMA, fano_A=A_BAR, fano_B=B_BAR, fano_box=box, **opts)


def _oracle_fit(w, box=0.1, a=0, b=None, max_iter=20, tol=1e-6, y=None):
    """The oracle's converged box optimum, with its run capped like the GPU's
    (``max_iter``, ``tol``) under "capped"."""
    y = w["y"][a:b] if y is None else y
    conv = oracle.fano_fit_batch(y, G.tooth_x, w["q"], GAMMA, A_BAR, B_BAR, box=box, converged=True)
    conv["capped"] = oracle.fano_fit_batch(y, G.tooth_x, w["q"], GAMMA, A_BAR, B_BAR, box=box,
                                           max_iter=max_iter, tol=tol)
    return conv


def _compare(o, ref, label, box=0.1):
    # every frame judged: status as the oracle's capped run, centre against
    # the converged optimum (or, unconverged, the capped result)
    st = o["status"]
    ok = W.judge_fit(o["params"], st, ref["capped"], ref, CENTER_TOL, label)
    pr, rp = o["params"], ref["params"]
    dc = np.abs(pr[ok, 0] - rp[ok, 0])
    dA = np.abs(pr[ok, 2] - rp[ok, 1])
    dB = np.abs(pr[ok, 3] - rp[ok, 2])
    print(f"\n[{label}] centre err max {dc.max():.1f} Hz, A err {dA.max():.2e}, B err {dB.max():.2e}, "
          f"mean iters {o['iters'].mean():.2f}, converged {np.mean((st & 3) == 0):.4f}")
    assert np.all(dc <= CENTER_TOL)
    assert np.all(dA <= AB_TOL) and np.all(dB <= AB_TOL)
    assert np.all(pr[ok, 1] == np.float32(GAMMA))
    # every fitted scale and offset lies in its box (the float32 bounds)
    lo_a, hi_a = np.float32(A_BAR * (1 - box)), np.float32(A_BAR * (1 + box))
    lo_b, hi_b = np.float32(B_BAR * (1 - box)), np.float32(B_BAR * (1 + box))
    assert np.all((pr[:, 2] >= lo_a) & (pr[:, 2] <= hi_a))
    assert np.all((pr[:, 3] >= lo_b) & (pr[:, 3] <= hi_b))
    return ok


def _process(p, w, dev, a=0, b=None):
    fr = torch.from_numpy(w["frames"][a:b]).to(dev)
    out = p.process(fr)
    cg.cg_check_device(p.handle)
    return {k: v.cpu().numpy() for k, v in out.items() if v is not None}


@pytest.mark.parametrize("q", [0.3, -0.5])
def test_fano_process_parity(dev, q):
    w = _w(q)
    with _plan(w) as p:
        assert p.info["path"] == cg.PATH_PIPELINE
        o = _process(p, w, dev)
    _compare(o, _oracle_fit(w), f"fano q={q}")


def test_fano_q0_is_the_lorentzian_dip(dev):
    # q = 0: B + A e^2 / (1 + e^2) = (A + B) - A g^2 / ((x - c)^2 + g^2)
    w = _w(0.0)
    with _plan(w) as p:
        o = _process(p, w, dev)
    _compare(o, _oracle_fit(w), "fano q=0")
    # the same centres as the oracle's Lorentzian fit with the width fixed
    # only to within the noise (not the same estimator), so no tighter bar
    lor = oracle.fit_batch(w["y"], G.tooth_x, converged=True)
    ok = (lor["status"] == 0) & ((o["status"] & 3) == 0)
    assert np.median(np.abs(o["params"][ok, 0] - lor["params"][ok, 0])) <= 0.01 * synth.FWHM_HZ


def test_fano_laser_power_past_the_box(dev):
    # a laser-power step: every spectrum 12 % brighter than the reference
    # (A and B 12 % above their averages, past the +-10 % box); both sides
    # run to a tight tolerance so that they meet at the box optimum
    w0 = _w(0.3)
    bins = oracle.tooth_bins(G.sample_rate, G.frame_len, G.tooth_freqs)
    ref = w0["ref"] / 1.12
    w = dict(w0, ref=ref, y=oracle.process(w0["frames"], bins, ref, G.tooth_x)["y"])
    with _plan(w, max_iter=200, tol=1e-10) as p:
        o = _process(p, w, dev)
    rf = _oracle_fit(w, max_iter=200, tol=1e-10)
    ok = _compare(o, rf, "fano laser power +12 %")
    # parameters on a bound in the oracle sit on the same float32 bound
    bounds = {1: (A_BAR * 0.9, A_BAR * 1.1, 2), 2: (B_BAR * 0.9, B_BAR * 1.1, 3)}
    n_on = np.zeros(len(ok), dtype=bool)
    for i, (lo, hi, col) in bounds.items():
        for edge in (lo, hi):
            on = np.abs(rf["params"][:, i] - edge) <= 1e-12 * edge
            n_on |= on
            assert np.all(o["params"][ok & on, col] == np.float32(edge)), (i, edge)
    assert n_on.mean() >= 0.9
    # a box wide enough frees them again
    with _plan(w, box=0.5) as p:
        o2 = _process(p, w, dev)
    _compare(o2, _oracle_fit(w, box=0.5), "fano laser power, box 0.5", box=0.5)


@pytest.mark.parametrize("lanes", [2, 4, 8])
def test_fano_lanes_per_frame(dev, lanes):
    w = _w(0.3)
    with _plan(w, lanes_per_frame=lanes) as p:
        assert p.info["lanes_per_frame"] == lanes
        o = _process(p, w, dev, 0, 1000)
    _compare(o, _oracle_fit(w, a=0, b=1000), f"fano lanes={lanes}")


def test_fano_ragged_single_and_empty(dev):
    w = _w(0.3)
    ref = _oracle_fit(w)
    with _plan(w) as p:
        for a, b in [(0, 1), (7, 8), (5, 262), (1001, 1514)]:
            o = _process(p, w, dev, a, b)
            sub = {k: v[a:b] for k, v in ref.items() if k != "capped"}
            sub["capped"] = {k: v[a:b] for k, v in ref["capped"].items()}
            _compare_small(o, sub)
        out = p.process(torch.from_numpy(w["frames"][:0]).to(dev))
        assert out["params"].shape == (0, 4)


def _compare_small(o, ref):
    ok = W.judge_fit(o["params"], o["status"], ref["capped"], ref, CENTER_TOL, "fano ragged")
    assert np.all(np.abs(o["params"][ok, 0] - ref["params"][ok, 0]) <= CENTER_TOL)
    assert np.all(np.abs(o["params"][ok, 2] - ref["params"][ok, 1]) <= AB_TOL)


def test_fano_cg_fit_on_given_spectra(dev):
    w = _w(-0.5)
    y = torch.from_numpy(w["y"][:1500].astype(np.float32)).to(dev)
    n = y.shape[0]
    with _plan(w) as p:
        params = torch.empty((n, 4), dtype=torch.float32, device=dev)
        rss = torch.empty(n, dtype=torch.float32, device=dev)
        iters = torch.empty(n, dtype=torch.int16, device=dev)
        status = torch.empty(n, dtype=torch.int16, device=dev)
        cg.cg_fit(p.handle, y, n, None, params, rss, iters, status, None)
        torch.cuda.synchronize()
        cg.cg_check_device(p.handle)
    o = dict(params=params.cpu().numpy(), status=status.cpu().numpy(), iters=iters.cpu().numpy())
    # the oracle on the same float32 spectra
    ref = _oracle_fit(w, y=w["y"][:1500].astype(np.float32))
    _compare(o, ref, "fano cg_fit")


def test_fano_refused_options(dev):
    w = _w(0.3)
    with pytest.raises(cg.CgError, match="CG_ERR_ARG"):
        cg.Plan(G.sample_rate, G.frame_len, G.tooth_freqs, G.tooth_x, w["ref"], model=cg.MODEL_FANO,
                fano_q=0.3, fano_gamma=0.0, fano_A=A_BAR, fano_B=B_BAR)
    with pytest.raises(cg.CgError, match="CG_ERR_ARG"):
        cg.Plan(G.sample_rate, G.frame_len, G.tooth_freqs, G.tooth_x, w["ref"], model=cg.MODEL_FANO,
                fano_q=0.3, fano_gamma=GAMMA, fano_A=0.0, fano_B=B_BAR)
    with pytest.raises(cg.CgError, match="CG_ERR_ARG"):
        cg.Plan(G.sample_rate, G.frame_len, G.tooth_freqs, G.tooth_x, w["ref"], model=7)
    with pytest.raises(cg.CgError, match="CG_ERR_UNSUPPORTED"):
        cg.Plan(G.sample_rate, G.frame_len, G.tooth_freqs, G.tooth_x, w["ref"], model=cg.MODEL_FANO,
                fano_q=0.3, fano_gamma=GAMMA, fano_A=A_BAR, fano_B=B_BAR, init=cg.INIT_MLP)
    with pytest.raises(cg.CgError, match="CG_ERR_UNSUPPORTED"):
        _plan(w, lanes_per_frame=32)


@pytest.mark.parametrize("opts", [dict(solve_f64=1), dict(readout=cg.READOUT_GEMM_SPLIT, sample_bits=12)])
def test_fano_fp64_solve_and_tensor_core_readout(dev, opts):
    # the FP64 3x3 solve (the GEMM readout's default) on one lane of the group
    w = _w(-0.5)
    with _plan(w, **opts) as p:
        o = _process(p, w, dev, 0, 1000)
    _compare(o, _oracle_fit(w, a=0, b=1000), f"fano {sorted(opts)}")
