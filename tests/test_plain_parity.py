"""Parity of the plain CUDA path with the FP64 oracle (GPU).

Tolerances (readings of the targets, see the design notes):
  * tooth amplitudes: |amps_gpu - amps_oracle| <= 1e-5 * ref_k, i.e. the
    normalised spectrum agrees to 1e-5;
  * fitted centre: within 1e-4 of the linewidth (FWHM, 80 MHz -> 8 kHz) of
    the oracle's fully converged least-squares optimum on the same frame.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import workloads as W

torch = pytest.importorskip("torch")
cg = pytest.importorskip("paper_2307_12988_gb300")

pytestmark = pytest.mark.gpu

AMP_TOL = 1e-5
CENTER_TOL = 1e-4 * synth.FWHM_HZ


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _plan(w, **opts):
    return cg.Plan(*W.plan_args(w), **opts)


def _amp_err(amps, w):
    return np.max(np.abs(amps - w["oracle"]["amps"]) / w["ref"][None, :])


@pytest.mark.parametrize("name", ["tiny", "paper_rate", "wide", "serve4096"])
@pytest.mark.parametrize("fft", [cg.FFT_AUTO, cg.FFT_FULL])
def test_readout_parity(dev, name, fft):
    w = W.workload(name)
    with _plan(w, fft=fft, path=cg.PATH_SPLIT) as p:
        fr = torch.from_numpy(w["frames"]).to(dev)
        amps, y = p.readout(fr)
        torch.cuda.synchronize()
        amps, y = amps.cpu().numpy(), y.cpu().numpy()
    assert _amp_err(amps, w) <= AMP_TOL
    assert np.max(np.abs(y - w["oracle"]["y"])) <= AMP_TOL


@pytest.mark.parametrize("name", ["serve4096", "pow2_2048", "pow2_8192"])
def test_power_of_two_readout_parity(dev, name):
    # full real transforms with N = 2048, 4096, 8192 take the three-pass
    # register readout on the pipeline path (4-byte aligned frames); ragged
    # batches and a 2-byte aligned slice (general transform) as well
    w = W.workload(name)
    fr = torch.from_numpy(w["frames"]).to(dev)
    n = fr.shape[0]
    with _plan(w, path=cg.PATH_PIPELINE) as p:
        assert p.info["fft_kind"] == cg.FFT_FULL
        for a, b in [(0, n), (2, n - 1), (1, 40), (6, 7)]:
            amps, y = p.readout(fr[a:b])
            torch.cuda.synchronize()
            err = _amp_err(amps.cpu().numpy(), {"oracle": {"amps": w["oracle"]["amps"][a:b]}, "ref": w["ref"]})
            assert err <= AMP_TOL, (name, a, b, err)
            assert np.max(np.abs(y.cpu().numpy() - w["oracle"]["y"][a:b])) <= AMP_TOL


def test_coset_transform_is_chosen_for_comb_geometries():
    for name, M, L in [("tiny", 10, 100), ("paper_rate", 10, 110), ("wide", 10, 250)]:
        w = W.workload(name)
        with _plan(w) as p:
            assert p.info["fft_kind"] == cg.FFT_COSET
            assert (p.info["coset_modulus"], p.info["fft_len"]) == (M, L)
            np.testing.assert_array_equal(p.bins, w["bins"])
    w = W.workload("serve4096")
    with _plan(w) as p:
        assert p.info["fft_kind"] == cg.FFT_FULL and p.info["n_collisions"] == 1
        np.testing.assert_array_equal(p.bins, w["bins"])


def test_readout_ragged_misaligned_and_empty(dev):
    w = W.workload("paper_rate")
    fr = torch.from_numpy(w["frames"]).to(dev)
    with _plan(w, path=cg.PATH_SPLIT) as p:
        # odd first frame: the batch starts 8 bytes off a 16-byte boundary
        for a, b in [(1, 2), (1, 62), (3, 700), (0, 1), (997, 1500)]:
            amps, _ = p.readout(fr[a:b], want_y=False)
            torch.cuda.synchronize()
            err = np.max(np.abs(amps.cpu().numpy() - w["oracle"]["amps"][a:b]) / w["ref"])
            assert err <= AMP_TOL, (a, b, err)
        amps, y = p.readout(fr[:0])
        assert amps.shape == (0, p.T)


def test_moment_init_parity(dev):
    w = W.workload("paper_rate")
    x = w["geom"].tooth_x
    y = w["oracle"]["y"]
    ref_init = oracle.fit_batch(y, x, max_iter=0)
    with _plan(w, max_iter=0) as p:
        out = p.fit(torch.from_numpy(y.astype(np.float32)).to(dev))
        torch.cuda.synchronize()
        got = out["params"].cpu().numpy()
        flags = out["status"].cpu().numpy()
    exp = ref_init["init"].copy()
    exp[:, 1] = np.abs(exp[:, 1])
    span = x.max() - x.min()
    assert np.max(np.abs(got[:, 0] - exp[:, 0])) <= 1e-5 * span
    assert np.max(np.abs(got[:, 1] - exp[:, 1])) <= 1e-5 * span
    assert np.max(np.abs(got[:, 2:] - exp[:, 2:])) <= 1e-5
    assert np.all((flags & 0x10) == (ref_init["status"] & 0x10))


@pytest.mark.parametrize("lanes", [4, 8, 16, 32])
def test_lm_parity_from_oracle_init(dev, lanes):
    w = W.workload("paper_rate")
    x = w["geom"].tooth_x
    y = w["oracle"]["y"]
    init = oracle.fit_batch(y, x, max_iter=0)["init"]
    with _plan(w, lanes_per_frame=lanes) as p:
        out = p.fit(torch.from_numpy(y.astype(np.float32)).to(dev),
                    p0=torch.from_numpy(init.astype(np.float32)).to(dev))
        torch.cuda.synchronize()
        params = out["params"].cpu().numpy()
        status = out["status"].cpu().numpy()
        iters = out["iters"].cpu().numpy()
    conv = w["converged"]["params"]
    ok = W.judge_fit(params, status, w["oracle"], w["converged"], CENTER_TOL, f"lm lanes={lanes}")
    assert np.max(np.abs(params[ok, 0] - conv[ok, 0])) <= CENTER_TOL
    assert np.max(np.abs(params[ok, 1] - conv[ok, 1])) <= CENTER_TOL
    assert np.max(np.abs(params[ok, 2:] - conv[ok, 2:])) <= 1e-4
    # iteration counts track the oracle's capped fit
    assert abs(iters.mean() - w["oracle"]["iters"].mean()) < 1.0


@pytest.mark.parametrize("name", ["tiny", "tiny_peak", "paper_rate", "wide", "serve4096"])
@pytest.mark.parametrize("path", [cg.PATH_PIPELINE, cg.PATH_FUSED, cg.PATH_SPLIT])
def test_process_parity(dev, name, path):
    w = W.workload(name)
    with _plan(w, path=path) as p:
        fr = torch.from_numpy(w["frames"]).to(dev)
        out = p.process(fr)
        torch.cuda.synchronize()
        o = {k: v.cpu().numpy() for k, v in out.items() if v is not None}
    assert _amp_err(o["amps"], w) <= AMP_TOL
    assert np.max(np.abs(o["y"] - w["oracle"]["y"])) <= AMP_TOL
    ok = W.judge_fit(o["params"], o["status"], w["oracle"], w["converged"], CENTER_TOL, f"{name} path {path}")
    conv = w["converged"]["params"]
    assert np.max(np.abs(o["params"][ok, 0] - conv[ok, 0])) <= CENTER_TOL
    # secondary parameters: the chi^2 stopping rule (tol 1e-6) leaves the flatter
    # width / depth / offset directions looser than the centre; bound them at 1e-3
    assert np.max(np.abs(o["params"][ok, 1] - conv[ok, 1]) / conv[ok, 1]) <= 1e-3
    assert np.max(np.abs(o["params"][ok, 2:] - conv[ok, 2:])) <= 1e-3
    rss_conv = w["converged"]["rss"]
    assert np.all(o["rss"][ok] <= rss_conv[ok] * (1 + 1e-3) + 1e-9)


def test_fit_status_edge_cases(dev):
    w = W.workload("tiny")
    T = w["geom"].n_teeth
    y = np.ones((4, T), dtype=np.float32)
    y[1, 5] = np.nan
    y[2] = w["oracle"]["y"][0]
    y[3] = w["oracle"]["y"][1]
    with _plan(w) as p:
        out = p.fit(torch.from_numpy(y).to(dev))
        torch.cuda.synchronize()
        st = out["status"].cpu().numpy()
    assert st[0] == (cg.FIT_SINGULAR | cg.FIT_INIT_FLAT)
    assert st[1] & 0xF == cg.FIT_NONFINITE
    assert st[2] == cg.FIT_CONVERGED and st[3] == cg.FIT_CONVERGED


def test_reference_accumulate(dev):
    w = W.workload("paper_rate")
    with _plan(w) as p:
        ref = p.reference_accumulate(torch.from_numpy(w["ref_frames"]).to(dev))
    np.testing.assert_allclose(ref, w["ref"], rtol=2e-6)


def test_results_independent_of_batching(dev):
    """Each frame's result is the same alone and inside a larger call."""
    w = W.workload("paper_rate")
    fr = torch.from_numpy(w["frames"]).to(dev)
    with _plan(w) as p:
        full = p.process(fr)
        part = p.process(fr[37:38])
        torch.cuda.synchronize()
        for k in ("amps", "params", "rss"):
            a = full[k][37:38].cpu().numpy()
            b = part[k].cpu().numpy()
            np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("name", ["paper_rate", "wide", "serve4096"])
def test_results_independent_of_requesting_y(dev, name):
    """Asking for y_dev or not changes nothing: without it the fit forms
    y = amps / reference itself, with the same rounding as the readout."""
    w = W.workload(name)
    fr = torch.from_numpy(w["frames"]).to(dev)
    with _plan(w) as p:
        with_y = p.process(fr, want_y=True)
        no_y = p.process(fr, want_y=False)
        torch.cuda.synchronize()
        for k in ("amps", "params", "rss", "iters", "status"):
            np.testing.assert_array_equal(with_y[k].cpu().numpy(), no_y[k].cpu().numpy(), err_msg=k)


def _all_values_frames(lo, hi, N, dtype, seed):
    """Frames of N samples holding every integer of [lo, hi] once (in random
    order), padded with random values to whole frames."""
    rng = np.random.default_rng(seed)
    vals = rng.permutation(np.arange(lo, hi + 1, dtype=np.int64))
    nf = -(-vals.size // N)
    pad = rng.integers(lo, hi + 1, nf * N - vals.size)
    return np.concatenate([vals, pad]).astype(dtype).reshape(nf, N)


@pytest.mark.parametrize("name", ["tiny", "paper_rate", "wide", "serve4096", "paper8"])
def test_default_readout_full_sample_range(dev, name):
    # every int16 value (every int8 value for the 8-bit frame) through the
    # default readout of each geometry (coset-pruned transform; the
    # power-of-two transform for 4096 samples): the cast is exact, so the
    # amplitudes meet the oracle's within the FP32 transform's rounding,
    # bounded here by 1e-5 of the frame's root-sum-square amplitude
    w = W.workload(name)
    g = w["geom"]
    if name == "paper8":
        fr = _all_values_frames(-128, 127, g.frame_len, np.int8, 19)
        fr = np.concatenate([fr] * 8)
    else:
        fr = _all_values_frames(-32768, 32767, g.frame_len, np.int16, 17)
    amps_o, _ = oracle.readout(fr, w["bins"])
    with _plan(w) as p:
        amps, _ = p.readout(torch.from_numpy(fr).to(dev), want_y=False)
        cg.cg_check_device(p.handle)
    scale = np.sqrt(g.frame_len * (fr.astype(np.float64) ** 2).sum(axis=1, keepdims=True))
    err = np.max(np.abs(amps.cpu().numpy() - amps_o) / scale)
    assert err <= 1e-5, (name, err)
