"""What the trained network gains over the moment guess (GPU).

Held-out frames of the learned-guess workload (wide geometry: 2.5 GS/s,
2500 samples, 221 teeth; per-frame centre U(+-100 MHz), FWHM U(60, 100) MHz,
SNR U(20, 40) dB; a stream seed and parameter seed the network never saw)
go through the plain plan (moment guess + LM, at most 20 steps) and through
the learned plan (network guess + 2 polish steps, fallback to the full LM).
Both are judged against the oracle's fully converged fit of the oracle's own
readout: the learned path must need markedly fewer LM steps per frame while
its centres stay within 1e-4 of each frame's linewidth as often as the
plain path's do.
"""
import os

import numpy as np
import pytest
import torch

import oracle
import paper_2307_12988_gb300 as cg
import synth

pytestmark = pytest.mark.gpu
BLOB = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2307_12988_gb300", "data", "mlp_wide_t221.cgmlp")
N_FRAMES = 20000


@pytest.fixture(scope="module")
def heldout():
    g = synth.WIDE
    stream = synth.make_stream(g, synth.BASE_SEED + 500)
    lp = synth.learned_params(N_FRAMES, seed=synth.BASE_SEED + 501)
    fr = synth.frames(stream, N_FRAMES, centers=lp["c"], fwhm_hz=lp["fwhm"], snr_db=lp["snr_db"])
    rf = synth.frames(stream, 2000, cavity=False, noise_stream=1, snr_db=30.0)
    bins = oracle.tooth_bins(g.sample_rate, g.frame_len, g.tooth_freqs)
    ref = oracle.reference(rf["frames"], bins)
    _, y = oracle.readout(fr["frames"], bins, ref)
    conv = oracle.fit_batch(y, g.tooth_x, converged=True)
    return dict(g=g, frames=fr["frames"], ref=ref, fwhm=lp["fwhm"], conv=conv)


def _run(h, **opts):
    g = h["g"]
    frames = torch.from_numpy(h["frames"]).cuda()
    with cg.Plan(g.sample_rate, g.frame_len, g.tooth_freqs, g.tooth_x, h["ref"], **opts) as plan:
        if opts.get("init") == cg.INIT_MLP:
            with open(BLOB, "rb") as f:
                plan.mlp_load(f.read())
        o = plan.process(frames)
        cg.cg_check_device(plan.handle)
    p = o["params"].cpu().numpy()
    st = o["status"].cpu().numpy()
    it = o["iters"].cpu().numpy().astype(np.float64)
    err = np.abs(p[:, 0] - h["conv"]["params"][:, 0])
    ok = h["conv"]["status"] == 0
    within = np.mean(err[ok] <= 1e-4 * h["fwhm"][ok])
    return dict(iters=it.mean(), within=within, converged=np.mean((st & 3) == 0),
                fallback=np.mean((st & cg.FIT_FALLBACK) != 0))


def test_learned_guess_cuts_lm_steps_at_equal_accuracy(heldout):
    plain = _run(heldout)
    learned = _run(heldout, init=cg.INIT_MLP)
    print(f"\n[plain]   mean LM steps {plain['iters']:.3f}  within 1e-4 FWHM {plain['within']:.5f}  "
          f"converged {plain['converged']:.5f}")
    print(f"[learned] mean LM steps {learned['iters']:.3f}  within 1e-4 FWHM {learned['within']:.5f}  "
          f"converged {learned['converged']:.5f}  fallback {learned['fallback']:.4f}")
    assert learned["iters"] <= 0.75 * plain["iters"]
    assert learned["within"] >= 0.999
    assert learned["within"] >= plain["within"] - 5e-4
    assert learned["converged"] >= plain["converged"] - 5e-4
    assert learned["fallback"] <= 0.10
