"""Training of the learned initial guess (test helper; run as a script on a GPU).

    python -m tests.mlp_train --n 2000000 --epochs 30 --out paper_2307_12988_gb300/data/mlp_wide_t221.cgmlp

Spectra: ``synth.tooth_domain_spectra`` on the wide geometry (2.5 GS/s, 2500
samples, 221 teeth at |51 + 10 k| MHz, k = -110..110): centres U(+-100 MHz),
FWHM U(60, 100) MHz, time-domain SNR U(20, 40) dB per spectrum.
Labels: the oracle's fully converged LM fit of each spectrum (c, |g|, A, B).
Left out: spectra whose converged fit reports no convergence, and the rare
degenerate optima outside the comb (|c| beyond the outermost tooth, g beyond
the span or below half a tooth spacing, |A| or |B| above 10), which a
starting guess should not imitate.
Training: the library's own kernels (``cg_mlp_train_epoch``: forward,
backward, Adam) with a cosine learning-rate schedule; inputs and labels are
standardised per feature and the standardisation is saved with the weights.
Only this helper, the tests and the benchmark's CPU leg touch ``oracle``.
"""
from __future__ import annotations

import argparse
import math
import time

import numpy as np

import oracle
import synth

TRAIN_SEED = synth.BASE_SEED + 400


def make_dataset(n: int, seed: int = TRAIN_SEED, geom=synth.WIDE, chunk: int = 200_000, log=print):
    ys, ps = [], []
    dropped = 0
    for i, s in enumerate(range(0, n, chunk)):
        m = min(chunk, n - s)
        d = synth.tooth_domain_spectra(geom, m, seed=seed + i)
        r = oracle.fit_batch(d["y"], geom.tooth_x, converged=True)
        p = r["params"].copy()
        p[:, 1] = np.abs(p[:, 1])
        span = float(geom.tooth_x.max() - geom.tooth_x.min())
        dx = span / (geom.n_teeth - 1)
        ok = ((r["status"] == 0) & (np.abs(p[:, 0]) <= 0.5 * span) & (p[:, 1] >= 0.5 * dx) &
              (p[:, 1] <= span) & (np.abs(p[:, 2]) <= 10.0) & (np.abs(p[:, 3]) <= 10.0))
        dropped += int(m - ok.sum())
        ys.append(d["y"][ok].astype(np.float32))
        ps.append(p[ok].astype(np.float32))
        log(f"  labelled {s + m}/{n}")
    return np.concatenate(ys), np.concatenate(ps), dropped


def train(y: np.ndarray, p: np.ndarray, *, epochs: int = 30, batch: int = 1024, lr: float = 1e-3,
          seed: int = 0, n_hidden: int = 256, log=print):
    import torch
    import paper_2307_12988_gb300 as cg
    n, T = y.shape
    in_mean = y.mean(axis=0)
    in_scale = 1.0 / np.maximum(y.std(axis=0), 1e-6)
    out_mean = p.mean(axis=0)
    out_scale = np.maximum(p.std(axis=0), 1e-12)
    x = ((y - in_mean) * in_scale).astype(np.float32)
    t = ((p - out_mean) / out_scale).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    td = torch.from_numpy(t).cuda()
    net = cg.Mlp(T, n_hidden, 4, max_batch=batch, seed=seed)
    rng = np.random.default_rng(seed)
    history = []
    for ep in range(epochs):
        lr_ep = lr * 0.5 * (1.0 + math.cos(math.pi * ep / epochs))
        perm = torch.from_numpy(rng.permutation(n).astype(np.int32)).cuda()
        losses = net.train_epoch(xd, td, perm, batch, lr_ep).cpu().numpy()
        history.append(float(losses.mean()))
        log(f"  epoch {ep:3d} lr {lr_ep:.2e} loss {history[-1]:.5f}")
    net.set_norm(in_mean.astype(np.float32), in_scale.astype(np.float32), out_mean.astype(np.float32),
                 out_scale.astype(np.float32))
    return net, history


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=2_000_000)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--out", required=True)
    a = ap.parse_args()
    t0 = time.time()
    y, p, dropped = make_dataset(a.n)
    print(f"dataset {y.shape} ({dropped} dropped) in {time.time() - t0:.1f} s", flush=True)
    t1 = time.time()
    net, hist = train(y, p, epochs=a.epochs, batch=a.batch, lr=a.lr)
    print(f"trained in {time.time() - t1:.1f} s; final loss {hist[-1]:.5f}", flush=True)
    with open(a.out, "wb") as f:
        f.write(net.save())


if __name__ == "__main__":
    main()
