"""Pins of the FP64 network reference (oracle/mlp.py) to facts outside itself (CPU only).

* the activation: tanh-form GELU against the published exact form
  z Phi(z) (Hendrycks & Gimpel 2016) to within the approximation's known
  error, and the odd-part identity gelu(z) - gelu(-z) = z;
* the backward pass: central finite differences of the loss, for every
  parameter block (a transposed operand, a dropped bias or a wrong
  activation derivative fails here);
* the forward pass: special weight settings with closed-form outputs;
* Adam: the first bias-corrected step moves every parameter by lr sign(g);
* BF16 rounding: torch's own conversion and hand-checked ties.
"""
import math

import numpy as np
import pytest
import torch

from oracle import mlp


def _erf_gelu(z):
    from scipy.special import erf
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def test_gelu_close_to_exact_form():
    z = np.linspace(-8.0, 8.0, 20001)
    assert np.max(np.abs(mlp.gelu(z) - _erf_gelu(z))) < 5e-4
    # and far from a plausible wrong constant (sqrt(pi/2) instead of sqrt(2/pi))
    t_bad = np.tanh(math.sqrt(math.pi / 2) * (z + 0.044715 * z ** 3))
    assert np.max(np.abs(0.5 * z * (1 + t_bad) - _erf_gelu(z))) > 1e-2


def test_gelu_odd_part_and_limits():
    z = np.linspace(-5, 5, 101)
    assert np.allclose(mlp.gelu(z) - mlp.gelu(-z), z, rtol=0, atol=1e-14)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert abs(mlp.gelu(np.array([30.0]))[0] - 30.0) < 1e-12
    assert abs(mlp.gelu(np.array([-30.0]))[0]) < 1e-12


def test_gelu_grad_matches_central_difference():
    z = np.linspace(-6, 6, 241)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.gelu_grad(z))) < 1e-8
    assert abs(mlp.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15


@pytest.mark.parametrize("shape", [(7, 9, 3), (5, 4, 4), (11, 6, 1)])
def test_gradient_matches_finite_differences(shape):
    n_in, H, n_out = shape
    rng = np.random.default_rng(11)
    npar = mlp.n_params(n_in, H, n_out)
    theta = rng.normal(0, 0.6, npar)
    x = rng.normal(0, 1, (6, n_in))
    t = rng.normal(0, 1, (6, n_out))
    _, g = mlp.loss_and_grad(theta, x, t, n_in, H, n_out)
    h = 1e-6
    fd = np.empty(npar)
    for i in range(npar):
        e = np.zeros(npar)
        e[i] = h
        fd[i] = (mlp.loss(theta + e, x, t, n_in, H, n_out) - mlp.loss(theta - e, x, t, n_in, H, n_out)) / (2 * h)
    assert np.max(np.abs(fd - g)) < 1e-7 * max(1.0, np.max(np.abs(g)))


def test_forward_closed_forms():
    n_in, H, n_out = 5, 6, 3
    rng = np.random.default_rng(3)
    x = rng.normal(0, 1, (4, n_in))
    p = {"W1": rng.normal(0, 1, (H, n_in)), "b1": rng.normal(0, 1, H),
         "W2": np.zeros((H, H)), "b2": np.zeros(H),
         "W3": rng.normal(0, 1, (n_out, H)), "b3": np.array([1.5, -2.0, 0.25])}
    pack = lambda d: np.concatenate([d[k].ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")])
    # a dead second layer (gelu(0) = 0): the output is the output bias
    out = mlp.forward(pack(p), x, n_in, H, n_out)
    assert np.array_equal(out, np.tile(p["b3"], (4, 1)))
    # W1 = 0 and a single W2 entry (row i, column j): z2 is nonzero only in
    # unit i, where it equals gelu(b1[j]); the output is W3[:, i] gelu(gelu(b1[j])) + b3
    p["W1"] = np.zeros((H, n_in))
    p["W2"] = np.zeros((H, H))
    i, j = 4, 1
    p["W2"][i, j] = 1.0
    out = mlp.forward(pack(p), x, n_in, H, n_out)
    a = 0.5 * p["b1"][j] * (1 + math.erf(p["b1"][j] / math.sqrt(2)))   # exact GELU, within 5e-4
    want = p["W3"][:, i] * _erf_gelu(np.array([a]))[0] + p["b3"]
    assert np.allclose(out, np.tile(want, (4, 1)), atol=2e-3 * np.max(np.abs(p["W3"])) + 1e-12)
    # and exactly the tanh form composed
    want_exact = p["W3"][:, i] * mlp.gelu(mlp.gelu(np.array([p["b1"][j]])))[0] + p["b3"]
    assert np.allclose(out, np.tile(want_exact, (4, 1)), rtol=1e-14, atol=1e-14)


def test_adam_first_step_is_sign_step():
    rng = np.random.default_rng(5)
    theta = rng.normal(0, 1, 50)
    g = rng.normal(0, 1, 50)
    new, m, v = mlp.adam_step(theta, g, np.zeros(50), np.zeros(50), 1, lr=0.01)
    # (the eps term shifts the step by lr eps / |g|, far below 1e-6 here)
    assert np.allclose(new, theta - 0.01 * np.sign(g), rtol=0, atol=1e-6)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_round_matches_torch_and_ties():
    rng = np.random.default_rng(9)
    a = np.concatenate([rng.normal(0, 1, 5000), rng.normal(0, 1e-3, 1000), rng.normal(0, 1e3, 1000)])
    want = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(a), want)
    assert mlp.bf16_round(np.array([1.0 + 2.0 ** -8]))[0] == 1.0             # tie -> even
    assert mlp.bf16_round(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6   # tie -> even (up)
