"""FP64 reference of the learned initial-guess network (TEST INFRASTRUCTURE ONLY).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
module; the library never imports it.

The network is a multilayer perceptron in -> H -> H -> out with GELU hidden
activations in their tanh form (Hendrycks & Gimpel, "Gaussian Error Linear
Units", 2016):

    gelu(z) = z/2 * (1 + tanh(k (z + 0.044715 z^3))),  k = sqrt(2/pi),

a linear output layer, and the mean-squared-error loss
L = mean over the batch and the outputs of (out - target)^2.  Written with
plain numpy matrix products in FP64.  Pinned in the tests by central finite
differences of the loss (the backward pass), by the closed forms of special
weight settings (the forward pass), and by the published erf form of GELU
(the activation).

Flat parameter layout, shared with the library's parameter vector:
W1 [H, in], b1 [H], W2 [H, H], b2 [H], W3 [out, H], b3 [out], row-major.
"""
from __future__ import annotations

import math

import numpy as np

_K = math.sqrt(2.0 / math.pi)
_C = 0.044715


def gelu(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * z * (1.0 + np.tanh(_K * (z + _C * z ** 3)))


def gelu_grad(z: np.ndarray) -> np.ndarray:
    """d gelu / dz of the tanh form."""
    z = np.asarray(z, dtype=np.float64)
    t = np.tanh(_K * (z + _C * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * _K * (1.0 + 3.0 * _C * z * z)


def n_params(n_in: int, n_hidden: int, n_out: int) -> int:
    return n_hidden * n_in + n_hidden + n_hidden * n_hidden + n_hidden + n_out * n_hidden + n_out


def unpack(theta: np.ndarray, n_in: int, n_hidden: int, n_out: int) -> dict:
    theta = np.asarray(theta, dtype=np.float64)
    shapes = [("W1", (n_hidden, n_in)), ("b1", (n_hidden,)), ("W2", (n_hidden, n_hidden)),
              ("b2", (n_hidden,)), ("W3", (n_out, n_hidden)), ("b3", (n_out,))]
    out, o = {}, 0
    for name, shp in shapes:
        size = int(np.prod(shp))
        out[name] = theta[o:o + size].reshape(shp)
        o += size
    if o != theta.size:
        raise ValueError("parameter vector has the wrong length")
    return out


def forward(theta, x, n_in, n_hidden, n_out, keep=False, operand_round=None):
    """Network output for the rows of x.

    operand_round, if given, is applied to both operands of every matrix
    product (weights and activations), so that the result of a kernel which
    stores its operands in a narrower type can be compared with FP64
    arithmetic on exactly the operands it used.
    """
    p = unpack(theta, n_in, n_hidden, n_out)
    rnd = operand_round if operand_round is not None else (lambda a: a)
    x = np.asarray(x, dtype=np.float64)
    z1 = rnd(x) @ rnd(p["W1"]).T + p["b1"]
    a1 = gelu(z1)
    z2 = rnd(a1) @ rnd(p["W2"]).T + p["b2"]
    a2 = gelu(z2)
    out = a2 @ p["W3"].T + p["b3"]
    if keep:
        return out, dict(x=x, z1=z1, a1=a1, z2=z2, a2=a2, p=p)
    return out


def loss(theta, x, target, n_in, n_hidden, n_out) -> float:
    d = forward(theta, x, n_in, n_hidden, n_out) - np.asarray(target, dtype=np.float64)
    return float(np.mean(d * d))


def loss_and_grad(theta, x, target, n_in, n_hidden, n_out):
    """MSE loss and its gradient with respect to the flat parameter vector
    (reverse-mode differentiation of forward(), layer by layer)."""
    out, c = forward(theta, x, n_in, n_hidden, n_out, keep=True)
    t = np.asarray(target, dtype=np.float64)
    n = out.shape[0]
    diff = out - t
    value = float(np.mean(diff * diff))
    g_out = 2.0 * diff / (n * n_out)
    p = c["p"]
    gW3 = g_out.T @ c["a2"]
    gb3 = g_out.sum(axis=0)
    g_z2 = (g_out @ p["W3"]) * gelu_grad(c["z2"])
    gW2 = g_z2.T @ c["a1"]
    gb2 = g_z2.sum(axis=0)
    g_z1 = (g_z2 @ p["W2"]) * gelu_grad(c["z1"])
    gW1 = g_z1.T @ c["x"]
    gb1 = g_z1.sum(axis=0)
    grad = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return value, grad


def adam_step(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) with bias-corrected
    moments; step counts from 1.  Returns the new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as FP64: the FP32
    value's low 16 bits are rounded away by integer arithmetic on its bits."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
