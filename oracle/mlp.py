"""FP64 oracle for the warm-start network: a 3-hidden-layer, width-64 MLP.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper has no network; this is the learned warm start of the Robbins-
Monro iteration.  The paper's reason it can work: the slopes a_k are
intrinsic (volume independent) quantities, Sec. 2.2 eq. (2.5) and the
appendix, eqs. (A.11)-(A.13), so a map (L, E/6V, dE) -> a learned on small
volumes predicts larger ones; Sec. 2.4 says a good initial a only needs to be
close to the result.

Definition (both the oracle and the CUDA kernels implement exactly this):
  features  x = ((1/V, E/6V, dE/6V) - mean) / std   (V = L^4; training-set statistics;
            1/V because the finite-volume corrections of a_k are O(1/V), eq. (A.12))
  h1 = gelu(x W1 + b1)      W1: 3x64
  h2 = gelu(h1 W2 + b2)     W2: 64x64
  h3 = gelu(h2 W3 + b3)     W3: 64x64
  y  = h3 W4 + b4           W4: 64x1
  gelu(z) = z * Phi(z) = z (1 + erf(z / sqrt 2)) / 2
  loss = mean over the batch of (y - t)^2
  Adam (Kingma & Ba 2015) with bias correction.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

WIDTH = 64
N_IN = 3
SHAPES = [(N_IN, WIDTH), (WIDTH,), (WIDTH, WIDTH), (WIDTH,), (WIDTH, WIDTH), (WIDTH,),
          (WIDTH, 1), (1,)]


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)


def init_params(seed: int):
    """Deterministic init from a seeded numpy generator (an input, not method arithmetic)."""
    rng = np.random.default_rng(seed)
    p = []
    for s in SHAPES:
        if len(s) == 2:
            p.append(rng.normal(0.0, 1.0 / math.sqrt(s[0]), size=s))
        else:
            p.append(np.zeros(s))
    return p


def forward(params, x):
    W1, b1, W2, b2, W3, b3, W4, b4 = params
    z1 = x @ W1 + b1
    h1 = gelu(z1)
    z2 = h1 @ W2 + b2
    h2 = gelu(z2)
    z3 = h2 @ W3 + b3
    h3 = gelu(z3)
    y = h3 @ W4 + b4
    return y[:, 0], (x, z1, h1, z2, h2, z3, h3)


def loss(params, x, t):
    y, _ = forward(params, x)
    return float(np.mean((y - t) ** 2))


def backward(params, x, t):
    """Gradients of the MSE loss with respect to every parameter."""
    W1, b1, W2, b2, W3, b3, W4, b4 = params
    y, (x, z1, h1, z2, h2, z3, h3) = forward(params, x)
    n = x.shape[0]
    dy = (2.0 / n) * (y - t)[:, None]
    gW4 = h3.T @ dy
    gb4 = dy.sum(axis=0)
    dz3 = (dy @ W4.T) * gelu_grad(z3)
    gW3 = h2.T @ dz3
    gb3 = dz3.sum(axis=0)
    dz2 = (dz3 @ W3.T) * gelu_grad(z2)
    gW2 = h1.T @ dz2
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2.T) * gelu_grad(z1)
    gW1 = x.T @ dz1
    gb1 = dz1.sum(axis=0)
    return [gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4]


class Adam:
    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = [np.zeros_like(p) for p in params]
        self.v = [np.zeros_like(p) for p in params]
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        c1 = 1.0 - self.b1 ** self.t
        c2 = 1.0 - self.b2 ** self.t
        out = []
        for p, g, m, v in zip(params, grads, self.m, self.v):
            m[...] = self.b1 * m + (1.0 - self.b1) * g
            v[...] = self.b2 * v + (1.0 - self.b2) * g * g
            out.append(p - self.lr * (m / c1) / (np.sqrt(v / c2) + self.eps))
        return out


def features(L, e6v, dE6v):
    return np.stack([1.0 / np.asarray(L, dtype=np.float64) ** 4, np.asarray(e6v, dtype=np.float64),
                     np.asarray(dE6v, dtype=np.float64)], axis=1)


def standardise(raw, mean=None, std=None):
    if mean is None:
        mean = raw.mean(axis=0)
        std = raw.std(axis=0)
        std = np.where(std > 0, std, 1.0)
    return (raw - mean) / std, mean, std
