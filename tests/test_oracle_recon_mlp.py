"""Pins of the FP64 reconstruction and MLP oracles against closed forms."""
import math

import numpy as np
import pytest

from oracle import mlp, recon


# ---------------------------------------------------------------- reconstruction
def test_trapezium_is_exact_for_linear_slope():
    """eq. (2.6): the trapezium rule integrates a linear a(E) exactly."""
    c = np.sort(np.random.default_rng(1).uniform(100.0, 300.0, 40))
    a0, a1 = -1.3, 2.5e-3
    ln = recon.lnrho_at_centres(c, a0 + a1 * c)
    exact = a0 * (c - c[0]) + 0.5 * a1 * (c ** 2 - c[0] ** 2)
    assert np.max(np.abs(ln - exact)) < 1e-9


def test_gaussian_density_observables():
    """ln rho = -(E-mu)^2/(2 s^2): <E>_beta = mu + beta s^2 and C_V = s^2 (eqs. (2.46)-(2.47))."""
    mu, s = 900.0, 12.0
    c = np.linspace(mu - 40 * s, mu + 40 * s, 8001)
    a = -(c - mu) / s ** 2
    for beta in [-0.7, 0.0, 0.3, 1.1]:
        lnZ, E1, E2 = recon.moments(c, a, beta)
        assert abs(E1 - (mu + beta * s * s)) < 1e-8
        assert abs((E2 - E1 ** 2) - s * s) < 1e-7
        # ln Z up to the additive constant ln rho(c_0): compare two betas
    lz0 = recon.moments(c, a, 0.0)[0]
    lz1 = recon.moments(c, a, 0.4)[0]
    assert abs((lz1 - lz0) - (0.4 * mu + 0.5 * 0.4 ** 2 * s ** 2)) < 1e-8


def test_cv_peak_of_two_state_mixture():
    """rho = g1 N(mu1, s) + g2 N(mu2, s): C_V = s^2 + D^2 p (1-p), maximal at
    beta_c = ln(g1/g2) / D with C_V = s^2 + D^2 / 4."""
    mu1, mu2, s, g1, g2 = 0.0, 30.0, 2.0, 5.0, 1.0
    D = mu2 - mu1
    c = np.linspace(-40.0, 70.0, 22001)

    def lnrho(E):
        return np.logaddexp(math.log(g1) - (E - mu1) ** 2 / (2 * s * s),
                            math.log(g2) - (E - mu2) ** 2 / (2 * s * s))

    h = 1e-5
    a = (lnrho(c + h) - lnrho(c - h)) / (2 * h)
    b, cv = recon.cv_peak(c, a, 0.0, 0.2, n_grid=401)
    assert abs(b - math.log(g1 / g2) / D) < 1e-5
    assert abs(cv - (s * s + D * D / 4)) < 1e-4


# ---------------------------------------------------------------- MLP
def test_gelu_identities():
    z = np.linspace(-6, 6, 101)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert np.max(np.abs(mlp.gelu(z) - mlp.gelu(-z) - z)) < 1e-14   # Phi(z)+Phi(-z)=1
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.gelu_grad(z))) < 1e-8


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(3)
    p = mlp.init_params(7)
    p = [q + 0.1 * rng.normal(size=q.shape) for q in p]
    x = rng.normal(size=(33, 3))
    t = rng.normal(size=33)
    g = mlp.backward(p, x, t)
    h = 1e-6
    for k in range(len(p)):
        flat = p[k].reshape(-1)
        for j in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[j]
            flat[j] = old + h
            lp = mlp.loss(p, x, t)
            flat[j] = old - h
            lm = mlp.loss(p, x, t)
            flat[j] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[j]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-9


def test_zero_network_outputs_bias():
    p = [np.zeros(s) for s in mlp.SHAPES]
    p[-1][0] = -0.97
    y, _ = mlp.forward(p, np.ones((5, 3)))
    assert np.all(y == -0.97)


def test_adam_first_step_is_signed_lr():
    p = [np.array([1.0, -2.0, 3.0])]
    g = [np.array([0.5, -4.0, 1e-3])]
    opt = mlp.Adam(p, lr=0.01, eps=1e-12)
    out = opt.step(p, g)[0]
    assert np.allclose(out, p[0] - 0.01 * np.sign(g[0]), atol=1e-10)
