"""Pins of the oracle's multicanonical reweighting (Sec. 2.6, eq. (2.56)) and
of its tunnelling count, against results fixed without the formula itself:
a Gaussian density sampled flat, a two-state system in closed form, and a
second, independent way of counting tunnellings."""
import numpy as np
import pytest

import oracle
from oracle import recon


def test_flat_samples_of_a_gaussian_density_reweight_to_the_canonical_gaussian():
    """rho(E) = exp(-E^2 / (2 s^2)) has the canonical distribution
    rho(E) e^{beta E} ~ N(beta s^2, s^2).  A multicanonical run with
    W = 1/rho walks flat in E, so uniform samples on [-R, R] stand for its
    samples; ln rho~ is the piecewise-linear table of eq. (2.10) whose slope
    in each interval is the chord slope of -E^2 / (2 s^2).  Reweighted to
    beta, the samples give the Gaussian's mean and variance within their
    statistical error and the table's O(de^2) error.  Dropping ln rho~, its
    sign or the sign of beta moves the mean by many standard errors."""
    s, R, n_int = 3.0, 24.0, 480
    de = 2 * R / n_int
    c = -R + de * (np.arange(n_int) + 0.5)
    a = -c / s ** 2                                   # chord slopes of the parabola
    w = oracle.MucaWeight(-R, de, a)
    rng = np.random.default_rng(11)
    E = rng.uniform(-R, R, 400_000)
    lr = np.array([w.lnrho(x) for x in E])
    lr0 = -R ** 2 / (2 * s ** 2)                      # the table is 0 at e0 = -R
    assert np.allclose(lr[:50] + lr0, -E[:50] ** 2 / (2 * s ** 2), atol=de ** 2 / (8 * s ** 2) + 1e-12)
    for beta in (-0.4, 0.0, 0.25, 0.6):
        m1, m2 = recon.muca_moments(E, lr, beta)
        var = m2 - m1 * m1
        # effective sample size of uniform samples for N(mu, s^2): n * sqrt(pi) s / R
        n_eff = E.size * np.sqrt(np.pi) * s / R
        assert abs(m1 - beta * s ** 2) < 5 * s / np.sqrt(n_eff), (beta, m1)
        assert abs(var / s ** 2 - 1.0) < 5 * np.sqrt(2.0 / n_eff), (beta, var)
        assert abs(recon.muca_specific_heat(E, lr, beta) - var) < 1e-9 * var


@pytest.mark.parametrize("dl", [0.0, 0.8, -2.5])
def test_two_states_reweight_in_closed_form(dl):
    """Samples at two energies E1 < E2 in equal numbers (the flat histogram of
    a two-state system) with ln rho~ = L1, L2 there: reweighted to beta the
    weight of E2 is p = 1 / (1 + exp(-(beta (E2 - E1) + L2 - L1))), so
    <E> = E1 + (E2 - E1) p and C_V = (E2 - E1)^2 p (1 - p), whose maximum
    (E2 - E1)^2 / 4 lies at beta = -(L2 - L1) / (E2 - E1).  (The maximum is
    flat to second order, so its location is pinned to ~1e-6.)"""
    E1, E2, L1 = -2.0, 4.0, 3.0
    L2 = L1 + dl
    E = np.array([E1, E2] * 50)
    lr = np.array([L1, L2] * 50)
    g = E2 - E1
    for beta in (-0.7, -0.1, 0.0, 0.3):
        p = 1.0 / (1.0 + np.exp(-(beta * g + dl)))
        m1, m2 = recon.muca_moments(E, lr, beta)
        assert m1 == pytest.approx(E1 + g * p, rel=0, abs=1e-9)
        assert m2 - m1 * m1 == pytest.approx(g * g * p * (1 - p), rel=1e-6, abs=1e-7)
    b, cv = recon.muca_cv_peak(E, lr, -1.0, 1.0, n_grid=201, tol=1e-12)
    assert b == pytest.approx(-dl / g, abs=1e-6)
    assert cv == pytest.approx(g * g / 4.0, rel=1e-9)


def _tunnellings_by_compression(E_chain, lo, hi):
    """The same count another way: the sequence of end regions visited,
    consecutive repeats merged; every change of region is one passage."""
    regions = [(-1 if e < lo else 1) for e in E_chain if e < lo or e > hi]
    merged = [r for i, r in enumerate(regions) if i == 0 or r != regions[i - 1]]
    return max(len(merged) - 1, 0)


def test_tunnelling_count():
    lo, hi = 1.0, 9.0
    assert recon.tunnellings([5, 0, 5, 10, 5, 0, 10], lo, hi) == 3
    assert recon.tunnellings([5, 5, 5], lo, hi) == 0
    assert recon.tunnellings([0, 0, 10, 10, 0], lo, hi) == 2
    assert recon.tunnellings([10, 1.0, 9.0, 0.5], lo, hi) == 1     # the ends themselves do not count
    rng = np.random.default_rng(5)
    for _ in range(200):
        walk = np.cumsum(rng.normal(0.0, 1.5, rng.integers(0, 300))) + 5.0
        assert recon.tunnellings(walk, lo, hi) == _tunnellings_by_compression(walk, lo, hi)
