"""Closed forms and quadratures that pin the oracle.

Two-dimensional U(1) with open boundaries has independent plaquettes: in a
maximal tree gauge every plaquette angle is one free link, so under the Haar
measure the plaquette angles are independent and uniform (Sec. 3.1 for the
model; the appendix, eq. (A.3), gives the density of a sum of independent
domains).  Hence

* one plaquette at weight exp(beta cos p): <cos p> = I1(beta)/I0(beta);
* two plaquettes: E = cos p1 + cos p2 with p1, p2 uniform, so every
  restricted, reweighted moment of eqs. (2.13)-(2.15) is a two-dimensional
  integral over (p1, p2) that quadrature evaluates to ~1e-10.

Nothing here calls the oracle.
"""
from __future__ import annotations

import numpy as np
from scipy import integrate, optimize, special


def bessel_ratio(beta: float) -> float:
    """<cos p> for one plaquette at weight exp(beta cos p)."""
    return float(special.i1(beta) / special.i0(beta))


def restricted_moments_2plaq(lo: float, hi: float, a: float, kmax: int = 2):
    """Integrals  int dp1 dp2 / pi^2  E^k exp(-a E) 1[lo <= E <= hi],  k = 0..kmax,
    with E = cos p1 + cos p2 and p1, p2 uniform on [0, pi] (by symmetry)."""
    out = np.zeros(kmax + 1)

    def inner(u, k):
        cu = np.cos(u)
        top, bot = hi - cu, lo - cu   # need cos v in [bot, top]
        if top < -1.0 or bot > 1.0:
            return 0.0
        v1 = np.arccos(min(1.0, top))
        v2 = np.arccos(max(-1.0, bot))
        f = lambda v: (cu + np.cos(v)) ** k * np.exp(-a * (cu + np.cos(v)))
        return integrate.quad(f, v1, v2, epsabs=1e-14, epsrel=1e-12)[0]

    for k in range(kmax + 1):
        out[k] = integrate.quad(lambda u: inner(u, k), 0.0, np.pi, epsabs=1e-13,
                                epsrel=1e-11, limit=500)[0] / np.pi ** 2
    return out


def restricted_mean_2plaq(lo, hi, a):
    m = restricted_moments_2plaq(lo, hi, a, 1)
    return m[1] / m[0]


def llr_root_2plaq(lo, hi, bracket=(-30.0, 30.0)):
    """The a solving <<E - lo - dE/2>>(a) = 0 (eq. (2.17)) for two plaquettes."""
    c = 0.5 * (lo + hi)
    return optimize.brentq(lambda a: restricted_mean_2plaq(lo, hi, a) - c, *bracket,
                           xtol=1e-12)


def batch_means(x, nbatch: int = 50):
    """Mean and its standard error from batch means (autocorrelated chain)."""
    x = np.asarray(x, dtype=np.float64)
    n = (len(x) // nbatch) * nbatch
    b = x[:n].reshape(nbatch, -1).mean(axis=1)
    return float(x[:n].mean()), float(b.std(ddof=1) / np.sqrt(nbatch))


def restricted_moments_3plaq(lo: float, hi: float, a: float, kmax: int = 1, n_outer=600,
                             n_inner=48):
    """The same integrals for E = cos p1 + cos p2 + cos p3 (three independent
    uniform plaquettes): Gauss-Legendre over (p1, p2) in [0, pi]^2 and, for each,
    Gauss-Legendre over the p3 interval on which E lies in the window."""
    xo, wo = np.polynomial.legendre.leggauss(n_outer)
    xi, wi = np.polynomial.legendre.leggauss(n_inner)
    u = 0.5 * np.pi * (xo + 1.0)
    wu = 0.5 * np.pi * wo
    cu = np.cos(u)
    c = cu[:, None] + cu[None, :]
    w2 = wu[:, None] * wu[None, :]
    top = np.clip(hi - c, -1.0, 1.0)
    bot = np.clip(lo - c, -1.0, 1.0)
    ok = (hi - c >= -1.0) & (lo - c <= 1.0)
    v1 = np.arccos(top)
    v2 = np.arccos(bot)
    half = 0.5 * (v2 - v1)
    mid = 0.5 * (v2 + v1)
    v = mid[..., None] + half[..., None] * xi[None, None, :]
    E = c[..., None] + np.cos(v)
    out = np.zeros(kmax + 1)
    for k in range(kmax + 1):
        f = E ** k * np.exp(-a * E)
        inner = (f * wi[None, None, :]).sum(axis=-1) * half
        out[k] = (w2 * np.where(ok, inner, 0.0)).sum() / np.pi ** 3
    return out


def restricted_mean_3plaq(lo, hi, a):
    m = restricted_moments_3plaq(lo, hi, a, 1)
    return m[1] / m[0]


def density_2plaq(E: float) -> float:
    """Density of E = cos p1 + cos p2 for independent uniform plaquette angles
    (normalised: its integral over E is 1): the convolution of two
    arcsine densities 1 / (pi sqrt(1 - e^2)), evaluated with the endpoint
    singularities as an algebraic quadrature weight.  0 < |E| < 2."""
    E = abs(E)
    lo, hi = E - 1.0, 1.0
    f = lambda e: 1.0 / np.sqrt((1.0 + e) * (1.0 + E - e))
    val = integrate.quad(f, lo, hi, weight="alg", wvar=(-0.5, -0.5), epsabs=1e-13,
                         epsrel=1e-12, limit=200)[0]
    return float(val / np.pi ** 2)
