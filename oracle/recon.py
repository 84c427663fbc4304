"""FP64 oracle for the reconstruction of ln rho and of action observables.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Follows Sec. 2.2 and Sec. 2.3 of Langfeld, Lucini, Pellegrini, Rago
(arXiv:1509.08391):

* eq. (2.6) / (2.7): the trapezium rule on the slopes a_k gives
  ln rho at consecutive interval centres,
  ln rho(c_{k+1}) - ln rho(c_k) = (c_{k+1} - c_k) (a_k + a_{k+1}) / 2,
  fixed up to an additive constant by ln rho(c_0) = 0.  For contiguous
  intervals c_{k+1} - c_k = dE, which is the paper's form.
* eq. (2.46) / (2.47): action observables as sums over the centres,
  Z(beta) = sum_k w exp(ln rho(c_k) + beta c_k) and
  <E^m> = sum_k w c_k^m exp(ln rho(c_k) + beta c_k) / Z, with w the spacing
  of the (uniformly spaced) centres.
* Sec. 3.4: C_V(beta) = <E^2> - <E>^2 and beta_c = argmax C_V, located by a
  grid scan and golden-section refinement.

Everything is evaluated in log space (log-sum-exp) in FP64.
"""
from __future__ import annotations

import numpy as np


def lnrho_at_centres(c, a):
    c = np.asarray(c, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    out = np.zeros_like(c)
    for k in range(len(c) - 1):
        out[k + 1] = out[k] + 0.5 * (c[k + 1] - c[k]) * (a[k] + a[k + 1])
    return out


def moments(c, a, beta):
    """(ln Z, <E>, <E^2>) at one beta from eqs. (2.46)-(2.47)."""
    c = np.asarray(c, dtype=np.float64)
    w = (c[-1] - c[0]) / (len(c) - 1) if len(c) > 1 else 1.0
    x = lnrho_at_centres(c, a) + beta * c
    m = x.max()
    e = np.exp(x - m)
    s0 = e.sum()
    lnZ = m + np.log(w * s0)
    E1 = (c * e).sum() / s0
    E2 = (c * c * e).sum() / s0
    return lnZ, E1, E2


def specific_heat(c, a, beta):
    _, E1, E2 = moments(c, a, beta)
    return E2 - E1 * E1


def cv_peak(c, a, beta_lo, beta_hi, n_grid=2001, tol=1e-12):
    """beta_c and C_V(beta_c): grid scan, then golden-section search."""
    betas = np.linspace(beta_lo, beta_hi, n_grid)
    cv = np.array([specific_heat(c, a, b) for b in betas])
    i = int(np.argmax(cv))
    lo = betas[max(i - 1, 0)]
    hi = betas[min(i + 1, n_grid - 1)]
    g = (np.sqrt(5.0) - 1.0) / 2.0
    x1 = hi - g * (hi - lo)
    x2 = lo + g * (hi - lo)
    f1 = specific_heat(c, a, x1)
    f2 = specific_heat(c, a, x2)
    while hi - lo > tol:
        if f1 < f2:
            lo, x1, f1 = x1, x2, f2
            x2 = lo + g * (hi - lo)
            f2 = specific_heat(c, a, x2)
        else:
            hi, x2, f2 = x2, x1, f1
            x1 = hi - g * (hi - lo)
            f1 = specific_heat(c, a, x1)
    b = 0.5 * (lo + hi)
    return b, specific_heat(c, a, b)
