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
* Sec. 2.6, eq. (2.56): canonical averages from the samples E_i of a
  multicanonical run with weight W = 1/rho~: sample i carries
  exp(beta E_i) / W(E_i) = exp(beta E_i + ln rho~(E_i)), so
  <E^m>(beta) = sum_i E_i^m exp(beta E_i + ln rho~(E_i)) / sum_i exp(...).
  The ergodicity check of the same section counts tunnellings: passages of
  a chain from the lowest to the highest part of the range or back.

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
    return _peak(lambda b: specific_heat(c, a, b), beta_lo, beta_hi, n_grid, tol)


def _peak(f, beta_lo, beta_hi, n_grid, tol):
    """Maximum of f on [beta_lo, beta_hi]: the best of n_grid equally spaced
    points, then golden-section search between its two neighbours."""
    betas = np.linspace(beta_lo, beta_hi, n_grid)
    cv = np.array([f(b) for b in betas])
    i = int(np.argmax(cv))
    lo = betas[max(i - 1, 0)]
    hi = betas[min(i + 1, n_grid - 1)]
    g = (np.sqrt(5.0) - 1.0) / 2.0
    x1 = hi - g * (hi - lo)
    x2 = lo + g * (hi - lo)
    f1 = f(x1)
    f2 = f(x2)
    while hi - lo > tol:
        if f1 < f2:
            lo, x1, f1 = x1, x2, f2
            x2 = lo + g * (hi - lo)
            f2 = f(x2)
        else:
            hi, x2, f2 = x2, x1, f1
            x1 = hi - g * (hi - lo)
            f1 = f(x1)
    b = 0.5 * (lo + hi)
    return b, f(b)


def muca_moments(E, lnrho_E, beta):
    """(<E>, <E^2>) at coupling beta from multicanonical samples E (any
    shape), eq. (2.56); lnrho_E holds ln rho~ at each sample."""
    E = np.asarray(E, dtype=np.float64).ravel()
    lr = np.asarray(lnrho_E, dtype=np.float64).ravel()
    x = beta * E + lr
    w = np.exp(x - x.max())
    s0 = w.sum()
    return (w * E).sum() / s0, (w * E * E).sum() / s0


def muca_specific_heat(E, lnrho_E, beta):
    E1, E2 = muca_moments(E, lnrho_E, beta)
    return E2 - E1 * E1


def muca_cv_peak(E, lnrho_E, beta_lo, beta_hi, n_grid=401, tol=1e-10):
    """beta_c and C_V(beta_c) of the reweighted samples (Sec. 2.6 with
    Sec. 3.4): grid scan, then golden-section search."""
    return _peak(lambda b: muca_specific_heat(E, lnrho_E, b), beta_lo, beta_hi, n_grid, tol)


def tunnellings(E_chain, lo, hi):
    """Number of tunnellings of one chain (Sec. 2.6): its energies in time
    order; each passage from E < lo to E > hi, or from E > hi to E < lo,
    counts once."""
    count = 0
    last = 0            # -1: last seen below lo, +1: above hi, 0: neither yet
    for e in E_chain:
        if e < lo:
            if last == 1:
                count += 1
            last = -1
        elif e > hi:
            if last == -1:
                count += 1
            last = 1
    return count
