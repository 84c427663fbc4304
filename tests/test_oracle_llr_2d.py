"""The whole LLR method on a system with a known density of states: the 2-D
open strip of two plaquettes (7 links), whose plaquette angles are
independent and uniform, so rho(E) is the convolution of two arcsine
densities (appendix, the independent-plaquette form), with a logarithmic
spike at E = 0.

- Algorithm 1 with eq. (2.30) over 6 contiguous intervals of dE = 0.5 on
  [-1.4, 1.6]: every slope agrees with the exact root of eq. (2.17) (by
  quadrature) within its statistical error, and <E>(beta) reconstructed from
  the slopes (eqs. (2.6), (2.46), (2.47)) agrees with the same reconstruction
  from the exact roots within the propagated statistical error.
- The reconstruction's own error (exact roots against the exact canonical
  mean over the same range) is O(dE^2) where rho is smooth (Sec. 2.3):
  on [0.1, 1.6] halving dE divides it by ~4.  (Across the spike at E = 0 the
  slope diverges and the trapezium rule for ln rho loses that order.)"""
import os

import numpy as np

import oracle
from oracle import recon
from tests import exact2d


def _roots(lo, de, n):
    return np.array([exact2d.llr_root_2plaq(lo + k * de, lo + (k + 1) * de) for k in range(n)])


def _exact_truncated_mean(lo, de, n, beta):
    """<E> at coupling beta over [lo, lo + n de]: the exact restricted moments
    of every interval at a = -beta, summed."""
    m0 = m1 = 0.0
    for k in range(n):
        z = exact2d.restricted_moments_2plaq(lo + k * de, lo + (k + 1) * de, -beta, 1)
        m0 += z[0]
        m1 += z[1]
    return m1 / m0


def test_llr_slopes_and_their_reconstruction_on_two_plaquettes():
    LO, DE, N, R = -1.4, 0.5, 6, 8
    g = oracle.Geom([3, 2], periodic=False)
    lo = [LO + k * DE for k in range(N) for _ in range(R)]
    iid = [k for k in range(N) for _ in range(R)]
    rid = [r for _ in range(N) for r in range(R)]
    out = oracle.batch_run(g, 31337, iid, rid, lo, [DE] * len(lo), [-1.0] * len(lo), n_or=1,
                           block=1, n_therm=5, n_meas=100, n_rm=400,
                           n_threads=min(8, os.cpu_count() or 1))
    assert np.all(out["status"] == 0)
    a = out["a"].reshape(N, R)
    a_mean = a.mean(axis=1)
    a_err = a.std(axis=1, ddof=1) / np.sqrt(R)
    exact = _roots(LO, DE, N)
    z = (a_mean - exact) / a_err
    assert np.all(np.abs(z) < 4.0), z
    assert np.sum(z ** 2) < N + 4.0 * np.sqrt(2.0 * N)          # chi^2 of N d.o.f.
    c = LO + DE * (np.arange(N) + 0.5)
    for beta in (-0.5, 0.5, 1.5):
        ref = recon.moments(c, exact, beta)[1]
        per_rep = np.array([recon.moments(c, a[:, r], beta)[1] for r in range(R)])
        stat = per_rep.std(ddof=1) / np.sqrt(R)
        got = recon.moments(c, a_mean, beta)[1]
        assert abs(got - ref) < 4.0 * stat, (beta, got, ref, stat)


def test_reconstruction_error_is_second_order_in_the_interval_width():
    LO, HI = 0.1, 1.6
    for beta in (-0.5, 1.5):
        err = []
        for de in (0.5, 0.25):
            n = int(round((HI - LO) / de))
            c = LO + de * (np.arange(n) + 0.5)
            err.append(recon.moments(c, _roots(LO, de, n), beta)[1]
                       - _exact_truncated_mean(LO, de, n, beta))
        assert abs(err[0]) < 0.05
        assert 0.15 < err[1] / err[0] < 0.35, (beta, err)      # (1/2)^2 = 0.25
