"""Pins of the oracle's multicanonical update (Sec. 2.6, eq. (2.50)): the
weight 1/rho~ with rho~ the piecewise-exponential density of eq. (2.10),
heat-bath proposals at a fixed slope a0 corrected by Metropolis-Hastings.

* With a linear ln rho~ (one slope a everywhere) the weight is exp(-a E),
  so the chain is the canonical ensemble at beta = -a whatever a0 is: on the
  2-D open strip of two independent plaquettes <E> = 2 I1(beta)/I0(beta).
* With ln rho~ interpolating the exact two-plaquette ln rho, the energy
  histogram is flat between the ends of the table (the random walk in E the
  weight is built for)."""
import numpy as np

import oracle
from tests import exact2d


def _strip():
    g = oracle.Geom([3, 2], periodic=False)
    assert g.nplaq == 2
    return g


def test_linear_weight_is_the_canonical_ensemble_for_any_proposal_slope():
    g = _strip()
    a_t = -1.3
    for a0 in (a_t, a_t + 0.9, a_t - 0.7):
        w = oracle.MucaWeight(-2.0, 0.25, np.full(16, a_t))
        t = oracle.Lattice(g, 97, 1, 0, -2.0, 4.0, n_or=1, block=1)
        t.hot_start()
        es = oracle.muca_sweep(t, w, a0, 60000)[1000:]
        m, err = exact2d.batch_means(es)
        want = 2.0 * exact2d.bessel_ratio(-a_t)
        assert abs(m - want) < 4 * err, (a0, m, want, err)
        if a0 != a_t:
            st = t.stats()
            assert st["hb_acc"] < st["hb_tot"]     # the correction is doing work


def test_exact_inverse_density_gives_a_flat_energy_histogram():
    g = _strip()
    e0, de, n = 0.15, 0.05, 32                     # table over E in [0.15, 1.75]
    edges = e0 + de * np.arange(n + 1)
    lnr = np.log([exact2d.density_2plaq(e) for e in edges])
    a = np.diff(lnr) / de                          # exact ln rho at every edge
    w = oracle.MucaWeight(e0, de, a)
    t = oracle.Lattice(g, 4242, 2, 0, e0, n * de, n_or=1, block=1)
    t.hot_start()
    assert t.approach(10000) >= 0
    es = oracle.muca_sweep(t, w, float(np.median(a)), 200000)
    bins = np.linspace(0.3, 1.6, 14)               # inner range, away from the tails
    h, _ = np.histogram(es, bins=bins)
    frac = h / h.mean()
    # 13 bins of ~13000 correlated samples: a few % of noise; the canonical
    # density would vary by a factor ~1.5 over this range
    assert np.all(np.abs(frac - 1.0) < 0.08), frac
    # the chain walks across the table: many round trips between its ends
    lo_hit = es < 0.4
    hi_hit = es > 1.5
    trips, state = 0, None
    for l, hh in zip(lo_hit, hi_hit):
        if l and state != "lo":
            trips += state == "hi"
            state = "lo"
        elif hh and state != "hi":
            trips += state == "lo"
            state = "hi"
    assert trips > 100
