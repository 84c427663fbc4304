"""Pins of the oracle's replica exchange between overlapping intervals
(Sec. 2.5): the exchange must leave the product of the two restricted
ensembles (eqs. (2.13)-(2.15)) invariant, so with exchanges every interval still
samples its own restricted density exactly, and the exchange rate is the
expectation of the Metropolis probability under that product."""
import numpy as np

import oracle
from tests import exact2d


def _strip():
    g = oracle.Geom([3, 2], periodic=False)
    assert g.nplaq == 2
    return g


def _product_swap_rate(w1, w2, a1, a2, n=4_000_000, seed=11):
    """E[1(E1, E2 in the common region) min(1, exp((a1 - a2)(E1 - E2)))] with
    E1, E2 independent exact samples of the two restricted two-plaquette
    densities (plaquette angles uniform, Sec. 3.1; rejection sampling)."""
    rng = np.random.default_rng(seed)

    def draw(lo, hi, a):
        p = rng.uniform(0.0, np.pi, size=(n, 2))
        E = np.cos(p).sum(axis=1)
        E = E[(E >= lo) & (E <= hi)]
        bound = max(-a * lo, -a * hi)
        keep = rng.uniform(size=E.size) < np.exp(-a * E - bound)
        return E[keep]

    E1, E2 = draw(*w1, a1), draw(*w2, a2)
    m = min(E1.size, E2.size)
    E1, E2 = E1[:m], E2[:m]
    lo, hi = max(w1[0], w2[0]), min(w1[1], w2[1])
    both = (E1 >= lo) & (E1 <= hi) & (E2 >= lo) & (E2 <= hi)
    p = np.where(both, np.minimum(1.0, np.exp((a1 - a2) * (E1 - E2))), 0.0)
    return float(p.mean()), float(p.std() / np.sqrt(m))


def test_exchange_keeps_each_restricted_ensemble_exact():
    """Two overlapping windows on the 2-plaquette strip at very different
    slopes, one composite sweep of each chain and one exchange attempt per
    round: each window's mean energy equals the quadrature of eq. (2.15), and the
    exchange rate equals its expectation under the product ensemble."""
    g = _strip()
    w1, w2 = (0.3, 0.9), (0.6, 1.2)
    a = np.array([-4.0, 4.0])
    lats = []
    for k, (lo, hi) in enumerate((w1, w2)):
        t = oracle.Lattice(g, 2468, k, 0, lo, hi - lo, n_or=1, block=1)
        t.hot_start()
        assert t.approach(10000) >= 0
        lats.append(t)
    n_rounds = 40000
    es = np.zeros((n_rounds, 2))
    acc = np.zeros(n_rounds)
    for r in range(n_rounds):
        for k, t in enumerate(lats):
            t.sweep(a[k], 1)
        acc[r] = oracle.replica_exchange(lats, [0, 1], a, r)[0]
        es[r] = [lats[0].E, lats[1].E]
    assert np.all(es[:, 0] >= w1[0] - 1e-12) and np.all(es[:, 0] <= w1[1] + 1e-12)
    assert np.all(es[:, 1] >= w2[0] - 1e-12) and np.all(es[:, 1] <= w2[1] + 1e-12)
    for k, (lo, hi) in enumerate((w1, w2)):
        m, err = exact2d.batch_means(es[:, k])
        assert abs(m - exact2d.restricted_mean_2plaq(lo, hi, a[k])) < 4 * err
    rate, rate_err = exact2d.batch_means(acc)
    want, want_err = _product_swap_rate(w1, w2, a[0], a[1])
    assert 0.05 < want < 0.95   # the exchange is doing real work here
    assert abs(rate - want) < 4 * np.hypot(rate_err, want_err)


def test_exchange_outside_the_common_region_is_never_taken():
    """A configuration outside the other window is never exchanged, whatever
    the slopes, and an exchange swaps the links and energies exactly."""
    g = _strip()
    t1 = oracle.Lattice(g, 1357, 0, 0, 0.3, 0.6, n_or=1)
    t2 = oracle.Lattice(g, 1357, 1, 0, 0.6, 0.6, n_or=1)
    for t in (t1, t2):
        t.hot_start()
        assert t.approach(10000) >= 0
    seen_swap = seen_block = False
    for r in range(4000):
        t1.sweep(0.0, 1)
        t2.sweep(0.0, 1)
        th1, th2, E1, E2 = t1.links(), t2.links(), t1.E, t2.E
        inside = 0.6 <= E1 <= 0.9 and 0.6 <= E2 <= 0.9
        acc = oracle.replica_exchange([t1, t2], [0, 1], [5.0, -5.0], r)[0]
        if not inside:
            assert not acc
            seen_block = True
        if acc:
            seen_swap = True
            assert np.array_equal(t1.links(), th2) and np.array_equal(t2.links(), th1)
            assert t1.E == E2 and t2.E == E1
        else:
            assert np.array_equal(t1.links(), th1) and t1.E == E1
    assert seen_swap and seen_block
