"""Pins of the FP64 oracle against results fixed by the paper and by mathematics.

Each test is chosen so that a plausible mistake in the oracle (a dropped
staple term, a wrong sign or index, a transposed link in a plaquette, a wrong
Robbins-Monro sign or offset, a mis-drawn von Mises variate, a window that is
not closed) fails at least one of them.
"""
import os

import numpy as np
import pytest
from scipy import stats

import oracle
from tests import exact2d

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_uniform_is_open_and_exact():
    assert oracle.uniform(0) == 2.0 ** -24
    assert oracle.uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert oracle.uniform(0x80000000) == 0.5 + 2.0 ** -24
    # every value is an odd multiple of 2^-24 -> exact in float32 too
    for w in [1, 12345678, 0xDEADBEEF]:
        u = oracle.uniform(w)
        assert np.float32(u) == u


# ---------------------------------------------------------------- energy
def _lat(L=4, d=4, periodic=True, **kw):
    g = oracle.Geom([L] * d, periodic)
    t = oracle.Lattice(g, kw.pop("seed", 11), kw.pop("iid", 0), kw.pop("rid", 0),
                       kw.pop("E_lo", -1e9), kw.pop("dE", 2e9), **kw)
    return g, t


@pytest.mark.parametrize("L", [2, 4, 6])
def test_cold_start_energy_is_6V(L):
    g, t = _lat(L)
    t.set_links(np.zeros(g.nslot))
    assert g.nplaq == 6 * L ** 4
    assert t.energy() == 6 * L ** 4


@pytest.mark.parametrize("L", [4, 6])
def test_pi_flux_energy_is_minus_6V(L):
    """theta_mu(x) = pi * sum_{i<mu} x_i makes every plaquette angle pi."""
    g, t = _lat(L)
    V = L ** 4
    th = np.zeros(g.nslot)
    for s in range(V):
        x = [(s // L ** i) % L for i in range(4)]
        for mu in range(4):
            th[mu * V + s] = np.pi * sum(x[:mu])
    t.set_links(th)
    assert abs(t.energy() + 6 * V) < 1e-9


def _gauge_transform(th, lam, L):
    V = L ** 4
    out = th.copy()
    for s in range(V):
        x = [(s // L ** i) % L for i in range(4)]
        for mu in range(4):
            y = list(x)
            y[mu] = (y[mu] + 1) % L
            sp = sum(y[i] * L ** i for i in range(4))
            out[mu * V + s] = th[mu * V + s] - lam[s] + lam[sp]
    return out


def test_gauge_invariance_of_energy_and_staples():
    """U_mu(x) -> conj(Lambda(x)) U_mu(x) Lambda(x+mu) leaves E and |S| unchanged (Sec. 3.1)."""
    L = 4
    g, t = _lat(L)
    rng = np.random.default_rng(5)
    th = rng.uniform(-np.pi, np.pi, g.nslot)
    t.set_links(th)
    E0 = t.energy()
    S0 = np.array([t.staple(l)[0] for l in range(0, g.nslot, 7)])
    lam = rng.uniform(-np.pi, np.pi, L ** 4)
    t.set_links(_gauge_transform(th, lam, L))
    assert abs(t.energy() - E0) < 1e-11
    S1 = np.array([t.staple(l)[0] for l in range(0, g.nslot, 7)])
    assert np.max(np.abs(S1 - S0)) < 1e-12


def test_staple_gives_exact_local_energy_change():
    """E(theta_l + delta) - E(theta_l) = |S| (cos(theta_l + delta + alpha) - cos(theta_l + alpha))."""
    g, t = _lat(4)
    rng = np.random.default_rng(6)
    th = rng.uniform(-np.pi, np.pi, g.nslot)
    for l in [0, 17, 300, 511, 777, 1023]:
        t.set_links(th)
        E0 = t.energy()
        S, alpha = t.staple(l)
        th2 = th.copy()
        th2[l] += 0.7
        t.set_links(th2)
        pred = S * (np.cos(th[l] + 0.7 + alpha) - np.cos(th[l] + alpha))
        assert abs((t.energy() - E0) - pred) < 1e-11


def test_overrelaxation_preserves_energy_and_is_an_involution():
    g, t = _lat(4)
    rng = np.random.default_rng(7)
    th = rng.uniform(-np.pi, np.pi, g.nslot)
    t.set_links(th)
    E0 = t.energy()
    for cls in range(8):
        before = t.links()
        t.class_pass(cls, 1)
        assert abs(t.energy() - E0) < 1e-11
        assert abs(t.E - E0) < 1e-11
        t.class_pass(cls, 1)  # reflect again with the same staples -> identity
        d = np.angle(np.exp(1j * (t.links() - before)))
        assert np.max(np.abs(d)) < 1e-12
    t.single_pass(1)
    assert abs(t.energy() - E0) < 1e-10


def test_tracked_energy_equals_fresh_sum():
    L = 4
    six = 6 * L ** 4
    g, t = _lat(L, E_lo=0.6 * six, dE=4.0)
    t.hot_start()
    assert t.approach(1000) >= 0
    for _ in range(20):
        t.single_pass(0, -1.0)
        t.single_pass(1)
        assert abs(t.E - t.energy()) < 1e-9
    t.sweep(-1.0, 5)
    assert t.stats()["max_drift"] < 1e-9


# ---------------------------------------------------------------- sampler
@pytest.mark.parametrize("kappa", [0.05, 0.8, 3.0, 11.0, -2.5])
def test_von_mises_sampler_distribution(kappa):
    key = [0x1234, 0x5678]
    n = 20000
    xs = np.array([oracle.vonmises(kappa, key, i, 3, 0)[0] for i in range(n)])
    assert np.all(xs >= -np.pi) and np.all(xs < np.pi)
    if kappa > 0:
        ks = stats.kstest(xs, stats.vonmises(kappa, loc=0.0).cdf)
    else:
        ks = stats.kstest(np.mod(xs, 2 * np.pi), stats.vonmises(-kappa, loc=np.pi).cdf)
    assert ks.pvalue > 1e-4
    m = np.cos(xs).mean()
    exact = np.sign(kappa) * exact2d.bessel_ratio(abs(kappa))
    assert abs(m - exact) < 5 * np.cos(xs).std() / np.sqrt(n)


# ---------------------------------------------------------------- 2D exact
def test_unrestricted_heat_bath_2d_open_gives_I1_over_I0():
    """2-D open lattice: independent plaquettes, <cos p> = I1(beta)/I0(beta)."""
    beta = 1.3
    g = oracle.Geom([6, 6], periodic=False)
    t = oracle.Lattice(g, 99, 0, 0, -1e9, 2e9, n_or=1)
    t.hot_start()
    t.sweep(-beta, 100)
    es = []
    for _ in range(4000):
        t.sweep(-beta, 1)
        es.append(t.E / g.nplaq)
    m, err = exact2d.batch_means(es)
    assert abs(m - exact2d.bessel_ratio(beta)) < 4 * err + 1e-12


def test_three_plaquette_quadrature_is_self_consistent():
    """The 3-plaquette quadrature reduces to known limits: the unrestricted mean
    at weight exp(-aE) is 3 I1(-a)/I0(-a), and a window covering everything
    gives the same."""
    from scipy import special
    a = -0.8
    m = exact2d.restricted_moments_3plaq(-3.5, 3.5, a, 1)
    assert abs(m[1] / m[0] - 3 * special.i1(-a) / special.i0(-a)) < 1e-6
    assert abs(m[0] - special.i0(-a) ** 3) < 1e-6


def test_three_plaquette_blocks_of_two_are_exact():
    """4x2 open strip (3 plaquettes): a slab of one class holds two links, so
    with B = 2 the window decides two-link blocks; the chain still reproduces
    the restricted mean of eq. (2.15)."""
    lo, hi, a = 0.9, 1.6, -1.0
    g = oracle.Geom([4, 2], periodic=False)
    assert g.nplaq == 3
    t = oracle.Lattice(g, 4321, 2, 0, lo, hi - lo, n_or=1, block=2)
    t.hot_start()
    assert t.approach(10000) >= 0
    es = []
    for _ in range(40000):
        t.sweep(a, 1)
        es.append(t.E)
    es = np.array(es)
    assert np.all(es >= lo - 1e-12) and np.all(es <= hi + 1e-12)
    m, err = exact2d.batch_means(es)
    assert abs(m - exact2d.restricted_mean_3plaq(lo, hi, a)) < 4 * err


@pytest.mark.parametrize("block,a", [(1, -1.0), (2, 2.0), (1, 4.0)])
def test_two_plaquette_restricted_mean_is_exact(block, a):
    """2x1 plaquette strip (7 links): the restricted chain reproduces eq. (2.15)."""
    lo, hi = 0.5, 1.1
    g = oracle.Geom([3, 2], periodic=False)
    assert g.nplaq == 2 and int(g.exists().sum()) == 7
    t = oracle.Lattice(g, 1234, 5, block, lo, hi - lo, n_or=1, block=block)
    t.hot_start()
    assert t.approach(10000) >= 0
    es = []
    for _ in range(40000):
        t.sweep(a, 1)
        es.append(t.E)
    es = np.array(es)
    assert np.all(es >= lo - 1e-12) and np.all(es <= hi + 1e-12)
    m, err = exact2d.batch_means(es)
    exact = exact2d.restricted_mean_2plaq(lo, hi, a)
    assert abs(m - exact) < 4 * err


def test_two_plaquette_robbins_monro_converges_to_root():
    """Algorithm 1 with eq. (2.30) on the strip converges to the root of eq. (2.17)."""
    lo, hi = 0.5, 1.1
    root = exact2d.llr_root_2plaq(lo, hi)
    g = oracle.Geom([3, 2], periodic=False)
    R = 16
    out = oracle.batch_run(g, 777, [0] * R, list(range(R)), [lo] * R, [hi - lo] * R,
                           [-1.0] * R, n_or=1, block=1, n_therm=5, n_meas=100, n_rm=300,
                           n_threads=min(8, os.cpu_count() or 1))
    assert np.all(out["status"] == 0)
    a = out["a"]
    err = a.std(ddof=1) / np.sqrt(R)
    assert abs(a.mean() - root) < 4 * err + 2e-3
    # a wrong sign or a dropped 1/(n+1) would leave the replicas far apart or far away
    assert a.std(ddof=1) < 0.2


@pytest.mark.parametrize("side", ["below", "above"])
def test_approach_reaches_window_and_stays(side):
    L = 4
    six = 6 * L ** 4
    E_lo = 0.62 * six if side == "below" else -0.05 * six
    g, t = _lat(L, seed=3)   # unrestricted first
    t.hot_start()
    if side == "above":
        t.sweep(-1.5, 5)  # move E far above the window first
        assert t.E > E_lo + 4.0
    t.set_window(E_lo, 4.0)
    n = t.approach(1000)
    assert n > 0
    for _ in range(10):
        t.sweep(-1.0, 1)
        assert E_lo <= t.E <= E_lo + 4.0


def test_robbins_monro_step_matches_eq_kk21_on_the_exact_mean():
    """One Robbins-Monro step from a = root + 0.5 on the 2-plaquette strip, the
    chain equilibrated at that a first: averaged over replicas, the step equals
    12 (<<E>>(a) - E_lo - dE/2) / (dE^2 (n + 1)) with <<E>>(a) from the
    quadrature of eq. (2.15), for n = 0 and n = 3.  A wrong gain constant, sign
    or step offset moves the mean step by a factor of 2 or more."""
    lo, hi = 0.5, 1.1
    dE = hi - lo
    root = exact2d.llr_root_2plaq(lo, hi)
    a0 = root + 0.5
    exact_mean = exact2d.restricted_mean_2plaq(lo, hi, a0)
    g = oracle.Geom([3, 2], periodic=False)
    for n in (0, 3):
        want = 12.0 * (exact_mean - lo - 0.5 * dE) / (dE * dE * (n + 1))
        steps = []
        for r in range(64):
            t = oracle.Lattice(g, 2024, 3, r, lo, dE, n_or=1, block=1)
            t.hot_start()
            assert t.approach(10000) >= 0
            a1, _ = t.rm_step(a0, 200, 1600, n)
            steps.append(a1 - a0)
        steps = np.array(steps)
        err = steps.std(ddof=1) / np.sqrt(steps.size)
        assert abs(steps.mean() - want) < 4 * err + 0.02 * abs(want), (n, steps.mean(), want, err)
        assert 4 * err < 0.25 * abs(want)        # resolves a factor-2 error in the gain


def test_robbins_monro_spread_follows_the_asymptotic_variance():
    """The spread of a_n across independent replicas (Sec. 2.4): for the
    iteration a <- a + c <<dE>> / (n + 1) with c = 12 / dE^2, near the root
    <<dE>> has slope -M' in a (M' the window variance of E at the root, by
    quadrature of eq. (2.15)) and per-step noise sigma^2 (measured at the
    root), so Var(a_n) -> c^2 sigma^2 / ((2 c M' - 1) n).  Checked on the
    2-plaquette strip at n = 100 and 400 with 128 replicas: both within the
    sampling error of a variance (measured ratios ~1.05 and ~0.93), and the 1/n
    decay between them.  A gain without the 1/(n+1) leaves the spread constant
    and fails the decay; the gain constant itself is pinned by the one-step
    test above (a factor 2 moves this variance by only ~1/3)."""
    lo, hi = 0.5, 1.1
    dE = hi - lo
    c = 12.0 / (dE * dE)
    root = exact2d.llr_root_2plaq(lo, hi)
    z, s1, s2 = exact2d.restricted_moments_2plaq(lo, hi, root)[:3]
    Mp = s2 / z - (s1 / z) ** 2
    assert 2.0 * c * Mp - 1.0 > 0.2          # the regime where the 1/n law holds
    g = oracle.Geom([3, 2], periodic=False)
    n_therm, n_meas = 5, 50
    # sigma^2: variance of one step's <<dE>> estimate at a = root
    xi = []
    for r in range(64):
        t = oracle.Lattice(g, 4242, 5, r, lo, dE, n_or=1, block=1)
        t.hot_start()
        assert t.approach(10000) >= 0
        for k in range(40):
            a1, m = t.rm_step(root, n_therm, n_meas, 10 ** 9)    # a huge n: a stays put
            xi.append(m)
    sigma2 = float(np.var(xi, ddof=1))
    v_inf = c * c * sigma2 / (2.0 * c * Mp - 1.0)
    R = 128
    var = {}
    for n_rm in (100, 400):
        out = oracle.batch_run(g, 9090, [0] * R, list(range(R)), [lo] * R, [dE] * R,
                               [root] * R, n_or=1, block=1, n_therm=n_therm, n_meas=n_meas,
                               n_rm=n_rm, n_threads=min(8, os.cpu_count() or 1))
        assert np.all(out["status"] == 0)
        var[n_rm] = float(np.var(out["a"], ddof=1))
        # a sample variance of R values has relative sd sqrt(2 / (R - 1)) = 0.125
        ratio = var[n_rm] / (v_inf / n_rm)
        assert 0.6 < ratio < 1.5, (n_rm, ratio)
    assert 0.15 < var[400] / var[100] < 0.45


def test_strong_coupling_slope_in_four_dimensions():
    """At small E/6V (strong coupling) the 4-D plaquettes are nearly
    independent: <cos theta_P>(beta) = I1(beta)/I0(beta) up to O(u^5)
    corrections (u = I1/I0, 4e-5 at u = 0.1), so the slope of ln rho is
    a(E) = -beta(E) with I1(beta)/I0(beta) = E/6V (appendix, the cumulant
    form of a_k), up to O(1/V).  Algorithm 1 on the 4^4 lattice at
    E/6V = 0.05 and 0.10 must land there within its statistical error plus
    2e-3 (those corrections); a flipped sign, a factor 2 in E or the 1 - cos
    convention fail it by many errors.  The pi-flux map E -> -E (which the
    configuration pins check) makes rho(E) = rho(-E), so the slope at
    E/6V = -0.05 is +beta(0.05): the mirror image at the level of Algorithm 1."""
    from scipy import optimize, special
    L, dE, R = 4, 4.0, 4
    six_v = 6 * L ** 4
    es = (-0.05, 0.05, 0.10)
    g = oracle.Geom([L] * 4)
    lo = [e * six_v - dE / 2 for e in es for _ in range(R)]
    iid = [k for k in range(len(es)) for _ in range(R)]
    rid = [r for _ in es for r in range(R)]
    out = oracle.batch_run(g, 555, iid, rid, lo, [dE] * len(lo), [0.0] * len(lo), n_or=4,
                           block=1, n_therm=10, n_meas=50, n_rm=100,
                           n_threads=min(8, os.cpu_count() or 1))
    assert np.all(out["status"] == 0)
    a = out["a"].reshape(len(es), R)
    for k, e in enumerate(es):
        beta = optimize.brentq(lambda b: special.i1(b) / special.i0(b) - abs(e), 1e-6, 5.0)
        want = -beta if e > 0 else beta
        err = a[k].std(ddof=1) / np.sqrt(R)
        assert abs(a[k].mean() - want) < 4 * err + 2e-3, (e, a[k].mean(), want, err)
        assert err < 0.25 * beta          # resolves a factor 2 in the slope
    # the mirror pair directly
    err2 = np.hypot(a[0].std(ddof=1), a[1].std(ddof=1)) / np.sqrt(R)
    assert abs(a[0].mean() + a[1].mean()) < 4 * err2 + 2e-3
