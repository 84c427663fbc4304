"""GPU multicanonical reweighting (Sec. 2.6, eq. (2.56)), its C_V peak and the
tunnelling count against the oracle, on seeded synthetic samples shaped like
the multicanonical runs (energies spread over the paper's L = 10 range and
beyond it, a 64-interval table of slopes near -1), at a small size, at the
benchmark's size (512 chains x 4000 thinned sweeps) and in closed form."""
import numpy as np
import pytest

import oracle
from oracle import recon
from paper_1509_08391_gb300 import llr

pytestmark = pytest.mark.gpu

SIX_V = 6.0 * 10 ** 4


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1509_08391_gb300 import build
    build.build()


def _table(n_int=64, seed=1):
    rng = np.random.default_rng(seed)
    e0, e1 = 0.59 * SIX_V, 0.687777 * SIX_V
    de = (e1 - e0) / n_int
    a = -1.0095 + 0.004 * np.sin(np.linspace(0, 3, n_int)) + 1e-4 * rng.standard_normal(n_int)
    return e0, de, a


def _samples(n, e0, de, n_int, seed=2):
    """Flat in E over the table and a little beyond it on both sides."""
    rng = np.random.default_rng(seed)
    span = n_int * de
    return rng.uniform(e0 - 0.03 * span, e0 + 1.03 * span, n)


def _oracle_lnrho(E, e0, de, a):
    w = oracle.MucaWeight(e0, de, a)
    return np.array([w.lnrho(x) for x in np.ravel(E)])


def test_reweighted_moments_match_the_oracle():
    e0, de, a = _table()
    E = _samples(150_000, e0, de, a.size)
    lr = _oracle_lnrho(E, e0, de, a)
    betas = np.linspace(1.0, 1.016, 33)
    g1, g2 = llr.muca_reweight(E, e0, de, a, betas)
    for b, x1, x2 in zip(betas, g1, g2):
        o1, o2 = recon.muca_moments(E, lr, b)
        assert x1 == pytest.approx(o1, rel=1e-12, abs=0)
        # the variance is the small difference of the two; compare it too
        assert x2 - x1 * x1 == pytest.approx(o2 - o1 * o1, rel=1e-7)


def test_reweighted_cv_peak_matches_the_oracle():
    e0, de, a = _table(seed=3)
    # two clusters of samples (the two phases) with some in between, so the
    # reweighted C_V has a clear peak
    rng = np.random.default_rng(4)
    E = np.concatenate([rng.normal(0.605 * SIX_V, 250.0, 40_000),
                        rng.normal(0.645 * SIX_V, 250.0, 40_000),
                        rng.uniform(0.6 * SIX_V, 0.65 * SIX_V, 20_000)])
    lr = _oracle_lnrho(E, e0, de, a)
    bg, cg = llr.muca_cv_peak(E, e0, de, a, 1.0, 1.016, n_grid=161, tol=1e-10)
    bo, co = recon.muca_cv_peak(E, lr, 1.0, 1.016, n_grid=161, tol=1e-10)
    assert bg == pytest.approx(bo, abs=1e-8)
    assert cg == pytest.approx(co, rel=1e-8)
    assert 1.0 < bg < 1.016


def test_two_states_in_closed_form_on_the_gpu():
    """Equal numbers of samples at E1 and E2 inside one interval of slope 0
    (ln rho~ equal at both): the reweighted C_V peaks at beta = 0 with
    (E2 - E1)^2 / 4, and <E> is E1 + (E2 - E1) / (1 + exp(-beta (E2 - E1)))."""
    e0, de, a = 0.0, 10.0, np.zeros(3)
    E = np.array([12.0, 18.0] * 64)
    b, cv = llr.muca_cv_peak(E, e0, de, a, -1.0, 1.0, n_grid=201, tol=1e-12)
    assert b == pytest.approx(0.0, abs=1e-6)
    assert cv == pytest.approx(9.0, rel=1e-10)
    betas = np.array([-0.3, 0.0, 0.2])
    e1, _ = llr.muca_reweight(E, e0, de, a, betas)
    assert np.allclose(e1, 12.0 + 6.0 / (1.0 + np.exp(-6.0 * betas)), rtol=0, atol=1e-12)


def test_reweighting_at_the_benchmark_size():
    """512 chains x 4000 thinned sweeps (the L = 12 multicanonical run's
    sample count), the launch configuration the benchmark uses."""
    e0, de, a = _table(seed=5)
    E = _samples(512 * 4000, e0, de, a.size, seed=6)
    lr = _oracle_lnrho(E, e0, de, a)
    betas = np.array([1.004, 1.0094, 1.014])
    g1, g2 = llr.muca_reweight(E, e0, de, a, betas)
    for b, x1, x2 in zip(betas, g1, g2):
        o1, o2 = recon.muca_moments(E, lr, b)
        assert x1 == pytest.approx(o1, rel=1e-12, abs=0)
        assert x2 - x1 * x1 == pytest.approx(o2 - o1 * o1, rel=1e-6)


def test_tunnellings_match_the_oracle():
    rng = np.random.default_rng(7)
    n_steps, n_chains = 3000, 96
    walk = np.cumsum(rng.normal(0.0, 1.0, (n_steps, n_chains)), axis=0)
    walk = np.round(walk)                       # integer energies: samples exactly at lo and hi
    lo, hi = -10.0, 10.0
    got = llr.muca_tunnellings(walk, lo, hi)
    ref = [recon.tunnellings(walk[:, c], lo, hi) for c in range(n_chains)]
    assert got.tolist() == ref
    assert sum(ref) > 0
    assert llr.muca_tunnellings(np.zeros((0, 5)), lo, hi).tolist() == [0] * 5


def test_bad_arguments_are_refused():
    e0, de, a = _table()
    E = _samples(10, e0, de, a.size)
    with pytest.raises(llr.LLRError):
        llr.muca_reweight(E[:0], e0, de, a, [1.0])
    with pytest.raises(llr.LLRError):
        llr.muca_reweight(E, e0, -1.0, a, [1.0])
    with pytest.raises(llr.LLRError):
        llr.muca_cv_peak(E, e0, de, a, 1.0, 1.0)
    with pytest.raises(llr.LLRError):
        llr.muca_tunnellings(np.zeros((3, 2)), 1.0, -1.0)
