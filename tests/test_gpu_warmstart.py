"""What the learned warm start gains over the method without it (small volumes).

Training data are the method's own slopes at L = 8 ... 16 from a short
uneven-batch run over E/6V in [0.50, 0.75], across the transition; the
network predicts the slopes at L = 20 and starts the Robbins-Monro iteration
there with the gain offset n0.  Compared with the naive start a = -1, n0 = 0
(Sec. 2.4 allows either): the predicted start is closer to the long
reference run, it stays closer over the first steps, and the warm-started
slopes still agree with the reference within 3 sigma.  Near the transition
alone (E/6V around 0.6-0.66) the slopes are all close to -1, so there the
naive start is itself within ~0.01-0.02 and the comparison says little; the
wider range is where a start matters.
"""
import numpy as np
import pytest

from paper_1509_08391_gb300 import warmstart, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1509_08391_gb300 import build
    build.build()


def test_warm_start_beats_naive_start_at_L20():
    rng = dict(e_lo=0.50, e_hi=0.75)
    data = warmstart.training_set(n_int=12, replicas=2, n_rm=30, n_therm=2, n_meas=6, **rng)
    assert np.all(np.isfinite(data["a"]))
    net, eps, loss = warmstart.fit_network(data, epochs=2000)
    assert eps < 0.05
    target = workloads.warm_start_targets(20, replicas=4, n_int=8, **rng)
    n_rm = 16
    res = warmstart.compare(target, net, eps, n_rm, 2, 6)
    net.close()
    assert np.mean(res.agree_warm) >= 0.75      # converged slopes agree with the reference
    # distance to the reference: the predicted start is closer than a = -1, and
    # the warm-started iteration stays ahead over the first steps
    assert res.err_warm[0] < res.err_naive[0]
    assert np.mean(res.err_warm[:6]) < np.mean(res.err_naive[:6])
    warm = [s for s in res.warm_steps if s is not None]
    naive = [s for s in res.naive_steps if s is not None]
    assert len(warm) >= len(naive)
    if warm and naive:
        assert np.median(warm) <= np.median(naive)


def test_learned_start_gains_at_the_top_of_the_c4_range_at_L20():
    """The learned start as configured for C4: the network is trained on the
    method's own slopes at L = 8 ... 16 over E/6V in [0.58, 0.68] and starts
    the Robbins-Monro iteration at L = 20 (R = 4, dE = 50).  Tested on the top
    of that range (E/6V in [0.655, 0.68], 8 intervals), where the slope has
    moved away from the naive a = -1 (a_ref ~ -1.02): the learned start is
    closer to the reference run and the iteration stays closer over its first
    steps.  The full measurement (128 intervals at L = 20 and L = 24) also
    shows where it does not gain: in the middle of the range, where
    a ~ -1.00 ... -1.01, a = -1 is as close, and at L = 24 the network
    extrapolates worse than a = -1."""
    data = warmstart.training_set(n_int=24, replicas=2, n_rm=40, n_therm=2, n_meas=8)
    net, eps, loss = warmstart.fit_network(data)
    target = workloads.warm_start_targets(20, replicas=4, n_int=8, e_lo=0.655, e_hi=0.68)
    warm, naive, ref_a, ref_err, n0 = warmstart.converge_arms(target, net, eps, 20, 2, 8)
    net.close()
    print("\n[c4 top] start error learned %.4f naive %.4f; mean over 6 steps %.4f / %.4f"
          % (warm.err_curve[0], naive.err_curve[0], np.mean(warm.err_curve[:6]),
             np.mean(naive.err_curve[:6])))
    assert np.all(np.isfinite(ref_a)) and np.mean(ref_a) < -1.01
    assert warm.err_curve[0] < 0.6 * naive.err_curve[0]
    assert np.mean(warm.err_curve[:6]) < np.mean(naive.err_curve[:6])
