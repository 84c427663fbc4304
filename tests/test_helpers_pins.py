"""The GPU tests' helpers pinned against the oracle (CPU only): the numpy
staple table, the overrelaxation update order and the class order that the
per-link tolerances are built from, and the sampler-attempt trace."""
import numpy as np
import pytest

import oracle
from tests import gpu_helpers as gh


@pytest.fixture(scope="module")
def lat4():
    g = oracle.Geom([4] * 4)
    o = oracle.Lattice(g, 7, 3, 1, 0.0, 1.0)
    o.hot_start()
    return g, o


def test_numpy_staples_match_oracle(lat4):
    g, o = lat4
    th = o.links()
    S_abs, alpha = gh.staples(th, 4)
    S_o = o.staple_moduli()
    assert np.allclose(S_abs, S_o, atol=1e-12, rtol=0)
    for l in range(0, th.size, 37):
        m, al = o.staple(l)
        assert abs(m - S_abs[l]) < 1e-12
        assert abs(gh.wrapped_diff(al, alpha[l])) < 1e-10
    sub = np.array([5, 300, 777, 1023])
    s2, a2 = gh.staples(th, 4, sub)
    assert np.array_equal(s2, S_abs[sub]) and np.array_equal(a2, alpha[sub])


def test_class_order_matches_oracle(lat4):
    g, o = lat4
    th = o.links()
    for cls in range(8):
        o2 = oracle.Lattice(g, 7, 3, 1, -1e9, 2e9)
        o2.set_links(th)
        tr = o2.class_trace(cls, 1, 0.0)
        assert np.array_equal(tr["th_old"], th[gh.class_links(4, cls)])


def test_overrelaxation_order_matches_oracle(lat4):
    """Each link's reflection, recomputed from the state at its update time
    (neighbours earlier in or_update_key at their new angles), reproduces the
    oracle's whole overrelaxation pass; a wrong order moves links by O(1)."""
    g, o = lat4
    th0 = o.links()
    o2 = oracle.Lattice(g, 7, 3, 1, -1e9, 2e9)
    o2.set_links(th0)
    o2.single_pass(1, 0.0)
    th1 = o2.links()
    nbr = gh.neighbours(4)
    key = gh.or_update_key(4)
    earlier = key[nbr] < key[:, None]
    vals = np.where(earlier, th1[nbr], th0[nbr])
    _, alpha = gh.staples(None, 4, vals=vals)
    refl = np.angle(np.exp(1j * (-th0 - 2 * alpha)))
    assert np.max(np.abs(gh.wrapped_diff(refl, th1))) < 1e-9
    # the propagation tolerance of identical passes is the bare one
    tol, S = gh.or_pass_tolerance(4, th0, th1, np.zeros_like(th0))
    assert np.allclose(tol, gh.TOL_RAD + 2 * gh.COND_ABS / S)


def test_sampler_attempt_trace_matches_the_sampler():
    key = [123, 456]
    for kappa in (0.3, 1.7, -2.5, 6.0):
        for link in range(20):
            X, att = oracle.vonmises(kappa, key, link, 5, 0)
            Xs, m1, m2 = oracle.vonmises_attempts(kappa, key, link, 5, 0, n_max=att + 2)
            taken = (m1 > 0) | (m2 >= 0)
            j = int(np.argmax(taken))
            assert j == att - 1 and Xs[j] == X
            # the oracle's own variate is never a near tie of itself
            assert not gh.sampler_near_tie(key, link, 5, kappa, X, 1e-9)


def _clone(g, w, th, E, sweep):
    o = oracle.Lattice(g, w.seed, w.interval_id[0], w.replica_id[0], w.E_lo[0], w.dE[0])
    o.set_links(th)
    o.E = E
    o.sweep_counter = sweep
    return o


def test_class_checker_accepts_the_oracle_and_rejects_planted_mistakes():
    """compare_class fed the oracle's own class update (rounded to float32)
    passes with no near tie; a link moved by 1e-3 rad, or a taken proposal
    replaced by its old angle away from the window edges, fails it."""
    from paper_1509_08391_gb300 import workloads
    w = workloads.small_l4()
    g = oracle.Geom([4] * 4)
    base = _clone(g, w, np.zeros(1024), 0.0, 0)
    base.hot_start()
    assert base.approach(1000) >= 0
    base.sweep(-1.0, 1)
    th, E0, sw = base.links(), base.E, base.sweep_counter
    for kind in (0, 1):
        for cls in (0, 5):
            tr = _clone(g, w, th, E0, sw).class_trace(cls, kind, -1.0)
            o2 = _clone(g, w, th, E0, sw)
            o2.class_pass(cls, kind, -1.0)
            gl = o2.links().astype(np.float32)
            order = gh.class_links(4, cls)
            S, al = gh.staples(th, 4, order)
            rep = gh.compare_class(w, 0, kind, -1.0, cls, gl, tr, S, al, sw, E0)
            assert rep["links"] == 128 and rep.get("window_ties", 0) == 0
            bad = gl.copy()
            bad[order[10]] += 1e-3
            with pytest.raises(AssertionError):
                gh.compare_class(w, 0, kind, -1.0, cls, bad, tr, S, al, sw, E0)
            if kind == 0:
                lo, hi = w.E_lo[0], w.E_lo[0] + w.dE[0]
                cand = np.asarray(tr["E_before"]) + np.asarray(tr["dE"])
                far = np.minimum.reduce([np.abs(cand - lo), np.abs(cand - hi),
                                         np.abs(np.asarray(tr["E_before"]) - lo),
                                         np.abs(np.asarray(tr["E_before"]) - hi)]) > 0.05
                moved = np.abs(gh.wrapped_diff(tr["th_prop"], tr["th_old"])) > 1e-2
                k = int(np.nonzero(far & moved & np.asarray(tr["accepted"]))[0][0])
                flipped = gl.copy()
                flipped[order[k]] = np.float32(tr["th_old"][k])
                with pytest.raises(AssertionError):
                    gh.compare_class(w, 0, kind, -1.0, cls, flipped, tr, S, al, sw, E0)
