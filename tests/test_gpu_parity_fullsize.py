"""GPU path against the FP64 oracle where the full-size code paths run.

* Class-by-class updates at L = 8 and L = 12 (10 and 47 chunks of 224 links
  per class: the producer/consumer ring wraps, the consumer carries the
  running energy across chunks) and at L = 20 (the benchmark's lattices and
  launch shape, all 8 classes), with the workloads' own windows, so blocks
  are refused: every link within its float32 tolerance, every window
  decision identical except near ties (tests/gpu_helpers.py).
* A trajectory of three composite sweeps (1 heat-bath + 4 overrelaxation
  passes) stepped class by class and pass by pass from the GPU's state, every
  link compared at every step; the stepped GPU run is bit-identical to the
  free-running one, so the comparison covers the real trajectory.
* FP64 energies of the L = 20 lattices within 1e-9 relative on identical
  angles.
* The L = 4 workload exactly as configured (8 intervals x 4 replicas, dE = 4,
  50 + 100 sweeps, 20 Robbins-Monro steps) on both sides: slopes within the
  combined 3 sigma, and ln rho and the specific-heat peak reconstructed from
  each side's own chains statistically consistent.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import recon
from paper_1509_08391_gb300 import llr, workloads
from tests import gpu_helpers as gh

pytestmark = pytest.mark.gpu

TOL_E_REL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1509_08391_gb300 import build
    build.build()
    oracle.build()


def _report(name, rep):
    print("\n[parity] %s: %s" % (name, {k: (round(v, 9) if isinstance(v, float) else v)
                                        for k, v in sorted(rep.items())}))


def _lattices_of(w, L, picks):
    idx = [i for i in range(w.n_lattices) if w.L[i] == L]
    return workloads.subset(w, [idx[k] for k in picks])


@pytest.mark.parametrize("L,threads", [(8, 128), (8, 256), (8, 512), (12, 256)])
def test_multichunk_class_updates_match_oracle(L, threads):
    if L == 8:
        w = workloads.subset(workloads.l8_batch(replicas=1), [3, 17, 29])
    else:
        w = _lattices_of(workloads.uneven_batch(), 12, [10, 40])
    a = np.linspace(-1.02, -0.98, w.n_lattices)
    with llr.Batch.from_workload(w, max_approach=5000) as b:
        b.set_kernel_config(threads, True)
        b.sweep(a, 2)
        rep = gh.check_class_updates(b, w, range(w.n_lattices), a)
    _report("L=%d threads=%d" % (L, threads), rep)
    assert rep["links"] == 2 * w.n_lattices * 4 * L ** 4
    assert rep["refused"] > 0, "no window refusals: the scan was not exercised"
    assert gh.near_ties_are_rare(rep), rep


def test_l20_all_classes_match_oracle_in_the_window():
    """The benchmark's L = 20 lattices, launch shape and windows (dE = 12),
    after the approach: all 8 classes of a heat-bath and of an
    overrelaxation pass, every link."""
    w = workloads.subset(workloads.l20_critical(), [700, 1500])
    a = np.array([-1.011, -1.009])
    with llr.Batch.from_workload(w, max_approach=2000) as b:
        b.set_kernel_config(256, True)
        b.sweep(a, 2)
        rep = gh.check_class_updates(b, w, range(w.n_lattices), a)
    _report("L=20", rep)
    assert rep["links"] == 2 * w.n_lattices * 4 * 20 ** 4
    assert rep["refused"] > 0
    assert gh.near_ties_are_rare(rep), rep


def test_l20_fp64_energy_matches_oracle_on_same_angles():
    w = workloads.subset(workloads.l20_critical(), [0, 777, 2047])
    with llr.Batch.from_workload(w, max_approach=2000) as b:
        b.set_kernel_config(256, True)
        b.sweep(np.full(w.n_lattices, -1.01), 1)
        E = b.energy()
        for i in range(w.n_lattices):
            o = gh.oracle_mirror(b, w, i)
            assert abs(E[i] - o.energy()) <= TOL_E_REL * abs(E[i]), (i, E[i], o.energy())


def _check_or_pass(b, w, a, rep):
    """One whole overrelaxation pass (slab by slab, the 8 classes within a
    slab) on both sides from the GPU's state: every link within the
    propagation tolerance of or_pass_tolerance; no refusal on either side
    (the energies sit away from the window edges), and the running energy is
    left as it was on both sides (R19)."""
    trk = b.tracked_energy()
    mirrors = [gh.oracle_mirror(b, w, i, tracked=trk[i]) for i in range(w.n_lattices)]
    before = [o.links() for o in mirrors]
    st0 = b.stats()
    b.single_pass(1, a)
    st1 = b.stats()
    trk1 = b.tracked_energy()
    for i, o in enumerate(mirrors):
        s0 = o.stats()
        o.single_pass(1, a[i])
        s1 = o.stats()
        assert s1["or_acc"] - s0["or_acc"] == s1["or_tot"] - s0["or_tot"]
        assert st1["or_acc"][i] - st0["or_acc"][i] == st1["or_tot"][i] - st0["or_tot"][i]
        g = b.get_links(i).astype(np.float64)
        th1 = o.links()
        d = np.abs(gh.wrapped_diff(g, th1))
        tol, S = gh.or_pass_tolerance(w.L[i], before[i], th1, d)
        bad = np.nonzero(d > tol)[0]
        assert bad.size == 0, ("overrelaxation pass", i, int(bad[0]), float(d[bad[0]]),
                               float(tol[bad[0]]), float(S[bad[0]]))
        rep["or_links"] = rep.get("or_links", 0) + d.size
        rep["or_worst_rad"] = max(rep.get("or_worst_rad", 0.0), float(d.max()))
        # overrelaxation leaves the running energy on both sides (R19)
        assert trk1[i] == trk[i] and o.E == trk[i], (i, trk1[i], trk[i], o.E)


def test_stepped_trajectory_matches_oracle_link_by_link():
    """Three composite sweeps of the L = 4 workload: each heat-bath class and
    each whole overrelaxation pass compared link by link with the oracle from
    the GPU's state, the end of each sweep (resync, sweep counter) as its own
    launch; a second batch runs the same three sweeps free (llr_sweep) and
    must end bit-identical, links, running energies and counters."""
    w = workloads.small_l4()
    n = w.n_lattices
    a = np.linspace(-1.1, -0.9, n)
    rep = {}
    with llr.Batch.from_workload(w, max_approach=1000) as b1, \
            llr.Batch.from_workload(w, max_approach=1000) as b2:
        b1.sweep(a, 1)
        b2.sweep(a, 1)
        for _ in range(3):
            gh.check_class_updates(b1, w, range(n), a, kinds=(0,), report=rep)
            for _ in range(w.n_or):
                _check_or_pass(b1, w, a, rep)
            b1.single_pass(3)
        b2.sweep(a, 3)
        for i in range(n):
            assert np.array_equal(b1.get_links(i), b2.get_links(i)), i
            assert b1.get_sweep_counter(i) == b2.get_sweep_counter(i)
        assert np.array_equal(b1.tracked_energy(), b2.tracked_energy())
    _report("stepped trajectory L=4", rep)
    assert rep["links"] == 3 * 8 * n * 128
    assert gh.near_ties_are_rare(rep), rep


# ---------------------------------------------------------------------------
# The L = 4 workload as configured, both sides, and the reconstruction
# ---------------------------------------------------------------------------
R = 4


@pytest.fixture(scope="module")
def c0_runs():
    w = workloads.small_l4(replicas=R)
    nth, nme, n_rm = w.n_therm, w.n_meas, w.n_rm
    assert (nth, nme, n_rm) == (50, 100, 20)
    a = np.full(w.n_lattices, w.a0)
    with llr.Batch.from_workload(w, max_approach=1000) as b:
        for n in range(n_rm):
            a, _ = b.rm_step(a, nth, nme, n)
        assert np.all(b.status() == 0)
    out = oracle.batch_run(oracle.Geom([4] * 4), w.seed, w.interval_id, w.replica_id, w.E_lo,
                           w.dE, np.full(w.n_lattices, w.a0), n_or=w.n_or, block=w.block,
                           n_therm=nth, n_meas=nme, n_rm=n_rm, max_approach=1000,
                           beta_up=w.beta_up, beta_dn=w.beta_dn,
                           n_threads=min(16, os.cpu_count() or 1))
    assert np.all(out["status"] == 0)
    n_int = w.n_lattices // R
    c = np.asarray(w.E_lo[::R]) + 0.5 * w.dE[0]
    return c, a.reshape(n_int, R), np.asarray(out["a"]).reshape(n_int, R)


def _consistent(name, g, o, k=3.0):
    """Means of per-replica values g, o within k combined standard errors."""
    g, o = np.asarray(g, np.float64), np.asarray(o, np.float64)
    sig = np.sqrt(g.var(ddof=1) / g.size + o.var(ddof=1) / o.size)
    diff = abs(g.mean() - o.mean())
    print("\n[parity] %s: gpu %.6g oracle %.6g diff %.3g sigma %.3g" %
          (name, g.mean(), o.mean(), diff, sig))
    assert diff <= k * sig, (name, diff, sig)


def test_c0_slopes_agree_with_oracle_within_3_sigma(c0_runs):
    """a_k after 20 Robbins-Monro steps, replica means, within the combined
    3 sigma of the replica spreads.  The spread after n steps of eq. (2.30) is
    set by the gain 12/dE^2 and the window (Sec. 2.2, eq. (2.28)), the same for
    every interval here, so the per-side variance is pooled over the 8
    intervals (24 degrees of freedom instead of 3)."""
    c, ga, oa = c0_runs
    s2 = ga.var(axis=1, ddof=1).mean() + oa.var(axis=1, ddof=1).mean()
    sig = np.sqrt(s2 / R)
    diff = np.abs(ga.mean(axis=1) - oa.mean(axis=1))
    print("\n[parity] C0 slopes: gpu %s\n oracle %s\n diff/sigma %s" %
          (np.round(ga.mean(axis=1), 5), np.round(oa.mean(axis=1), 5), np.round(diff / sig, 2)))
    assert np.all(diff <= 3 * sig), (diff, sig)


def test_c0_reconstruction_consistent_with_oracle(c0_runs):
    """ln rho (trapezium over the centres, eqs. (2.6)/(2.7)) and the
    specific-heat peak (Sec. 3.4) reconstructed per replica from the GPU's
    chains by the GPU kernels and from the oracle's chains by the oracle's
    numpy reconstruction: the replica means agree within the combined 3
    sigma, and the peak lies inside the coupling range on both sides."""
    c, ga, oa = c0_runs
    lg = [llr.reconstruct_lnrho(c, ga[:, r])[-1] for r in range(R)]
    lo_ = [recon.lnrho_at_centres(c, oa[:, r])[-1] for r in range(R)]
    _consistent("ln rho(c_last) - ln rho(c_0)", lg, lo_)
    b_lo, b_hi = 0.6, 1.6
    pg = [llr.cv_peak(c, ga[:, r], b_lo, b_hi, 2001, 1e-10) for r in range(R)]
    po = [recon.cv_peak(c, oa[:, r], b_lo, b_hi, 2001, 1e-10) for r in range(R)]
    for (bg, _), (bo, _) in zip(pg, po):
        assert b_lo + 1e-3 < bg < b_hi - 1e-3 and b_lo + 1e-3 < bo < b_hi - 1e-3
    _consistent("beta at the C_V peak", [p[0] for p in pg], [p[0] for p in po])
    _consistent("C_V peak", [p[1] for p in pg], [p[1] for p in po])
