"""GPU path (CUDA library through the C ABI) against the FP64 oracle at L = 4.

Tolerances (tests/gpu_helpers.py): every link of a class update within
2e-5 rad + c 4e-6/|S| of the oracle from an identical state (c = 1 heat-bath,
2 overrelaxation), every link of a whole overrelaxation pass within the same
bound plus the propagated deviations of its earlier-updated neighbours;
window decisions identical except near ties; FP64 energies within 1e-9
relative on identical angles.  The full-size cases, the stepped trajectory
and the Robbins-Monro statistics are in test_gpu_parity_fullsize.py.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import recon
from paper_1509_08391_gb300 import llr, workloads
from tests.gpu_helpers import check_class_updates, near_ties_are_rare, oracle_mirror
from tests.test_gpu_parity_fullsize import _check_or_pass

pytestmark = pytest.mark.gpu

TOL_E_REL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1509_08391_gb300 import build
    build.build()
    oracle.build()


def _batch(w, **kw):
    return llr.Batch.from_workload(w, **kw)


def test_hot_start_is_bit_identical_to_oracle():
    w = workloads.small_l4()
    with _batch(w, max_approach=0) as b:
        g = oracle.Geom([4] * 4)
        for i in range(w.n_lattices):
            o = oracle.Lattice(g, w.seed, w.interval_id[i], w.replica_id[i], w.E_lo[i], w.dE[i])
            o.hot_start()
            assert np.array_equal(b.get_links(i), o.links().astype(np.float32))


@pytest.mark.parametrize("L", [4, 6, 8])
def test_fp64_energy_matches_oracle_on_same_angles(L):
    w = workloads.Workload("e", [L] * 3, [0.0] * 3, [1.0] * 3, [0, 1, 2], [0, 0, 0], 42)
    with _batch(w, max_approach=0) as b:
        b.sweep(np.full(3, -1.0), 2)    # unrestricted-ish: window far away, dist rule
        E = b.energy()
        for i in range(3):
            o = oracle_mirror(b, w, i)
            assert abs(E[i] - o.energy()) <= TOL_E_REL * max(1.0, abs(E[i]))


def test_tracked_energy_close_to_fresh():
    w = workloads.small_l4()
    with _batch(w, max_approach=1000) as b:
        b.sweep(np.full(w.n_lattices, -1.0), 5)
        trk, fresh = b.tracked_energy(), b.energy()
        assert np.max(np.abs(trk - fresh)) < 1e-4
        st = b.stats()
        assert np.all(st["max_drift"] < 1e-3)
        assert np.all(st["status"] == 0)


def test_running_energy_does_not_drift_over_heat_bath_passes():
    """The window decisions of a heat-bath pass use the running energy (fresh
    energy at the last resync plus the accepted dE in float32); over one pass
    it must follow the FP64 energy of the links without a systematic drift,
    or the window the chain enforces is shifted against the one the
    measurement of eq. (2.16) assumes, and every a_k with it.  256 L = 8
    lattices in their windows, 8 heat-bath passes each: the mean drift per pass
    is bounded far below the -4.8e-4 a per-move bias of -3.5e-8 produced."""
    w = workloads.subset(workloads.paper_volume_study(8, replicas=1), range(0, 512, 2))
    a = np.full(w.n_lattices, -1.007)
    drift = []
    with _batch(w, max_approach=5000) as b:
        b.sweep(a, 4)
        for _ in range(8):
            b.sweep(a, 1)
            t0, f0 = b.tracked_energy(), b.energy()
            b.single_pass(0, a)
            t1, f1 = b.tracked_energy(), b.energy()
            drift.append((t1 - f1) - (t0 - f0))
    drift = np.concatenate(drift)
    err = drift.std() / np.sqrt(drift.size)
    assert abs(drift.mean()) < 2e-5 + 5 * err, (drift.mean(), err)


@pytest.mark.parametrize("block", [1, 4])
def test_each_class_update_matches_oracle_link_by_link(block):
    """One checkerboard class at a time (heat-bath, then overrelaxation) from an
    identical state: every link within 2e-5 rad plus its FP32 conditioning
    term, and the same window decisions."""
    w = workloads.small_l4()
    w.block = block
    a = np.linspace(-1.1, -0.9, w.n_lattices)
    with _batch(w, max_approach=1000) as b:
        b.sweep(a, 1)
        rep = check_class_updates(b, w, range(w.n_lattices), a)
    assert rep["links"] == 2 * w.n_lattices * 1024 and rep["refused"] > 0
    assert near_ties_are_rare(rep), rep


def test_class_updates_match_oracle_at_zero_and_positive_slope():
    """The sampler's other branches: a = 0 (kappa = 0, uniform proposal) and
    a > 0 (kappa < 0, X -> X + pi), one class at a time from an identical state."""
    w = workloads.small_l4()
    a = np.linspace(0.0, 1.2, w.n_lattices)
    with _batch(w, max_approach=1000) as b:
        b.sweep(np.full(w.n_lattices, -1.0), 1)
        rep = check_class_updates(b, w, range(w.n_lattices), a, kinds=(0,))
    assert rep["links"] == w.n_lattices * 1024
    assert near_ties_are_rare(rep), rep


def test_full_overrelaxation_pass_matches_oracle_link_by_link():
    """Two whole overrelaxation passes (slab by slab of x3; in a slab the 8
    classes mu = 0..3, parity 0, 1 in order), each from the GPU's state: every
    link within its tolerance, including the float32 deviations of the
    neighbours updated before it in the same pass (any other order of the
    groups moves links by O(1)); no refusals, and the running energies agree."""
    w = workloads.small_l4()
    a = np.full(w.n_lattices, -1.0)
    rep = {}
    with _batch(w, max_approach=1000) as b:
        b.sweep(a, 1)
        for _ in range(2):
            _check_or_pass(b, w, a, rep)
    assert rep["or_links"] == 2 * w.n_lattices * 1024


def _oracle_composite_sweep(o, a, n_or, lo, hi):
    """One composite sweep of the oracle lattice, heat-bath pass class by class
    with its decision trace.  Returns the smallest distance of a heat-bath
    candidate energy to a window edge (how close the closest call was)."""
    margin = np.inf
    for cls in range(8):
        tr = o.class_trace(cls, 0, a)
        cand = np.asarray(tr["E_before"]) + np.asarray(tr["dE"])
        if cand.size:
            margin = min(margin, float(np.min(np.minimum(np.abs(cand - lo), np.abs(cand - hi)))))
    for _ in range(n_or):
        o.single_pass(1, a)
    o.E = o.energy()
    o.sweep_counter = o.sweep_counter + 1
    return margin


def test_composite_sweeps_conserve_the_oracle_energies():
    """Full 1 HB + 4 OR sweeps: the links diverge chaotically through the
    overrelaxation passes, but overrelaxation conserves E and the heat-bath
    decisions stay identical, so the energies after each sweep agree.  A
    heat-bath decision may flip only at a near tie (an oracle candidate energy
    within 1e-3 of a window edge, the float32 error of the GPU's running
    energy); at most one lattice-sweep may show one."""
    w = workloads.small_l4()
    a = np.full(w.n_lattices, -1.0)
    flips = 0
    with _batch(w, max_approach=1000) as b:
        mirrors = [oracle_mirror(b, w, i) for i in range(w.n_lattices)]
        for _ in range(2):
            hb_gpu0 = b.stats()["hb_acc"].copy()
            b.sweep(a, 1)
            E = b.tracked_energy()
            hb_gpu = b.stats()["hb_acc"] - hb_gpu0
            for i, o in enumerate(mirrors):
                lo, hi = w.E_lo[i], w.E_lo[i] + w.dE[i]
                hb0 = o.stats()["hb_acc"]
                margin = _oracle_composite_sweep(o, a[i], w.n_or, lo, hi)
                same = o.stats()["hb_acc"] - hb0 == hb_gpu[i] and abs(E[i] - o.E) < 1e-3
                if not same:
                    assert margin < 1e-3, (i, E[i], o.E, margin)
                    flips += 1
                assert lo <= E[i] <= hi
                # continue both from the GPU state: one sweep at a time
                o.set_links(b.get_links(i).astype(np.float64))
                o.sweep_counter = b.get_sweep_counter(i)
    assert flips <= 1


def test_approach_reaches_every_window():
    w = workloads.small_l4()
    with _batch(w, max_approach=0) as b:
        n_gpu = b.approach(1000)
        E = b.energy()
        assert np.all(b.status() == 0)
    g = oracle.Geom([4] * 4)
    for i in range(w.n_lattices):
        o = oracle.Lattice(g, w.seed, w.interval_id[i], w.replica_id[i], w.E_lo[i], w.dE[i],
                           beta_up=w.beta_up, beta_dn=w.beta_dn)
        o.hot_start()
        n = o.approach(1000)
        assert abs(n - n_gpu[i]) <= 2
        assert w.E_lo[i] - 1e-5 <= E[i] <= w.E_lo[i] + w.dE[i] + 1e-5


def test_plain_form_equals_batched_form():
    """Same machine code, one launch per pass versus one persistent launch:
    bit-identical slopes, measurements and links."""
    w = workloads.subset(workloads.small_l4(), range(3))
    a0 = np.full(w.n_lattices, -1.0)
    with _batch(w, max_approach=1000) as b1, _batch(w, max_approach=1000) as b2:
        a1, m1 = b1.rm_step(a0, 2, 3, 0)
        a2, m2 = b2.rm_step_plain(a0, 2, 3, 0)
        assert np.array_equal(a1, a2) and np.array_equal(m1, m2)
        for i in range(w.n_lattices):
            assert np.array_equal(b1.get_links(i), b2.get_links(i))


def test_reconstruction_matches_oracle():
    rng = np.random.default_rng(0)
    c = np.linspace(900.0, 1100.0, 257)
    a = -1.0 + 0.002 * (c - 1000.0) + 0.01 * rng.normal(size=c.size)
    ln_g = llr.reconstruct_lnrho(c, a)
    ln_o = recon.lnrho_at_centres(c, a)
    assert np.max(np.abs(ln_g - ln_o)) < 1e-10 * max(1.0, np.max(np.abs(ln_o)))
    betas = np.linspace(0.5, 1.5, 11)
    lz, e1, e2 = llr.observables(c, a, betas)
    for k, bt in enumerate(betas):
        z, E1, E2 = recon.moments(c, a, bt)
        assert abs(lz[k] - z) < 1e-9 * max(1.0, abs(z))
        assert abs(e1[k] - E1) < 1e-9 * abs(E1)
        assert abs((e2[k] - e1[k] ** 2) - (E2 - E1 ** 2)) < 1e-6 * max(1.0, E2 - E1 ** 2)
    bg, cg = llr.cv_peak(c, a, 0.5, 1.5, 2001, 1e-12)
    bo, co = recon.cv_peak(c, a, 0.5, 1.5, 2001, 1e-12)
    assert abs(bg - bo) < 1e-8 and abs(cg - co) < 1e-8 * max(1.0, co)
