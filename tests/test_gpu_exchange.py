"""Replica exchange between overlapping intervals on the GPU (Sec. 2.5)
against the FP64 oracle: the same decisions on the same states, exchanges
that move link arrays and energies exactly, a checkpoint that carries the
exchanged arrangement, and Robbins-Monro slopes that exchanges leave
unchanged in distribution."""
import numpy as np
import pytest

import oracle
from paper_1509_08391_gb300 import llr, workloads
from tests.gpu_helpers import oracle_mirror

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1509_08391_gb300 import build
    build.build()


def _swap_draw(w, i, rnd):
    """The 53-bit uniform deciding a pair whose first lattice is i (oracle's Philox)."""
    key0 = (w.seed & 0xFFFFFFFF) ^ (w.interval_id[i] & 0xFFFFFFFF)
    key1 = ((w.seed >> 32) & 0xFFFFFFFF) ^ (w.replica_id[i] & 0xFFFFFFFF)
    x = oracle.philox4x32_10([0, rnd, 13, 0], [key0, key1])
    return (float(x[0] >> 11) * 4294967296.0 + float(x[1])) / 9007199254740992.0


def test_exchange_decisions_and_moves_match_oracle():
    w = workloads.overlapping_l4(replicas=2)
    n = w.n_lattices
    a = np.random.default_rng(5).uniform(-1.6, -0.4, n)
    tried = taken = flips = 0
    with llr.Batch.from_workload(w, max_approach=2000) as b:
        for rnd in range(30):
            b.sweep(a, 1)
            mirrors = [oracle_mirror(b, w, i) for i in range(n)]
            E0 = b.tracked_energy()
            links0 = [b.get_links(i) for i in range(n)]
            pairs = workloads.exchange_pairs(w, rnd)
            acc_g = b.replica_exchange(pairs, a, rnd)
            acc_o = oracle.replica_exchange(mirrors, pairs, a, rnd)
            E1 = b.tracked_energy()
            for k, (i, j) in enumerate(pairs):
                lo = max(w.E_lo[i], w.E_lo[j])
                hi = min(w.E_lo[i] + w.dE[i], w.E_lo[j] + w.dE[j])
                Ei, Ej = E0[i], E0[j]
                inside = lo <= Ei <= hi and lo <= Ej <= hi
                tried += inside
                if acc_g[k] != acc_o[k]:
                    # only a near tie may be decided differently
                    edge = min(abs(Ei - lo), abs(Ei - hi), abs(Ej - lo), abs(Ej - hi))
                    p = np.exp((a[i] - a[j]) * (Ei - Ej))
                    assert edge < 1e-4 or abs(_swap_draw(w, i, rnd) - p) < 1e-4, (rnd, i, j)
                    flips += 1
                if acc_g[k]:
                    taken += 1
                    assert inside
                    assert np.array_equal(b.get_links(i), links0[j])
                    assert np.array_equal(b.get_links(j), links0[i])
                    assert E1[i] == E0[j] and E1[j] == E0[i]
                else:
                    assert np.array_equal(b.get_links(i), links0[i])
                    assert E1[i] == E0[i] and E1[j] == E0[j]
            # the moved arrays are the ones the next sweeps update
            assert np.all(b.status() == 0)
        assert np.allclose(b.energy(), b.tracked_energy(), rtol=0, atol=1e-3)
    assert tried >= 20 and 0 < taken < tried
    assert flips <= 1


def test_checkpoint_after_exchanges_resumes_bit_identically():
    w = workloads.overlapping_l4(replicas=1)
    n = w.n_lattices
    a = np.full(n, -1.0)
    with llr.Batch.from_workload(w, max_approach=2000) as b:
        moved = 0
        for rnd in range(12):
            a, _ = b.rm_step(a, 1, 3, rnd)
            moved += int(b.replica_exchange(workloads.exchange_pairs(w, rnd), a, rnd).sum())
        assert moved > 0
        blob, a_ck = b.save_state(), a.copy()
        for rnd in range(12, 15):
            a, _ = b.rm_step(a, 1, 3, rnd)
            b.replica_exchange(workloads.exchange_pairs(w, rnd), a, rnd)
        ref = (a.copy(), [b.get_links(i) for i in range(n)])
    with llr.Batch.from_workload(w, max_approach=0) as c:
        c.load_state(blob)
        a = a_ck
        for rnd in range(12, 15):
            a, _ = c.rm_step(a, 1, 3, rnd)
            c.replica_exchange(workloads.exchange_pairs(w, rnd), a, rnd)
        assert np.array_equal(a, ref[0])
        for i in range(n):
            assert np.array_equal(c.get_links(i), ref[1][i])


def test_bad_pairs_are_rejected():
    w = workloads.overlapping_l4(replicas=1)
    with llr.Batch.from_workload(w, max_approach=0) as b:
        a = np.full(w.n_lattices, -1.0)
        for pairs in ([(0, 0)], [(0, 1), (1, 2)], [(0, w.n_lattices)]):
            with pytest.raises(llr.LLRError) as e:
                b.replica_exchange(pairs, a, 0)
            assert e.value.code == llr.LLR_ERR_ARG


def test_slopes_with_exchange_agree_with_slopes_without():
    """Exchanges change how chains move between windows, not the root of
    eq. (2.17): per interval the replica-mean slope after the same Robbins-Monro
    schedule agrees with and without exchanges within the combined spread."""
    R = 6
    w = workloads.overlapping_l4(replicas=R)
    n = w.n_lattices
    n_rm = 30
    res = {}
    for exch in (False, True):
        a = np.full(n, -1.0)
        with llr.Batch.from_workload(w, max_approach=2000) as b:
            taken = 0
            for rnd in range(n_rm):
                a, _ = b.rm_step(a, w.n_therm, w.n_meas, rnd)
                if exch:
                    taken += int(b.replica_exchange(workloads.exchange_pairs(w, rnd), a,
                                                    rnd).sum())
            assert np.all(b.status() == 0)
        if exch:
            assert taken > n_rm
        res[exch] = a.reshape(-1, R)
    for k in range(res[False].shape[0]):
        m0, m1 = res[False][k].mean(), res[True][k].mean()
        s = np.hypot(res[False][k].std(ddof=1), res[True][k].std(ddof=1)) / np.sqrt(R)
        assert abs(m0 - m1) < 4 * s + 2e-3, (k, m0, m1, s)
