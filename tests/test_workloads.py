"""Input generators and host-side helpers (no GPU): the interval layouts the
tests and the benchmark use, the replica-exchange pairing schedule, and the
benchmark's reweighting table."""
import numpy as np

from paper_1509_08391_gb300 import workloads


def test_paper_volume_study_has_contiguous_intervals_over_the_table_range():
    """Table 1 at L = 8: 512 intervals of width (E_max - E_min) / 512 that
    tile [E_min, E_max] with no gap and no overlap (Sec. 2.4, E_k = E_min + k dE)."""
    w = workloads.paper_volume_study(8, replicas=3)
    six_v = 6 * 8 ** 4
    lo = np.asarray(w.E_lo).reshape(512, 3)
    assert np.all(lo == lo[:, :1])                       # replicas share the window
    dE = w.dE[0]
    assert abs(dE - six_v * (0.67 - 0.5722222) / 512) < 1e-12
    assert np.allclose(np.diff(lo[:, 0]), dE, rtol=0, atol=1e-9)
    assert abs(lo[0, 0] - 0.5722222 * six_v) < 1e-9
    assert abs(lo[-1, 0] + dE - 0.67 * six_v) < 1e-9
    assert len(set(w.interval_id)) == 512 and w.n_rm == 600


def test_discretisation_study_keeps_the_range():
    for n in (32, 128):
        w = workloads.paper_volume_study(8, replicas=1, n_int=n)
        six_v = 6 * 8 ** 4
        assert w.n_lattices == n
        assert abs(w.E_lo[0] - 0.5722222 * six_v) < 1e-9
        assert abs(w.E_lo[-1] + w.dE[0] - 0.67 * six_v) < 1e-9


def test_exchange_pairs_are_disjoint_overlapping_neighbours():
    w = workloads.overlapping_l4(replicas=3, n_int=7)
    seen_pairs = set()
    for parity in (0, 1):
        pairs = workloads.exchange_pairs(w, parity)
        used = [i for p in pairs for i in p]
        assert len(used) == len(set(used))              # one round: each lattice once
        for i, j in pairs:
            assert w.L[i] == w.L[j] and w.replica_id[i] == w.replica_id[j]
            assert w.E_lo[i] < w.E_lo[j] < w.E_lo[i] + w.dE[i]   # overlapping windows
            seen_pairs.add((i, j))
    # the two parities together try every neighbouring pair once
    assert len(seen_pairs) == 3 * (7 - 1)
