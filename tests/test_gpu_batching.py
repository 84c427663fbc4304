"""Batching, persistent launch and CUDA-graph replay of the Robbins-Monro loop.

A lattice's chain does not depend on which other lattices share the launch,
on the order the persistent kernel picks up work items, or on whether the
steps are launched one by one or replayed from a captured graph: all of these
must give bit-identical slopes.
"""
import numpy as np
import pytest

import oracle
from paper_1509_08391_gb300 import llr, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1509_08391_gb300 import build
    build.build()
    oracle.build()


def _uneven(n_int=3):
    base = workloads.uneven_batch()
    L, lo, de, iid, rid = [], [], [], [], []
    for Lg in (8, 12, 16):
        dE = 8.0 * (Lg / 8) ** 2
        E = workloads.place_intervals(Lg, n_int, 0.58, 0.68, dE)
        for k in range(n_int):
            L.append(Lg)
            lo.append(float(E[k]))
            de.append(dE)
            iid.append(Lg * 100 + k)
            rid.append(0)
    return workloads.Workload("uneven_small", L, lo, de, iid, rid, base.seed, n_therm=1,
                              n_meas=2)


def test_graph_replay_equals_stepwise_launches():
    torch = pytest.importorskip("torch")
    w = workloads.subset(workloads.small_l4(replicas=2), range(8))
    n_rm = 4
    a0 = np.linspace(-1.1, -0.9, w.n_lattices)
    dev = torch.device("cuda", 0)
    with llr.Batch.from_workload(w, max_approach=1000) as b1, \
            llr.Batch.from_workload(w, max_approach=1000) as b2:
        a = a0.copy()
        hist1 = []
        for n in range(n_rm + 1):
            a, _ = b1.rm_step(a, 2, 3, 5 + n)
            hist1.append(a.copy())
        ad = torch.tensor(a0, dtype=torch.float64, device=dev)
        hd = torch.zeros((n_rm, w.n_lattices), dtype=torch.float64, device=dev)
        b2.rm_run(ad, 2, 3, 5, n_rm, hd)
        torch.cuda.synchronize()
        hist2 = hd.cpu().numpy()
        assert np.array_equal(np.array(hist1[:n_rm]), hist2)
        assert np.array_equal(ad.cpu().numpy(), hist2[-1])
        # a further replay continues the same chain
        b2.rm_run(ad, 2, 3, 5 + n_rm, 1, None)
        torch.cuda.synchronize()
        assert np.array_equal(ad.cpu().numpy(), hist1[n_rm])


def test_uneven_batch_equals_separate_batches():
    """L = 8, 12, 16 in one persistent launch versus one batch per L."""
    w = _uneven()
    with llr.Batch.from_workload(w, max_approach=1000) as b:
        a_all, m_all = b.rm_step(np.full(w.n_lattices, -1.0), 1, 2, 0)
        st = b.status()
        links_all = [b.get_links(i) for i in range(w.n_lattices)]
    assert np.all(st == 0)
    for Lg in (8, 12, 16):
        idx = [i for i in range(w.n_lattices) if w.L[i] == Lg]
        ws = workloads.subset(w, idx)
        with llr.Batch.from_workload(ws, max_approach=1000) as bs:
            a_s, m_s = bs.rm_step(np.full(ws.n_lattices, -1.0), 1, 2, 0)
            assert np.array_equal(a_s, a_all[idx]) and np.array_equal(m_s, m_all[idx])
            for k, i in enumerate(idx):
                assert np.array_equal(bs.get_links(k), links_all[i])


def test_kernel_shapes_give_identical_chains():
    """Every CTA shape (128 ... 512 threads) runs the same per-link arithmetic."""
    w = workloads.subset(workloads.small_l4(), range(4))
    outs = []
    for t in (128, 160, 192, 256, 512):
        with llr.Batch.from_workload(w, max_approach=0) as b:
            b.set_kernel_config(t, True)
            b.approach(1000)
            a, m = b.rm_step(np.full(w.n_lattices, -1.0), 1, 2, 0)
            outs.append((a, m, b.get_links(0)))
    for a, m, l0 in outs[1:]:
        assert np.array_equal(a, outs[0][0]) and np.array_equal(l0, outs[0][2])
