"""Checkpoint and resume: the chain state saved after k Robbins-Monro steps and
loaded into a fresh handle continues bit-identically (random numbers are keyed
by the per-lattice sweep counter, not by a consumed stream)."""
import numpy as np
import pytest

from paper_1509_08391_gb300 import llr, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1509_08391_gb300 import build
    build.build()


def test_resume_is_bit_identical():
    w = workloads.subset(workloads.l8_batch(), range(6))
    a = np.full(w.n_lattices, -1.0)
    with llr.Batch.from_workload(w, max_approach=1000) as b:
        for n in range(2):
            a, _ = b.rm_step(a, 1, 2, n)
        blob = b.save_state()
        a_ckpt = a.copy()
        for n in range(2, 4):
            a, m = b.rm_step(a, 1, 2, n)
        ref = (a.copy(), m.copy(), [b.get_links(i) for i in range(w.n_lattices)])
    with llr.Batch.from_workload(w, max_approach=0) as c:
        c.load_state(blob)
        a = a_ckpt
        for n in range(2, 4):
            a, m = c.rm_step(a, 1, 2, n)
        assert np.array_equal(a, ref[0]) and np.array_equal(m, ref[1])
        for i in range(w.n_lattices):
            assert np.array_equal(c.get_links(i), ref[2][i])


def test_state_from_another_configuration_is_rejected():
    w1 = workloads.subset(workloads.l8_batch(), [0])
    w2 = workloads.subset(workloads.l8_batch(), [1])
    with llr.Batch.from_workload(w1, max_approach=0) as b1, \
            llr.Batch.from_workload(w2, max_approach=0) as b2:
        with pytest.raises(llr.LLRError) as e:
            b2.load_state(b1.save_state())
        assert e.value.code == llr.LLR_ERR_ARG
