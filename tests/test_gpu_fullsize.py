"""Full-size checks in the launch configuration the benchmark times
(L = 20, 2048 lattices of the critical-region workload, 256 threads per
CTA, fast math): per-link outputs the oracle recomputes one by one, and
properties that hold at any size."""
import numpy as np
import pytest

import oracle
from paper_1509_08391_gb300 import llr, workloads
from tests.gpu_helpers import check_class_updates

pytestmark = pytest.mark.gpu

BENCH_THREADS = 256
BENCH_FAST = True


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1509_08391_gb300 import build
    build.build()
    oracle.build()


def test_l20_class_updates_match_oracle_link_by_link():
    """A window wide enough that no decision can flip makes every link of an
    L=20 class update an independent output; each class of a heat-bath and of
    an overrelaxation pass is checked from an identical state."""
    full = workloads.l20_critical()
    w = workloads.subset(full, [0, 1])
    w.E_lo = [-1.0e7] * 2
    w.dE = [2.0e7] * 2
    with llr.Batch.from_workload(w, max_approach=0) as b:
        b.set_kernel_config(BENCH_THREADS, BENCH_FAST)
        b.sweep(np.full(2, -1.0), 2)         # leave the hot start
        a = np.array([-1.011, -0.99])
        worst, flips = check_class_updates(b, w, [1], a, classes=[0, 5])
        assert flips == 0


def test_l20_full_batch_properties():
    """The whole 2048-lattice batch: approach, one Robbins-Monro step of
    1 + 2 sweeps; every energy stays in its window, tracked and FP64 energies
    agree, acceptances are sane and nothing is NaN."""
    w = workloads.l20_critical()
    with llr.Batch.from_workload(w, max_approach=0) as b:
        b.set_kernel_config(BENCH_THREADS, BENCH_FAST)
        n = b.approach(500)
        assert np.all(n < 500)
        a = np.full(w.n_lattices, -1.01)
        b.stats(reset=True)
        a1, mean = b.rm_step(a, 1, 2, 0)
        assert np.all(np.isfinite(a1)) and np.all(b.status() == 0)
        E = b.energy()
        Et = b.tracked_energy()
        lo = np.asarray(w.E_lo)
        hi = lo + np.asarray(w.dE)
        assert np.all(E >= lo - 0.05) and np.all(E <= hi + 0.05)
        assert np.max(np.abs(E - Et)) < 1e-2
        st = b.stats()
        assert np.all(st["max_drift"] < 0.05)
        hb = st["hb_acc"].sum() / st["hb_tot"].sum()
        orr = st["or_acc"].sum() / st["or_tot"].sum()
        assert 0.5 < hb < 1.0 and orr > 0.99
        assert np.all(np.abs(mean) <= 0.5 * np.asarray(w.dE) + 0.05)
