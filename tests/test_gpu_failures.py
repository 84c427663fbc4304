"""Failure detection without faulting the GPU: bounded device waits that run
out return an error status the host reads (the context stays usable), an
unreachable window and a non-finite slope are reported as errors."""
import numpy as np
import pytest

from paper_1509_08391_gb300 import llr, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1509_08391_gb300 import build
    build.build()


def test_bounded_wait_runs_out_and_context_survives():
    w = workloads.subset(workloads.l8_batch(), [0])
    with llr.Batch.from_workload(w, max_approach=1000) as b:
        before = b.get_links(0)
        b.set_wait_limit(0)            # no wait allowed: sweep 2 cannot wait for sweep 1
        with pytest.raises(llr.LLRError) as e:
            b.sweep(np.array([-1.0]), 3)
        assert e.value.code == llr.LLR_ERR_TIMEOUT
        # the skipped sweeps left the lattice alone: exactly one sweep was applied
        assert b.stats()["sweeps"][0] >= 1
        b.set_wait_limit(20_000_000_000)
        b.sweep(np.array([-1.0]), 2)   # the context and the handle still work
        assert np.all(b.status() == 0)
        assert not np.array_equal(before, b.get_links(0))


def test_unreachable_window_is_reported():
    L = 4
    six_v = 6.0 * L ** 4
    w = workloads.Workload("unreachable", [L], [six_v + 10.0], [4.0], [0], [0], 1)
    with pytest.raises(llr.LLRError) as e:
        llr.Batch.from_workload(w, max_approach=5)
    assert e.value.code == llr.LLR_ERR_WINDOW


def test_non_finite_slope_is_reported():
    w = workloads.subset(workloads.small_l4(), [0, 1])
    with llr.Batch.from_workload(w, max_approach=1000) as b:
        with pytest.raises(llr.LLRError) as e:
            b.rm_step(np.array([np.nan, -1.0]), 1, 1, 0)
        assert e.value.code == llr.LLR_ERR_NUMERIC


def test_one_timed_out_wait_does_not_stall_the_rest_of_the_launch():
    """Once a bounded wait has run out, every later work item that would wait
    skips at once instead of waiting out its own limit: 100000 sweeps of one
    L = 16 lattice with a 5 ms limit (less than one sweep of one CTA) return
    within about one sweep, where waiting out the limit item by item would
    take ~(items / resident CTAs) x 5 ms, over a second."""
    import time
    full = workloads.uneven_batch()
    w = workloads.subset(full, [next(i for i in range(full.n_lattices) if full.L[i] == 16)])
    with llr.Batch.from_workload(w, max_approach=0) as b:
        b.set_wait_limit(5_000_000)
        t0 = time.perf_counter()
        with pytest.raises(llr.LLRError) as e:
            b.sweep(np.array([-1.0]), 100000)
        dt = time.perf_counter() - t0
        assert e.value.code == llr.LLR_ERR_TIMEOUT
        assert dt < 0.4, dt
        done = b.stats()["sweeps"][0]
        assert 1 <= done < 100
        # the error was read and cleared; the handle keeps working
        b.set_wait_limit(20_000_000_000)
        b.sweep(np.array([-1.0]), 2)
        assert np.all(b.status() == 0)
        assert b.stats()["sweeps"][0] == done + 2
