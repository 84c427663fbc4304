"""The autotuner of the batched sweep kernel (threads per CTA, ring stages,
shared-memory carve-out): the shape it picks is the one the next launches use,
and the chains do not depend on the shape -- a run with the tuned shape and a
run with a different value of every knob give bit-identical slopes and links."""
import numpy as np
import pytest

from paper_1509_08391_gb300 import autotune, llr
from tests.test_gpu_batching import _uneven

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1509_08391_gb300 import build
    build.build()


def test_tuned_shape_is_launched_and_leaves_the_chains_unchanged():
    w = _uneven(n_int=3)
    shape = autotune.tune(w, use_cache=False)
    assert shape["threads"] in autotune.SHAPES
    assert shape["ring"] in autotune.RINGS and shape["carveout"] in autotune.CARVEOUTS
    other = {"threads": 128 if shape["threads"] != 128 else 512,
             "ring": 1 if shape["ring"] != 1 else 4,
             "carveout": 100 if shape["carveout"] != 100 else -1}
    a0 = np.linspace(-1.05, -0.95, w.n_lattices)
    runs = []
    for sh in (shape, other):
        with llr.Batch.from_workload(w, max_approach=2000) as b:
            autotune.apply(b, sh)
            a = a0.copy()
            for n in range(3):
                a, _ = b.rm_step(a, 1, 2, n)
            last = b.last_launch()
            assert (last["threads"], last["ring"], last["carveout"]) == \
                (sh["threads"], sh["ring"], sh["carveout"]), (last, sh)
            assert last["fast_math"] == 1 and 0 < last["grid"] <= 3 * w.n_lattices
            runs.append((a, [b.get_links(i) for i in range(w.n_lattices)], b.tracked_energy()))
    assert np.array_equal(runs[0][0], runs[1][0])
    assert np.array_equal(runs[0][2], runs[1][2])
    assert all(np.array_equal(x, y) for x, y in zip(runs[0][1], runs[1][1]))
    # the cache holds the candidate timings the choice came from
    entry = next(v for k, v in autotune._load().items() if k.endswith("|n=%d" % w.n_lattices))
    assert entry["shape"] == shape and len(entry["ms_per_2_sweeps"]) >= 5
