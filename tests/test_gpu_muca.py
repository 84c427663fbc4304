"""The multicanonical run (Sec. 2.6, eq. (2.50)) on the GPU against the FP64
oracle: each heat-bath class of the weight 1/rho~ from an identical state
(same proposals, same Metropolis-Hastings decisions except near ties), the
canonical limit of a linear ln rho~ for any proposal slope, and the errors."""
import numpy as np
import pytest

import oracle
from paper_1509_08391_gb300 import llr, workloads
from tests.gpu_helpers import class_links, link_tolerance, oracle_mirror, wrapped_diff

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1509_08391_gb300 import build
    build.build()
    oracle.build()


def _table(L):
    six_v = 6.0 * L ** 4
    n = 16
    e0 = 0.5 * six_v
    de = 0.25 * six_v / n
    a = -0.85 - 0.02 * np.arange(n)          # a smooth, decreasing slope
    return e0, de, a


def test_each_multicanonical_class_matches_oracle():
    w = workloads.small_l4()
    e0, de, a = _table(4)
    a0 = -1.0
    weight = oracle.MucaWeight(e0, de, a)
    flips = taken = total = 0
    with llr.Batch.from_workload(w, max_approach=1000) as b:
        b.sweep(np.full(w.n_lattices, -1.0), 1)
        b.set_muca_weight(e0, de, a, a0)
        for cls in range(8):
            mirrors = {i: oracle_mirror(b, w, i) for i in range(w.n_lattices)}
            S = {i: mirrors[i].staple_moduli() for i in mirrors}
            b.single_pass(2, None, class_mask=1 << cls)
            for i, o in mirrors.items():
                tr = oracle.muca_class_trace(o, weight, cls, a0)
                order = class_links(w.L[i], cls)
                g = b.get_links(i).astype(np.float64)
                d = np.abs(wrapped_diff(g, o.links()))[order]
                tol = link_tolerance(S[i])[order]
                bad = np.nonzero(d > tol)[0]
                taken += int(tr["accepted"].sum())
                total += tr["accepted"].size
                if bad.size:
                    k = int(bad[0])
                    # the first difference must be a decision at a near tie
                    margin = abs(np.log(tr["u"][k]) - tr["x"][k])
                    assert margin < 1e-4, (cls, i, k, float(d[k]), margin)
                    flips += 1
    assert flips <= 2
    assert 0.3 * total < taken < total       # Metropolis-Hastings is doing work


def test_linear_weight_gives_the_same_ensemble_for_any_proposal_slope():
    """ln rho~ linear with slope a_t: the weight is exp(-a_t E), so proposals
    at a0 = a_t (always taken) and at a0 = a_t + 0.4 (corrected) sample the
    same canonical ensemble: equal mean energies."""
    w = workloads.subset(workloads.l8_batch(), range(32))
    w.L = [4] * 32
    six_v = 6.0 * 4 ** 4
    w.E_lo = [0.3 * six_v] * 32
    w.dE = [0.5 * six_v] * 32
    a_t = -1.0
    means, errs = [], []
    for a0 in (a_t, a_t + 0.4):
        with llr.Batch.from_workload(w, max_approach=1000) as b:
            b.set_muca_weight(-six_v, 2 * six_v / 64, np.full(64, a_t), a0)
            b.muca_sweep(200, history=False)
            E = b.muca_sweep(1500)
            st = b.stats()
        per_chain = E.mean(axis=0)
        means.append(per_chain.mean())
        errs.append(per_chain.std(ddof=1) / np.sqrt(per_chain.size))
        if a0 != a_t:
            assert st["hb_acc"].sum() < st["hb_tot"].sum()
    assert abs(means[0] - means[1]) < 4 * np.hypot(*errs) + 1e-3 * abs(means[0]), (means, errs)


def test_muca_calls_need_a_weight():
    w = workloads.subset(workloads.small_l4(), range(1))
    with llr.Batch.from_workload(w, max_approach=0) as b:
        for f in (lambda: b.muca_sweep(1), lambda: b.single_pass(2, None)):
            with pytest.raises(llr.LLRError) as e:
                f()
            assert e.value.code == llr.LLR_ERR_ARG
        with pytest.raises(llr.LLRError):
            b.set_muca_weight(0.0, -1.0, [1.0], -1.0)
