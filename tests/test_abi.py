"""The C ABI library loads and exports every entry point include/llr.h declares (no GPU)."""
import ctypes
import os
import re

import pytest

from paper_1509_08391_gb300 import build as b
from paper_1509_08391_gb300 import llr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "llr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(llr_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    b.build()
    return ctypes.CDLL(b.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["llr_init_lattice", "llr_sweep", "llr_rm_step", "llr_reconstruct_lnrho"]:
        assert n in names
    assert sorted(llr.EXPORTS) == names


def test_library_exports_every_declared_symbol(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_binding_loads_and_rejects_bad_config_without_gpu():
    L = llr.load()
    # argument validation happens before any CUDA call
    with pytest.raises(llr.LLRError) as e:
        llr.Batch([5], [0.0], [1.0], [0], [0], 1)
    assert e.value.code == llr.LLR_ERR_ARG
    with pytest.raises(llr.LLRError) as e:
        llr.Batch([4], [0.0], [-1.0], [0], [0], 1)
    assert e.value.code == llr.LLR_ERR_ARG
    with pytest.raises(llr.LLRError) as e:
        llr.Batch([4], [0.0], [1.0], [0], [0], 1, block=3)
    assert e.value.code == llr.LLR_ERR_ARG
    assert L.llr_last_error().decode() != ""


def test_reconstruction_rejects_unsorted_centres_without_gpu():
    with pytest.raises(llr.LLRError) as e:
        llr.reconstruct_lnrho([2.0, 1.0], [0.0, 0.0])
    assert e.value.code == llr.LLR_ERR_ARG


def test_multicanonical_analysis_rejects_bad_input_without_gpu():
    """llr_muca_reweight / llr_muca_cv_peak / llr_muca_tunnellings check their
    arguments on the host before any device work (Sec. 2.6 analysis)."""
    import numpy as np
    from paper_1509_08391_gb300 import llr
    a = np.full(4, -1.0)
    E = np.linspace(10.0, 20.0, 16)
    bad = E.copy()
    bad[3] = np.nan
    for call in (lambda: llr.muca_reweight(bad, 10.0, 2.5, a, [1.0]),
                 lambda: llr.muca_reweight(E, 10.0, 0.0, a, [1.0]),
                 lambda: llr.muca_reweight(E, 10.0, 2.5, a, [np.inf]),
                 lambda: llr.muca_cv_peak(E, 10.0, 2.5, a, 1.0, 0.5),
                 lambda: llr.muca_tunnellings(np.zeros((3, 2)), 1.0, -1.0)):
        with pytest.raises(llr.LLRError) as exc:
            call()
        assert exc.value.code == llr.LLR_ERR_ARG


def test_bench_issue_roofline_arithmetic(monkeypatch):
    """bench.issue_roofline: warp instructions per update x updates/s against
    4 warp instructions per SM per clock; None without a matching record."""
    import bench
    monkeypatch.setattr(bench, "kernel_profile", lambda: {"warp_instructions_per_update": 10.0})
    r = bench.issue_roofline(5e10, 152, 2000.0)
    assert r["bound"] == "issue"
    assert r["achieved"] == pytest.approx(5e10 * 10.0 / 1e9)
    assert r["peak"] == pytest.approx(4 * 152 * 2000.0e6 / 1e9)
    assert r["frac"] == pytest.approx(500.0 / 1216.0)
    monkeypatch.setattr(bench, "kernel_profile", lambda: None)
    assert bench.issue_roofline(5e10, 152, 2000.0) is None

