"""llr_observables_noalloc: the observables entry point for callers that cannot
allocate device memory (an application that owns all device memory in its
own pool, or code that must not call cudaMalloc/cudaFree while it runs).

It must give the same ln Z, <E>, <E^2> as llr_observables, the allocating
entry point, on two calls in a row (the second one reusing the fixed scratch
array the first left behind).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1509_08391_gb300 import llr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    from paper_1509_08391_gb300 import build
    build.build()
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    return torch


def _case(seed, n):
    rng = np.random.default_rng(seed)
    c = np.linspace(1400.0, 1700.0, n)
    a = -1.05 + 0.0012 * (c - 1550.0) + 0.02 * rng.normal(size=n)
    betas = np.linspace(0.8, 1.3, 17)
    return c, a, betas


def test_noalloc_matches_allocating_entry_point_twice(torch_cuda):
    torch = torch_cuda
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    for call, (seed, n) in enumerate([(1, 300), (2, 257)]):   # a smaller second call
        c, a, betas = _case(seed, n)
        lz_ref, e1_ref, e2_ref = llr.observables(c, a, betas)
        dc = torch.tensor(c, dtype=torch.float64, device=dev)
        da = torch.tensor(a, dtype=torch.float64, device=dev)
        db = torch.tensor(betas, dtype=torch.float64, device=dev)
        lz = torch.full_like(db, float("nan"))
        e1 = torch.full_like(db, float("nan"))
        e2 = torch.full_like(db, float("nan"))
        torch.cuda.synchronize(dev)
        llr.observables_noalloc(dc, da, db, lz, e1, e2, stream=stream.cuda_stream)
        stream.synchronize()
        lz, e1, e2 = lz.cpu().numpy(), e1.cpu().numpy(), e2.cpu().numpy()
        assert np.all(np.abs(lz - lz_ref) <= 1e-9 * np.maximum(1.0, np.abs(lz_ref))), call
        assert np.all(np.abs(e1 - e1_ref) <= 1e-9 * np.abs(e1_ref)), call
        cv, cv_ref = e2 - e1 ** 2, e2_ref - e1_ref ** 2
        assert np.all(np.abs(cv - cv_ref) <= 1e-6 * np.maximum(1.0, cv_ref)), call


def test_noalloc_rejects_more_centres_than_its_scratch(torch_cuda):
    torch = torch_cuda
    dev = torch.device("cuda", 0)
    n = llr.NOALLOC_MAX_CENTRES + 1
    lib = llr.load()
    buf = torch.zeros(4, dtype=torch.float64, device=dev)
    p = ctypes.c_void_p(buf.data_ptr())
    code = lib.llr_observables_noalloc(n, p, p, 1, p, p, p, p, None)
    assert code == llr.LLR_ERR_ARG
    assert b"65536" in lib.llr_last_error()
