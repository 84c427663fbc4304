"""Autotuner of the batched sweep kernel's launch shape.

The CTA shapes (128, 160, 192, 256, 512 threads; one consumer warp, the rest
producers) run identical per-link arithmetic, so the choice changes speed
only, never results.  For a workload the tuner builds a scratch batch of the
same lattices (the caller's chains are not advanced), times one composite
sweep per shape with CUDA events after a warm-up sweep, and caches the
fastest shape per (GPU, lattice sizes, batch size) in a JSON file.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import llr, workloads

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "autotune.json")
SHAPES = (128, 160, 192, 256, 512)


def _key(w: workloads.Workload, gpu: str) -> str:
    Ls = sorted(set(int(x) for x in w.L))
    return "%s|L=%s|n=%d" % (gpu, ",".join(map(str, Ls)), w.n_lattices)


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def _save(d):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".%d.tmp" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def tune(w: workloads.Workload, shapes=SHAPES, use_cache=True, verbose=False):
    """Best threads-per-CTA for this workload (fast math on)."""
    import torch
    gpu = torch.cuda.get_device_name()
    key = _key(w, gpu)
    cache = _load()
    if use_cache and key in cache:
        return int(cache[key]["threads"])
    times = {}
    stream = torch.cuda.Stream()
    with llr.Batch.from_workload(w, stream=stream.cuda_stream, max_approach=1000) as b:
        a = np.full(w.n_lattices, w.a0)
        for t in shapes:
            b.set_kernel_config(t, True)
            b.sweep(a, 1)                      # warm-up
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.sweep(a, 1)
            e1.record(stream)
            e1.synchronize()
            times[t] = e0.elapsed_time(e1)
            if verbose:
                print("autotune %s: %d threads %.2f ms" % (key, t, times[t]), flush=True)
    best = min(times, key=times.get)
    cache[key] = {"threads": int(best), "ms_per_sweep": times}
    _save(cache)
    return int(best)
