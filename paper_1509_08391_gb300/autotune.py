"""Autotuner of the batched sweep kernel's launch shape.

Knobs (none changes the chains: every shape runs the same per-link
arithmetic in the same order, so the choice changes speed only):
  * threads per CTA: 128, 160, 192, 256, 512 (one warp takes the window
    decisions, the others propose; the chunk of a heat-bath pass is the
    proposing warps x 32 links, so this also sets the chunk size);
  * ring: stages of the producer/consumer ring in use (1, 2, 4), how many
    chunks the proposing warps may run ahead of the deciding warp;
  * carveout: the shared-memory share of the SM's unified L1/shared storage
    (driver default, 50, 75 or 100 percent).
The order of the overrelaxation groups (slab by slab of x3) is not a knob:
it is part of the update order of the Markov chain (reading R1), so another
grouping would be another chain.

For a workload the tuner builds a scratch batch of the same lattices (the
caller's chains are not advanced), times two composite sweeps per candidate
with CUDA events after a warm-up sweep, searching one knob at a time (threads,
then ring, then carve-out) from the defaults, and caches the fastest shape per
(GPU, lattice sizes, batch size) in a JSON file.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import llr, workloads

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "autotune.json")
SHAPES = (128, 160, 192, 256, 512)
RINGS = (1, 2, 4)
CARVEOUTS = (-1, 50, 75, 100)
DEFAULT = {"threads": 256, "ring": 4, "carveout": -1}


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


def apply(batch: "llr.Batch", shape: dict, fast_math: bool = True):
    batch.set_kernel_shape(shape["threads"], fast_math, shape["ring"], shape["carveout"])


def tune(w: workloads.Workload, use_cache=True, verbose=False, sweeps=2):
    """Fastest launch shape {threads, ring, carveout} for this workload (fast
    math on); the per-candidate times are kept in the cache entry."""
    import torch
    gpu = torch.cuda.get_device_name()
    key = _key(w, gpu)
    cache = _load()
    if use_cache and key in cache and "shape" in cache[key]:
        return dict(cache[key]["shape"])
    times = {}
    stream = torch.cuda.Stream()
    best = dict(DEFAULT)
    with llr.Batch.from_workload(w, stream=stream.cuda_stream, max_approach=5000) as b:
        a = np.full(w.n_lattices, w.a0)

        def run(shape):
            name = "t%d_r%d_c%d" % (shape["threads"], shape["ring"], shape["carveout"])
            if name in times:
                return times[name]
            apply(b, shape)
            b.sweep(a, 1)                      # warm-up
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.sweep(a, sweeps)
            e1.record(stream)
            e1.synchronize()
            times[name] = e0.elapsed_time(e1)
            if verbose:
                print("autotune %s: %s %.2f ms" % (key, name, times[name]), flush=True)
            return times[name]

        for knob, values in (("threads", SHAPES), ("ring", RINGS), ("carveout", CARVEOUTS)):
            scores = {}
            for v in values:
                cand = dict(best, **{knob: v})
                scores[v] = run(cand)
            best[knob] = min(scores, key=scores.get)
    cache[key] = {"shape": best, "ms_per_%d_sweeps" % sweeps: times}
    _save(cache)
    return dict(best)
