"""Seeded synthetic workloads (inputs only; none of the method's arithmetic).

Both the CUDA path and the oracle take their inputs from here.  A workload is
a batch of independent (interval, replica) Markov chains: for each one the
lattice side L, the window [E_lo, E_lo + dE] of the action E = sum cos
theta_P, the Philox key words (interval id, replica id) and a seed.

Interval placement: n intervals of width dE inside [e_lo, e_hi] * 6V, the
first starting at e_lo * 6V and the last ending at e_hi * 6V, equally spaced
(they overlap or leave gaps depending on n * dE versus the span).  With
n * dE equal to the span they are the paper's contiguous intervals
E_k = E_min + k dE (Sec. 2.4, Algorithm 1).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np

SEED_BASE = 20260101


def place_intervals(L: int, n: int, e_lo: float, e_hi: float, dE: float) -> np.ndarray:
    six_v = 6.0 * L ** 4
    if n == 1:
        return np.array([e_lo * six_v])
    step = (six_v * (e_hi - e_lo) - dE) / (n - 1)
    return e_lo * six_v + step * np.arange(n)


@dataclass
class Workload:
    name: str
    L: List[int]
    E_lo: List[float]
    dE: List[float]
    interval_id: List[int]
    replica_id: List[int]
    seed: int
    n_or: int = 4
    block: int = 1
    n_therm: int = 50
    n_meas: int = 100
    n_rm: int = 20
    a0: float = -1.0
    beta_up: float = 1.5
    beta_dn: float = 0.5
    max_approach: int = 10000
    notes: dict = field(default_factory=dict)

    @property
    def n_lattices(self) -> int:
        return len(self.L)

    def links_per_lattice(self) -> np.ndarray:
        return 4 * np.asarray(self.L, dtype=np.int64) ** 4


def _grid(name, Ls, n_int, e_lo, e_hi, dEs, replicas, seed, **kw) -> Workload:
    L, lo, de, iid, rid = [], [], [], [], []
    base = 0
    for Lg, dE in zip(Ls, dEs):
        E = place_intervals(Lg, n_int, e_lo, e_hi, dE)
        for k in range(n_int):
            for r in range(replicas):
                L.append(Lg)
                lo.append(float(E[k]))
                de.append(float(dE))
                iid.append(base + k)
                rid.append(r)
        base += n_int
    return Workload(name, L, lo, de, iid, rid, seed, **kw)


def small_l4(replicas: int = 1) -> Workload:
    """L=4, 8 intervals over E/6V in [0.55, 0.70], dE=4, 50 + 100 sweeps per
    Robbins-Monro step, 20 steps: the case the oracle finishes in seconds."""
    return _grid("u1_4d_L4_8int_dE4", [4], 8, 0.55, 0.70, [4.0], replicas, SEED_BASE + 0,
                 n_therm=50, n_meas=100, n_rm=20)


def l8_batch(replicas: int = 4) -> Workload:
    """L=8, 32 intervals over E/6V in [0.58, 0.68] x 4 replicas, dE=8, 1:4
    heat-bath:overrelaxation, 100 Robbins-Monro steps."""
    return _grid("u1_4d_L8_32int_x4_dE8", [8], 32, 0.58, 0.68, [8.0], replicas, SEED_BASE + 1,
                 n_therm=50, n_meas=100, n_rm=100)


def uneven_batch() -> Workload:
    """L = 8, 12, 16 with 64 intervals each over E/6V in [0.58, 0.68], dE
    scaled with sqrt(V): 8, 18, 32."""
    Ls = [8, 12, 16]
    dEs = [8.0 * (L / 8) ** 2 for L in Ls]
    return _grid("u1_4d_uneven_L8_12_16_64int", Ls, 64, 0.58, 0.68, dEs, 1, SEED_BASE + 2,
                 n_therm=50, n_meas=100, n_rm=100)


def l20_critical(replicas: int = 8, n_int: int = 256) -> Workload:
    """L=20 around the pseudo-critical coupling: 256 narrow intervals over E/6V
    in [0.62, 0.67], dE=12, 8 replicas each, 200 Robbins-Monro steps."""
    return _grid("u1_4d_L20_256int_x8_dE12", [20], n_int, 0.62, 0.67, [12.0], replicas,
                 SEED_BASE + 3, n_therm=10, n_meas=40, n_rm=200)


def warm_start_targets(L: int, replicas: int = 4, n_int: int = 128, e_lo: float = 0.58,
                       e_hi: float = 0.68) -> Workload:
    """Prediction targets of the learned warm start: 128 intervals over
    E/6V in [e_lo, e_hi] (default [0.58, 0.68]) at L = 20 or 24, dE scaled
    with sqrt(V)."""
    dE = 8.0 * (L / 8) ** 2
    return _grid("u1_4d_L%d_%dint_warm" % (L, n_int), [L], n_int, e_lo, e_hi, [dE], replicas,
                 SEED_BASE + 4, n_therm=10, n_meas=40, n_rm=100)


def overlapping_l4(replicas: int = 2, n_int: int = 6) -> Workload:
    """L=4 with overlapping windows for replica exchange (Sec. 2.5): n_int
    windows of width dE = 16 whose lower edges are 8 apart (half overlap),
    starting at E/6V = 0.58."""
    L, dE = 4, 16.0
    six_v = 6.0 * L ** 4
    e_hi = (0.58 * six_v + 8.0 * (n_int - 1) + dE) / six_v
    return _grid("u1_4d_L4_%dint_overlap" % n_int, [L], n_int, 0.58, e_hi, [dE], replicas,
                 SEED_BASE + 5, n_therm=5, n_meas=20, n_rm=20)


def exchange_pairs(w: Workload, parity: int):
    """The lattice pairs tried in one replica-exchange round: neighbouring
    windows (k, k+1) with k = parity mod 2, same L and same replica, in
    ascending order of the window edge.  Index bookkeeping only."""
    by_key = {}
    for i in range(w.n_lattices):
        by_key.setdefault((w.L[i], w.replica_id[i]), []).append(i)
    pairs = []
    for key in sorted(by_key):
        idx = sorted(by_key[key], key=lambda i: w.E_lo[i])
        for k in range(parity & 1, len(idx) - 1, 2):
            pairs.append((idx[k], idx[k + 1]))
    return pairs


def subset(w: Workload, idx) -> Workload:
    idx = list(idx)
    pick = lambda xs: [xs[i] for i in idx]
    return Workload(w.name + "_subset", pick(w.L), pick(w.E_lo), pick(w.dE),
                    pick(w.interval_id), pick(w.replica_id), w.seed, w.n_or, w.block,
                    w.n_therm, w.n_meas, w.n_rm, w.a0, w.beta_up, w.beta_dn, w.max_approach,
                    dict(w.notes))


# Energy ranges of the paper's volume study (Table 1): E/6V from E_min
# to E_max in 512 contiguous intervals; N_SW sweeps and N_RM Robbins-Monro
# iterations per interval.
PAPER_VOLUME_STUDY = {
    8: (0.5722222, 0.67, 250, 600),
    10: (0.59, 0.687777, 200, 400),
    12: (0.59, 0.687777, 200, 400),
    14: (0.59, 0.687777, 200, 400),
    16: (0.59, 0.687777, 200, 400),
    18: (0.59, 0.687777, 200, 400),
    20: (0.59, 0.687777, 200, 400),
}


def paper_volume_study(L: int, replicas: int = 8, n_therm: int = 5, n_meas: int = 20,
                       n_rm: int = 0, n_int: int = 512) -> Workload:
    """The paper's L^4 study (Table 1): n_int (512) contiguous intervals of
    width dE = (E_max - E_min) / n_int over its E/6V range (other n_int: the
    discretisation study, Table 7), `replicas` independent chains per
    interval (the paper repeats each run N_B = 20 times), N_RM Robbins-Monro
    iterations (the paper's value when n_rm = 0).  Sweeps per iteration are
    composite sweeps (1 heat-bath + 4 overrelaxation passes)."""
    e_lo, e_hi, _n_sw, n_rm_paper = PAPER_VOLUME_STUDY[L]
    dE = 6.0 * L ** 4 * (e_hi - e_lo) / n_int
    return _grid("u1_4d_L%d_%dint_x%d_paper" % (L, n_int, replicas), [L], n_int, e_lo, e_hi, [dE],
                 replicas, SEED_BASE + 10 + L, n_therm=n_therm, n_meas=n_meas,
                 n_rm=n_rm if n_rm > 0 else n_rm_paper)
