"""Learned warm start of the Robbins-Monro iteration and the convergence measure.

Orchestration only: every computation (sweeps, Robbins-Monro updates, MLP
training and inference) runs in the CUDA library through the C ABI.  PyTorch
provides device buffers and streams.

Protocol
  1. Training data: the method's own slopes at small volumes.  One uneven
     batch (L = 8, 10, 12, 14, 16) runs Robbins-Monro in one persistent
     launch per step (graph replays); the slope of each interval is the
     replica mean of a over the last quarter of the steps.
  2. The network (3 x 64 GELU) learns a(1/V, E/6V, dE/6V); its error eps on a
     held-out volume sets the gain offset n0: a start that is off by eps is
     worth (s / eps)^2 Robbins-Monro steps, s = 12 sigma / dE^2 being the
     spread of one step's estimate of a (sigma the noise of <<dE>>).
  3. At the target volume, the Robbins-Monro iteration starts from the
     prediction with the gain 12 / (dE^2 (n + n0 + 1)) (eq. (2.30) with the
     step count shifted by n0, still a Robbins-Monro schedule: sum c_n
     diverges, sum c_n^2 converges, Sec. 2.2).  The plain form starts from a
     naive a = -1 with n0 = 0 (Sec. 2.4 allows any initial a).
  4. Convergence (Sec. 2.4's stopping rule): the replica-mean step
     |a^(n+1) - a^(n)| <= eps_stop for `hold` consecutive steps; a converged
     slope must also agree with a long plain reference run within the
     combined 3 sigma of the replica spreads.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np

from . import llr, workloads


def _torch():
    import torch
    return torch


def run_rm(batch: "llr.Batch", a0, n_therm, n_meas, n_rm, rm_offset=0, device=None):
    """n_rm Robbins-Monro steps of every lattice (graph replays); returns the
    history a^(1..n_rm) as an (n_rm, n_lattices) array and the device time."""
    torch = _torch()
    dev = device or torch.device("cuda", torch.cuda.current_device())
    a = torch.tensor(np.asarray(a0, dtype=np.float64), device=dev)
    hist = torch.empty((max(n_rm, 1), batch.n), dtype=torch.float64, device=dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    batch.rm_run(a, n_therm, n_meas, rm_offset, n_rm, hist)
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    return hist[:n_rm].cpu().numpy(), dt


def interval_features(w: workloads.Workload):
    L = np.asarray(w.L, dtype=np.float64)
    six_v = 6.0 * L ** 4
    centre = np.asarray(w.E_lo) + 0.5 * np.asarray(w.dE)
    return L, centre / six_v, np.asarray(w.dE) / six_v


def slopes_by_interval(w: workloads.Workload, a_lat):
    """Replica means and standard errors per interval id."""
    ids = np.asarray(w.interval_id)
    uniq = np.unique(ids)
    mean = np.array([a_lat[ids == k].mean() for k in uniq])
    err = np.array([a_lat[ids == k].std(ddof=1) / math.sqrt((ids == k).sum())
                    if (ids == k).sum() > 1 else 0.0 for k in uniq])
    first = np.array([np.nonzero(ids == k)[0][0] for k in uniq])
    return uniq, mean, err, first


def training_set(n_int=24, replicas=2, n_rm=40, n_therm=2, n_meas=8, seed=None, stream=None,
                 Ls=(8, 10, 12, 14, 16), e_lo=0.58, e_hi=0.68):
    """The method's own slopes at small volumes (one uneven batch) for
    intervals over E/6V in [e_lo, e_hi]."""
    base = workloads.uneven_batch()
    L, lo, de, iid, rid = [], [], [], [], []
    for g, Lg in enumerate(Ls):
        dE = 8.0 * (Lg / 8) ** 2
        E = workloads.place_intervals(Lg, n_int, e_lo, e_hi, dE)
        for k in range(n_int):
            for r in range(replicas):
                L.append(Lg)
                lo.append(float(E[k]))
                de.append(dE)
                iid.append(g * 1000 + k)
                rid.append(r)
    w = workloads.Workload("u1_4d_train_L" + "_".join(str(x) for x in Ls), L, lo, de, iid, rid,
                           seed if seed is not None else base.seed, n_therm=n_therm,
                           n_meas=n_meas, n_rm=n_rm)
    t0 = time.perf_counter()
    with llr.Batch.from_workload(w, stream=stream, max_approach=1000) as b:
        hist, _ = run_rm(b, np.full(w.n_lattices, w.a0), n_therm, n_meas, n_rm)
    tail = hist[-max(1, n_rm // 4):].mean(axis=0)
    uniq, a_mean, a_err, first = slopes_by_interval(w, tail)
    Lf, ef, df = interval_features(w)
    return dict(L=Lf[first], e6v=ef[first], dE6v=df[first], a=a_mean, err=a_err,
                seconds=time.perf_counter() - t0, workload=w)


def fit_network(data, epochs=4000, lr=2e-3, seed=3, holdout_L=16):
    """Train on all volumes but one to measure the held-out error eps, then on
    all of them.  Returns (network, eps)."""
    keep = data["L"] != holdout_L
    with llr.MLP(seed=seed) as probe:
        probe.fit(data["L"][keep], data["e6v"][keep], data["dE6v"][keep], data["a"][keep],
                  epochs=epochs, lr=lr, standardise=True)
        pred = probe.predict(data["L"][~keep], data["e6v"][~keep], data["dE6v"][~keep])
        eps = float(np.sqrt(np.mean((pred - data["a"][~keep]) ** 2)))
    net = llr.MLP(seed=seed)
    loss = net.fit(data["L"], data["e6v"], data["dE6v"], data["a"], epochs=epochs, lr=lr,
                   standardise=True)
    return net, eps, loss


def gain_offset(dE, n_meas, eps, n_rm):
    """n0 = (s / eps)^2, the number of Robbins-Monro steps a start that is off by
    eps is worth: one step estimates a with spread s = 12 sigma / dE^2, sigma =
    dE / sqrt(12 n_meas) the noise of <<dE>> at the root (flat window), and n
    averaged steps have spread s / sqrt(n).  Capped at n_rm / 2."""
    sigma = dE / math.sqrt(12.0 * n_meas)
    s = 12.0 * sigma / (dE * dE)
    n0 = round((s / max(eps, 1e-12)) ** 2)
    return int(max(0, min(n0, n_rm // 2)))


def converged_step(hist_mean, eps_stop=1e-4, hold=3):
    """First n (1-based count of steps) after which the replica-mean step stays
    <= eps_stop for `hold` consecutive steps; None if never."""
    steps = np.abs(np.diff(hist_mean, axis=0))
    n_steps = steps.shape[0]
    out = []
    for k in range(hist_mean.shape[1]):
        ok = steps[:, k] <= eps_stop
        found = None
        run = 0
        for n in range(n_steps):
            run = run + 1 if ok[n] else 0
            if run >= hold:
                found = n + 2 - hold   # steps are between a^(n+1) and a^(n+2)
                break
        out.append(found)
    return out


def replica_mean_history(w, hist):
    ids = np.asarray(w.interval_id)
    uniq = np.unique(ids)
    return uniq, np.stack([hist[:, ids == k].mean(axis=1) for k in uniq], axis=1)


@dataclass
class CompareResult:
    naive_steps: list
    warm_steps: list
    agree_naive: np.ndarray
    agree_warm: np.ndarray
    seconds_per_step: float
    n0: int
    eps: float
    err_naive: np.ndarray   # mean over intervals of |replica-mean a^(n) - reference|, n = 0..n_rm
    err_warm: np.ndarray


def compare(target: workloads.Workload, net, eps, n_rm, n_therm, n_meas, eps_stop=1e-4, hold=3,
            ref_factor=2, stream=None):
    """Naive plain-schedule start versus learned warm start at the target volume."""
    L, e6v, d6v = interval_features(target)
    a_warm = net.predict(L, e6v, d6v)
    n0 = gain_offset(float(np.median(target.dE)), n_meas, eps, n_rm)
    a_naive = np.full(target.n_lattices, target.a0)
    with llr.Batch.from_workload(target, stream=stream, max_approach=1000) as b:
        h_naive, t_naive = run_rm(b, a_naive, n_therm, n_meas, ref_factor * n_rm)
    with llr.Batch.from_workload(target, stream=stream, max_approach=1000) as b:
        h_warm, t_warm = run_rm(b, a_warm, n_therm, n_meas, n_rm, rm_offset=n0)
    _, m_naive = replica_mean_history(target, np.vstack([a_naive[None, :], h_naive]))
    _, m_warm = replica_mean_history(target, np.vstack([a_warm[None, :], h_warm]))
    # reference: the long plain run's final replica means and errors
    _, ref_a, jerr, _ = slopes_by_interval(target, h_naive[-1])
    _, aw, werr, _ = slopes_by_interval(target, h_warm[-1])
    _, an, nerr, _ = slopes_by_interval(target, h_naive[n_rm - 1])
    agree_w = np.abs(aw - ref_a) <= 3.0 * np.sqrt(werr ** 2 + jerr ** 2) + 1e-12
    agree_n = np.abs(an - ref_a) <= 3.0 * np.sqrt(nerr ** 2 + jerr ** 2) + 1e-12
    err_n = np.abs(m_naive[:n_rm + 1] - ref_a[None, :]).mean(axis=1)
    err_w = np.abs(m_warm - ref_a[None, :]).mean(axis=1)
    return CompareResult(converged_step(m_naive[:n_rm + 1], eps_stop, hold),
                         converged_step(m_warm, eps_stop, hold), agree_n, agree_w,
                         t_warm / n_rm, n0, eps, err_n, err_w)


@dataclass
class ArmResult:
    steps: list              # per interval: steps to the stopping rule (None: not met)
    seconds_per_step: float  # device time of one Robbins-Monro step of the arm's batch
    err_at_stop: np.ndarray  # per interval: |replica-mean a at its stopping step - a_ref|
    err_curve: np.ndarray    # mean over intervals of |replica-mean a^(n) - a_ref|, n = 0..n_rm
    hist: np.ndarray         # a after each step, (steps, lattices)

    def converged(self):
        return [s for s in self.steps if s is not None]

    def intervals_per_s(self, n_rm):
        """Intervals that met the rule, over the time until the last of them did
        (all n_rm steps if some never did)."""
        done = self.converged()
        if not done:
            return 0.0
        n = max(done) if len(done) == len(self.steps) else n_rm
        return len(done) / (self.seconds_per_step * n)


def converge_arms(target: workloads.Workload, net, eps, n_rm, n_therm, n_meas, eps_stop=1e-4,
                  hold=3, stream=None):
    """The batched Robbins-Monro iteration at the target volume from the
    learned warm start (gain offset n0) and from the naive start a = -1
    (n0 = 0), every (interval, replica) chain in one persistent launch per
    step (graph replays).  The naive run continues to 2 n_rm steps; its
    final replica means are the reference a_ref (with their standard errors).
    Returns (warm arm, naive arm, a_ref, a_ref standard errors, n0)."""
    L, e6v, d6v = interval_features(target)
    a_warm = net.predict(L, e6v, d6v)
    n0 = gain_offset(float(np.median(target.dE)), n_meas, eps, n_rm)
    a_naive = np.full(target.n_lattices, target.a0)
    with llr.Batch.from_workload(target, stream=stream, max_approach=1000) as b:
        h_naive, t_naive = run_rm(b, a_naive, n_therm, n_meas, 2 * n_rm)
    with llr.Batch.from_workload(target, stream=stream, max_approach=1000) as b:
        h_warm, t_warm = run_rm(b, a_warm, n_therm, n_meas, n_rm, rm_offset=n0)
    _, ref_a, ref_err, _ = slopes_by_interval(target, h_naive[-1])
    arms = []
    for a0, hist, t, steps_run in ((a_warm, h_warm, t_warm, n_rm),
                                   (a_naive, h_naive[:n_rm], t_naive, 2 * n_rm)):
        _, m = replica_mean_history(target, np.vstack([a0[None, :], hist]))
        stop = converged_step(m, eps_stop, hold)
        at = np.array([abs(m[s if s is not None else n_rm, k] - ref_a[k])
                       for k, s in enumerate(stop)])
        arms.append(ArmResult(stop, t / steps_run, at, np.abs(m - ref_a[None, :]).mean(axis=1),
                              hist))
    return arms[0], arms[1], ref_a, ref_err, n0


def plain_arm(target: workloads.Workload, interval_index, n_steps, n_therm, n_meas,
              stream=None):
    """The plain form (one lattice at a time, one launch per pass, no graph,
    naive start) on the replicas of one interval for n_steps Robbins-Monro
    steps, timed on the host clock.  Returns (final a of the replicas, wall
    seconds)."""
    import time as _time
    ids = np.asarray(target.interval_id)
    k = np.unique(ids)[interval_index]
    sub = workloads.subset(target, list(np.nonzero(ids == k)[0]))
    with llr.Batch.from_workload(sub, stream=stream, max_approach=1000) as b:
        a = np.full(sub.n_lattices, sub.a0)
        t0 = _time.perf_counter()
        for n in range(n_steps):
            a, _ = b.rm_step_plain(a, n_therm, n_meas, n)
        dt = _time.perf_counter() - t0
    return a, dt
