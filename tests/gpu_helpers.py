"""Shared helpers for the GPU parity tests (GPU path vs FP64 oracle)."""
import numpy as np

import oracle
from paper_1509_08391_gb300 import llr


def wrapped_diff(a, b):
    return np.angle(np.exp(1j * (np.asarray(a, np.float64) - np.asarray(b, np.float64))))


def oracle_mirror(batch: "llr.Batch", w, i, geoms={}):
    """An oracle lattice holding exactly the GPU lattice i's current state."""
    L = w.L[i]
    if L not in geoms:
        geoms[L] = oracle.Geom([L] * 4)
    o = oracle.Lattice(geoms[L], w.seed, w.interval_id[i], w.replica_id[i], w.E_lo[i], w.dE[i],
                       n_or=w.n_or, block=w.block, beta_up=w.beta_up, beta_dn=w.beta_dn)
    o.set_links(batch.get_links(i).astype(np.float64))
    o.sweep_counter = batch.get_sweep_counter(i)
    return o


def first_mismatch_class(d, L, tol):
    """Index (in the oracle's class order mu, parity) of the first class containing a
    mismatching link, or None."""
    V = L ** 4
    s = np.arange(V)
    x = [(s // L ** k) % L for k in range(4)]
    par = (x[0] + x[1] + x[2] + x[3]) & 1
    bad = np.abs(d) > tol
    for mu in range(4):
        for p in range(2):
            if np.any(bad[mu * V:(mu + 1) * V][par == p]):
                return 2 * mu + p
    return None


# FP32 conditioning of a link update: alpha = arg(S) moves by ~|dS| / |S| when
# the staple sum S carries float32 errors |dS| (six sincos of angle sums,
# ~1e-6), and the reflection theta' = -theta - 2 alpha doubles it.
TOL_RAD = 2e-5
COND_ABS = 4e-6


def link_tolerance(S_abs):
    return TOL_RAD + COND_ABS / np.maximum(S_abs, 1e-12)


def class_links(L, cls):
    """Canonical link indices (mu V + s) of class cls = 2 mu + parity."""
    V = L ** 4
    mu, p = cls >> 1, cls & 1
    s = np.arange(V)
    x = [(s // L ** k) % L for k in range(4)]
    par = (x[0] + x[1] + x[2] + x[3]) & 1
    return mu * V + s[par == p]


def check_class_updates(b, w, lattices, a, kinds=(0, 1), classes=range(8), e_tie=1e-3):
    """Update one class at a time on the GPU and in the oracle from the same
    state.  Walking the class in update order, every link agrees within its
    tolerance up to the first window decision that differs; that decision
    must be a near tie (the oracle's candidate energy within e_tie of a window
    edge, below the float32 error the GPU's running energy carries), and the
    rest of that class is then not compared.  Returns (worst deviation, flips)."""
    worst, flips = 0.0, 0
    for kind in kinds:
        for cls in classes:
            mirrors = {i: oracle_mirror(b, w, i) for i in lattices}
            S = {i: mirrors[i].staple_moduli() for i in lattices}
            b.single_pass(kind, a, class_mask=1 << cls)
            for i, o in mirrors.items():
                tr = o.class_trace(cls, kind, a[i])
                order = class_links(w.L[i], cls)
                g = b.get_links(i).astype(np.float64)
                d_all = np.abs(wrapped_diff(g, o.links()))
                tol_all = link_tolerance(S[i])
                # links outside the class must be untouched on both sides
                outside = np.ones(g.size, bool)
                outside[order] = False
                assert np.all(d_all[outside] == 0.0) or np.all(d_all[outside] < 1e-7)
                d = d_all[order]
                tol = tol_all[order]
                bad = np.nonzero(d > tol)[0]
                if bad.size:
                    k = int(bad[0])
                    gk = g[order][k]
                    took_old = abs(wrapped_diff(gk, tr["th_old"][k])) <= tol[k]
                    took_new = abs(wrapped_diff(gk, tr["th_prop"][k])) <= tol[k]
                    flipped = (took_old and tr["accepted"][k]) or (took_new and not tr["accepted"][k])
                    lo, hi = w.E_lo[i], w.E_lo[i] + w.dE[i]
                    cand = tr["E_before"][k] + tr["dE"][k]
                    margin = min(abs(cand - lo), abs(cand - hi))
                    assert flipped and margin < e_tie, (
                        "kind", kind, "class", cls, "lattice", i, "link", k, "dev", float(d[k]),
                        "|S|", float(S[i][order][k]), "flipped", flipped, "margin", margin)
                    flips += 1
                    d = d[:k]
                worst = max(worst, float(d.max()) if d.size else 0.0)
    return worst, flips
