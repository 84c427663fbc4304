"""Shared helpers for the GPU parity tests (GPU path vs FP64 oracle).

Tolerances, derived from the float32 arithmetic of the GPU path:
  * a link updated from an identical state: TOL_RAD + c * COND_ABS / |S|.  The
    heat-bath proposal is X - alpha (alpha = arg S); float32 staples carry
    ~1e-6 absolute error in S, so alpha carries ~1e-6 / |S| (c = 1).  The
    reflection theta' = -theta - 2 alpha doubles it (c = 2).  TOL_RAD covers the
    float32 rounding of the angle and of the sampler's variate.
  * a link of a whole overrelaxation pass, whose neighbours were updated
    earlier in the same pass: the errors of those neighbours enter S,
    |dS| <= sum of their angle errors, so the tolerance adds
    2 * sum(d_neighbours updated before it) / |S| (or_pass_tolerance).
  * window decisions: identical except near ties, where the oracle's candidate
    energy (or the energy before the block) lies within e_tie of an edge.  The
    two running energies start a class equal and then differ by the float32
    error of each move's dE (evaluated at the GPU's stored angle, which is
    itself within the link tolerance of the oracle's): ~5e-6 per move, a
    random walk, so at the k-th link e_tie = 1e-4 + 5 * 5e-6 * sqrt(k + 1).
  * sampler decisions: identical except near ties of the Best-Fisher accept
    test, where a margin of the attempt at which the two samplers part lies
    within SAMPLER_EPS of zero.
"""
import numpy as np

import oracle
from paper_1509_08391_gb300 import llr


def wrapped_diff(a, b):
    return np.angle(np.exp(1j * (np.asarray(a, np.float64) - np.asarray(b, np.float64))))


def oracle_mirror(batch: "llr.Batch", w, i, geoms={}, tracked=None):
    """An oracle lattice holding exactly the GPU lattice i's current state
    (links, sweep counter and, if given, the GPU's running energy)."""
    L = w.L[i]
    if L not in geoms:
        geoms[L] = oracle.Geom([L] * 4)
    o = oracle.Lattice(geoms[L], w.seed, w.interval_id[i], w.replica_id[i], w.E_lo[i], w.dE[i],
                       n_or=w.n_or, block=w.block, beta_up=w.beta_up, beta_dn=w.beta_dn)
    o.set_links(batch.get_links(i).astype(np.float64))
    o.sweep_counter = batch.get_sweep_counter(i)
    if tracked is not None:
        o.E = float(tracked)
    return o


TOL_RAD = 2e-5
COND_ABS = 4e-6
SAMPLER_EPS = 1e-4
E_TIE0 = 1e-4
E_TIE_MOVE = 2.5e-5


def e_tie_at(k):
    """Near-tie margin of the window decision at the k-th link of a class."""
    return E_TIE0 + E_TIE_MOVE * np.sqrt(k + 1.0)


def link_tolerance(S_abs, kind=0):
    c = 2.0 if kind == 1 else 1.0
    return TOL_RAD + c * COND_ABS / np.maximum(S_abs, 1e-12)


def site_coords(L):
    s = np.arange(L ** 4)
    return s, [(s // L ** k) % L for k in range(4)]


def class_links(L, cls):
    """Canonical link indices (mu V + s) of class cls = 2 mu + parity, in
    update order (ascending site)."""
    V = L ** 4
    mu, p = cls >> 1, cls & 1
    s, x = site_coords(L)
    par = (x[0] + x[1] + x[2] + x[3]) & 1
    return mu * V + s[par == p]


def neighbours(L, links=None):
    """int[n, 18]: for link theta_mu(x) (canonical index mu V + s; all links,
    or the given ones) the canonical indices of the 18 angles of its six
    staples, per nu != mu: theta_nu(x+mu), theta_mu(x+nu), theta_nu(x)
    (forward, phi = a - b - c) and theta_nu(x-nu+mu), theta_mu(x-nu),
    theta_nu(x-nu) (backward, phi = -a - b + c), from the plaquette
    definition of Sec. 3.1."""
    V = L ** 4
    links = np.arange(4 * V) if links is None else np.asarray(links, dtype=np.int64)
    mu_l, s = links // V, links % V
    x = [(s // L ** k) % L for k in range(4)]

    def site(xs):
        return ((xs[3] * L + xs[2]) * L + xs[1]) * L + xs[0]

    def sh(base, d, k):
        y = list(base)
        y[d] = (y[d] + k) % L
        return y

    out = np.zeros((links.size, 18), dtype=np.int64)
    for mu in range(4):
        sel = np.nonzero(mu_l == mu)[0]
        if sel.size == 0:
            continue
        xs = [c[sel] for c in x]
        ss = s[sel]
        cols = []
        for nu in range(4):
            if nu == mu:
                continue
            xpm, xpn, xmn = sh(xs, mu, 1), sh(xs, nu, 1), sh(xs, nu, -1)
            xmnpm = sh(xmn, mu, 1)
            cols += [nu * V + site(xpm), mu * V + site(xpn), nu * V + ss,
                     nu * V + site(xmnpm), mu * V + site(xmn), nu * V + site(xmn)]
        out[sel] = np.stack(cols, axis=1)
    return out


def staples(th, L, links=None, vals=None):
    """(|S|, alpha) of the given links (default: all, canonical order) from
    angles th (canonical layout), FP64; vals ([n, 18]) overrides the
    neighbour angles."""
    v = np.asarray(th, np.float64)[neighbours(L, links)] if vals is None else vals
    S = np.zeros(v.shape[0], dtype=np.complex128)
    for j in range(3):
        a, b, c, d, e, f = (v[:, 6 * j + k] for k in range(6))
        S += np.exp(1j * (a - b - c)) + np.exp(1j * (-d - e + f))
    return np.abs(S), np.angle(S)


def or_update_key(L):
    """Position of every link in an overrelaxation pass: slab x3, then class
    2 mu + parity, then site (the order of reading R1)."""
    V = L ** 4
    s, x = site_coords(L)
    par = (x[0] + x[1] + x[2] + x[3]) & 1
    key = np.zeros(4 * V, dtype=np.int64)
    for mu in range(4):
        key[mu * V:(mu + 1) * V] = (x[3] * 8 + 2 * mu + par) * V + s
    return key


def or_pass_tolerance(L, th_before, th_after, d):
    """Per-link tolerance of a whole overrelaxation pass from an identical
    state: |S| at the moment the link is updated (neighbours updated earlier
    in the pass at their new angles, the others at their old ones) and the
    deviations d of those earlier neighbours."""
    nbr = neighbours(L)
    key = or_update_key(L)
    earlier = key[nbr] < key[:, None]
    vals = np.where(earlier, np.asarray(th_after, np.float64)[nbr],
                    np.asarray(th_before, np.float64)[nbr])
    S_abs, _ = staples(None, L, vals=vals)
    prop = np.sum(np.where(earlier, np.asarray(d)[nbr], 0.0), axis=1)
    return TOL_RAD + 2.0 * (COND_ABS + prop) / np.maximum(S_abs, 1e-12), S_abs


def lattice_key(w, i):
    seed = int(w.seed) & (2 ** 64 - 1)
    return [(seed & 0xFFFFFFFF) ^ (int(w.interval_id[i]) & 0xFFFFFFFF),
            (seed >> 32) ^ (int(w.replica_id[i]) & 0xFFFFFFFF)]


def sampler_near_tie(key, link, sweep, kappa, target_X, tol, eps=SAMPLER_EPS):
    """Whether a float32 sampler could have produced the variate target_X
    where the FP64 sampler took another attempt.  With margin = max(m1, m2)
    (an attempt is taken iff m1 > 0 or m2 >= 0), j_o the oracle's attempt and
    j an attempt giving target_X: if j < j_o the oracle refused j, so its
    margin there must be within eps of zero; if j > j_o the GPU refused j_o
    (margin within eps), refused the attempts between (margins below eps) and
    took j (margin above -eps)."""
    X, m1, m2 = oracle.vonmises_attempts(kappa, key, int(link), int(sweep), 0, n_max=16)
    if X.size == 0:
        return False
    margin = np.maximum(m1, m2)
    taken = (m1 > 0) | (m2 >= 0)
    if not taken.any():
        return False
    j_o = int(np.argmax(taken))
    for j in np.nonzero(np.abs(wrapped_diff(X, target_X)) <= tol)[0]:
        j = int(j)
        if j == j_o:
            continue
        if j < j_o and abs(margin[j]) < eps:
            return True
        if j > j_o and abs(margin[j_o]) < eps and np.all(margin[j_o + 1:j] < eps) \
                and margin[j] > -eps:
            return True
    return False


def _dist(E, lo, hi):
    return np.where(E < lo, lo - E, np.where(E > hi, E - hi, 0.0))


def window_rule(kind, E, d, lo, hi):
    """The window decision of a block (R2 heat-bath, R19 overrelaxation)."""
    if kind == 1:
        return (_dist(E, lo, hi) > 0) | (_dist(E + d, lo, hi) == 0)
    return _dist(E + d, lo, hi) <= _dist(E, lo, hi)


def compare_class(w, i, kind, a_i, cls, g, tr, S_cls, alpha_cls, sweep, E0, report=None):
    """Compare one class update of lattice i (GPU links g, canonical) with the
    oracle's trace of the same update from the same state (S_cls, alpha_cls:
    staple modulus and angle of the class's links in update order, FP64; E0:
    the running energy both started from).

    Every link must be, within its tolerance, the oracle's proposal or its old
    angle -- or, for the heat-bath, another attempt of the sampler at a near
    tie (sampler_near_tie).  Every block decision is then replayed in link
    order with the FP64 dE of the candidates, the running energy following
    the GPU's decisions (overrelaxation leaves it, R19): each decision must
    equal the window rule's, except
    near ties (the energy before or after the block within e_tie_at of an
    edge).  Until the first near tie the replayed energies must equal the
    oracle's own."""
    L, B = w.L[i], w.block
    order = class_links(L, cls)
    n = order.size
    tol = link_tolerance(S_cls, kind)
    gk = np.asarray(g, np.float64)[order]
    th_old, th_prop = np.asarray(tr["th_old"]), np.asarray(tr["th_prop"])
    d_new = np.abs(wrapped_diff(gk, th_prop))
    d_old = np.abs(wrapped_diff(gk, th_old))
    took_new, took_old = d_new <= tol, d_old <= tol
    lo, hi = w.E_lo[i], w.E_lo[i] + w.dE[i]
    key = lattice_key(w, i)
    rep = report if report is not None else {}
    # FP64 dE of the candidates (local energy |S| cos(theta + alpha))
    e_old = S_cls * np.cos(th_old + alpha_cls)
    d_prop = S_cls * np.cos(th_prop + alpha_cls) - e_old
    d_gpu = S_cls * np.cos(gk + alpha_cls) - e_old
    alt = np.zeros(n, bool)
    for k in np.nonzero(~took_new & ~took_old)[0]:
        ok = kind == 0 and sampler_near_tie(key, int(order[k]), sweep, -a_i * S_cls[k],
                                            gk[k] + alpha_cls[k], tol[k])
        assert ok, ("link mismatch", "kind", kind, "class", cls, "lattice", i, "position",
                    int(k), "dev new", float(d_new[k]), "dev old", float(d_old[k]),
                    "tol", float(tol[k]), "|S|", float(S_cls[k]))
        alt[k] = True
    both = took_new & took_old
    taken = (took_new & ~both) | alt
    kept = took_old & ~took_new & ~alt
    nb = (n + B - 1) // B
    blk = np.arange(n) // B
    taken_b = np.bincount(blk, weights=taken, minlength=nb) > 0
    kept_b = np.bincount(blk, weights=kept, minlength=nb) > 0
    assert not np.any(taken_b & kept_b), ("a block taken in part", kind, cls, i)
    alt_b = np.bincount(blk, weights=alt, minlength=nb) > 0
    amb_b = ~taken_b & ~kept_b          # every link's proposal within tol of its old angle
    d_prop_b = np.bincount(blk, weights=d_prop, minlength=nb)
    d_gpu_b = np.bincount(blk, weights=np.where(alt, d_gpu, d_prop), minlength=nb)
    acc_tr = np.asarray(tr["accepted"])[::B][:nb]
    step = np.where(taken_b | (amb_b & acc_tr), d_gpu_b, 0.0)
    if kind == 1:
        step[:] = 0.0        # R19: overrelaxation does not move the running energy
    E_b = E0 + np.concatenate([[0.0], np.cumsum(step)[:-1]])
    rule = window_rule(kind, E_b, d_prop_b, lo, hi)
    decided = ~amb_b & ~alt_b
    flip = decided & (rule != taken_b)
    k0 = np.arange(nb) * B
    margin = np.minimum.reduce([np.abs(E_b - lo), np.abs(E_b - hi),
                                np.abs(E_b + d_prop_b - lo), np.abs(E_b + d_prop_b - hi)])
    far = flip & (margin >= e_tie_at(k0))
    assert not far.any(), ("window decision differs away from an edge", kind, cls, i,
                           int(np.argmax(far)), float(margin[np.argmax(far)]))
    # the replay is the oracle's own chain until the first decision that differs
    first = int(np.argmax(flip | alt_b)) if (flip | alt_b).any() else nb
    Eo = np.asarray(tr["E_before"])[::B][:nb]
    assert np.allclose(E_b[:first], Eo[:first], rtol=0, atol=1e-8 + 1e-12 * abs(E0)), \
        ("replayed energies differ from the oracle's", kind, cls, i)
    dev = np.where(taken, np.where(alt, 0.0, d_new), np.where(kept, d_old, 0.0))
    rep["links"] = rep.get("links", 0) + n
    rep["decisions"] = rep.get("decisions", 0) + int(decided.sum())
    rep["refused"] = rep.get("refused", 0) + int(kept_b.sum())
    rep["window_ties"] = rep.get("window_ties", 0) + int(flip.sum())
    rep["sampler_ties"] = rep.get("sampler_ties", 0) + int(alt.sum())
    rep["worst_rad"] = max(rep.get("worst_rad", 0.0), float(dev.max()))
    rep["worst_cond"] = max(rep.get("worst_cond", 0.0), float(np.max((dev - TOL_RAD) * S_cls)))
    if flip.any():
        rep["worst_tie_margin"] = max(rep.get("worst_tie_margin", 0.0),
                                      float(margin[flip].max()))
    return rep


def near_ties_are_rare(rep):
    """Near ties are decisions within the float32 error of the running energy
    of an edge, or sampler attempts within 1e-4 of their accept threshold:
    a small fraction of all decisions (a real mismatch fails compare_class)."""
    return (rep.get("window_ties", 0) <= 2 + 1e-4 * rep["decisions"]
            and rep.get("sampler_ties", 0) <= 2 + 1e-5 * rep["links"])


def check_class_updates(b, w, lattices, a, kinds=(0, 1), classes=range(8), report=None):
    """Update one class at a time on the GPU and in the oracle from the same
    state (links, sweep counter and the GPU's running energy) and compare
    every link and every decision (compare_class).  Links outside the class
    must be untouched on both sides.  Returns a report: links and decisions
    compared, refusals seen, the worst deviation and conditioning constant,
    and the near ties met."""
    rep = report if report is not None else {}
    for kind in kinds:
        for cls in classes:
            trk = b.tracked_energy()
            mirrors = {i: oracle_mirror(b, w, i, tracked=trk[i]) for i in lattices}
            st = {i: staples(mirrors[i].links(), w.L[i], class_links(w.L[i], cls))
                  for i in lattices}
            sweeps = {i: mirrors[i].sweep_counter for i in lattices}
            b.single_pass(kind, a, class_mask=1 << cls)
            for i, o in mirrors.items():
                before = o.links()
                tr = o.class_trace(cls, kind, a[i])
                g = b.get_links(i).astype(np.float64)
                outside = np.ones(g.size, bool)
                outside[class_links(w.L[i], cls)] = False
                assert np.array_equal(g[outside], before[outside]), \
                    ("links outside the class changed", kind, cls, i)
                compare_class(w, i, kind, a[i], cls, g, tr, st[i][0], st[i][1], sweeps[i],
                              trk[i], report=rep)
    return rep
