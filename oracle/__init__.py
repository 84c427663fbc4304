"""FP64 CPU oracle for the LLR window-restricted Monte Carlo of compact U(1).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  It shares no code with the CUDA library: the Markov chain is
plain C (``llr_oracle.c``, compiled with gcc), the reconstruction and the MLP
are plain numpy (``recon.py``, ``mlp.py``).

Paper: Langfeld, Lucini, Pellegrini, Rago, "An efficient algorithm for
numerical computations of continuous densities of states" (arXiv:1509.08391).
The C file's header lists the sections and equations each part follows and
the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "llr_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (IEEE FP64, no contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared",
           "-fPIC", "-pthread", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P, I, D, U32, U64 = (ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                 ctypes.c_uint32, ctypes.c_uint64)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            up = ctypes.POINTER(ctypes.c_uint32)
            sig = {
                "orc_philox4x32_10": (None, [up, up, up]),
                "orc_uniform": (D, [U32]),
                "orc_geom_new": (P, [I, ip, I]),
                "orc_geom_free": (None, [P]),
                "orc_geom_nslot": (I, [P]),
                "orc_geom_nplaq": (I, [P]),
                "orc_geom_nsite": (I, [P]),
                "orc_geom_link_exists": (I, [P, I]),
                "orc_lat_new": (P, [P, U64, I, I, D, D, I, I, D, D]),
                "orc_lat_free": (None, [P]),
                "orc_energy": (D, [P]),
                "orc_lat_set_links": (None, [P, dp]),
                "orc_lat_get_links": (None, [P, dp]),
                "orc_lat_get_E": (D, [P]),
                "orc_lat_set_E": (None, [P, D]),
                "orc_lat_get_sweep": (U32, [P]),
                "orc_lat_set_sweep": (None, [P, U32]),
                "orc_lat_set_window": (None, [P, D, D]),
                "orc_lat_stats": (None, [P, dp]),
                "orc_lat_hot_start": (None, [P]),
                "orc_vonmises": (I, [D, up, U32, U32, U32, dp]),
                "orc_vonmises_attempts": (I, [D, up, U32, U32, U32, I, dp, dp, dp]),
                "orc_lat_sweep": (None, [P, D, I]),
                "orc_lat_pass": (None, [P, I, D]),
                "orc_lat_class_pass": (None, [P, I, I, D]),
                "orc_lat_class_trace": (I, [P, I, I, D, dp, dp, dp, dp, ip]),
                "orc_lat_approach": (I, [P, I]),
                "orc_lat_rm_step": (D, [P, D, I, I, I, dp]),
                "orc_lat_staple": (None, [P, I, dp]),
                "orc_lat_staple_moduli": (None, [P, dp]),
                "orc_batch_run": (I, [P, I, U64, ip, ip, dp, dp, dp, dp, I, I, I, I, I, I, I,
                                      D, D, I, ip, dp]),
                "orc_batch_sweeps": (None, [P, dp, I, I, I]),
                "orc_replica_exchange": (I, [P, I, ip, dp, U32, ip]),
                "orc_muca_new": (P, [I, D, D, dp]),
                "orc_muca_free": (None, [P]),
                "orc_muca_lnrho": (D, [P, D]),
                "orc_lat_muca_sweep": (None, [P, P, D, I, dp]),
                "orc_lat_muca_class_trace": (I, [P, P, I, D, dp, dp, dp, dp, ip]),
                "orc_batch_approach": (None, [P, ip, I, I, I]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _up(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def philox4x32_10(ctr, key):
    """Philox4x32-10 block function (Salmon et al., SC'11)."""
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_up(c), _up(k), _up(out))
    return out


def uniform(w: int) -> float:
    return lib().orc_uniform(int(w) & 0xFFFFFFFF)


def vonmises(kappa, key, c0, c1, c2):
    """One von Mises variate (Best & Fisher 1979).  Returns (X, attempts)."""
    k = np.asarray(key, dtype=np.uint32).copy()
    x = ctypes.c_double(0.0)
    att = lib().orc_vonmises(float(kappa), _up(k), c0, c1, c2, ctypes.byref(x))
    return x.value, att


def vonmises_attempts(kappa, key, c0, c1, c2, n_max=8):
    """Every sampler attempt: (X if taken, margin m1, margin m2) arrays."""
    k = np.asarray(key, dtype=np.uint32).copy()
    X, m1, m2 = np.zeros(n_max), np.zeros(n_max), np.zeros(n_max)
    n = lib().orc_vonmises_attempts(float(kappa), _up(k), c0, c1, c2, int(n_max), _dp(X),
                                    _dp(m1), _dp(m2))
    return X[:n], m1[:n], m2[:n]


class Geom:
    """d-dimensional hypercubic lattice, periodic or open (Sec. 3.1)."""

    def __init__(self, dims, periodic=True):
        dims = [int(d) for d in dims]
        arr = (ctypes.c_int * 4)(*(dims + [1] * (4 - len(dims))))
        self._h = lib().orc_geom_new(len(dims), arr, 1 if periodic else 0)
        if not self._h:
            raise ValueError("bad geometry")
        self.dims = dims
        self.d = len(dims)
        self.periodic = periodic
        self.nslot = lib().orc_geom_nslot(self._h)
        self.nplaq = lib().orc_geom_nplaq(self._h)
        self.nsite = lib().orc_geom_nsite(self._h)

    def exists(self):
        return np.array([lib().orc_geom_link_exists(self._h, i) for i in range(self.nslot)],
                        dtype=bool)

    def __del__(self):
        try:
            if self._h:
                lib().orc_geom_free(self._h)
        except Exception:
            pass


class Lattice:
    """One (interval, replica) Markov chain of the restricted ensemble."""

    def __init__(self, geom: Geom, seed: int, interval_id: int, replica_id: int,
                 E_lo: float, dE: float, n_or: int = 4, block: int = 1,
                 beta_up: float = 1.5, beta_dn: float = 0.5):
        self.geom = geom
        self._h = lib().orc_lat_new(geom._h, int(seed) & (2 ** 64 - 1), int(interval_id),
                                    int(replica_id), float(E_lo), float(dE), int(n_or),
                                    int(block), float(beta_up), float(beta_dn))

    def __del__(self):
        try:
            if self._h:
                lib().orc_lat_free(self._h)
        except Exception:
            pass

    # state
    def hot_start(self):
        lib().orc_lat_hot_start(self._h)

    def set_links(self, th):
        th = np.ascontiguousarray(th, dtype=np.float64)
        assert th.size == self.geom.nslot
        lib().orc_lat_set_links(self._h, _dp(th))

    def links(self):
        out = np.zeros(self.geom.nslot)
        lib().orc_lat_get_links(self._h, _dp(out))
        return out

    @property
    def E(self):
        return lib().orc_lat_get_E(self._h)

    @E.setter
    def E(self, v):
        lib().orc_lat_set_E(self._h, float(v))

    @property
    def sweep_counter(self):
        return lib().orc_lat_get_sweep(self._h)

    @sweep_counter.setter
    def sweep_counter(self, v):
        lib().orc_lat_set_sweep(self._h, int(v))

    def set_window(self, E_lo, dE):
        lib().orc_lat_set_window(self._h, float(E_lo), float(dE))

    def stats(self):
        out = np.zeros(6)
        lib().orc_lat_stats(self._h, _dp(out))
        return dict(hb_acc=out[0], hb_tot=out[1], or_acc=out[2], or_tot=out[3],
                    caps=out[4], max_drift=out[5])

    def energy(self):
        return lib().orc_energy(self._h)

    def staple(self, link):
        out = np.zeros(2)
        lib().orc_lat_staple(self._h, int(link), _dp(out))
        return out

    def staple_moduli(self):
        out = np.zeros(self.geom.nslot)
        lib().orc_lat_staple_moduli(self._h, _dp(out))
        return out

    # dynamics
    def sweep(self, a, n=1):
        lib().orc_lat_sweep(self._h, float(a), int(n))

    def single_pass(self, mode, a=0.0):
        lib().orc_lat_pass(self._h, int(mode), float(a))

    def class_pass(self, cls, mode, a=0.0):
        lib().orc_lat_class_pass(self._h, int(cls), int(mode), float(a))

    def class_trace(self, cls, mode, a=0.0):
        """class_pass plus, per link in update order: old angle, proposal, energy
        before its block, the block's dE and the accept decision."""
        n = self.geom.nslot
        bufs = [np.zeros(n) for _ in range(4)]
        acc = np.zeros(n, dtype=np.int32)
        m = lib().orc_lat_class_trace(self._h, int(cls), int(mode), float(a), _dp(bufs[0]),
                                      _dp(bufs[1]), _dp(bufs[2]), _dp(bufs[3]), _ip(acc))
        return dict(th_old=bufs[0][:m], th_prop=bufs[1][:m], E_before=bufs[2][:m],
                    dE=bufs[3][:m], accepted=acc[:m].astype(bool))

    def approach(self, max_sweeps):
        return lib().orc_lat_approach(self._h, int(max_sweeps))

    def rm_step(self, a, n_therm, n_meas, rm_index):
        m = ctypes.c_double(0.0)
        a_new = lib().orc_lat_rm_step(self._h, float(a), int(n_therm), int(n_meas),
                                      int(rm_index), ctypes.byref(m))
        return a_new, m.value


class MucaWeight:
    """ln rho~ of eq. (2.10) from the slopes of n contiguous intervals of width
    de starting at e0, continued linearly beyond them: the weight 1/rho~ of the
    multicanonical run (Sec. 2.6, eq. (2.50))."""

    def __init__(self, e0, de, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        self._a = a
        self._h = lib().orc_muca_new(len(a), float(e0), float(de), _dp(a))
        if not self._h:
            raise ValueError("bad multicanonical table")

    def lnrho(self, E):
        return lib().orc_muca_lnrho(self._h, float(E))

    def __del__(self):
        try:
            if self._h:
                lib().orc_muca_free(self._h)
        except Exception:
            pass


def muca_sweep(lattice, weight, a0, n_sweeps):
    """n multicanonical composite sweeps; returns the energy after each."""
    out = np.zeros(int(n_sweeps))
    lib().orc_lat_muca_sweep(lattice._h, weight._h, float(a0), int(n_sweeps), _dp(out))
    return out


def muca_class_trace(lattice, weight, cls, a0):
    """One multicanonical heat-bath class: per link (update order) the energy
    before it, its dE, the uniform u, the exponent x and the decision."""
    n = lattice.geom.nslot
    bufs = [np.zeros(n) for _ in range(4)]
    acc = np.zeros(n, dtype=np.int32)
    m = lib().orc_lat_muca_class_trace(lattice._h, weight._h, int(cls), float(a0), _dp(bufs[0]),
                                       _dp(bufs[1]), _dp(bufs[2]), _dp(bufs[3]), _ip(acc))
    return dict(E_before=bufs[0][:m], dE=bufs[1][:m], u=bufs[2][:m], x=bufs[3][:m],
                accepted=acc[:m].astype(bool))


def batch_run(geom: Geom, seed, interval_id, replica_id, E_lo, dE, a0, n_or=4, block=1,
              n_therm=50, n_meas=100, n_rm=20, rm_offset=0, max_approach=10000,
              beta_up=1.5, beta_dn=0.5, n_threads=1, history=False):
    """Independent LLR runs (Algorithm 1) for many lattices on host threads."""
    n = len(E_lo)
    iid = np.ascontiguousarray(interval_id, dtype=np.int32)
    rid = np.ascontiguousarray(replica_id, dtype=np.int32)
    elo = np.ascontiguousarray(E_lo, dtype=np.float64)
    de = np.ascontiguousarray(dE, dtype=np.float64)
    a = np.ascontiguousarray(a0, dtype=np.float64).copy()
    hist = np.zeros((n, n_rm)) if history else None
    status = np.zeros(n, dtype=np.int32)
    upd = np.zeros(n)
    lib().orc_batch_run(geom._h, n, int(seed) & (2 ** 64 - 1), _ip(iid), _ip(rid), _dp(elo),
                        _dp(de), _dp(a), _dp(hist) if hist is not None else None, n_or, block,
                        n_therm, n_meas, n_rm, rm_offset, max_approach, float(beta_up),
                        float(beta_dn), int(n_threads), _ip(status), _dp(upd))
    return dict(a=a, history=hist, status=status, updates=upd)


def parallel_sweeps(lattices, a, n_sweeps, n_threads):
    """n_sweeps composite sweeps on each lattice, lattices spread over host threads."""
    n = len(lattices)
    arr = (ctypes.c_void_p * n)(*[t._h for t in lattices])
    av = np.ascontiguousarray(np.broadcast_to(a, (n,)), dtype=np.float64)
    lib().orc_batch_sweeps(ctypes.cast(arr, ctypes.c_void_p), _dp(av), n, int(n_sweeps),
                           int(n_threads))


def replica_exchange(lattices, pairs, a, round_):
    """One replica-exchange round over the given pairs of lattices of
    overlapping intervals (Sec. 2.5).  Returns the accepted flags."""
    n = len(lattices)
    arr = (ctypes.c_void_p * n)(*[t._h for t in lattices])
    pr = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1)
    av = np.ascontiguousarray(np.broadcast_to(a, (n,)), dtype=np.float64)
    acc = np.zeros(max(len(pr) // 2, 1), dtype=np.int32)
    lib().orc_replica_exchange(ctypes.cast(arr, ctypes.c_void_p), len(pr) // 2, _ip(pr), _dp(av),
                               int(round_) & 0xFFFFFFFF, _ip(acc))
    return acc[:len(pr) // 2].astype(bool)


def parallel_approach(lattices, max_sweeps, n_threads):
    n = len(lattices)
    arr = (ctypes.c_void_p * n)(*[t._h for t in lattices])
    st = np.zeros(n, dtype=np.int32)
    lib().orc_batch_approach(ctypes.cast(arr, ctypes.c_void_p), _ip(st), n, int(max_sweeps),
                             int(n_threads))
    return st
