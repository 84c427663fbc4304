"""Thin ctypes binding of the C ABI in ``include/llr.h`` (argument marshalling only).

Every computation runs in the CUDA library ``_lib/libllr_gb300.so``; there is
no CPU fallback.  ``load()`` raises if the library is missing or cannot be
loaded.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libllr_gb300.so")

LLR_OK = 0
LLR_ERR_ARG = -1
LLR_ERR_CUDA = -2
LLR_ERR_WINDOW = -3
LLR_ERR_TIMEOUT = -4
LLR_ERR_NUMERIC = -5

# Every entry point declared in include/llr.h.
EXPORTS = [
    "llr_init_lattice", "llr_approach", "llr_sweep", "llr_pass", "llr_rm_step", "llr_rm_run", "llr_rm_step_dev",
    "llr_rm_step_plain", "llr_energy", "llr_tracked_energy", "llr_get_links", "llr_set_links",
    "llr_get_sweep_counter", "llr_set_sweep_counter", "llr_stats", "llr_status",
    "llr_reconstruct_lnrho", "llr_observables", "llr_cv_peak", "llr_set_kernel_config",
    "llr_destroy", "llr_last_error", "llr_observables_noalloc",
    "llr_mlp_create", "llr_mlp_num_params", "llr_mlp_get_params", "llr_mlp_set_params",
    "llr_mlp_set_norm", "llr_mlp_get_norm", "llr_mlp_predict", "llr_mlp_grad", "llr_mlp_fit",
    "llr_mlp_destroy", "llr_set_wait_limit", "llr_state_bytes", "llr_save_state",
    "llr_load_state", "llr_replica_exchange", "llr_set_muca_weight", "llr_muca_sweep",
    "llr_set_kernel_shape", "llr_get_last_launch", "llr_muca_reweight", "llr_muca_cv_peak",
    "llr_muca_tunnellings",
]
NOALLOC_MAX_CENTRES = 65536

_lib = None


class LLRError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (code %d)" % (msg, code))
        self.code = code


class _Config(ctypes.Structure):
    _fields_ = [
        ("n_lattices", ctypes.c_int),
        ("L", ctypes.POINTER(ctypes.c_int)),
        ("E_lo", ctypes.POINTER(ctypes.c_double)),
        ("dE", ctypes.POINTER(ctypes.c_double)),
        ("interval_id", ctypes.POINTER(ctypes.c_int)),
        ("replica_id", ctypes.POINTER(ctypes.c_int)),
        ("seed", ctypes.c_uint64),
        ("n_or", ctypes.c_int),
        ("accept_block", ctypes.c_int),
        ("beta_up", ctypes.c_double),
        ("beta_dn", ctypes.c_double),
        ("max_approach", ctypes.c_int),
    ]


def load(path: str = LIB_PATH):
    """Load the CUDA library (no fallback: raises if it is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("CUDA library %s is missing: run __graft_entry__.build() "
                           "(or python -m paper_1509_08391_gb300.build)" % path)
    L = ctypes.CDLL(path)
    P, I, D, U32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint32
    sig = {
        "llr_init_lattice": [ctypes.POINTER(P), ctypes.POINTER(_Config), P],
        "llr_approach": [P, I, P],
        "llr_sweep": [P, P, I, I, P],
        "llr_pass": [P, I, P, I],
        "llr_rm_step": [P, I, I, I, P, P],
        "llr_rm_step_dev": [P, I, I, I, P, P, P],
        "llr_rm_run": [P, I, I, I, I, P, P],
        "llr_rm_step_plain": [P, I, I, I, P, P],
        "llr_energy": [P, P],
        "llr_tracked_energy": [P, P],
        "llr_get_links": [P, I, P],
        "llr_set_links": [P, I, P],
        "llr_get_sweep_counter": [P, I, ctypes.POINTER(U32)],
        "llr_set_sweep_counter": [P, I, U32],
        "llr_stats": [P, P, I],
        "llr_status": [P, P],
        "llr_reconstruct_lnrho": [I, P, P, P],
        "llr_observables": [I, P, P, I, P, P, P, P],
        "llr_cv_peak": [I, P, P, D, D, I, D, P],
        "llr_muca_reweight": [ctypes.c_longlong, P, I, D, D, P, I, P, P, P],
        "llr_muca_cv_peak": [ctypes.c_longlong, P, I, D, D, P, D, D, I, D, P],
        "llr_muca_tunnellings": [I, I, P, D, D, P],
        "llr_set_kernel_config": [P, I, I],
        "llr_set_kernel_shape": [P, I, I, I, I],
        "llr_get_last_launch": [P, P],
        "llr_destroy": [P],
        "llr_observables_noalloc": [I, P, P, I, P, P, P, P, P],
        "llr_mlp_create": [ctypes.POINTER(P), ctypes.c_uint64, P],
        "llr_mlp_num_params": [],
        "llr_mlp_get_params": [P, P],
        "llr_mlp_set_params": [P, P],
        "llr_mlp_set_norm": [P, P, P],
        "llr_mlp_get_norm": [P, P, P],
        "llr_mlp_predict": [P, I, P, P, P, P],
        "llr_mlp_grad": [P, I, P, P, P, P, P, P],
        "llr_mlp_fit": [P, I, P, P, P, P, I, D, I, P],
        "llr_mlp_destroy": [P],
        "llr_set_wait_limit": [P, ctypes.c_ulonglong],
        "llr_save_state": [P, P],
        "llr_load_state": [P, P],
        "llr_replica_exchange": [P, I, P, P, U32, P],
        "llr_set_muca_weight": [P, I, D, D, P, D],
        "llr_muca_sweep": [P, I, P],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = I
    L.llr_state_bytes.argtypes = [P]
    L.llr_state_bytes.restype = ctypes.c_size_t
    L.llr_last_error.argtypes = []
    L.llr_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(code):
    if code != LLR_OK:
        raise LLRError(code, load().llr_last_error().decode())


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dev_ptr(x):
    """Device pointer of a torch CUDA tensor (or a raw int)."""
    if x is None:
        return None
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    return ctypes.c_void_p(x.data_ptr())


class Batch:
    """A batch of independent (interval, replica) lattices on one GPU."""

    def __init__(self, L, E_lo, dE, interval_id, replica_id, seed, n_or=4, block=1,
                 beta_up=1.5, beta_dn=0.5, max_approach=0, stream=None):
        lib = load()
        self.n = len(L)
        self._L = np.ascontiguousarray(L, dtype=np.int32)
        self._lo = np.ascontiguousarray(E_lo, dtype=np.float64)
        self._de = np.ascontiguousarray(dE, dtype=np.float64)
        self._iid = np.ascontiguousarray(interval_id, dtype=np.int32)
        self._rid = np.ascontiguousarray(replica_id, dtype=np.int32)
        cfg = _Config(self.n, self._L.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                      self._lo.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                      self._de.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                      self._iid.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                      self._rid.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                      int(seed) & (2 ** 64 - 1), int(n_or), int(block), float(beta_up),
                      float(beta_dn), int(max_approach))
        h = ctypes.c_void_p()
        code = lib.llr_init_lattice(ctypes.byref(h), ctypes.byref(cfg),
                                    ctypes.c_void_p(stream) if stream else None)
        self._h = h
        _check(code)

    @classmethod
    def from_workload(cls, w, stream=None, max_approach=None):
        return cls(w.L, w.E_lo, w.dE, w.interval_id, w.replica_id, w.seed, n_or=w.n_or,
                   block=w.block, beta_up=w.beta_up, beta_dn=w.beta_dn,
                   max_approach=w.max_approach if max_approach is None else max_approach,
                   stream=stream)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().llr_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -------------------------------------------------------------- dynamics
    def set_kernel_config(self, threads=256, fast_math=True):
        _check(load().llr_set_kernel_config(self._h, int(threads), 1 if fast_math else 0))

    def set_kernel_shape(self, threads=256, fast_math=True, ring=4, carveout=-1):
        _check(load().llr_set_kernel_shape(self._h, int(threads), 1 if fast_math else 0,
                                           int(ring), int(carveout)))

    def last_launch(self):
        """{threads, fast_math, ring, carveout, grid} of the last batched launch."""
        out = np.zeros(5, dtype=np.int32)
        _check(load().llr_get_last_launch(self._h, _ptr(out)))
        return dict(zip(("threads", "fast_math", "ring", "carveout", "grid"),
                        (int(v) for v in out)))

    def approach(self, max_sweeps):
        out = np.zeros(self.n, dtype=np.int32)
        _check(load().llr_approach(self._h, int(max_sweeps), _ptr(out)))
        return out

    def sweep(self, a, n_sweeps=1, measure=False):
        a = np.ascontiguousarray(np.broadcast_to(a, (self.n,)), dtype=np.float64)
        out = np.zeros(self.n)
        _check(load().llr_sweep(self._h, _ptr(a), int(n_sweeps), 1 if measure else 0, _ptr(out)))
        return out

    def single_pass(self, kind, a=None, class_mask=0xFF):
        if a is not None:
            a = np.ascontiguousarray(np.broadcast_to(a, (self.n,)), dtype=np.float64)
        _check(load().llr_pass(self._h, int(kind), _ptr(a) if a is not None else None,
                               int(class_mask)))

    def rm_step(self, a, n_therm, n_meas, rm_index):
        a = np.ascontiguousarray(np.broadcast_to(a, (self.n,)), dtype=np.float64).copy()
        mean = np.zeros(self.n)
        _check(load().llr_rm_step(self._h, int(n_therm), int(n_meas), int(rm_index), _ptr(a),
                                  _ptr(mean)))
        return a, mean

    def rm_step_dev(self, a_in, a_out, n_therm, n_meas, rm_index, mean_out=None):
        _check(load().llr_rm_step_dev(self._h, int(n_therm), int(n_meas), int(rm_index),
                                      _dev_ptr(a_in), _dev_ptr(a_out), _dev_ptr(mean_out)))

    def rm_run(self, a_dev, n_therm, n_meas, rm_index0, n_steps, hist_dev=None):
        """n_steps graph-replayed Robbins-Monro iterations on device buffers."""
        _check(load().llr_rm_run(self._h, int(n_therm), int(n_meas), int(rm_index0),
                                 int(n_steps), _dev_ptr(a_dev), _dev_ptr(hist_dev)))

    def rm_step_plain(self, a, n_therm, n_meas, rm_index):
        a = np.ascontiguousarray(np.broadcast_to(a, (self.n,)), dtype=np.float64).copy()
        mean = np.zeros(self.n)
        _check(load().llr_rm_step_plain(self._h, int(n_therm), int(n_meas), int(rm_index),
                                        _ptr(a), _ptr(mean)))
        return a, mean

    def replica_exchange(self, pairs, a, round_):
        """One replica-exchange round over pairs of lattices of overlapping
        intervals (llr_replica_exchange); returns the exchanged flags."""
        pr = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1)
        a = np.ascontiguousarray(np.broadcast_to(a, (self.n,)), dtype=np.float64)
        acc = np.zeros(max(pr.size // 2, 1), dtype=np.int32)
        _check(load().llr_replica_exchange(self._h, pr.size // 2, _ptr(pr), _ptr(a),
                                           int(round_) & 0xFFFFFFFF, _ptr(acc)))
        return acc[:pr.size // 2].astype(bool)

    def set_muca_weight(self, e0, de, a, a0):
        """The multicanonical weight 1/rho~ (llr_set_muca_weight)."""
        a = np.ascontiguousarray(a, dtype=np.float64)
        _check(load().llr_set_muca_weight(self._h, a.size, float(e0), float(de), _ptr(a),
                                          float(a0)))

    def muca_sweep(self, n_sweeps, history=True):
        """n multicanonical composite sweeps; the energies after each sweep as
        an (n_sweeps, n_lattices) array (or None)."""
        out = np.zeros((int(n_sweeps), self.n)) if history else None
        _check(load().llr_muca_sweep(self._h, int(n_sweeps),
                                     _ptr(out) if out is not None else None))
        return out

    # ------------------------------------------------------------ inspection
    def energy(self):
        out = np.zeros(self.n)
        _check(load().llr_energy(self._h, _ptr(out)))
        return out

    def tracked_energy(self):
        out = np.zeros(self.n)
        _check(load().llr_tracked_energy(self._h, _ptr(out)))
        return out

    def get_links(self, i):
        out = np.zeros(4 * int(self._L[i]) ** 4, dtype=np.float32)
        _check(load().llr_get_links(self._h, int(i), _ptr(out)))
        return out

    def set_links(self, i, th):
        th = np.ascontiguousarray(th, dtype=np.float32)
        assert th.size == 4 * int(self._L[i]) ** 4
        _check(load().llr_set_links(self._h, int(i), _ptr(th)))

    def get_sweep_counter(self, i):
        v = ctypes.c_uint32(0)
        _check(load().llr_get_sweep_counter(self._h, int(i), ctypes.byref(v)))
        return v.value

    def set_sweep_counter(self, i, value):
        _check(load().llr_set_sweep_counter(self._h, int(i), int(value) & 0xFFFFFFFF))

    def stats(self, reset=False):
        out = np.zeros((self.n, 8))
        _check(load().llr_stats(self._h, _ptr(out), 1 if reset else 0))
        keys = ["hb_acc", "hb_tot", "or_acc", "or_tot", "caps", "max_drift", "sweeps", "status"]
        return {k: out[:, j] for j, k in enumerate(keys)}

    def status(self):
        out = np.zeros(self.n, dtype=np.int32)
        _check(load().llr_status(self._h, _ptr(out)))
        return out

    def set_wait_limit(self, ns):
        _check(load().llr_set_wait_limit(self._h, int(ns)))

    def save_state(self):
        """The chain state of every lattice as bytes (checkpoint)."""
        buf = np.zeros(load().llr_state_bytes(self._h), dtype=np.uint8)
        _check(load().llr_save_state(self._h, _ptr(buf)))
        return buf.tobytes()

    def load_state(self, blob):
        buf = np.frombuffer(blob, dtype=np.uint8).copy()
        assert buf.size == load().llr_state_bytes(self._h)
        _check(load().llr_load_state(self._h, _ptr(buf)))


def reconstruct_lnrho(centres, a):
    c = np.ascontiguousarray(centres, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    out = np.zeros_like(c)
    _check(load().llr_reconstruct_lnrho(len(c), _ptr(c), _ptr(a), _ptr(out)))
    return out


def observables(centres, a, betas):
    c = np.ascontiguousarray(centres, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(np.atleast_1d(betas), dtype=np.float64)
    lz, e1, e2 = np.zeros_like(b), np.zeros_like(b), np.zeros_like(b)
    _check(load().llr_observables(len(c), _ptr(c), _ptr(a), len(b), _ptr(b), _ptr(lz), _ptr(e1),
                                  _ptr(e2)))
    return lz, e1, e2


def cv_peak(centres, a, beta_lo, beta_hi, n_grid=2001, tol=1e-12):
    c = np.ascontiguousarray(centres, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    out = np.zeros(2)
    _check(load().llr_cv_peak(len(c), _ptr(c), _ptr(a), float(beta_lo), float(beta_hi),
                              int(n_grid), float(tol), _ptr(out)))
    return float(out[0]), float(out[1])


def muca_reweight(E, e0, de, a, betas):
    """<E>, <E^2> of multicanonical samples E (any shape, pooled) reweighted
    to each coupling (llr_muca_reweight, eq. (2.56))."""
    x = np.ascontiguousarray(np.ravel(E), dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(np.atleast_1d(betas), dtype=np.float64)
    e1, e2 = np.zeros_like(b), np.zeros_like(b)
    _check(load().llr_muca_reweight(x.size, _ptr(x), len(a), float(e0), float(de), _ptr(a),
                                    len(b), _ptr(b), _ptr(e1), _ptr(e2)))
    return e1, e2


def muca_cv_peak(E, e0, de, a, beta_lo, beta_hi, n_grid=401, tol=1e-10):
    """(beta_c, C_V(beta_c)) of reweighted multicanonical samples (llr_muca_cv_peak)."""
    x = np.ascontiguousarray(np.ravel(E), dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    out = np.zeros(2)
    _check(load().llr_muca_cv_peak(x.size, _ptr(x), len(a), float(e0), float(de), _ptr(a),
                                   float(beta_lo), float(beta_hi), int(n_grid), float(tol),
                                   _ptr(out)))
    return float(out[0]), float(out[1])


def muca_tunnellings(E, lo, hi):
    """Tunnellings per chain of E[step][chain] between E < lo and E > hi
    (llr_muca_tunnellings)."""
    x = np.ascontiguousarray(np.atleast_2d(E), dtype=np.float64)
    out = np.zeros(x.shape[1], dtype=np.int32)
    _check(load().llr_muca_tunnellings(x.shape[0], x.shape[1], _ptr(x), float(lo), float(hi),
                                       _ptr(out)))
    return out


def observables_noalloc(centres_dev, a_dev, beta_dev, lnZ_dev, E_dev, E2_dev, stream=None):
    """llr_observables_noalloc on caller-owned device buffers (torch tensors or
    raw device pointers); enqueues on `stream` and allocates nothing."""
    n = centres_dev.numel() if hasattr(centres_dev, "numel") else None
    nb = beta_dev.numel() if hasattr(beta_dev, "numel") else None
    _check(load().llr_observables_noalloc(int(n), _dev_ptr(centres_dev), _dev_ptr(a_dev),
                                          int(nb), _dev_ptr(beta_dev), _dev_ptr(lnZ_dev),
                                          _dev_ptr(E_dev), _dev_ptr(E2_dev),
                                          ctypes.c_void_p(stream) if stream else None))


class MLP:
    """The warm-start network (llr_mlp_* entry points)."""

    def __init__(self, seed=1, stream=None):
        lib = load()
        h = ctypes.c_void_p()
        code = lib.llr_mlp_create(ctypes.byref(h), int(seed) & (2 ** 64 - 1),
                                  ctypes.c_void_p(stream) if stream else None)
        self._h = h
        _check(code)
        self.n_params = lib.llr_mlp_num_params()

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().llr_mlp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @staticmethod
    def _in(L, e, d):
        return [np.ascontiguousarray(x, dtype=np.float64) for x in (L, e, d)]

    def get_params(self):
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(load().llr_mlp_get_params(self._h, _ptr(out)))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.n_params
        _check(load().llr_mlp_set_params(self._h, _ptr(p)))

    def set_norm(self, mean, std):
        m = np.ascontiguousarray(mean, dtype=np.float64)
        s = np.ascontiguousarray(std, dtype=np.float64)
        _check(load().llr_mlp_set_norm(self._h, _ptr(m), _ptr(s)))

    def get_norm(self):
        m, s = np.zeros(3), np.zeros(3)
        _check(load().llr_mlp_get_norm(self._h, _ptr(m), _ptr(s)))
        return m, s

    def predict(self, L, e6v, dE6v):
        L, e, d = self._in(L, e6v, dE6v)
        out = np.zeros(L.size)
        _check(load().llr_mlp_predict(self._h, L.size, _ptr(L), _ptr(e), _ptr(d), _ptr(out)))
        return out

    def grad(self, L, e6v, dE6v, target):
        L, e, d = self._in(L, e6v, dE6v)
        t = np.ascontiguousarray(target, dtype=np.float64)
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = ctypes.c_double(0.0)
        _check(load().llr_mlp_grad(self._h, L.size, _ptr(L), _ptr(e), _ptr(d), _ptr(t), _ptr(g),
                                   ctypes.byref(loss)))
        return g, loss.value

    def fit(self, L, e6v, dE6v, target, epochs, lr=1e-3, standardise=True):
        L, e, d = self._in(L, e6v, dE6v)
        t = np.ascontiguousarray(target, dtype=np.float64)
        loss = ctypes.c_double(0.0)
        _check(load().llr_mlp_fit(self._h, L.size, _ptr(L), _ptr(e), _ptr(d), _ptr(t),
                                  int(epochs), float(lr), 1 if standardise else 0,
                                  ctypes.byref(loss)))
        return loss.value
