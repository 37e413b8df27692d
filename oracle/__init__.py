"""CPU oracle for arXiv:1604.07515 (Parallel Local Graph Clustering).

TEST INFRASTRUCTURE ONLY: a plain, slow, single-threaded restatement of the
paper's algorithms, used to check the CUDA library.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  The library itself never loads it and
shares no code with it.

The arithmetic lives in ``oracle.cpp`` (built with ``-ffp-contract=off``);
this module only compiles it on demand and marshals numpy arrays through
ctypes.  Functions and the paper passages they follow:

* ``prnibble``        Sec. 3.3, Fig. alg:pr-nibble / alg:pr-nibble2 (synchronous)
* ``prnibble_queue``  Sec. 3.3, sequential FIFO push (push counts only)
* ``nibble``          Sec. 3.2, Fig. alg:nibble
* ``hkpr``            Sec. 3.4, Fig. alg:hkpr (level-synchronous)
* ``hkpr_queue``      Sec. 3.4, sequential queue over (vertex, level)
* ``hkpr_psi``        Sec. 3.4, the psi_k coefficients
* ``rand_hkpr``       Sec. 3.5 (walk endpoints and p = counts / walks)
* ``sweep``           Sec. 3.1, sequential sweep cut
* ``sweep_zpath``     Sec. 3.1, Theorem thm:sweep (the Z array construction)
* ``philox4x32_10``   Salmon et al., SC'11 (random stream of ``rand_hkpr``)

parity: every function is pinned by the ``-m "not gpu"`` tests; the Philox
words against cuRAND's host-side Philox4x32-10 generator (a library routine)
on the counter words ``rand_hkpr`` uses.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# field ids, kinds and stat slots (mirror the enums in oracle.cpp)
IDX, VAL, IDX2, VAL2, TRACE, TRACE_N, ORDER, VOL, CUT, ENDPT = range(10)
Z1, Z2, ZS1, ZS2, ZSUM, PUSHED = range(10, 16)
_I32, _I64, _F64 = 0, 1, 2
ST_ROUNDS, ST_PUSHES, ST_PUSHED_EDGES, ST_TOUCHED, ST_STATUS, ST_BEST, ST_BEST_VOL, ST_BEST_CUT = range(8)


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so (no FMA contraction)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64, i32, f64, ci = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_int
        lib.orc_len.restype = i64
        lib.orc_len.argtypes = [P, ci, ci]
        lib.orc_copy.argtypes = [P, ci, ci, P]
        lib.orc_stats.argtypes = [P, P]
        lib.orc_conductance.restype = f64
        lib.orc_conductance.argtypes = [P]
        lib.orc_free.argtypes = [P]
        lib.orc_philox4x32_10.argtypes = [P, P, P]
        lib.orc_hkpr_psi.argtypes = [f64, ci, P]
        g = [i64, P, P]
        for name, extra in [
            ("orc_prnibble", [i32, f64, f64, ci, i64, ci]),
            ("orc_prnibble_queue", [i32, f64, f64, ci]),
            ("orc_prnibble_set", [i64, P, P, f64, f64, ci, f64, i64, ci]),
            ("orc_nibble", [i32, ci, f64, ci]),
            ("orc_hkpr", [i32, f64, ci, f64, ci]),
            ("orc_hkpr_signed", [i32, f64, ci, f64, ci, ci]),
            ("orc_hkpr_queue", [i32, f64, ci, f64]),
            ("orc_rand_hkpr", [i32, f64, ci, i64, ctypes.c_uint64]),
            ("orc_sweep", [i64, P, P]),
            ("orc_sweep_zpath", [i64, P]),
        ]:
            fn = getattr(lib, name)
            fn.restype = P
            fn.argtypes = g + extra
        _lib = lib
    return _lib


@dataclass
class Result:
    """Arrays and counters returned by one oracle call."""
    idx: np.ndarray = None
    val: np.ndarray = None
    idx2: np.ndarray = None
    val2: np.ndarray = None
    trace: list = field(default_factory=list)   # per-round frontiers (ascending)
    pushed_per_round: np.ndarray = None
    rounds: int = 0
    pushes: int = 0
    pushed_edges: int = 0
    touched: int = 0
    status: int = 0
    # sweep
    order: np.ndarray = None
    vol: np.ndarray = None
    cut: np.ndarray = None
    best: int = 0
    best_vol: int = 0
    best_cut: int = 0
    conductance: float = float("inf")
    # rand-HK-PR
    endpoints: np.ndarray = None
    # Z path
    z: np.ndarray = None
    z_sorted: np.ndarray = None
    z_summed: np.ndarray = None

    @property
    def cluster(self) -> np.ndarray:
        return self.order[: self.best] if self.order is not None else None


def _arr(lib, h, fld, kind):
    n = lib.orc_len(h, fld, kind)
    dt = {_I32: np.int32, _I64: np.int64, _F64: np.float64}[kind]
    a = np.empty(n, dtype=dt)
    if n:
        lib.orc_copy(h, fld, kind, a.ctypes.data)
    return a


def _collect(h) -> Result:
    lib = _load()
    st = np.zeros(8, dtype=np.int64)
    lib.orc_stats(h, st.ctypes.data)
    r = Result()
    r.idx, r.val = _arr(lib, h, IDX, _I32), _arr(lib, h, VAL, _F64)
    r.idx2, r.val2 = _arr(lib, h, IDX2, _I32), _arr(lib, h, VAL2, _F64)
    tr, trn = _arr(lib, h, TRACE, _I32), _arr(lib, h, TRACE_N, _I64)
    pos = np.concatenate([[0], np.cumsum(trn)]).astype(np.int64)
    r.trace = [tr[pos[k]:pos[k + 1]] for k in range(len(trn))]
    r.pushed_per_round = _arr(lib, h, PUSHED, _I64)
    (r.rounds, r.pushes, r.pushed_edges, r.touched, r.status,
     r.best, r.best_vol, r.best_cut) = (int(x) for x in st)
    r.order = _arr(lib, h, ORDER, _I32)
    r.vol, r.cut = _arr(lib, h, VOL, _I64), _arr(lib, h, CUT, _I64)
    r.conductance = lib.orc_conductance(h)
    r.endpoints = _arr(lib, h, ENDPT, _I32)
    z1, z2 = _arr(lib, h, Z1, _I64), _arr(lib, h, Z2, _I64)
    r.z = np.stack([z1, z2], axis=1) if len(z1) else None
    zs1, zs2 = _arr(lib, h, ZS1, _I64), _arr(lib, h, ZS2, _I64)
    r.z_sorted = np.stack([zs1, zs2], axis=1) if len(zs1) else None
    zsum = _arr(lib, h, ZSUM, _I64)
    r.z_summed = np.stack([zsum, zs2], axis=1) if len(zsum) else None
    lib.orc_free(h)
    return r


def _g(off, col):
    off = np.ascontiguousarray(off, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    return off, col, len(off) - 1


def prnibble(off, col, seed, alpha, eps, rule=0, max_rounds=1 << 40, trace=False) -> Result:
    off, col, n = _g(off, col)
    h = _load().orc_prnibble(n, off.ctypes.data, col.ctypes.data, int(seed), float(alpha),
                             float(eps), int(rule), int(max_rounds), int(bool(trace)))
    return _collect(h)


def prnibble_set(off, col, seeds, weights, alpha, eps, rule=0, beta=1.0,
                 max_rounds=1 << 40, trace=False) -> Result:
    """PR-Nibble from a weighted seed set with beta-fraction rounds
    (orc_prnibble_set)."""
    off, col, n = _g(off, col)
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    weights = np.ascontiguousarray(np.broadcast_to(np.asarray(weights, dtype=np.float64),
                                                   seeds.shape))
    h = _load().orc_prnibble_set(n, off.ctypes.data, col.ctypes.data, len(seeds),
                                 seeds.ctypes.data, weights.ctypes.data, float(alpha),
                                 float(eps), int(rule), float(beta), int(max_rounds),
                                 int(bool(trace)))
    return _collect(h)


def prnibble_queue(off, col, seed, alpha, eps, rule=0) -> Result:
    off, col, n = _g(off, col)
    h = _load().orc_prnibble_queue(n, off.ctypes.data, col.ctypes.data, int(seed),
                                   float(alpha), float(eps), int(rule))
    return _collect(h)


def nibble(off, col, seed, T, eps, trace=False) -> Result:
    off, col, n = _g(off, col)
    h = _load().orc_nibble(n, off.ctypes.data, col.ctypes.data, int(seed), int(T), float(eps),
                           int(bool(trace)))
    return _collect(h)


def hkpr(off, col, seed, t, N, eps, trace=False, threshold_sign=1) -> Result:
    """threshold_sign -1: the entry thresholds with e^{-t} (Sec. 3.4's
    sequential description) instead of the parallel figure's e^{t}."""
    off, col, n = _g(off, col)
    h = _load().orc_hkpr_signed(n, off.ctypes.data, col.ctypes.data, int(seed), float(t),
                                int(N), float(eps), int(bool(trace)),
                                -1 if threshold_sign < 0 else 1)
    return _collect(h)


def hkpr_queue(off, col, seed, t, N, eps) -> Result:
    off, col, n = _g(off, col)
    h = _load().orc_hkpr_queue(n, off.ctypes.data, col.ctypes.data, int(seed), float(t),
                               int(N), float(eps))
    return _collect(h)


def hkpr_psi(t, N) -> np.ndarray:
    psi = np.zeros(N + 1, dtype=np.float64)
    _load().orc_hkpr_psi(float(t), int(N), psi.ctypes.data)
    return psi


def rand_hkpr(off, col, seed, t, K, n_walks, rng_seed) -> Result:
    off, col, n = _g(off, col)
    h = _load().orc_rand_hkpr(n, off.ctypes.data, col.ctypes.data, int(seed), float(t), int(K),
                              int(n_walks), int(rng_seed) & ((1 << 64) - 1))
    return _collect(h)


def sweep(off, col, idx, val) -> Result:
    off, col, n = _g(off, col)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    h = _load().orc_sweep(n, off.ctypes.data, col.ctypes.data, len(idx), idx.ctypes.data,
                          val.ctypes.data)
    return _collect(h)


def sweep_zpath(off, col, order) -> Result:
    off, col, n = _g(off, col)
    order = np.ascontiguousarray(order, dtype=np.int32)
    h = _load().orc_sweep_zpath(n, off.ctypes.data, col.ctypes.data, len(order),
                                order.ctypes.data)
    return _collect(h)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out
