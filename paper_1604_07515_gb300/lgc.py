"""ctypes binding of liblgc (include/lgc.h): argument marshalling only.

Every step of every method runs in the library's CUDA kernels; this module
converts numpy / torch buffers to pointers and back.  There is no CPU
fallback: if the library cannot be loaded or no GPU is present, calls raise.

Names follow the C ABI without the ``lgc_`` prefix::

    ctx = Context(0)                       # lgc_ctx_create
    g = Graph(ctx, off, col)               # lgc_graph_create (host or CUDA tensors)
    p, st = prnibble(g, seed, alpha=0.01, eps=1e-6, mode="det")
    c = sweep(g, p)                        # lgc_sweep
"""
from __future__ import annotations

import ctypes
import os
import threading
import weakref
from ctypes import POINTER, byref, c_double, c_int, c_int32, c_int64, c_uint64, c_void_p

import numpy as np

from . import build as _build

LGC_OK, LGC_PENDING = 0, 1
LGC_EINVAL, LGC_ENOMEM, LGC_ETABLEFULL, LGC_EMAXROUNDS = -1, -2, -3, -4
LGC_ECUDA, LGC_EBUSY, LGC_ENOTFOUND, LGC_ETIMEOUT = -5, -6, -7, -8
OPT_RESULT_ON_DEVICE, OPT_TRACE, OPT_SERVE_MEM_BUDGET, OPT_SERVE_MAX_BATCH = 1, 2, 3, 4
GRAPH_VALIDATE, GRAPH_DEVICE_INPUT = 1, 2
ALGO_PRNIBBLE, ALGO_NIBBLE, ALGO_HKPR, ALGO_RAND_HKPR = 0, 1, 2, 3
_RULES = {"opt": 0, "orig": 1, 0: 0, 1: 1}
_MODES = {"atomic": 0, "det": 1, 0: 0, 1: 1}


class LgcError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {_lib_or_none_strerror(status)} ({status})")
        self.status = status


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class AllocFns(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", ctypes.c_void_p)]


def torch_allocator(device: int):
    """(alloc, free) callables that take the library's device memory from
    PyTorch's caching allocator (stream-ordered per stream)."""
    import torch

    def alloc(nbytes, stream):
        return torch.cuda.caching_allocator_alloc(nbytes, device, stream)

    def free(ptr, stream):
        torch.cuda.caching_allocator_delete(ptr)

    return alloc, free


class Svec(ctypes.Structure):
    _fields_ = [("nnz", c_int64), ("idx", c_void_p), ("val", c_void_p), ("on_device", c_int)]


class Cluster(ctypes.Structure):
    _fields_ = [("size", c_int64), ("ids", c_void_p), ("vol", c_int64), ("cut", c_int64),
                ("conductance", c_double), ("on_device", c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("rounds", c_int64), ("pushes", c_int64), ("pushed_edges", c_int64),
                ("touched", c_int64), ("table_capacity", c_int64), ("status_detail", c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class PRNibbleParams(ctypes.Structure):
    _fields_ = [("alpha", c_double), ("eps", c_double), ("rule", c_int), ("mode", c_int),
                ("max_rounds", c_int64)]


class NibbleParams(ctypes.Structure):
    _fields_ = [("T", c_int), ("eps", c_double), ("mode", c_int)]


class HKPRParams(ctypes.Structure):
    _fields_ = [("t", c_double), ("eps", c_double), ("N", c_int), ("mode", c_int)]


class RandHKPRParams(ctypes.Structure):
    _fields_ = [("t", c_double), ("K", c_int), ("n_walks", c_int64), ("rng_seed", c_uint64)]


class Request(ctypes.Structure):
    _fields_ = [("algo", c_int), ("seed", c_int32), ("want_sweep", c_int),
                ("pr", PRNibbleParams), ("nb", NibbleParams), ("hk", HKPRParams),
                ("rh", RandHKPRParams)]


class Result(ctypes.Structure):
    _fields_ = [("status", c_int), ("p", POINTER(Svec)), ("cluster", POINTER(Cluster)),
                ("stats", Stats), ("submit_s", c_double), ("start_s", c_double),
                ("end_s", c_double)]


_lib = None
_lock = threading.Lock()

# every symbol the header declares, with (restype, argtypes)
_P = c_void_p
SIGNATURES = {
    "lgc_ctx_create": (c_int, [c_int, _P, POINTER(_P)]),
    "lgc_ctx_create_with_alloc": (c_int, [c_int, POINTER(AllocFns), _P, POINTER(_P)]),
    "lgc_set_trace": (c_int, [_P, c_int]),
    "lgc_ctx_destroy": (None, [_P]),
    "lgc_ctx_set_option": (c_int, [_P, c_int, c_int64]),
    "lgc_ctx_synchronize": (c_int, [_P]),
    "lgc_graph_create": (c_int, [_P, c_int64, _P, _P, c_int, POINTER(_P)]),
    "lgc_graph_destroy": (None, [_P]),
    "lgc_graph_num_vertices": (c_int64, [_P]),
    "lgc_graph_batch_handoff": (c_int64, [_P]),
    "lgc_graph_pull_light": (c_int, [_P]),
    "lgc_graph_set_pull_light": (c_int, [_P, c_int]),
    "lgc_graph_num_entries": (c_int64, [_P]),
    "lgc_prnibble": (c_int, [_P, c_int32, POINTER(PRNibbleParams), POINTER(POINTER(Svec)),
                             POINTER(Stats)]),
    "lgc_nibble": (c_int, [_P, c_int32, POINTER(NibbleParams), POINTER(POINTER(Svec)),
                           POINTER(Stats)]),
    "lgc_hkpr": (c_int, [_P, c_int32, POINTER(HKPRParams), POINTER(POINTER(Svec)),
                         POINTER(Stats)]),
    "lgc_rand_hkpr": (c_int, [_P, c_int32, POINTER(RandHKPRParams), POINTER(POINTER(Svec)),
                              POINTER(Stats)]),
    "lgc_rand_hkpr_endpoints": (c_int, [_P, _P, c_int64]),
    "lgc_sweep": (c_int, [_P, POINTER(Svec), POINTER(POINTER(Cluster))]),
    "lgc_sweep_batch": (c_int, [_P, c_int64, _P, _P]),
    "lgc_graph_autotune": (c_int, [_P, POINTER(c_int), POINTER(c_int), POINTER(c_int)]),
    "lgc_get_trace": (c_int, [_P, POINTER(c_int64), _P, c_int64, _P, c_int64]),
    "lgc_prnibble_residual": (c_int, [_P, POINTER(POINTER(Svec))]),
    "lgc_submit": (c_int, [_P, _P, POINTER(Request), POINTER(c_uint64)]),
    "lgc_poll": (c_int, [_P, c_uint64, POINTER(POINTER(Result))]),
    "lgc_wait": (c_int, [_P, c_uint64, POINTER(POINTER(Result))]),
    "lgc_svec_free": (None, [POINTER(Svec)]),
    "lgc_cluster_free": (None, [POINTER(Cluster)]),
    "lgc_result_free": (None, [POINTER(Result)]),
    "lgc_strerror": (ctypes.c_char_p, [c_int]),
    "lgc_sweep_noalloc": (c_int, [_P, c_int64, _P, _P, _P, POINTER(Cluster)]),
    "lgc_prnibble_batch": (c_int, [_P, c_int64, _P, _P, _P, _P]),
    "lgc_prnibble_set": (c_int, [_P, c_int64, _P, _P, c_double, POINTER(PRNibbleParams),
                                 POINTER(POINTER(Svec)), POINTER(Stats)]),
    "lgc_launch_count": (c_int64, [_P]),
    "lgc_profile_read": (c_int, [_P, c_int, _P]),
    "lgc_profile_reset": (c_int, [_P]),
}

OPT_PROFILE = 5
OPT_TABLE_FORM = 6
OPT_PULL = 7
OPT_DEVICE_ROUNDS = 8
OPT_PULL_BATCH = 9
OPT_PULL_GROUP = 10
OPT_PULL_SHARE = 11
OPT_BATCH_HANDOFF = 12
OPT_HK_THRESHOLD_SIGN = 13
OPT_SERVE_LANE = 14
OPT_SWEEP_CROSS = 15
PROF_EDGEMAP, PROF_VERTEXMAP, PROF_DET_EDGE, PROF_WALK, PROF_SWEEP, PROF_PULL = range(6)
PROF_NAMES = {PROF_EDGEMAP: "edgemap_push", PROF_VERTEXMAP: "vertexmap",
              PROF_DET_EDGE: "det_edge", PROF_WALK: "walk", PROF_SWEEP: "sweep_cross",
              PROF_PULL: "edgemap_pull"}


class KernelProfile(ctypes.Structure):
    _fields_ = [("launches", c_int64), ("ms", c_double), ("bytes", c_double)]


def library_path() -> str:
    return _build.OUT


def load(auto_build: bool = True):
    """Loads liblgc.so, compiling it first if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not _build.up_to_date():
            if not auto_build:
                raise ImportError(f"liblgc.so missing or stale at {_build.OUT}; run build()")
            _build.build()
        lib = ctypes.CDLL(_build.OUT)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _lib_or_none_strerror(status: int) -> str:
    try:
        return load(auto_build=False).lgc_strerror(status).decode()
    except Exception:
        return "status"


def _check(status: int, what: str, ok=(LGC_OK,)) -> int:
    if status not in ok:
        raise LgcError(status, what)
    return status


def _ptr(a) -> int:
    """Data pointer of a numpy array or a torch tensor."""
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


class Context:
    """lgc_ctx: one CUDA stream (the caller's, e.g. torch's current stream)."""

    def __init__(self, device: int = 0, stream=None, allocator=None):
        """allocator: None (the device's stream-ordered pool), "torch"
        (PyTorch's caching allocator), or a pair of callables
        alloc(nbytes, stream) -> int pointer (0 on failure) and
        free(ptr, stream) (lgc_ctx_create_with_alloc)."""
        lib = load()
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        h = c_void_p()
        self._alloc_fns = None
        if allocator is None:
            _check(lib.lgc_ctx_create(device, stream, byref(h)), "lgc_ctx_create")
        else:
            a, f = torch_allocator(device) if allocator == "torch" else allocator

            def c_alloc(nbytes, strm, user):
                try:
                    return a(int(nbytes), int(strm or 0)) or None
                except Exception:
                    return None  # the library reports LGC_ENOMEM

            def c_free(ptr, strm, user):
                try:
                    f(int(ptr), int(strm or 0))
                except Exception:
                    pass

            # the callbacks live as long as the context
            self._alloc_fns = AllocFns(ALLOC_FN(c_alloc), FREE_FN(c_free), None)
            _check(lib.lgc_ctx_create_with_alloc(device, byref(self._alloc_fns), stream,
                                                 byref(h)), "lgc_ctx_create_with_alloc")
        self.handle = h
        self.device = device
        self._graphs = weakref.WeakSet()  # graphs must be destroyed before the context

    def set_option(self, option: int, value: int):
        _check(load().lgc_ctx_set_option(self.handle, option, int(value)), "lgc_ctx_set_option")

    def set_trace(self, flags: int = 1):
        """lgc_set_trace: 1 records every round's frontier, 0 stops."""
        _check(load().lgc_set_trace(self.handle, int(flags)), "lgc_set_trace")

    def synchronize(self):
        _check(load().lgc_ctx_synchronize(self.handle), "lgc_ctx_synchronize")

    def trace(self) -> list[np.ndarray]:
        lib = load()
        rounds = c_int64()
        _check(lib.lgc_get_trace(self.handle, byref(rounds), None, 0, None, 0), "lgc_get_trace")
        sizes = np.zeros(rounds.value, np.int64)
        total = 0
        if rounds.value:
            _check(lib.lgc_get_trace(self.handle, byref(rounds), sizes.ctypes.data,
                                     rounds.value, None, 0), "lgc_get_trace")
            total = int(sizes.sum())
        ids = np.zeros(total, np.int32)
        if total:
            _check(lib.lgc_get_trace(self.handle, byref(rounds), None, 0, ids.ctypes.data,
                                     total), "lgc_get_trace")
        pos = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        return [ids[pos[k]:pos[k + 1]] for k in range(rounds.value)]

    def residual(self):
        r = POINTER(Svec)()
        _check(load().lgc_prnibble_residual(self.handle, byref(r)), "lgc_prnibble_residual")
        return _take_svec(r)

    def rand_hkpr_endpoints(self, n_walks: int) -> np.ndarray:
        out = np.zeros(n_walks, np.int32)
        _check(load().lgc_rand_hkpr_endpoints(self.handle, out.ctypes.data, n_walks),
               "lgc_rand_hkpr_endpoints")
        return out

    def launch_count(self) -> int:
        return load().lgc_launch_count(self.handle)

    def profile(self, kernel: int) -> dict:
        out = KernelProfile()
        _check(load().lgc_profile_read(self.handle, kernel, ctypes.addressof(out)),
               "lgc_profile_read")
        return {"launches": out.launches, "ms": out.ms, "bytes": out.bytes}

    def profile_reset(self):
        _check(load().lgc_profile_reset(self.handle), "lgc_profile_reset")

    def _own(self, obj):
        """Registers a graph or device-resident result released before the context."""
        self._graphs.add(obj)

    def close(self):
        if getattr(self, "handle", None):
            for obj in list(self._graphs):  # results first, then graphs
                if not isinstance(obj, Graph):
                    obj.close()
            for obj in list(self._graphs):
                obj.close()
            load().lgc_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    """lgc_graph: device copy of an undirected CSR (int64 offsets, int32 cols).

    off/col may be numpy arrays (host) or CUDA torch tensors (device)."""

    def __init__(self, ctx: Context, off, col, validate: bool = False):
        lib = load()
        dev = hasattr(off, "is_cuda") and off.is_cuda
        if not dev:
            off = np.ascontiguousarray(off, dtype=np.int64)
            col = np.ascontiguousarray(col, dtype=np.int32)
        n = (off.shape[0] if hasattr(off, "shape") else len(off)) - 1
        flags = (GRAPH_VALIDATE if validate else 0) | (GRAPH_DEVICE_INPUT if dev else 0)
        h = c_void_p()
        _check(lib.lgc_graph_create(ctx.handle, n, _ptr(off), _ptr(col), flags, byref(h)),
               "lgc_graph_create")
        self.handle = h
        self.ctx = ctx
        self.n = n
        self.nnz = lib.lgc_graph_num_entries(h)
        ctx._own(self)

    def autotune(self) -> tuple:
        """lgc_graph_autotune: times the heavy-vertex pull gather's shapes on
        this graph and keeps the fastest; returns (batch depth, lanes per item,
        bytes per gathered share)."""
        b, gr, sb = c_int(), c_int(), c_int()
        _check(load().lgc_graph_autotune(self.handle, byref(b), byref(gr), byref(sb)),
               "lgc_graph_autotune")
        return b.value, gr.value, sb.value

    def pull_light(self) -> int:
        """lgc_graph_pull_light: the degree bin of the pull rounds."""
        return load().lgc_graph_pull_light(self.handle)

    def set_pull_light(self, light: int):
        """lgc_graph_set_pull_light: rebuild the pull lists for another bin."""
        _check(load().lgc_graph_set_pull_light(self.handle, int(light)),
               "lgc_graph_set_pull_light")

    def batch_handoff(self) -> int:
        """lgc_graph_batch_handoff: the frontier size (edges) at which a seed
        leaves a batch and finishes alone (2**63 - 1: never)."""
        return load().lgc_graph_batch_handoff(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            if getattr(self.ctx, "handle", None):  # the context destroys nothing of ours
                load().lgc_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _HostResult:
    """Owns a library host result (page-locked memory from the library's
    pool); the numpy views of its arrays keep it alive and the last one to go
    releases it."""

    def __init__(self, ptr, free_name: str):
        self._ptr = ptr
        self._free = free_name

    def __del__(self):
        try:
            if self._ptr is not None:
                getattr(load(), self._free)(self._ptr)
                self._ptr = None
        except Exception:
            pass


class _View:
    """Array interface over library memory; numpy keeps it as the array's base."""

    def __init__(self, addr: int, n: int, typestr: str, owner: _HostResult):
        self.__array_interface__ = {"shape": (n,), "typestr": typestr,
                                    "data": (addr, False), "version": 3}
        self.owner = owner


def _host_array(addr, n: int, dtype, owner: _HostResult) -> np.ndarray:
    if n == 0:
        return np.zeros(0, dtype)
    return np.asarray(_View(addr, n, np.dtype(dtype).str, owner))


class SparseVec:
    """A library sparse vector.  Host results are numpy views (idx, val) of
    the library's page-locked result memory, released when the last view
    goes; device results keep the library handle."""

    def __init__(self, ptr, ctx: Context | None = None):
        self._ptr = ptr
        s = ptr.contents
        self.nnz = s.nnz
        self.on_device = bool(s.on_device)
        if not self.on_device:
            owner = _HostResult(ptr, "lgc_svec_free")
            self.idx = _host_array(s.idx, s.nnz, np.int32, owner)
            self.val = _host_array(s.val, s.nnz, np.float64, owner)
            self._ptr = None
        elif ctx is not None:
            self._ctx = ctx  # keeps the context alive while this result is
            ctx._own(self)

    def c_struct(self):
        """Pointer to an lgc_svec describing this vector (for lgc_sweep)."""
        if self._ptr is not None:
            return self._ptr
        self._keep = Svec(self.nnz, self.idx.ctypes.data, self.val.ctypes.data, 0)
        return ctypes.pointer(self._keep)

    def close(self):
        if getattr(self, "_ptr", None) is not None:
            ctx = getattr(self, "_ctx", None)
            if ctx is None or getattr(ctx, "handle", None):  # never after the context
                load().lgc_svec_free(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def host_svec(idx, val) -> SparseVec:
    """A host SparseVec from numpy arrays (idx ascending)."""
    v = SparseVec.__new__(SparseVec)
    v._ptr = None
    v.idx = np.ascontiguousarray(idx, dtype=np.int32)
    v.val = np.ascontiguousarray(val, dtype=np.float64)
    v.nnz = len(v.idx)
    v.on_device = False
    return v


def _take_svec(ptr) -> SparseVec:
    return SparseVec(ptr)


class ClusterResult:
    def __init__(self, ptr, ctx: Context | None = None):
        c = ptr.contents
        self.size, self.vol, self.cut = c.size, c.vol, c.cut
        self.conductance = c.conductance
        self.on_device = bool(c.on_device)
        self._ptr = ptr
        if not self.on_device:
            self.ids = _host_array(c.ids, c.size, np.int32, _HostResult(ptr, "lgc_cluster_free"))
            self._ptr = None
        elif ctx is not None:
            self._ctx = ctx
            ctx._own(self)

    def close(self):
        if getattr(self, "_ptr", None) is not None:
            ctx = getattr(self, "_ctx", None)
            if ctx is None or getattr(ctx, "handle", None):
                load().lgc_cluster_free(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def prnibble(g: Graph, seed: int, alpha: float, eps: float, rule="opt", mode="atomic",
             max_rounds: int = 0):
    prm = PRNibbleParams(alpha, eps, _RULES[rule], _MODES[mode], max_rounds)
    out, st = POINTER(Svec)(), Stats()
    s = load().lgc_prnibble(g.handle, seed, byref(prm), byref(out), byref(st))
    _check(s, "lgc_prnibble", ok=(LGC_OK, LGC_EMAXROUNDS))
    return SparseVec(out, g.ctx), st


def prnibble_set(g: Graph, seeds, alpha: float, eps: float, weights=None, beta: float = 1.0,
                 rule="opt", mode="atomic", max_rounds: int = 0):
    """PR-Nibble from a seed set (weights: None for all 1) with beta-fraction
    rounds (lgc_prnibble_set)."""
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    w = None if weights is None else np.ascontiguousarray(
        np.broadcast_to(np.asarray(weights, dtype=np.float64), seeds.shape))
    prm = PRNibbleParams(alpha, eps, _RULES[rule], _MODES[mode], max_rounds)
    out, st = POINTER(Svec)(), Stats()
    s = load().lgc_prnibble_set(g.handle, len(seeds), seeds.ctypes.data,
                                None if w is None else w.ctypes.data, float(beta), byref(prm),
                                byref(out), byref(st))
    _check(s, "lgc_prnibble_set", ok=(LGC_OK, LGC_EMAXROUNDS))
    return SparseVec(out, g.ctx), st


def nibble(g: Graph, seed: int, T: int, eps: float, mode="atomic"):
    prm = NibbleParams(T, eps, _MODES[mode])
    out, st = POINTER(Svec)(), Stats()
    _check(load().lgc_nibble(g.handle, seed, byref(prm), byref(out), byref(st)), "lgc_nibble")
    return SparseVec(out, g.ctx), st


def hkpr(g: Graph, seed: int, t: float, N: int, eps: float, mode="atomic"):
    prm = HKPRParams(t, eps, N, _MODES[mode])
    out, st = POINTER(Svec)(), Stats()
    _check(load().lgc_hkpr(g.handle, seed, byref(prm), byref(out), byref(st)), "lgc_hkpr")
    return SparseVec(out, g.ctx), st


def rand_hkpr(g: Graph, seed: int, t: float, K: int, n_walks: int, rng_seed: int):
    prm = RandHKPRParams(t, K, n_walks, rng_seed & ((1 << 64) - 1))
    out, st = POINTER(Svec)(), Stats()
    _check(load().lgc_rand_hkpr(g.handle, seed, byref(prm), byref(out), byref(st)),
           "lgc_rand_hkpr")
    return SparseVec(out, g.ctx), st


def sweep(g: Graph, p: SparseVec) -> ClusterResult:
    out = POINTER(Cluster)()
    _check(load().lgc_sweep(g.handle, p.c_struct(), byref(out)), "lgc_sweep")
    return ClusterResult(out, g.ctx)


def sweep_batch(g: Graph, ps) -> list:
    """Sweep cuts of many vectors in one pass (lgc_sweep_batch); the same
    clusters as sweep() on each."""
    ps = list(ps)
    B = len(ps)
    if B == 0:
        return []
    ptrs = (POINTER(Svec) * B)(*[p.c_struct() for p in ps])
    outs = (POINTER(Cluster) * B)()
    _check(load().lgc_sweep_batch(g.handle, B, ctypes.addressof(ptrs), ctypes.addressof(outs)),
           "lgc_sweep_batch")
    return [ClusterResult(outs[b], g.ctx) for b in range(B)]


def make_request(algo: int, seed: int, want_sweep: bool = True, **kw) -> Request:
    r = Request()
    r.algo, r.seed, r.want_sweep = algo, seed, int(want_sweep)
    if algo == ALGO_PRNIBBLE:
        r.pr = PRNibbleParams(kw["alpha"], kw["eps"], _RULES[kw.get("rule", "opt")],
                              _MODES[kw.get("mode", "atomic")], kw.get("max_rounds", 0))
    elif algo == ALGO_NIBBLE:
        r.nb = NibbleParams(kw["T"], kw["eps"], _MODES[kw.get("mode", "atomic")])
    elif algo == ALGO_HKPR:
        r.hk = HKPRParams(kw["t"], kw["eps"], kw["N"], _MODES[kw.get("mode", "atomic")])
    else:
        r.rh = RandHKPRParams(kw["t"], kw["K"], kw["n_walks"], kw.get("rng_seed", 0))
    return r


def submit(ctx: Context, g: Graph, req: Request) -> int:
    t = c_uint64()
    _check(load().lgc_submit(ctx.handle, g.handle, byref(req), byref(t)), "lgc_submit")
    return t.value


def poll(ctx: Context, ticket: int):
    """None while pending, else a dict with the host results and timings."""
    out = POINTER(Result)()
    s = load().lgc_poll(ctx.handle, ticket, byref(out))
    if s == LGC_PENDING:
        return None
    _check(s, "lgc_poll")
    return _take_result(out)


def wait(ctx: Context, ticket: int):
    """Block until the request is done (lgc_wait); the same dict as poll."""
    out = POINTER(Result)()
    _check(load().lgc_wait(ctx.handle, ticket, byref(out)), "lgc_wait")
    return _take_result(out)


def _take_result(out):
    r = out.contents
    res = {"status": r.status, "stats": r.stats.as_dict(), "submit_s": r.submit_s,
           "start_s": r.start_s, "end_s": r.end_s, "idx": None, "val": None, "cluster": None}
    if r.p:
        sv = r.p.contents
        res["idx"] = (np.ctypeslib.as_array((c_int32 * sv.nnz).from_address(sv.idx)).copy()
                      if sv.nnz else np.zeros(0, np.int32))
        res["val"] = (np.ctypeslib.as_array((c_double * sv.nnz).from_address(sv.val)).copy()
                      if sv.nnz else np.zeros(0))
    if r.cluster:
        c = r.cluster.contents
        res["cluster"] = {"size": c.size, "vol": c.vol, "cut": c.cut,
                          "conductance": c.conductance,
                          "ids": (np.ctypeslib.as_array((c_int32 * c.size).from_address(c.ids)).copy()
                                  if c.size else np.zeros(0, np.int32))}
    load().lgc_result_free(out)
    return res


def prnibble_batch(g: Graph, seeds, alpha, eps, rule="opt", mode="atomic", max_rounds=0):
    """PR-Nibble for many seeds in one batch (lgc_prnibble_batch).  alpha and
    eps may be scalars or one value per seed.  Returns (list of SparseVec,
    list of Stats)."""
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    B = len(seeds)
    alpha = np.broadcast_to(np.asarray(alpha, dtype=np.float64), (B,))
    eps = np.broadcast_to(np.asarray(eps, dtype=np.float64), (B,))
    prm = (PRNibbleParams * B)()
    for b in range(B):
        prm[b] = PRNibbleParams(float(alpha[b]), float(eps[b]), _RULES[rule], _MODES[mode],
                                max_rounds)
    outs = (POINTER(Svec) * B)()
    sts = (Stats * B)()
    _check(load().lgc_prnibble_batch(g.handle, B, seeds.ctypes.data, ctypes.addressof(prm),
                                     ctypes.addressof(outs), ctypes.addressof(sts)),
           "lgc_prnibble_batch")
    return [SparseVec(outs[b], g.ctx) for b in range(B)], [sts[b] for b in range(B)]
