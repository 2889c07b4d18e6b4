"""ctypes binding of ``libfiuncho.so``: one Python function per C entry
point, same names, argument marshalling only.  All computation happens in
the library's CUDA kernels; if the shared object is missing the import of
any entry point raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfiuncho.so")

FC_OK = 0
FC_EINVAL = -1
FC_ERANGE = -2
FC_ENOMEM = -3
FC_ECUDA = -4
FC_ETIMEOUT = -5
FC_ENODEV = -6
FC_KMAX_SEARCH = 6
FC_KMAX_BATCH = 4
FC_KMAX_TABLES = 6
FC_MAX_LIST = 4096

_lock = threading.Lock()
_lib = None

P = ctypes.c_void_p
i64 = ctypes.c_int64
u64 = ctypes.c_uint64
i32 = ctypes.c_int

_SIGNATURES = {
    "fc_load": ([P, i64, i64, P, P], i32),
    "fc_load_device": ([P, i64, i64, P, P], i32),
    "fc_set_stream": ([P, P], i32),
    "fc_search": ([P, i32, i64, P, P, P], i32),
    "fc_search_static": ([P, i32, i64, P, P, P], i32),
    "fc_tables": ([P, i32, P, i64, P], i32),
    "fc_scores": ([P, i32, u64, i64, P], i32),
    "fc_info": ([P, P, P, P, P], i32),
    "fc_log2_approx": ([P, i64, P], i32),
    "fc_pairs_dense": ([P, P, P], i32),
    "fc_triples_dense": ([P, P, P], i32),
    "fc_tuples_dense": ([P, i32, P, P], i32),
    "fc_search_range": ([P, i32, i64, u64, u64, P, P, P], i32),
    "fc_load_batch": ([i32, P, P, P, P, i32, P], i32),
    "fc_search_batch": ([P, i32, i64, P, P, P], i32),
    "fc_search_job": ([P, i32, i32, i64, P, P, P], i32),
    "fc_batch_info": ([P, P, P, P], i32),
    "fc_batch_job_kind": ([P, i32], i32),
    "fc_last_search_kind": ([P], i32),
    "fc_triples_form": ([P], i32),
    "fc_sweep_tables": ([P, i32, u64, i64, P], i32),
    "fc_timing": ([P, i32, P, P, P], i32),
    "fc_free": ([P], None),
    "fc_strerror": ([i32], ctypes.c_char_p),
    "fc_last_error": ([], ctypes.c_char_p),
    "fc_num_combinations": ([i64, i32], i64),
    "fc_unrank": ([i64, i32, u64, P], i32),
    "fc_rank": ([i64, i32, P, P], i32),
}


class FiunchoError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = library()
        msg = lib.fc_strerror(status).decode()
        detail = lib.fc_last_error().decode()
        super().__init__(f"{where}: {msg} ({status}): {detail}")
        self.status = status


def library():
    """Load the shared library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: run paper_2201_03331_gb300.build.build()")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in _SIGNATURES.items():
                fn = getattr(lib, name, None)
                if fn is None:
                    continue
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def _check(status: int, where: str):
    if status != FC_OK:
        raise FiunchoError(status, where)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(P)


class Handle:
    """Owns an ``fc_handle *``; freed by :func:`fc_free` or garbage collection."""

    def __init__(self, ptr: int):
        self._ptr = ptr

    @property
    def ptr(self):
        if not self._ptr:
            raise ValueError("handle already freed")
        return self._ptr

    def __del__(self):
        try:
            fc_free(self)
        except Exception:
            pass


def fc_load(genotypes: np.ndarray, phenotype: np.ndarray) -> Handle:
    """Pack host ``uint8[S][M]`` genotypes and ``uint8[M]`` phenotype."""
    G = np.ascontiguousarray(genotypes, dtype=np.uint8)
    ph = np.ascontiguousarray(phenotype, dtype=np.uint8)
    if G.ndim != 2 or ph.ndim != 1 or ph.shape[0] != G.shape[1]:
        raise ValueError("genotypes must be [S][M] and phenotype [M]")
    out = ctypes.c_void_p()
    _check(library().fc_load(_ptr(G), G.shape[0], G.shape[1], _ptr(ph), ctypes.byref(out)), "fc_load")
    return Handle(out.value)


def fc_load_device(genotypes, phenotype) -> Handle:
    """Pack device (torch CUDA ``uint8``) genotypes ``[S][M]`` and phenotype ``[M]``."""
    import torch
    if not (genotypes.is_cuda and phenotype.is_cuda):
        raise ValueError("fc_load_device takes CUDA tensors")
    G = genotypes.contiguous()
    ph = phenotype.contiguous()
    if G.dtype != torch.uint8 or ph.dtype != torch.uint8:
        raise ValueError("uint8 tensors expected")
    out = ctypes.c_void_p()
    _check(library().fc_load_device(G.data_ptr(), G.shape[0], G.shape[1], ph.data_ptr(),
                                    ctypes.byref(out)), "fc_load_device")
    return Handle(out.value)


def fc_set_stream(h: Handle, stream) -> None:
    """``stream``: a ``torch.cuda.Stream``, a raw ``cudaStream_t`` int, or None."""
    raw = getattr(stream, "cuda_stream", stream)
    _check(library().fc_set_stream(h.ptr, ctypes.c_void_p(raw or 0)), "fc_set_stream")


def fc_search(h: Handle, k: int, top_n: int):
    """Returns ``(idx uint32[c][k], score float64[c])``, best first."""
    idx = np.zeros((max(top_n, 1), k), dtype=np.uint32)
    score = np.zeros(max(top_n, 1), dtype=np.float64)
    cnt = ctypes.c_int64(0)
    _check(library().fc_search(h.ptr, k, top_n, _ptr(idx), _ptr(score), ctypes.byref(cnt)), "fc_search")
    n = cnt.value
    return idx[:n], score[:n]


def fc_search_static(h: Handle, k: int, top_n: int):
    """As :func:`fc_search`, through the entry point that allocates no
    device memory (fixed 8 MiB work area in the library's device image)."""
    idx = np.zeros((max(top_n, 1), k), dtype=np.uint32)
    score = np.zeros(max(top_n, 1), dtype=np.float64)
    cnt = ctypes.c_int64(0)
    _check(library().fc_search_static(h.ptr, k, top_n, _ptr(idx), _ptr(score), ctypes.byref(cnt)),
           "fc_search_static")
    n = cnt.value
    return idx[:n], score[:n]


def fc_tables(h: Handle, k: int, combos) -> np.ndarray:
    """Exact ``uint32[n][3^k][2]`` tables of the given combinations."""
    c = np.ascontiguousarray(np.asarray(combos, dtype=np.uint32).reshape(-1, k))
    out = np.zeros((c.shape[0], 3 ** k, 2), dtype=np.uint32)
    _check(library().fc_tables(h.ptr, k, _ptr(c), c.shape[0], _ptr(out)), "fc_tables")
    return out


def fc_log2_approx(n) -> np.ndarray:
    """The epilogue's hardware base-2 logarithm of ``max(n, 1)`` (float32)."""
    a = np.ascontiguousarray(np.asarray(n, dtype=np.uint32).ravel())
    out = np.zeros(a.shape[0], dtype=np.float32)
    _check(library().fc_log2_approx(_ptr(a), a.shape[0], _ptr(out)), "fc_log2_approx")
    return out


def fc_scores(h: Handle, k: int, rank_begin: int, n: int) -> np.ndarray:
    """FP32 sweep scores of ranks ``[rank_begin, rank_begin + n)``."""
    out = np.zeros(n, dtype=np.float32)
    _check(library().fc_scores(h.ptr, k, rank_begin, n, _ptr(out)), "fc_scores")
    return out


def fc_pairs_dense(h: Handle, scores: bool = True, tables: bool = False):
    """Dense order-2 output of the tensor-core kernel: ``(scores float32[S][S]
    or None, tables uint32[S][S][9][2] or None)`` (entries with i < j)."""
    S = fc_info(h)[0]
    sc = np.zeros((S, S), dtype=np.float32) if scores else None
    tb = np.zeros((S, S, 9, 2), dtype=np.uint32) if tables else None
    _check(library().fc_pairs_dense(h.ptr, _ptr(sc) if sc is not None else None,
                                    _ptr(tb) if tb is not None else None), "fc_pairs_dense")
    return sc, tb


def fc_triples_dense(h: Handle, scores: bool = True, tables: bool = False):
    """Dense order-3 output of the tensor-core kernel, indexed by
    lexicographic rank: ``(scores float32[C(S,3)] or None, tables
    uint32[C(S,3)][27][2] or None)``."""
    S = fc_info(h)[0]
    n = S * (S - 1) * (S - 2) // 6
    sc = np.zeros(n, dtype=np.float32) if scores else None
    tb = np.zeros((n, 27, 2), dtype=np.uint32) if tables else None
    _check(library().fc_triples_dense(h.ptr, _ptr(sc) if sc is not None else None,
                                      _ptr(tb) if tb is not None else None), "fc_triples_dense")
    return sc, tb


def fc_search_range(h: Handle, k: int, top_n: int, rank_begin: int, rank_end: int):
    """Exact top-N among the combinations of lexicographic ranks
    [rank_begin, rank_end): ``(indices uint32[n][k], scores float64[n])``."""
    n_max = max(0, min(top_n, rank_end - rank_begin))
    idx = np.zeros((max(n_max, 1), k), dtype=np.uint32)
    sc = np.zeros(max(n_max, 1), dtype=np.float64)
    cnt = ctypes.c_int64(0)
    _check(library().fc_search_range(h.ptr, k, top_n, rank_begin, rank_end, _ptr(idx), _ptr(sc),
                                     ctypes.byref(cnt)), "fc_search_range")
    return idx[:cnt.value], sc[:cnt.value]


def fc_tuples_dense(h: Handle, k: int, scores: bool = True, tables: bool = False):
    """Dense output of order k = 4..6 of the tensor-core tuple kernel,
    indexed by lexicographic rank: ``(scores float32[C(S,k)] or None, tables
    uint32[C(S,k)][3^k][2] or None)``."""
    S = fc_info(h)[0]
    n = math.comb(S, k)
    sc = np.zeros(n, dtype=np.float32) if scores else None
    tb = np.zeros((n, 3 ** k, 2), dtype=np.uint32) if tables else None
    _check(library().fc_tuples_dense(h.ptr, k, _ptr(sc) if sc is not None else None,
                                     _ptr(tb) if tb is not None else None), "fc_tuples_dense")
    return sc, tb


def fc_load_batch(genotypes, phenotypes) -> Handle:
    """``genotypes``: list of host ``uint8[S_d][M_d]``; ``phenotypes``: list of
    host ``uint8[R][M_d]`` (same R for every data set).  Job ``d*R + r`` is
    data set d with phenotype row r."""
    n = len(genotypes)
    if n == 0 or len(phenotypes) != n:
        raise ValueError("one phenotype block per data set")
    Gs = [np.ascontiguousarray(g, dtype=np.uint8) for g in genotypes]
    Ps = [np.ascontiguousarray(np.atleast_2d(p), dtype=np.uint8) for p in phenotypes]
    R = Ps[0].shape[0]
    for g, p in zip(Gs, Ps):
        if g.ndim != 2 or p.shape != (R, g.shape[1]):
            raise ValueError("genotypes [S][M] and phenotypes [R][M] per data set")
    gptr = (ctypes.c_void_p * n)(*[g.ctypes.data for g in Gs])
    pptr = (ctypes.c_void_p * n)(*[p.ctypes.data for p in Ps])
    S = np.array([g.shape[0] for g in Gs], dtype=np.int64)
    M = np.array([g.shape[1] for g in Gs], dtype=np.int64)
    out = ctypes.c_void_p()
    _check(library().fc_load_batch(n, gptr, _ptr(S), _ptr(M), pptr, R, ctypes.byref(out)), "fc_load_batch")
    h = Handle(out.value)
    h._n_jobs = n * R
    return h


def fc_batch_job_kind(h: Handle, job: int) -> int:
    """Path of the last batched search for ``job`` (fc_last_search_kind values)."""
    r = library().fc_batch_job_kind(h.ptr, job)
    if r < 0:
        _check(r, "fc_batch_job_kind")
    return r


def fc_batch_info(h: Handle):
    v = [ctypes.c_int(0) for _ in range(3)]
    _check(library().fc_batch_info(h.ptr, *[ctypes.byref(x) for x in v]), "fc_batch_info")
    return tuple(x.value for x in v)


def fc_search_batch(h: Handle, k: int, top_n: int):
    """Returns ``(idx uint32[jobs][top_n][k], score float64[jobs][top_n],
    count int64[jobs])``."""
    jobs = fc_batch_info(h)[2]
    idx = np.zeros((jobs, max(top_n, 1), k), dtype=np.uint32)
    score = np.zeros((jobs, max(top_n, 1)), dtype=np.float64)
    cnt = np.zeros(jobs, dtype=np.int64)
    _check(library().fc_search_batch(h.ptr, k, top_n, _ptr(idx), _ptr(score), _ptr(cnt)), "fc_search_batch")
    return idx[:, :top_n], score[:, :top_n], cnt


def fc_search_job(h: Handle, job: int, k: int, top_n: int):
    """fc_search on one job of a batch handle: ``(idx, score)``."""
    idx = np.zeros((max(top_n, 1), k), dtype=np.uint32)
    score = np.zeros(max(top_n, 1), dtype=np.float64)
    cnt = ctypes.c_int64(0)
    _check(library().fc_search_job(h.ptr, job, k, top_n, _ptr(idx), _ptr(score), ctypes.byref(cnt)),
           "fc_search_job")
    n = cnt.value
    return idx[:n], score[:n]


def fc_sweep_tables(h: Handle, k: int, rank_begin: int, n: int) -> np.ndarray:
    """Exact ``uint32[n][3^k][2]`` tables built by the sweep kernel for ranks
    ``[rank_begin, rank_begin + n)``."""
    out = np.zeros((n, 3 ** k, 2), dtype=np.uint32)
    _check(library().fc_sweep_tables(h.ptr, k, rank_begin, n, _ptr(out)), "fc_sweep_tables")
    return out


def fc_triples_form(h: Handle) -> int:
    """Form of the order-3 tensor-core kernel for this data set: 1 one
    accumulator (cases + 4096 controls), 0 one per class, -1 none."""
    r = library().fc_triples_form(h.ptr)
    if r < -1:
        _check(r, "fc_triples_form")
    return int(r)


def fc_last_search_kind(h: Handle) -> int:
    """0 none, 1 full 3^k AND/POPC sweep, 2 tensor-core order-2 pairs,
    3 inclusion-exclusion AND/POPC sweep."""
    r = library().fc_last_search_kind(h.ptr)
    if r < 0:
        _check(r, "fc_last_search_kind")
    return int(r)


def fc_info(h: Handle):
    v = [ctypes.c_int64(0) for _ in range(4)]
    _check(library().fc_info(h.ptr, *[ctypes.byref(x) for x in v]), "fc_info")
    return tuple(x.value for x in v)


def fc_timing(h: Handle, enable: int = -1):
    """Returns ``(sweep_ms, sweeps, launches)`` accumulated so far, then resets
    and switches instrumentation on (1) / off (0); ``enable=-1`` only reads."""
    ms = ctypes.c_double(0)
    sw = ctypes.c_int64(0)
    la = ctypes.c_int64(0)
    _check(library().fc_timing(h.ptr, enable, ctypes.byref(ms), ctypes.byref(sw), ctypes.byref(la)),
           "fc_timing")
    return ms.value, sw.value, la.value


def fc_free(h: Handle) -> None:
    if h._ptr:
        library().fc_free(h._ptr)
        h._ptr = None


def fc_strerror(status: int) -> str:
    return library().fc_strerror(status).decode()


def fc_last_error() -> str:
    return library().fc_last_error().decode()


def fc_num_combinations(S: int, k: int) -> int:
    return int(library().fc_num_combinations(S, k))


def fc_unrank(S: int, k: int, rank: int) -> np.ndarray:
    out = np.zeros(k, dtype=np.uint32)
    _check(library().fc_unrank(S, k, rank, _ptr(out)), "fc_unrank")
    return out


def fc_rank(S: int, k: int, combo) -> int:
    c = np.ascontiguousarray(np.asarray(combo, dtype=np.uint32))
    r = ctypes.c_uint64(0)
    _check(library().fc_rank(S, k, _ptr(c), ctypes.byref(r)), "fc_rank")
    return int(r.value)
