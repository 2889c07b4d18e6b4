"""Python access to the CPU oracle (``oracle/oracle.c``).

TEST INFRASTRUCTURE: only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The library under
``paper_2201_03331_gb300`` never imports it and shares no code with it.

The shared object is compiled from ``oracle.c`` with the host C compiler on
first use (or by :func:`build`) and loaded with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
# FC_ORACLE_LIB names another build of oracle.c to load instead (the pin
# strength tests load copies with planted mistakes this way).
_LIB = os.environ.get("FC_ORACLE_LIB") or os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

KMAX = 10


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to the source (gcc, -O2, pthreads)."""
    if os.environ.get("FC_ORACLE_LIB"):
        return _LIB
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i64, i32 = ctypes.c_int64, ctypes.c_int
            lib.orc_binom.argtypes = [i64, i64]
            lib.orc_binom.restype = i64
            lib.orc_validate.argtypes = [P, i64, i64, P, i32]
            lib.orc_validate.restype = i32
            lib.orc_tables.argtypes = [P, i64, i64, P, i32, P, i64, P]
            lib.orc_tables.restype = i32
            lib.orc_mi.argtypes = [P, i64, i32, P]
            lib.orc_mi.restype = i32
            lib.orc_search.argtypes = [P, i64, i64, P, i32, i64, i32, i64, i64, P, P, P, P]
            lib.orc_search.restype = i32
            lib.orc_distribution.argtypes = [i64, i32, i32, P]
            lib.orc_distribution.restype = i32
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(f"{what} failed with status {rc}")


def binom(n: int, r: int) -> int:
    return int(_load().orc_binom(n, r))


def validate(G: np.ndarray, ph: np.ndarray, k: int) -> int:
    G = np.ascontiguousarray(G, dtype=np.uint8)
    ph = np.ascontiguousarray(ph, dtype=np.uint8)
    return int(_load().orc_validate(_ptr(G), G.shape[0], G.shape[1], _ptr(ph), k))


def tables(G: np.ndarray, ph: np.ndarray, k: int, combos) -> np.ndarray:
    """``uint32[n][3^k][2]`` contingency tables (column 0 = cases)."""
    G = np.ascontiguousarray(G, dtype=np.uint8)
    ph = np.ascontiguousarray(ph, dtype=np.uint8)
    c = np.ascontiguousarray(np.asarray(combos, dtype=np.uint32).reshape(-1, k))
    out = np.zeros((c.shape[0], 3 ** k, 2), dtype=np.uint32)
    _check(_load().orc_tables(_ptr(G), G.shape[0], G.shape[1], _ptr(ph), k,
                              _ptr(c), c.shape[0], _ptr(out)), "orc_tables")
    return out


def mi(tabs: np.ndarray, k: int) -> np.ndarray:
    """FP64 mutual information of ``[n][3^k][2]`` tables."""
    t = np.ascontiguousarray(np.asarray(tabs, dtype=np.uint32).reshape(-1, 3 ** k, 2))
    out = np.zeros(t.shape[0], dtype=np.float64)
    _check(_load().orc_mi(_ptr(t), t.shape[0], k, _ptr(out)), "orc_mi")
    return out


def search(G: np.ndarray, ph: np.ndarray, k: int, top_n: int, nthreads: int = 0,
           prefix_range=(0, -1)):
    """Exhaustive search (Algorithm 1).  Returns ``(idx uint32[c][k],
    score float64[c], tested)``, best first."""
    G = np.ascontiguousarray(G, dtype=np.uint8)
    ph = np.ascontiguousarray(ph, dtype=np.uint8)
    idx = np.zeros((max(top_n, 1), k), dtype=np.uint32)
    score = np.zeros(max(top_n, 1), dtype=np.float64)
    cnt = ctypes.c_int64(0)
    tested = ctypes.c_int64(0)
    _check(_load().orc_search(_ptr(G), G.shape[0], G.shape[1], _ptr(ph), k, top_n,
                              nthreads, prefix_range[0], prefix_range[1],
                              _ptr(idx), _ptr(score), ctypes.byref(cnt),
                              ctypes.byref(tested)), "orc_search")
    n = cnt.value
    return idx[:n].copy(), score[:n].copy(), tested.value


def distribution(n: int, k: int, p: int) -> np.ndarray:
    """Combinations per unit under the paper's static (k-1)-prefix
    round-robin distribution."""
    out = np.zeros(p, dtype=np.uint64)
    _check(_load().orc_distribution(n, k, p, _ptr(out)), "orc_distribution")
    return out
