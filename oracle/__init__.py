"""FP64 CPU oracle for the context-enhanced tensor join (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The product
path (``paper_2312_01476_gb300``) never imports it, and this package imports
nothing from the product path.

The arithmetic lives in ``ejoin_oracle.c`` (plain C, FP64, OpenMP over R rows):
the definition of the operator from Sec. III-A Eq. (Cosine Similarity) and
Sec. III-C Eq. (E-theta-Join) / Eq. (Selection), evaluated pair by pair.  This
module only compiles it with gcc and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ejoin_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_libs: dict = {}

OPS = {"<": 0, "<=": 1, ">": 2, ">=": 3, "==": 4, "!=": 5}


def lib_path(mutant: int = 0) -> str:
    name = "libejoin_oracle.so" if mutant == 0 else f"libejoin_oracle_mut{mutant}.so"
    return os.path.join(_BUILD, name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle (or one of its test mutants) with gcc; returns the .so path.

    -ffp-contract=off keeps every multiply and add separately rounded on both
    x86 and aarch64 hosts, so the oracle's bits do not depend on the host.
    """
    out = lib_path(mutant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = f"{out}.{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
           f"-DORACLE_MUTANT={int(mutant)}", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _load(mutant: int = 0):
    with _lock:
        if mutant in _libs:
            return _libs[mutant]
        lib = ctypes.CDLL(build(mutant))
        f32p = ctypes.POINTER(ctypes.c_float)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        f64p = ctypes.POINTER(ctypes.c_double)
        lib.oracle_join.restype = ctypes.c_int64
        lib.oracle_join.argtypes = [f32p, ctypes.c_int64, ctypes.c_int64,
                                    f32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                    i32p, ctypes.c_int32, ctypes.c_int32,
                                    i32p, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_float, i64p, ctypes.c_int64,
                                    u32p, u32p, f64p, ctypes.c_int64, ctypes.c_int32]
        lib.oracle_sim_pairs.restype = None
        lib.oracle_sim_pairs.argtypes = [f32p, ctypes.c_int64, f32p, ctypes.c_int64, ctypes.c_int32,
                                         u32p, u32p, ctypes.c_int64, f64p, ctypes.c_int32]
        lib.oracle_norm.restype = ctypes.c_double
        lib.oracle_norm.argtypes = [f32p, ctypes.c_int32]
        lib.oracle_sim.restype = ctypes.c_double
        lib.oracle_sim.argtypes = [f32p, f32p, ctypes.c_int32]
        lib.oracle_top1.restype = ctypes.c_int64
        lib.oracle_top1.argtypes = [f32p, ctypes.c_int64, ctypes.c_int64,
                                    f32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                    i32p, ctypes.c_int32, ctypes.c_int32,
                                    i32p, ctypes.c_int32, ctypes.c_int32,
                                    i64p, ctypes.c_int64, u32p, u32p, f64p, ctypes.c_int32]
        lib.oracle_topk.restype = ctypes.c_int64
        lib.oracle_topk.argtypes = [f32p, ctypes.c_int64, ctypes.c_int64,
                                    f32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                    i32p, ctypes.c_int32, ctypes.c_int32,
                                    i32p, ctypes.c_int32, ctypes.c_int32,
                                    i64p, ctypes.c_int64, u32p, u32p, f64p, ctypes.c_int32]
        lib.oracle_count_selected.restype = ctypes.c_int64
        lib.oracle_count_selected.argtypes = [i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64]
        _libs[mutant] = lib
        return lib


def _ptr(a: Optional[np.ndarray], ctype):
    if a is None:
        return ctypes.cast(None, ctypes.POINTER(ctype))
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _rows_f32(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x)
    if x.ndim == 2 and x.dtype == np.float32 and x.size == 0:
        return x  # no rows: callers return before touching the data
    if x.ndim == 2 and x.dtype == np.float32 and x.shape[0] == 1:
        x = np.ascontiguousarray(x)  # the row stride of a one-row array is arbitrary
    if x.dtype != np.float32 or x.ndim != 2 or x.strides[1] != 4:
        raise TypeError("relation must be a 2-D float32 array with contiguous rows")
    return x


class Selection:
    """A relational predicate ``attr op c`` on one relation (Sec. III-C, Eq. Selection)."""

    def __init__(self, attr: np.ndarray, op: str = "<", c: int = 0):
        self.attr = np.ascontiguousarray(attr, dtype=np.int32)
        self.op = OPS[op]
        self.c = int(c)


def join(R: np.ndarray, S: np.ndarray, eps: float, selR: Optional[Selection] = None,
         selS: Optional[Selection] = None, rows: Optional[Sequence[int]] = None,
         threads: int = 0, mutant: int = 0):
    """All (i, j, sim) with selR(i), selS(j) and sim(R_i, S_j) >= eps, sorted by (i, j).

    ``rows``: evaluate only these R rows (sampling of large workloads).
    Returns (i: uint32[n], j: uint32[n], sim: float64[n]).
    """
    lib = _load(mutant)
    R = _rows_f32(R)
    S = _rows_f32(S)
    if R.shape[1] != S.shape[1]:
        raise ValueError("R and S must have the same dimension")
    if R.shape[0] == 0 or S.shape[0] == 0:
        return np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.float64)
    d = R.shape[1]
    ldR = R.strides[0] // 4
    ldS = S.strides[0] // 4
    rows_arr = None
    if rows is not None:
        rows_arr = np.ascontiguousarray(np.sort(np.asarray(rows, dtype=np.int64)))
    eps32 = float(np.float32(eps))
    args_sel = []
    for sel in (selR, selS):
        if sel is None:
            args_sel += [_ptr(None, ctypes.c_int32), 0, 0]
        else:
            args_sel += [_ptr(sel.attr, ctypes.c_int32), sel.op, sel.c]
    cap = 0
    while True:
        oi = np.empty(max(cap, 1), dtype=np.uint32)
        oj = np.empty(max(cap, 1), dtype=np.uint32)
        os_ = np.empty(max(cap, 1), dtype=np.float64)
        n = lib.oracle_join(_ptr(R, ctypes.c_float), R.shape[0], ldR,
                            _ptr(S, ctypes.c_float), S.shape[0], ldS, d,
                            *args_sel, ctypes.c_float(eps32),
                            _ptr(rows_arr, ctypes.c_int64), 0 if rows_arr is None else len(rows_arr),
                            _ptr(oi, ctypes.c_uint32), _ptr(oj, ctypes.c_uint32),
                            _ptr(os_, ctypes.c_double), cap, int(threads))
        if n < 0:
            raise MemoryError("oracle_join: allocation failed")
        if n <= cap:
            return oi[:n].copy(), oj[:n].copy(), os_[:n].copy()
        cap = int(n)


def top1(R: np.ndarray, S: np.ndarray, selR: Optional[Selection] = None, selS: Optional[Selection] = None,
         rows: Optional[Sequence[int]] = None, threads: int = 0, mutant: int = 0):
    """Top-1 join condition (Sec. VI-E, top-k with k = 1): for every kept R row i, the kept S row j
    of largest similarity (ties: the smaller j).  Returns (i: uint32[n], j: uint32[n], sim: float64[n])
    in ascending i."""
    lib = _load(mutant)
    R = _rows_f32(R)
    S = _rows_f32(S)
    if R.shape[1] != S.shape[1]:
        raise ValueError("R and S must have the same dimension")
    if R.shape[0] == 0 or S.shape[0] == 0:
        return np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.float64)
    rows_arr = None
    if rows is not None:
        rows_arr = np.ascontiguousarray(np.sort(np.asarray(rows, dtype=np.int64)))
    n_eval = R.shape[0] if rows_arr is None else len(rows_arr)
    args_sel = []
    for sel in (selR, selS):
        if sel is None:
            args_sel += [_ptr(None, ctypes.c_int32), 0, 0]
        else:
            args_sel += [_ptr(sel.attr, ctypes.c_int32), sel.op, sel.c]
    oi = np.empty(max(n_eval, 1), dtype=np.uint32)
    oj = np.empty(max(n_eval, 1), dtype=np.uint32)
    os_ = np.empty(max(n_eval, 1), dtype=np.float64)
    n = lib.oracle_top1(_ptr(R, ctypes.c_float), R.shape[0], R.strides[0] // 4,
                        _ptr(S, ctypes.c_float), S.shape[0], S.strides[0] // 4, R.shape[1],
                        *args_sel, _ptr(rows_arr, ctypes.c_int64), 0 if rows_arr is None else len(rows_arr),
                        _ptr(oi, ctypes.c_uint32), _ptr(oj, ctypes.c_uint32), _ptr(os_, ctypes.c_double),
                        int(threads))
    if n < 0:
        raise MemoryError("oracle_top1: allocation failed")
    return oi[:n].copy(), oj[:n].copy(), os_[:n].copy()


def topk(R: np.ndarray, S: np.ndarray, k: int, selR: Optional[Selection] = None,
         selS: Optional[Selection] = None, rows: Optional[Sequence[int]] = None, threads: int = 0,
         mutant: int = 0):
    """Top-k join condition (Sec. VI-E): for every kept R row i, the min(k, kept S rows) kept S rows of
    largest similarity, in descending similarity (ties: the smaller j).  Returns (i, j, sim) arrays with
    each row's records consecutive, rows in ascending i."""
    lib = _load(mutant)
    R = _rows_f32(R)
    S = _rows_f32(S)
    if R.shape[1] != S.shape[1]:
        raise ValueError("R and S must have the same dimension")
    if k <= 0 or R.shape[0] == 0 or S.shape[0] == 0:
        return np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.float64)
    rows_arr = None
    if rows is not None:
        rows_arr = np.ascontiguousarray(np.sort(np.asarray(rows, dtype=np.int64)))
    n_eval = R.shape[0] if rows_arr is None else len(rows_arr)
    args_sel = []
    for sel in (selR, selS):
        if sel is None:
            args_sel += [_ptr(None, ctypes.c_int32), 0, 0]
        else:
            args_sel += [_ptr(sel.attr, ctypes.c_int32), sel.op, sel.c]
    cap = max(n_eval * int(k), 1)
    oi = np.empty(cap, dtype=np.uint32)
    oj = np.empty(cap, dtype=np.uint32)
    os_ = np.empty(cap, dtype=np.float64)
    n = lib.oracle_topk(_ptr(R, ctypes.c_float), R.shape[0], R.strides[0] // 4,
                        _ptr(S, ctypes.c_float), S.shape[0], S.strides[0] // 4, R.shape[1], int(k),
                        *args_sel, _ptr(rows_arr, ctypes.c_int64), 0 if rows_arr is None else len(rows_arr),
                        _ptr(oi, ctypes.c_uint32), _ptr(oj, ctypes.c_uint32), _ptr(os_, ctypes.c_double),
                        int(threads))
    if n < 0:
        raise MemoryError("oracle_topk: allocation failed")
    return oi[:n].copy(), oj[:n].copy(), os_[:n].copy()


def sim_pairs(R: np.ndarray, S: np.ndarray, i: np.ndarray, j: np.ndarray, threads: int = 0,
              mutant: int = 0) -> np.ndarray:
    """FP64 similarity of the given pairs, one by one (same arithmetic as ``join``)."""
    lib = _load(mutant)
    R = _rows_f32(R)
    S = _rows_f32(S)
    i = np.ascontiguousarray(i, dtype=np.uint32)
    j = np.ascontiguousarray(j, dtype=np.uint32)
    out = np.empty(len(i), dtype=np.float64)
    if len(i) == 0:
        return out
    lib.oracle_sim_pairs(_ptr(R, ctypes.c_float), R.strides[0] // 4, _ptr(S, ctypes.c_float),
                         S.strides[0] // 4, R.shape[1], _ptr(i, ctypes.c_uint32),
                         _ptr(j, ctypes.c_uint32), len(i), _ptr(out, ctypes.c_double), int(threads))
    return out


def norm(x: np.ndarray, mutant: int = 0) -> float:
    lib = _load(mutant)
    x = np.ascontiguousarray(x, dtype=np.float32)
    return lib.oracle_norm(_ptr(x, ctypes.c_float), x.shape[0])


def sim(a: np.ndarray, b: np.ndarray, mutant: int = 0) -> float:
    lib = _load(mutant)
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    return lib.oracle_sim(_ptr(a, ctypes.c_float), _ptr(b, ctypes.c_float), a.shape[0])


def count_selected(sel: Selection, mutant: int = 0) -> int:
    lib = _load(mutant)
    return int(lib.oracle_count_selected(_ptr(sel.attr, ctypes.c_int32), sel.op, sel.c,
                                         len(sel.attr)))
