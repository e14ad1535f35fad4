"""CPU oracle for exact selectivity computation and selection push-down.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the bench's ``cpu_baseline`` / ``--impl reference`` legs may import this
package.  It shares no code with the CUDA library and never imports it.

The arithmetic lives in ``oracle.c`` (a recursive row-by-row evaluator of the
uncompiled predicate tree, Ch3 §3.1 and Algorithm 1 ``Execute``); this module
only marshals the neutral predicate trees of ``datagen`` into the C structs of
that file and gathers projected columns of the selected rows
(``sigma_P(R)`` followed by ``pi_cols``, §3.1 / §3.3).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

O_AND, O_OR, O_NOT, O_CMP, O_BETWEEN, O_IN, O_LIKE, O_TRUE, O_FALSE = range(1, 10)
OPS = {"=": 0, "<>": 1, "<": 2, "<=": 3, ">": 4, ">=": 5}
TYPES = {"i32": 0, "i64": 1, "f32": 2, "date": 3, "dict": 4}


class ocol(C.Structure):
    _fields_ = [("type", C.c_int32), ("n_dict", C.c_int32), ("data", C.c_void_p),
                ("dict", C.POINTER(C.c_char_p))]


class onode(C.Structure):
    _fields_ = [("kind", C.c_int32), ("col", C.c_int32), ("op", C.c_int32), ("n_child", C.c_int32),
                ("child", C.POINTER(C.c_int32)), ("i0", C.c_int64), ("i1", C.c_int64),
                ("f0", C.c_float), ("f1", C.c_float), ("n_vals", C.c_int32),
                ("ivals", C.POINTER(C.c_int64)), ("fvals", C.POINTER(C.c_float)),
                ("prefix", C.c_char_p)]


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (plain gcc, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-fno-fast-math",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def load(path: Optional[str] = None):
    """Load the oracle library (``path`` lets tests load a deliberately mutated copy)."""
    global _lib
    if path is None and _lib is not None:
        return _lib
    with _lock:
        lib = C.CDLL(path or build())
        P = C.POINTER
        lib.oracle_count.restype = C.c_uint64
        lib.oracle_count.argtypes = [P(onode), C.c_int32, P(ocol), C.c_int64, C.c_int64]
        lib.oracle_count_mt.restype = C.c_uint64
        lib.oracle_count_mt.argtypes = [P(onode), C.c_int32, P(ocol), C.c_int64, C.c_int64, C.c_int32]
        lib.oracle_select.restype = C.c_int64
        lib.oracle_select.argtypes = [P(onode), C.c_int32, P(ocol), C.c_int64, C.c_int64,
                                      P(C.c_int64), C.c_int64]
        lib.oracle_select_mt.restype = C.c_int64
        lib.oracle_select_mt.argtypes = [P(onode), C.c_int32, P(ocol), C.c_int64, C.c_int64,
                                         P(C.c_int64), C.c_int64, C.c_int32]
        if path is None:
            _lib = lib
        return lib


class OTable:
    """Host view of a table: numpy arrays, type names and dictionaries."""

    def __init__(self, arrays: Sequence[np.ndarray], types: Sequence[str],
                 dicts: Sequence[Optional[List[bytes]]]):
        self.arrays = [np.ascontiguousarray(a) for a in arrays]
        self.types = list(types)
        self.dicts = list(dicts)
        self.n_rows = int(self.arrays[0].shape[0]) if self.arrays else 0
        self._keep = []
        cols = (ocol * max(1, len(self.arrays)))()
        for i, (a, t, d) in enumerate(zip(self.arrays, self.types, self.dicts)):
            cols[i].type = TYPES[t]
            cols[i].data = a.ctypes.data
            if d is not None:
                arr = (C.c_char_p * len(d))(*d)
                self._keep.append(arr)
                cols[i].dict = C.cast(arr, C.POINTER(C.c_char_p))
                cols[i].n_dict = len(d)
        self.cols = cols

    @classmethod
    def from_table(cls, table) -> "OTable":
        return cls([c.data.cpu().numpy() for c in table.columns], [c.type for c in table.columns],
                   [c.dictionary for c in table.columns])


def _f32_exact(v) -> float:
    f = np.float32(v)
    if float(f) != float(v):
        raise TypeError(f"constant {v!r} is not exactly representable as float32")
    return float(f)


def _int_const(v) -> int:
    if isinstance(v, (float, np.floating)):
        raise TypeError(f"integer-like column compared with float constant {v!r}")
    return int(v)


class Tree:
    """The neutral nested-tuple tree laid out as an array of oracle nodes."""

    def __init__(self, tree, types: Sequence[str]):
        self._keep = []
        self._nodes: List[dict] = []
        self.root = self._add(tree, types)
        arr = (onode * len(self._nodes))()
        for i, nd in enumerate(self._nodes):
            for k, v in nd.items():
                setattr(arr[i], k, v)
        self.nodes = arr

    def _add(self, t, types) -> int:
        k = t[0]
        nd = {"col": -1}
        if k in ("and", "or", "not"):
            kids = t[1] if k != "not" else [t[1]]
            idx = [self._add(c, types) for c in kids]
            carr = (C.c_int32 * max(1, len(idx)))(*idx)
            self._keep.append(carr)
            nd.update(kind={"and": O_AND, "or": O_OR, "not": O_NOT}[k], n_child=len(idx),
                      child=C.cast(carr, C.POINTER(C.c_int32)))
        elif k == "true":
            nd.update(kind=O_TRUE)
        elif k == "false":
            nd.update(kind=O_FALSE)
        else:
            col = int(t[1])
            if col < 0 or col >= len(types):
                raise IndexError(f"column {col} out of range")
            ty = types[col]
            nd["col"] = col
            isf = ty == "f32"
            if k == "cmp":
                nd.update(kind=O_CMP, op=OPS[t[2]])
                if isf:
                    nd["f0"] = _f32_exact(t[3])
                else:
                    nd["i0"] = _int_const(t[3])
            elif k == "between":
                nd.update(kind=O_BETWEEN)
                if isf:
                    nd.update(f0=_f32_exact(t[2]), f1=_f32_exact(t[3]))
                else:
                    nd.update(i0=_int_const(t[2]), i1=_int_const(t[3]))
            elif k == "in":
                vals = list(t[2])
                nd.update(kind=O_IN, n_vals=len(vals))
                if isf:
                    a = (C.c_float * max(1, len(vals)))(*[_f32_exact(v) for v in vals])
                    nd["fvals"] = C.cast(a, C.POINTER(C.c_float))
                else:
                    a = (C.c_int64 * max(1, len(vals)))(*[_int_const(v) for v in vals])
                    nd["ivals"] = C.cast(a, C.POINTER(C.c_int64))
                self._keep.append(a)
            elif k == "like":
                if ty != "dict":
                    raise TypeError("LIKE needs a dictionary column")
                b = t[2].encode() if isinstance(t[2], str) else bytes(t[2])
                nd.update(kind=O_LIKE, prefix=b)
                self._keep.append(b)
            else:
                raise ValueError(f"unknown node {k!r}")
        self._nodes.append(nd)
        return len(self._nodes) - 1


def _otable(table) -> OTable:
    return table if isinstance(table, OTable) else OTable.from_table(table)


def count(table, tree, row_begin: int = 0, row_end: Optional[int] = None, threads: int = 1,
          lib=None) -> int:
    """Exact |{i : P(R[i])}| over rows [row_begin, row_end)."""
    ot = _otable(table)
    lib = lib or load()
    tr = Tree(tree, ot.types)
    e = ot.n_rows if row_end is None else row_end
    if threads <= 1:
        return int(lib.oracle_count(tr.nodes, tr.root, ot.cols, row_begin, e))
    return int(lib.oracle_count_mt(tr.nodes, tr.root, ot.cols, row_begin, e, threads))


def select(table, tree, row_begin: int = 0, row_end: Optional[int] = None, threads: int = 1,
           lib=None) -> np.ndarray:
    """Ascending int64 row ids of the rows satisfying the predicate."""
    ot = _otable(table)
    lib = lib or load()
    tr = Tree(tree, ot.types)
    e = ot.n_rows if row_end is None else row_end
    n = count(ot, tree, row_begin, e, threads, lib)
    out = np.empty(max(1, n), dtype=np.int64)
    ptr = out.ctypes.data_as(C.POINTER(C.c_int64))
    if threads <= 1:
        k = lib.oracle_select(tr.nodes, tr.root, ot.cols, row_begin, e, ptr, n)
    else:
        k = lib.oracle_select_mt(tr.nodes, tr.root, ot.cols, row_begin, e, ptr, n, threads)
    assert k == n
    return out[:n]


def max_rows_for_ratio(n_rows: int, ratio: float) -> int:
    """maxSize = R.size * PUSH_DOWN_MAX_SELECTIVITY (Algorithm 1), floored in double."""
    return int(np.floor(float(n_rows) * float(ratio)))


def pushdown(table, tree, proj: Sequence[int], max_rows: int, threads: int = 1, lib=None):
    """Algorithm 1 Execute(compound, isSPD=true, maxSize): the COUNT first, reject
    when count > maxSize, else the projected rows of sigma_P(R) in row order.

    Returns (status, count, [projected column arrays], row ids); status is
    "OK" or "TOO_LARGE" (the paper's thrown exception)."""
    ot = _otable(table)
    n = count(ot, tree, 0, None, threads, lib)
    if n > max_rows:
        return "TOO_LARGE", n, None, None
    ids = select(ot, tree, 0, None, threads, lib)
    return "OK", n, [ot.arrays[c][ids] for c in proj], ids
