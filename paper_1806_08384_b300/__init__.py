"""Python binding of libsel.so (include/sel.h): argument marshalling only.

Every step of the hot path runs in the library's CUDA kernels; this module
converts predicate trees and torch-tensor tables into the C structs of the
ABI and calls it.  There is no fallback: if libsel.so is missing or fails to
load, importing this package raises.

Predicate trees use the neutral nested-tuple form (see ``tree_to_postfix``):
("and", [...]), ("or", [...]), ("not", x), ("cmp", col, op, v),
("between", col, lo, hi), ("in", col, [v...]), ("like", col, "prefix"),
("true",), ("false",).
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import List, Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsel.so")

SEL_OK, SEL_ERR_INVALID_ARG, SEL_ERR_TYPE, SEL_ERR_UNSUPPORTED, SEL_ERR_OOM, SEL_ERR_CUDA, \
    SEL_ERR_TOO_LARGE, SEL_ERR_TIMEOUT = range(8)
STATUS_NAMES = ["SEL_OK", "SEL_ERR_INVALID_ARG", "SEL_ERR_TYPE", "SEL_ERR_UNSUPPORTED", "SEL_ERR_OOM",
                "SEL_ERR_CUDA", "SEL_ERR_TOO_LARGE", "SEL_ERR_TIMEOUT"]
TYPE_CODES = {"i32": 0, "i64": 1, "f32": 2, "date": 3, "dict": 4}
TORCH_TYPES = {"i32": torch.int32, "i64": torch.int64, "f32": torch.float32, "date": torch.int32,
               "dict": torch.int32}
N_CMP, N_BETWEEN, N_IN, N_LIKE, N_AND, N_OR, N_NOT, N_TRUE, N_FALSE = range(1, 10)
OPS = {"=": 0, "<>": 1, "<": 2, "<=": 3, ">": 4, ">=": 5}
SEL_PD_AUTO, SEL_PD_TWO_PASS, SEL_PD_ONE_PASS = 0, 1, 2


class sel_column(C.Structure):
    _fields_ = [("type", C.c_int32), ("dict_size", C.c_int32), ("data", C.c_void_p),
                ("dict", C.POINTER(C.c_char_p))]


class sel_table(C.Structure):
    _fields_ = [("cols", C.POINTER(sel_column)), ("n_cols", C.c_int32), ("n_rows", C.c_int64)]


class sel_node(C.Structure):
    _fields_ = [("kind", C.c_int32), ("col", C.c_int32), ("op", C.c_int32), ("n_children", C.c_int32),
                ("i_lo", C.c_int64), ("i_hi", C.c_int64), ("f_lo", C.c_float), ("f_hi", C.c_float),
                ("n_values", C.c_int32), ("reserved", C.c_int32), ("values", C.c_void_p),
                ("prefix", C.c_char_p)]


class TrainCfg(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("seed", C.c_uint64), ("apply_update", C.c_int32),
                ("reserved", C.c_int32)]


def train_cfg(epochs=5, batch=4096, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, seed=0, apply_update=1) -> TrainCfg:
    return TrainCfg(epochs, batch, lr, beta1, beta2, eps, seed, apply_update, 0)


class sel_spd_relation(C.Structure):
    _fields_ = [("table", C.POINTER(sel_table)), ("pred", C.c_void_p), ("proj_cols", C.POINTER(C.c_int32)),
                ("n_proj", C.c_int32), ("dev_out_cols", C.POINTER(C.c_void_p)), ("dev_out_rowids", C.c_void_p)]


class sel_spd_cfg(C.Structure):
    _fields_ = [("min_table_size", C.c_uint64), ("max_selectivity", C.c_double), ("max_rows", C.c_uint64)]


SPD_PROBE, SPD_TOO_SMALL, SPD_NO_PREDICATE, SPD_PUSHED, SPD_REVERTED = range(5)
SPD_NAMES = ("probe", "too_small", "no_predicate", "pushed", "reverted")


class SelError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built (python {os.path.join(_HERE, 'build.py')})")
    lib = C.CDLL(LIB_PATH)
    P, V = C.POINTER, C.c_void_p
    sigs = {
        "sel_last_error": (C.c_char_p, []),
        "sel_status_str": (C.c_char_p, [C.c_int]),
        "sel_ctx_create": (C.c_int, [V, P(V)]),
        "sel_ctx_destroy": (None, [V]),
        "sel_compile_predicate": (C.c_int, [P(sel_table), P(sel_node), C.c_int32, P(V)]),
        "sel_pred_free": (None, [V]),
        "sel_pred_describe": (C.c_int, [V, C.c_char_p, C.c_int64]),
        "sel_count": (C.c_int, [V, V, P(sel_table), P(C.c_uint64)]),
        "sel_count_async": (C.c_int, [V, V, P(sel_table), V]),
        "sel_pushdown": (C.c_int, [V, V, P(sel_table), P(C.c_int32), C.c_int32, P(V), V, C.c_uint64,
                                   P(C.c_uint64)]),
        "sel_count_batch": (C.c_int, [V, P(V), P(P(sel_table)), C.c_int32, P(C.c_uint64)]),
        "sel_count_batch_async": (C.c_int, [V, P(V), P(P(sel_table)), C.c_int32, V]),
        "sel_pushdown_async": (C.c_int, [V, V, P(sel_table), P(C.c_int32), C.c_int32, P(V), V, C.c_uint64, V]),
        "sel_ctx_synchronize": (C.c_int, [V]),
        "sel_pushdown_noalloc": (C.c_int, [V, V, P(sel_table), P(C.c_int32), C.c_int32, P(V), V, C.c_uint64, V, V]),
        "sel_batch_plan_create": (C.c_int, [V, P(V), P(P(sel_table)), C.c_int32, C.c_int32, P(V)]),
        "sel_batch_plan_run": (C.c_int, [V, V, P(C.c_uint64)]),
        "sel_batch_plan_info": (C.c_int, [V, P(C.c_int32), P(C.c_int32), P(C.c_int32), P(C.c_float)]),
        "sel_batch_plan_variant": (C.c_int, [V, P(C.c_int32), P(C.c_int32)]),
        "sel_batch_plan_free": (None, [V]),
        "sel_batch_plan_kernel": (C.c_int, [V, P(C.c_int32)]),
        "sel_debug_fail_allocation": (C.c_int, [C.c_int64]),
        "sel_ctx_set_batch_kernel": (C.c_int, [V, C.c_int32]),
        "sel_debug_bucket_count_host": (C.c_int, [P(V), C.c_int32, P(sel_table), P(C.c_uint64), P(C.c_int32),
                                                  P(C.c_int32)]),
        "sel_ctx_set_scan_shape": (C.c_int, [V, C.c_int32, C.c_int32, C.c_int32]),
        "sel_ctx_set_scan_variant": (C.c_int, [V, C.c_int32, C.c_int32]),
        "sel_ctx_launch_count": (C.c_uint64, [V]),
        "sel_ctx_debug_pushdown_fault": (C.c_int, [V, C.c_int64, C.c_uint64]),
        "sel_ctx_set_pushdown_super_rows": (C.c_int, [V, C.c_int32]),
        "sel_ctx_set_pushdown_method": (C.c_int, [V, C.c_int32]),
        "sel_ctx_set_pushdown_split_event": (C.c_int, [V, V]),
        "sel_debug_gemm_bf16": (C.c_int, [V, V, V, C.c_int32, C.c_int32, C.c_int32, V, C.c_int32, V]),
        "sel_count_distinct": (C.c_int, [V, P(sel_table), C.c_int32, V, P(C.c_uint64), P(C.c_uint64)]),
        "sel_join_size_estimate": (C.c_double, [C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64]),
        "sel_join_count": (C.c_int, [V, P(sel_table), C.c_int32, V, P(sel_table), C.c_int32, V, P(C.c_uint64),
                                     P(C.c_uint64), P(C.c_uint64)]),
        "sel_evaluate_and_push_down": (C.c_int, [V, P(sel_spd_relation), C.c_int32, P(sel_spd_cfg), P(C.c_int32),
                                                 P(C.c_uint64), P(C.c_uint64)]),
        "sel_mlp_create": (C.c_int, [V, P(sel_table), C.c_int32, C.c_uint64, P(V)]),
        "sel_mlp_free": (None, [V]),
        "sel_mlp_featurize": (C.c_int, [V, V, P(V), C.c_int32, V, V]),
        "sel_mlp_forward": (C.c_int, [V, V, V, C.c_int32, V]),
        "sel_debug_mlp_fused": (C.c_int, [V, C.c_int32]),
        "sel_mlp_train_step": (C.c_int, [V, V, V, V, C.c_int32, P(TrainCfg), P(C.c_float)]),
        "sel_mlp_train": (C.c_int, [V, V, P(V), P(C.c_uint64), C.c_int64, P(TrainCfg), P(C.c_float)]),
        "sel_mlp_estimate": (C.c_int, [V, V, P(V), P(sel_table), C.c_int32, C.c_float, P(C.c_double),
                                       P(C.c_float), P(C.c_uint8)]),
        "sel_mlp_param_count": (C.c_int64, []),
        "sel_mlp_choose_tau": (C.c_int, [P(C.c_float), P(C.c_double), P(C.c_uint64), C.c_int64, C.c_double,
                                         C.c_double, P(C.c_float), P(C.c_double)]),
        "sel_mlp_get_params": (C.c_int, [V, P(C.c_float), C.c_int64]),
        "sel_mlp_set_params": (C.c_int, [V, V, P(C.c_float), C.c_int64]),
        "sel_mlp_get_grads": (C.c_int, [V, P(C.c_float), C.c_int64]),
        "sel_mlp_save": (C.c_int, [V, C.c_char_p]),
        "sel_mlp_load": (C.c_int, [V, C.c_char_p, P(V)]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def _check(status: int, where: str):
    if status != SEL_OK:
        raise SelError(status, where, lib.sel_last_error().decode(errors="replace"))


# ----------------------------------------------------------------------------
# tables
# ----------------------------------------------------------------------------

class Table:
    """A sel_table over torch tensors (device columns) plus host dictionaries.

    ``columns``: sequence of objects with ``.data`` (1-D torch tensor),
    ``.type`` (one of i32 i64 f32 date dict) and ``.dictionary`` (list of
    bytes or None) -- e.g. a ``datagen.Table``'s columns."""

    def __init__(self, columns, n_rows: Optional[int] = None):
        self.columns = list(columns)
        self.types = [c.type for c in self.columns]
        self._keep = []
        arr = (sel_column * max(1, len(self.columns)))()
        rows = None
        for i, c in enumerate(self.columns):
            t = c.data
            if t.dtype != TORCH_TYPES[c.type] or t.dim() != 1 or not t.is_contiguous():
                raise TypeError(f"column {i}: need a contiguous 1-D {TORCH_TYPES[c.type]} tensor")
            rows = t.numel() if rows is None else rows
            if t.numel() != rows:
                raise ValueError("columns differ in length")
            arr[i].type = TYPE_CODES[c.type]
            arr[i].data = t.data_ptr() if t.numel() else None
            d = getattr(c, "dictionary", None)
            if d is not None:
                darr = (C.c_char_p * len(d))(*d)
                self._keep.append(darr)
                arr[i].dict = C.cast(darr, C.POINTER(C.c_char_p))
                arr[i].dict_size = len(d)
        self.cols = arr
        self.n_rows = int(rows or 0) if n_rows is None else int(n_rows)
        self.desc = sel_table(C.cast(arr, C.POINTER(sel_column)), len(self.columns), self.n_rows)

    @classmethod
    def of(cls, t) -> "Table":
        return t if isinstance(t, Table) else cls(t.columns)

    def ref(self):
        return C.byref(self.desc)


# ----------------------------------------------------------------------------
# predicates
# ----------------------------------------------------------------------------

def _f32(v) -> float:
    f = np.float32(v)
    if not (float(f) == float(v) or (np.isnan(f) and np.isnan(float(v)))):
        raise TypeError(f"constant {v!r} is not exactly representable as float32")
    return float(f)


def _int(v) -> int:
    if isinstance(v, (float, np.floating)):
        raise TypeError(f"integer-like column compared with float constant {v!r}")
    return int(v)


def tree_to_postfix(tree, types: Sequence[str]):
    """Neutral tree -> (ctypes array of sel_node, keep-alive list)."""
    nodes, keep = [], []

    def leaf(kind, col):
        n = sel_node()
        n.kind, n.col = kind, int(col)
        return n

    def walk(t):
        k = t[0]
        if k in ("and", "or"):
            for c in t[1]:
                walk(c)
            if not t[1]:                      # empty AND is TRUE, empty OR is FALSE
                n = sel_node()
                n.kind = N_TRUE if k == "and" else N_FALSE
                nodes.append(n)
                return
            n = sel_node()
            n.kind, n.n_children = (N_AND if k == "and" else N_OR), len(t[1])
            nodes.append(n)
        elif k == "not":
            walk(t[1])
            n = sel_node()
            n.kind = N_NOT
            nodes.append(n)
        elif k in ("true", "false"):
            n = sel_node()
            n.kind = N_TRUE if k == "true" else N_FALSE
            nodes.append(n)
        else:
            col = int(t[1])
            isf = 0 <= col < len(types) and types[col] == "f32"
            if k == "cmp":
                n = leaf(N_CMP, col)
                n.op = OPS[t[2]]
                if isf:
                    n.f_lo = _f32(t[3])
                else:
                    n.i_lo = _int(t[3])
            elif k == "between":
                n = leaf(N_BETWEEN, col)
                if isf:
                    n.f_lo, n.f_hi = _f32(t[2]), _f32(t[3])
                else:
                    n.i_lo, n.i_hi = _int(t[2]), _int(t[3])
            elif k == "in":
                vals = list(t[2])
                n = leaf(N_IN, col)
                n.n_values = len(vals)
                if vals:
                    a = np.array([_f32(v) for v in vals], np.float32) if isf else \
                        np.array([_int(v) for v in vals], np.int64)
                    keep.append(a)
                    n.values = a.ctypes.data
            elif k == "like":
                n = leaf(N_LIKE, col)
                b = t[2].encode() if isinstance(t[2], str) else bytes(t[2])
                keep.append(b)
                n.prefix = b
            else:
                raise ValueError(f"unknown node {k!r}")
            nodes.append(n)

    walk(tree)
    arr = (sel_node * len(nodes))(*nodes)
    return arr, keep


class Predicate:
    """A compiled predicate (sel_pred); compiled against a table schema."""

    def __init__(self, schema, tree):
        schema = Table.of(schema)
        self.tree = tree
        arr, keep = tree_to_postfix(tree, schema.types)
        h = C.c_void_p()
        _check(lib.sel_compile_predicate(schema.ref(), arr, len(arr), C.byref(h)), "sel_compile_predicate")
        self.h = h

    def describe(self) -> str:
        buf = C.create_string_buffer(1 << 16)
        _check(lib.sel_pred_describe(self.h, buf, len(buf)), "sel_pred_describe")
        return buf.value.decode()

    def __del__(self):
        h = getattr(self, "h", None)
        if h and h.value and lib is not None:
            lib.sel_pred_free(h)
            self.h = None


def compile_predicate(schema, tree) -> Predicate:
    return Predicate(schema, tree)


# ----------------------------------------------------------------------------
# context and calls
# ----------------------------------------------------------------------------

class Context:
    """A sel_ctx bound to a CUDA stream (default: torch's current stream)."""

    def __init__(self, stream: Optional[torch.cuda.Stream] = None):
        self.stream = stream or torch.cuda.current_stream()
        h = C.c_void_p()
        _check(lib.sel_ctx_create(C.c_void_p(self.stream.cuda_stream), C.byref(h)), "sel_ctx_create")
        self.h = h

    def set_scan_shape(self, tile_rows=0, stages=0, ctas_per_sm=0):
        _check(lib.sel_ctx_set_scan_shape(self.h, tile_rows, stages, ctas_per_sm), "sel_ctx_set_scan_shape")

    def count_distinct(self, table, col: int, pred: Optional[Predicate] = None):
        """(V(sigma_P(R), col), |sigma_P(R)|): distinct values of a column over the selected rows."""
        table = Table.of(table)
        d, r = C.c_uint64(), C.c_uint64()
        _check(lib.sel_count_distinct(self.h, table.ref(), int(col), pred.h if pred is not None else None,
                                      C.byref(d), C.byref(r)), "sel_count_distinct")
        return int(d.value), int(r.value)

    def join_count(self, r, col_r: int, pred_r: Optional[Predicate], s, col_s: int, pred_s: Optional[Predicate]):
        """(COUNT(*) of sigma_P(R) join sigma_Q(S) on R.col_r = S.col_s, |sigma_P(R)|, |sigma_Q(S)|)."""
        r, s = Table.of(r), Table.of(s)
        c, nr, ns = C.c_uint64(), C.c_uint64(), C.c_uint64()
        _check(lib.sel_join_count(self.h, r.ref(), int(col_r), pred_r.h if pred_r is not None else None, s.ref(),
                                  int(col_s), pred_s.h if pred_s is not None else None, C.byref(c), C.byref(nr),
                                  C.byref(ns)), "sel_join_count")
        return int(c.value), int(nr.value), int(ns.value)

    def set_scan_variant(self, consumer_warps=0, chunks_per_pass=0):
        _check(lib.sel_ctx_set_scan_variant(self.h, consumer_warps, chunks_per_pass), "sel_ctx_set_scan_variant")

    def set_batch_kernel(self, mode: int):
        """0: the faster of both kernels, 1: interpreter only, 2: bucket kernel only."""
        _check(lib.sel_ctx_set_batch_kernel(self.h, int(mode)), "sel_ctx_set_batch_kernel")

    def set_pushdown_super_rows(self, rows: int):
        """Super-tile target of the persistent push-down (0: from the table size)."""
        _check(lib.sel_ctx_set_pushdown_super_rows(self.h, rows), "sel_ctx_set_pushdown_super_rows")

    def set_pushdown_method(self, method: int):
        """SEL_PD_AUTO (two passes), SEL_PD_TWO_PASS or SEL_PD_ONE_PASS."""
        _check(lib.sel_ctx_set_pushdown_method(self.h, int(method)), "sel_ctx_set_pushdown_method")

    def set_pushdown_split_event(self, event: Optional[torch.cuda.Event]):
        """Record `event` between the two passes of each later push-down (None: off).
        The event must have been recorded once (torch creates it lazily)."""
        h = C.c_void_p(event.cuda_event if event is not None else None)
        _check(lib.sel_ctx_set_pushdown_split_event(self.h, h), "sel_ctx_set_pushdown_split_event")

    def debug_pushdown_fault(self, skip_tile: int, wait_ns: int = 0):
        _check(lib.sel_ctx_debug_pushdown_fault(self.h, skip_tile, wait_ns), "sel_ctx_debug_pushdown_fault")

    @property
    def launches(self) -> int:
        return int(lib.sel_ctx_launch_count(self.h))

    def count(self, pred: Predicate, table) -> int:
        table = Table.of(table)
        out = C.c_uint64()
        _check(lib.sel_count(self.h, pred.h, table.ref(), C.byref(out)), "sel_count")
        return int(out.value)

    def count_async(self, pred: Predicate, table, out: torch.Tensor):
        """Enqueues the count into out (a 1-element int64 device tensor)."""
        table = Table.of(table)
        _check(lib.sel_count_async(self.h, pred.h, table.ref(), C.c_void_p(out.data_ptr())), "sel_count_async")

    def pushdown(self, pred: Predicate, table, proj: Sequence[int], max_rows: int, rowids: bool = True,
                 out_cols: Optional[List[torch.Tensor]] = None, out_rowids: Optional[torch.Tensor] = None,
                 raise_too_large: bool = False):
        """Selection push-down (Algorithm 1 Execute).  Returns (status, count,
        [projected columns truncated to count], row ids or None); status is
        SEL_OK or SEL_ERR_TOO_LARGE."""
        table = Table.of(table)
        dev = table.columns[0].data.device if table.columns else torch.device("cuda")
        cap = max(int(max_rows), 0)
        if out_cols is None:
            out_cols = [torch.empty(max(cap, 1), dtype=TORCH_TYPES[table.types[c]], device=dev) for c in proj]
        if rowids and out_rowids is None:
            out_rowids = torch.empty(max(cap, 1), dtype=torch.int64, device=dev)
        pc = (C.c_int32 * max(1, len(proj)))(*proj)
        po = (C.c_void_p * max(1, len(proj)))(*[t.data_ptr() for t in out_cols])
        out = C.c_uint64()
        st = lib.sel_pushdown(self.h, pred.h, table.ref(), pc, len(proj), po,
                              C.c_void_p(out_rowids.data_ptr()) if rowids else None, cap, C.byref(out))
        n = int(out.value)
        if st == SEL_ERR_TOO_LARGE and not raise_too_large:
            return st, n, None, None
        _check(st, "sel_pushdown")
        return st, n, [t[:n] for t in out_cols], (out_rowids[:n] if rowids else None)

    def pushdown_async(self, pred: Predicate, table, proj: Sequence[int], max_rows: int,
                       out_cols: List[torch.Tensor], out_rowids: Optional[torch.Tensor], out_count: torch.Tensor):
        """Enqueues the push-down; the exact count goes to out_count (int64 device tensor)."""
        table = Table.of(table)
        pc = (C.c_int32 * max(1, len(proj)))(*proj)
        po = (C.c_void_p * max(1, len(proj)))(*[t.data_ptr() for t in out_cols])
        _check(lib.sel_pushdown_async(self.h, pred.h, table.ref(), pc, len(proj), po,
                                      C.c_void_p(out_rowids.data_ptr()) if out_rowids is not None else None,
                                      int(max_rows), C.c_void_p(out_count.data_ptr())), "sel_pushdown_async")

    def count_batch_async(self, preds: Sequence[Predicate], tables, out: torch.Tensor):
        """Enqueues the batched counts into out (int64 device tensor of len(preds))."""
        tabs = [Table.of(t) for t in tables]
        n = len(preds)
        pa = (C.c_void_p * n)(*[p.h.value for p in preds])
        ta = (C.POINTER(sel_table) * n)(*[C.pointer(t.desc) for t in tabs])
        _check(lib.sel_count_batch_async(self.h, pa, ta, n, C.c_void_p(out.data_ptr())), "sel_count_batch_async")

    def synchronize(self):
        _check(lib.sel_ctx_synchronize(self.h), "sel_ctx_synchronize")

    def count_batch(self, preds: Sequence[Predicate], tables) -> List[int]:
        tabs = [Table.of(t) for t in tables]
        n = len(preds)
        pa = (C.c_void_p * n)(*[p.h.value for p in preds])
        ta = (C.POINTER(sel_table) * n)(*[C.pointer(t.desc) for t in tabs])
        out = (C.c_uint64 * n)()
        _check(lib.sel_count_batch(self.h, pa, ta, n, out), "sel_count_batch")
        return [int(x) for x in out]

    def __del__(self):
        h = getattr(self, "h", None)
        if h and h.value and lib is not None:
            lib.sel_ctx_destroy(h)
            self.h = None


def pushdown_noalloc(pred: Predicate, table, proj: Sequence[int], max_rows: int, out_cols: List[torch.Tensor],
                     out_rowids: Optional[torch.Tensor], out_count: torch.Tensor,
                     out_error: Optional[torch.Tensor], stream: Optional[torch.cuda.Stream] = None):
    """sel_pushdown_noalloc: the push-down with the library's fixed scratch and
    caller-owned outputs only (no context, no device allocation); enqueue only.
    out_error (int32, 1 element) is required; None is passed on as NULL and
    the library rejects it."""
    table = Table.of(table)
    stream = stream or torch.cuda.current_stream()
    pc = (C.c_int32 * max(1, len(proj)))(*proj)
    po = (C.c_void_p * max(1, len(proj)))(*[t.data_ptr() for t in out_cols])
    _check(lib.sel_pushdown_noalloc(C.c_void_p(stream.cuda_stream), pred.h, table.ref(), pc, len(proj), po,
                                    C.c_void_p(out_rowids.data_ptr()) if out_rowids is not None else None,
                                    int(max_rows), C.c_void_p(out_count.data_ptr()),
                                    C.c_void_p(out_error.data_ptr()) if out_error is not None else None),
           "sel_pushdown_noalloc")


def debug_gemm_bf16(A: torch.Tensor, B: torch.Tensor, k_splits: int = 1) -> torch.Tensor:
    """C = A @ B.T on the tensor cores (bf16 inputs, fp32 result); for tests."""
    M, K = A.shape
    N = B.shape[0]
    C_ = torch.empty(M, N, dtype=torch.float32, device=A.device)
    err = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check(lib.sel_debug_gemm_bf16(C.c_void_p(torch.cuda.current_stream().cuda_stream), C.c_void_p(A.data_ptr()),
                                   C.c_void_p(B.data_ptr()), M, N, K, C.c_void_p(C_.data_ptr()), k_splits,
                                   C.c_void_p(err.data_ptr())), "sel_debug_gemm_bf16")
    torch.cuda.synchronize()
    if int(err.item()):
        raise SelError(SEL_ERR_TIMEOUT, "sel_debug_gemm_bf16", "a bounded wait gave up")
    return C_


class BatchPlan:
    """sel_batch_plan: the predicates and tables must outlive the plan."""

    def __init__(self, ctx: Context, preds: Sequence[Predicate], tables, autotune: bool = True):
        self.ctx = ctx
        self.preds = list(preds)
        self.tables = [Table.of(t) for t in tables]
        n = len(self.preds)
        self.n = n
        pa = (C.c_void_p * n)(*[p.h.value for p in self.preds])
        ta = (C.POINTER(sel_table) * n)(*[C.pointer(t.desc) for t in self.tables])
        self._keep = (pa, ta)
        h = C.c_void_p()
        _check(lib.sel_batch_plan_create(ctx.h, pa, ta, n, 1 if autotune else 0, C.byref(h)),
               "sel_batch_plan_create")
        self.h = h

    def run(self, device_out: Optional[torch.Tensor] = None) -> Optional[List[int]]:
        if device_out is not None:
            _check(lib.sel_batch_plan_run(self.h, C.c_void_p(device_out.data_ptr()), None), "sel_batch_plan_run")
            return None
        out = (C.c_uint64 * self.n)()
        _check(lib.sel_batch_plan_run(self.h, None, out), "sel_batch_plan_run")
        return [int(x) for x in out]

    def info(self):
        tr, st, cp, ms = C.c_int32(), C.c_int32(), C.c_int32(), C.c_float()
        _check(lib.sel_batch_plan_info(self.h, C.byref(tr), C.byref(st), C.byref(cp), C.byref(ms)),
               "sel_batch_plan_info")
        w, g = C.c_int32(), C.c_int32()
        _check(lib.sel_batch_plan_variant(self.h, C.byref(w), C.byref(g)), "sel_batch_plan_variant")
        k = C.c_int32()
        _check(lib.sel_batch_plan_kernel(self.h, C.byref(k)), "sel_batch_plan_kernel")
        return {"tile_rows": tr.value, "stages": st.value, "ctas_per_sm": cp.value, "ms": ms.value,
                "consumer_warps": w.value, "chunks_per_pass": g.value,
                "kernel": ("interpreter", "bucket")[k.value]}

    def __del__(self):
        h = getattr(self, "h", None)
        if h and h.value and lib is not None:
            lib.sel_batch_plan_free(h)
            self.h = None


# ----------------------------------------------------------------------------
# learned estimator
# ----------------------------------------------------------------------------

N_FEATURES = 144


class PredicateList:
    """A fixed list of predicates with its C array of handles built once (for
    calls that pass the same predicates again and again)."""

    def __init__(self, preds: Sequence[Predicate]):
        self.preds = list(preds)
        self.handles = (C.c_void_p * max(1, len(self.preds)))(*[p.h.value for p in self.preds])

    def __len__(self):
        return len(self.preds)

    def __getitem__(self, i):
        return self.preds[i]


class Estimator:
    """sel_mlp: CDF-sampled features, a BF16 tensor-core MLP and the gated
    exact fallback (see include/sel.h)."""

    def __init__(self, ctx: "Context", table=None, sample_rows: int = 4096, seed: int = 0, _handle=None):
        self.ctx = ctx
        if _handle is not None:
            self.h = _handle
            return
        table = Table.of(table)
        h = C.c_void_p()
        _check(lib.sel_mlp_create(ctx.h, table.ref(), sample_rows, seed, C.byref(h)), "sel_mlp_create")
        self.h = h

    @classmethod
    def load(cls, ctx: "Context", path: str) -> "Estimator":
        h = C.c_void_p()
        _check(lib.sel_mlp_load(ctx.h, path.encode(), C.byref(h)), "sel_mlp_load")
        return cls(ctx, _handle=h)

    def save(self, path: str):
        _check(lib.sel_mlp_save(self.h, path.encode()), "sel_mlp_save")

    def featurize(self, preds, device="cuda"):
        """preds: a sequence of Predicate, or a PredicateList (its handle array is built once)."""
        n = len(preds)
        feat = torch.empty(n, N_FEATURES, dtype=torch.bfloat16, device=device)
        ok = torch.empty(n, dtype=torch.uint8, device=device)
        pa = preds.handles if isinstance(preds, PredicateList) else (C.c_void_p * n)(*[p.h.value for p in preds])
        _check(lib.sel_mlp_featurize(self.ctx.h, self.h, pa, n, C.c_void_p(feat.data_ptr()),
                                     C.c_void_p(ok.data_ptr())), "sel_mlp_featurize")
        return feat, ok

    def forward(self, feat: torch.Tensor) -> torch.Tensor:
        out = torch.empty(feat.shape[0], 2, dtype=torch.float32, device=feat.device)
        _check(lib.sel_mlp_forward(self.ctx.h, self.h, C.c_void_p(feat.data_ptr()), feat.shape[0],
                                   C.c_void_p(out.data_ptr())), "sel_mlp_forward")
        return out

    def set_fused(self, on: bool):
        """sel_debug_mlp_fused: inference in one kernel (default) or layer by layer."""
        _check(lib.sel_debug_mlp_fused(self.h, 1 if on else 0), "sel_debug_mlp_fused")

    def train_step(self, feat: torch.Tensor, y: torch.Tensor, cfg: TrainCfg) -> float:
        loss = C.c_float()
        _check(lib.sel_mlp_train_step(self.ctx.h, self.h, C.c_void_p(feat.data_ptr()), C.c_void_p(y.data_ptr()),
                                      feat.shape[0], C.byref(cfg), C.byref(loss)), "sel_mlp_train_step")
        return float(loss.value)

    def train(self, preds: Sequence[Predicate], counts, cfg: TrainCfg) -> float:
        n = len(preds)
        pa = (C.c_void_p * n)(*[p.h.value for p in preds])
        ca = np.ascontiguousarray(np.asarray(counts, dtype=np.uint64))
        loss = C.c_float()
        _check(lib.sel_mlp_train(self.ctx.h, self.h, pa, ca.ctypes.data_as(C.POINTER(C.c_uint64)), n, C.byref(cfg),
                                 C.byref(loss)), "sel_mlp_train")
        return float(loss.value)

    def estimate(self, preds: Sequence[Predicate], table, tau: float):
        table = Table.of(table)
        n = len(preds)
        pa = (C.c_void_p * n)(*[p.h.value for p in preds])
        est = np.zeros(n, np.float64)
        sig = np.zeros(n, np.float32)
        used = np.zeros(n, np.uint8)
        _check(lib.sel_mlp_estimate(self.ctx.h, self.h, pa, table.ref(), n, float(tau),
                                    est.ctypes.data_as(C.POINTER(C.c_double)),
                                    sig.ctypes.data_as(C.POINTER(C.c_float)),
                                    used.ctypes.data_as(C.POINTER(C.c_uint8))), "sel_mlp_estimate")
        return est, sig, used.astype(bool)

    def get_params(self) -> np.ndarray:
        n = int(lib.sel_mlp_param_count())
        a = np.zeros(n, np.float32)
        _check(lib.sel_mlp_get_params(self.h, a.ctypes.data_as(C.POINTER(C.c_float)), n), "sel_mlp_get_params")
        return a

    def get_grads(self) -> np.ndarray:
        n = int(lib.sel_mlp_param_count())
        a = np.zeros(n, np.float32)
        _check(lib.sel_mlp_get_grads(self.h, a.ctypes.data_as(C.POINTER(C.c_float)), n), "sel_mlp_get_grads")
        return a

    def set_params(self, flat: np.ndarray):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        _check(lib.sel_mlp_set_params(self.ctx.h, self.h, a.ctypes.data_as(C.POINTER(C.c_float)), a.size),
               "sel_mlp_set_params")

    def __del__(self):
        h = getattr(self, "h", None)
        if h and h.value and lib is not None:
            lib.sel_mlp_free(h)
            self.h = None


PARAM_LAYOUT = [("W1", (256, 144)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)), ("W3", (256, 256)),
                ("b3", (256,)), ("W4", (2, 256)), ("b4", (2,))]


def unflatten(flat: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in PARAM_LAYOUT:
        k = int(np.prod(shape))
        out[name] = flat[o:o + k].reshape(shape)
        o += k
    return out


def flatten(params: dict) -> np.ndarray:
    return np.concatenate([np.asarray(params[name], np.float32).ravel() for name, _ in PARAM_LAYOUT])


def count_many(ctx: "Context", preds: Sequence[Predicate], table, chunk: int = 256) -> List[int]:
    """Exact counts of many predicates over one table, in batch plans of
    `chunk` probes (256: one quad of the bucket kernel, 0.083 ms per label on
    config 2's 300M rows against 0.145 with 128; a plan of more probes runs
    as parts of 256 anyway)."""
    T = Table.of(table)
    out = []
    for i in range(0, len(preds), chunk):
        part = list(preds[i:i + chunk])
        out += BatchPlan(ctx, part, [T] * len(part), autotune=False).run()
    return out


def evaluate_and_push_down(ctx: "Context", relations, min_table_size: int = 0, max_selectivity: float = 0.0,
                           max_rows: int = 0, rowids: bool = True):
    """Algorithm 1 EvaluateAndPushDown over relations given as (table, predicate
    or None, projected columns).  Returns one dict per relation: decision,
    count, max_size, and for pushed relations the projected columns and row ids
    (device tensors truncated to the count)."""
    n = len(relations)
    tabs = [Table.of(t) for t, _, _ in relations]
    rels = (sel_spd_relation * max(1, n))()
    keep = []
    outs = []
    for i, ((_, pred, proj), T) in enumerate(zip(relations, tabs)):
        size = T.n_rows
        cap = max_rows if max_rows else int(math.floor(size * max_selectivity))
        dev = T.columns[0].data.device if T.columns else torch.device("cuda")
        cols = [torch.empty(max(cap, 1), dtype=TORCH_TYPES[T.types[c]], device=dev) for c in proj]
        ids = torch.empty(max(cap, 1), dtype=torch.int64, device=dev) if rowids else None
        pc = (C.c_int32 * max(1, len(proj)))(*proj)
        po = (C.c_void_p * max(1, len(proj)))(*[t.data_ptr() for t in cols])
        keep += [pc, po, T]
        outs.append((cols, ids))
        rels[i].table = C.pointer(T.desc)
        rels[i].pred = pred.h if pred is not None else None
        rels[i].proj_cols = pc
        rels[i].n_proj = len(proj)
        rels[i].dev_out_cols = po
        rels[i].dev_out_rowids = ids.data_ptr() if ids is not None else None
    cfg = sel_spd_cfg(int(min_table_size), float(max_selectivity), int(max_rows))
    dec = (C.c_int32 * max(1, n))()
    cnt = (C.c_uint64 * max(1, n))()
    msz = (C.c_uint64 * max(1, n))()
    _check(lib.sel_evaluate_and_push_down(ctx.h, rels, n, C.byref(cfg), dec, cnt, msz), "sel_evaluate_and_push_down")
    res = []
    for i in range(n):
        d = {"decision": SPD_NAMES[dec[i]], "count": int(cnt[i]), "max_size": int(msz[i])}
        if dec[i] == SPD_PUSHED:
            cols, ids = outs[i]
            d["columns"] = [c[:d["count"]] for c in cols]
            d["rowids"] = ids[:d["count"]] if ids is not None else None
        res.append(d)
    return res


def debug_fail_allocation(nth: int):
    """sel_debug_fail_allocation: the nth library allocation from now on fails (0 disarms)."""
    _check(lib.sel_debug_fail_allocation(int(nth)), "sel_debug_fail_allocation")


def debug_bucket_count_host(preds: Sequence[Predicate], table, with_quads: bool = False):
    """sel_debug_bucket_count_host: (counts, blocks) of the column-bucket form
    evaluated on the CPU, plus the number of quads when ``with_quads`` (0: the
    block form); ``table`` holds CPU tensors."""
    table = Table.of(table)
    n = len(preds)
    pa = (C.c_void_p * n)(*[p.h.value for p in preds])
    out = (C.c_uint64 * n)()
    nb, nq = C.c_int32(), C.c_int32()
    _check(lib.sel_debug_bucket_count_host(pa, n, table.ref(), out, C.byref(nb), C.byref(nq)),
           "sel_debug_bucket_count_host")
    if with_quads:
        return [int(x) for x in out], int(nb.value), int(nq.value)
    return [int(x) for x in out], int(nb.value)


def choose_tau(sigma, est, exact, max_q: float = 2.0, quantile: float = 95.0):
    """sel_mlp_choose_tau: (tau, answered fraction) chosen on held-out predicates."""
    sg = np.ascontiguousarray(np.asarray(sigma, np.float32))
    es = np.ascontiguousarray(np.asarray(est, np.float64))
    ex = np.ascontiguousarray(np.asarray(exact, np.uint64))
    n = int(sg.shape[0])
    if es.shape[0] != n or ex.shape[0] != n:
        raise ValueError("sigma, est and exact need the same length")
    tau = C.c_float(0.0)
    ans = C.c_double(0.0)
    _check(lib.sel_mlp_choose_tau(sg.ctypes.data_as(C.POINTER(C.c_float)), es.ctypes.data_as(C.POINTER(C.c_double)),
                                  ex.ctypes.data_as(C.POINTER(C.c_uint64)), n, float(max_q), float(quantile),
                                  C.byref(tau), C.byref(ans)), "sel_mlp_choose_tau")
    return float(tau.value), float(ans.value)


def join_size_estimate(rows_r: int, rows_s: int, distinct_r: int, distinct_s: int) -> float:
    """|R join S| = |R||S| / max(V(R,A), V(S,A)) (sel_join_size_estimate)."""
    return float(lib.sel_join_size_estimate(int(rows_r), int(rows_s), int(distinct_r), int(distinct_s)))
