"""Host model of a compiled device program, for CPU tests of the compiler.

Parses the text of ``sel_pred_describe`` and evaluates the postfix program
row by row with the same per-opcode arithmetic the scan kernels use (32/64-bit
wrap-around range tests, binary32 compares, bitmaps, multiply-shift hash
tables).  It models the
library's program format, not the paper: the tests compare its results with
the oracle, so a compiler bug (a wrong bound, a lost negation, a misplaced
operand) shows up without a GPU.
"""
from __future__ import annotations

import re
from typing import List

import numpy as np


def parse(text: str):
    lines = text.strip().splitlines()
    slots = [tuple(int(x) for x in s.split("/")) for s in lines[0].split(":")[1].split()]
    prog = []
    for ln in lines[3:]:
        parts = ln.split()
        op = parts[0]
        kv = dict(p.split("=", 1) for p in parts[1:] if "=" in p)
        # "+AND" / "+OR": the mask is combined into the top instead of pushed
        kv["comb"] = "AND" if "+AND" in parts[1:] else "OR" if "+OR" in parts[1:] else ""
        prog.append((op, kv))
    return slots, prog


def _u32(x):
    return np.asarray(x).astype(np.int64) & 0xFFFFFFFF


def _leaf_mask(op: str, kv: dict, col: np.ndarray) -> np.ndarray:
    n = col.shape[0]
    if op == "CONST":
        m = np.ones(n, bool)
    elif op == "RANGE32":
        lo, sp = int(kv["lo"]), int(kv["span"])
        m = ((col.astype(np.int64) - lo) & 0xFFFFFFFF) <= sp
    elif op == "RANGE64":
        lo, sp = int(kv["lo"]), int(kv["span"])
        d = (col.astype(np.int64).view(np.uint64) - np.uint64(lo & 0xFFFFFFFFFFFFFFFF))
        m = d <= np.uint64(sp)
    elif op == "RANGEF":
        a, b = (int(x, 16) for x in kv["bits"].split(","))
        lo = np.array([a], np.uint32).view(np.float32)[0]
        hi = np.array([b], np.uint32).view(np.float32)[0]
        m = (lo <= col) & (col <= hi)
    elif op in ("IN32", "IN64"):
        vals = [int(v) for v in kv["vals"].split(",")] if kv.get("vals") else []
        m = np.isin(col.astype(np.int64), np.array(vals, np.int64))
    elif op == "INF":
        vals = np.array([int(v, 16) for v in kv["vals"].split(",")], np.uint32).view(np.float32)
        m = np.zeros(n, bool)
        for v in vals:
            m |= col == v
    elif op == "BITMAP":
        lo, nb = int(kv["lo"]), int(kv["nbits"])
        words = np.array([int(w, 16) for w in kv["words"].split(",")], np.uint64)
        d = (col.astype(np.int64) - lo) & 0xFFFFFFFF
        inside = d < nb
        dd = np.where(inside, d, 0)
        m = inside & (((words[dd >> 5] >> (dd & 31).astype(np.uint64)) & np.uint64(1)) == 1)
    elif op == "MASK32":
        lo, word = int(kv["lo"]), int(kv["word"], 16)
        d = (col.astype(np.int64) - lo) & 0xFFFFFFFF
        dd = np.where(d < 32, d, 0)
        m = (d < 32) & (((word >> dd) & 1) == 1)
    elif op in ("HASH32", "HASH64"):
        mult, sh = int(kv["mult"], 16), int(kv["shift"])
        table = np.array([int(v) for v in kv["table"].split(",")], np.int64)
        x = col.astype(np.int64)
        u = x.view(np.uint64) if op == "HASH64" else (x & 0xFFFFFFFF).astype(np.uint64)
        key = (u & np.uint64(0xFFFFFFFF)) ^ ((u >> np.uint64(32)) if op == "HASH64" else np.uint64(0))
        h = ((key * np.uint64(mult)) & np.uint64(0xFFFFFFFF)) >> np.uint64(sh)
        m = table[h.astype(np.int64)] == x
    else:
        raise ValueError(op)
    if kv.get("neg") == "1":
        m = ~m
    return m


def evaluate(text: str, arrays: List[np.ndarray], n_rows: int) -> np.ndarray:
    slots, prog = parse(text)
    stack = []
    memo = {}
    for op, kv in prog:
        if op == "SAVE":
            memo[kv["m"]] = stack[-1]
            continue
        if op in ("AND", "OR"):
            b, a = stack.pop(), stack.pop()
            stack.append(a & b if op == "AND" else a | b)
            continue
        if op == "LOAD":
            v = memo[kv["m"]]
        else:
            col = arrays[slots[int(kv["slot"])][0]] if op != "CONST" else np.zeros(n_rows)
            v = _leaf_mask(op, kv, col)
        if kv["comb"]:
            a = stack.pop()
            stack.append(a & v if kv["comb"] == "AND" else a | v)
        else:
            stack.append(v)
    assert len(stack) == 1
    return stack[0]


def need(text: str) -> int:
    return int(re.search(r"need: (\d+)", text).group(1))
