"""CPU oracle for the concrete-instance race check (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never does, and this package imports nothing from it.

The oracle is a plain single-threaded C++ program (``oracle.cpp``) that
enumerates every access instance with nested loops, sorts the instance tuples
with ``std::sort`` and applies the race predicate cell by cell; see the header
of ``oracle.cpp`` for the definitions and the passages of the paper they follow.
This module writes a :class:`workloads.spec.Model` in the oracle's own text
format and calls the compiled library through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

FIELDS = [
    "status", "verdict", "racy_cells", "instances", "distinct",
    "w_array", "w_scope", "w_addr",
    "x_block", "x_thread", "x_phase", "x_kind",
    "y_block", "y_thread", "y_phase", "y_kind",
    "oob_stmt", "oob_access", "oob_gtid", "oob_dim",
    "x_wphase", "y_wphase",
]
STATUS_OK, STATUS_INVALID, STATUS_OOB = 0, 1, 3


def build(force: bool = False) -> str:
    """Compile ``oracle.cpp`` into ``oracle/_build/liboracle.so`` (host code, -O2)."""
    src = os.path.join(_HERE, "oracle.cpp")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, src], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            p64 = ctypes.POINTER(ctypes.c_int64)
            lib.oracle_check.argtypes = [ctypes.c_char_p, p64]
            lib.oracle_check.restype = ctypes.c_int
            lib.oracle_check_cells.argtypes = [ctypes.c_char_p, ctypes.c_int64, ctypes.c_int64, p64]
            lib.oracle_check_cells.restype = ctypes.c_int
            lib.oracle_check_part.argtypes = [ctypes.c_char_p, ctypes.c_int64, ctypes.c_int64, p64]
            lib.oracle_check_part.restype = ctypes.c_int
            lib.oracle_check_parallel.argtypes = [ctypes.c_char_p, ctypes.c_int, p64]
            lib.oracle_check_parallel.restype = ctypes.c_int
            lib.oracle_cell_count.argtypes = [ctypes.c_char_p]
            lib.oracle_cell_count.restype = ctypes.c_int64
            lib.oracle_brute.argtypes = [ctypes.c_char_p, p64]
            lib.oracle_brute.restype = ctypes.c_int
            lib.oracle_expand.argtypes = [ctypes.c_char_p, p64, ctypes.c_int64]
            lib.oracle_expand.restype = ctypes.c_int64
            lib.oracle_result_fields.restype = ctypes.c_int
            assert lib.oracle_result_fields() == len(FIELDS)
            _lib = lib
    return _lib


# ---------------------------------------------------------------------------
# text format
# ---------------------------------------------------------------------------

def _expr_text(e) -> str:
    op, a = e.op, e.args
    if op == "const":
        return str(int(a[0]))
    if op == "tid":
        return "t" + "xyz"[a[0]]
    if op == "bid":
        return "b" + "xyz"[a[0]]
    if op == "param":
        return f"p{a[0]}"
    if op == "iter":
        return f"i{a[0]}"
    if op == "add":
        return f"( + {_expr_text(a[0])} {_expr_text(a[1])} )"
    if op == "mul":
        return f"( * {int(a[0])} {_expr_text(a[1])} )"
    if op == "fdiv":
        return f"( / {_expr_text(a[0])} {int(a[1])} )"
    if op == "mod":
        return f"( % {_expr_text(a[0])} {int(a[1])} )"
    if op == "load":
        return f"( L {int(a[0])} {_expr_text(a[1])} )"
    raise ValueError(op)


def model_text(m) -> str:
    """The oracle's own text description of a model."""
    out = ["rcmodel 1",
           "grid %d %d %d" % tuple(m.grid),
           "block %d %d %d" % tuple(m.block),
           "params %d %s" % (len(m.params), " ".join(str(int(p)) for p in m.params)),
           "phases %d" % m.n_phases,
           "wphases %d" % getattr(m, "n_warp_phases", 1)]
    gp = list(getattr(m, "grid_phase", None) or [])
    out.append("gridphase %d %s" % (len(gp), " ".join(str(int(g)) for g in gp)))
    tables = list(getattr(m, "tables", None) or [])
    free = dict(getattr(m, "superset", None) or {})
    n_tab = max([len(tables)] + [int(t) + 1 for t in free])
    out.append("tables %d" % n_tab)
    for i in range(n_tab):
        if i in free:
            out.append("free %d %d" % (int(free[i][0]), int(free[i][1])))
        else:
            t = tables[i] if i < len(tables) else []
            out.append("%d %s" % (len(t), " ".join(str(int(v)) for v in t)))
    out.append("arrays %d" % len(m.arrays))
    for a in m.arrays:
        out.append("%s %d %s" % ("S" if a.scope == "shared" else "G", len(a.extents),
                                 " ".join(str(e) for e in a.extents)))
    out.append("stmts %d" % len(m.stmts))
    for s in m.stmts:
        out.append("stmt")
        out.append("phase " + _expr_text(s.phase))
        wp = getattr(s, "warp_phase", None)
        out.append("wphase " + (_expr_text(wp) if wp is not None else "0"))
        out.append("loops %d" % len(s.loops))
        for lp in s.loops:
            out.append("%s %s %d" % (_expr_text(lp.lower), _expr_text(lp.upper), lp.step))
        out.append("guards %d" % len(s.guards))
        for g in s.guards:
            out.append(_expr_text(g))
        out.append("accesses %d" % len(s.accesses))
        for ac in s.accesses:
            out.append("%s %d %d %s" % (ac.kind, ac.array, len(ac.index),
                                         " ".join(_expr_text(e) for e in ac.index)))
    out.append("end")
    return "\n".join(out) + "\n"


@dataclass
class OracleResult:
    status: int
    verdict: int
    racy_cells: int
    instances: int
    distinct: int
    w_array: int
    w_scope: int
    w_addr: int
    x_block: int
    x_thread: int
    x_phase: int
    x_kind: int
    y_block: int
    y_thread: int
    y_phase: int
    y_kind: int
    oob_stmt: int
    oob_access: int
    oob_gtid: int
    oob_dim: int
    x_wphase: int
    y_wphase: int

    @property
    def witness(self):
        """(array, scope instance, element, x=(b, p, t, k), y=(b, p, t, k)) or None."""
        if not self.verdict:
            return None
        return (self.w_array, self.w_scope, self.w_addr,
                (self.x_block, self.x_phase, self.x_thread, self.x_kind),
                (self.y_block, self.y_phase, self.y_thread, self.y_kind))


def _result(buf) -> OracleResult:
    return OracleResult(*[int(v) for v in buf])


def check(m) -> OracleResult:
    """Full oracle check of a model."""
    lib = _load()
    buf = (ctypes.c_int64 * len(FIELDS))()
    lib.oracle_check(model_text(m).encode(), buf)
    return _result(buf)


def check_text(text: str) -> OracleResult:
    lib = _load()
    buf = (ctypes.c_int64 * len(FIELDS))()
    lib.oracle_check(text.encode(), buf)
    return _result(buf)


def check_cells(m, lo: int, hi: int) -> OracleResult:
    """Oracle check restricted to the linear cells [lo, hi)."""
    lib = _load()
    buf = (ctypes.c_int64 * len(FIELDS))()
    lib.oracle_check_cells(model_text(m).encode(), int(lo), int(hi), buf)
    return _result(buf)


def check_part(m, part_count: int, part_index: int) -> OracleResult:
    """Oracle check restricted to the cells of one hash part (the check
    options' part_count, a power of two, and part_index)."""
    lib = _load()
    buf = (ctypes.c_int64 * len(FIELDS))()
    lib.oracle_check_part(model_text(m).encode(), int(part_count), int(part_index), buf)
    return _result(buf)


def check_parallel(m, n_threads: Optional[int] = None) -> OracleResult:
    """The full check on ``n_threads`` host threads (default: every core):
    equal cell ranges checked concurrently and merged (counts add up, the
    lowest racy range gives the witness)."""
    n = int(n_threads or os.cpu_count() or 1)
    buf = (ctypes.c_int64 * len(FIELDS))()
    _load().oracle_check_parallel(model_text(m).encode(), n, buf)
    return _result(buf)


def cell_count(m) -> int:
    return int(_load().oracle_cell_count(model_text(m).encode()))


def brute(m) -> OracleResult:
    """O(n^2) pairwise check of a small model."""
    lib = _load()
    buf = (ctypes.c_int64 * len(FIELDS))()
    lib.oracle_brute(model_text(m).encode(), buf)
    return _result(buf)


def expand(m, cap: Optional[int] = None) -> np.ndarray:
    """All in-bounds instances as an (n, 7) int64 array of (a, s, e, b, p, t, k),
    sorted, duplicates kept."""
    lib = _load()
    text = model_text(m).encode()
    if cap is None:
        n = lib.oracle_expand(text, (ctypes.c_int64 * 7)(), 0)
        if n < 0:
            raise ValueError("invalid model")
        cap = n
    out = np.zeros((max(cap, 1), 7), dtype=np.int64)
    n = lib.oracle_expand(text, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cap)
    if n < 0:
        raise ValueError("invalid model")
    return out[:min(n, cap)]
