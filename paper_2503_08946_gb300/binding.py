"""ctypes binding of the race-checker C ABI (include/rc.h).

Argument marshalling only: every step of the check runs in the CUDA library
``_build/librc.so``.  There is no fallback: if the library is missing or cannot
be loaded, :func:`load` raises.  PyTorch supplies device memory (the workspace
is a ``torch.uint8`` CUDA tensor) and streams.

Functions carry the C names: :func:`rc_model_create`, :func:`rc_model_destroy`,
:func:`rc_model_layout`, :func:`rc_workspace_size`, :func:`rc_check`,
:func:`rc_batch_workspace_size`, :func:`rc_check_batch`, :func:`rc_report`,
:func:`rc_expand_keys`, :func:`rc_sort_workspace_size`, :func:`rc_sort_keys`,
:func:`rc_status_str`, :func:`rc_get_limits`.
"""
from __future__ import annotations

import ctypes
import os
import threading
from ctypes import (POINTER, Structure, c_char_p, c_int, c_int32, c_int64, c_size_t, c_uint32,
                    c_uint64, c_void_p)
from dataclasses import dataclass
from typing import List, Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librc.so")

# status codes (rc_status)
RC_OK, RC_E_INVALID, RC_E_KEY_OVERFLOW, RC_E_OOB, RC_E_NOMEM, RC_E_TIMEOUT, RC_E_CUDA, \
    RC_E_NOT_READY, RC_E_UNSUPPORTED = range(9)
STATUS_NAMES = {RC_OK: "RC_OK", RC_E_INVALID: "RC_E_INVALID", RC_E_KEY_OVERFLOW: "RC_E_KEY_OVERFLOW",
                RC_E_OOB: "RC_E_OOB", RC_E_NOMEM: "RC_E_NOMEM", RC_E_TIMEOUT: "RC_E_TIMEOUT",
                RC_E_CUDA: "RC_E_CUDA", RC_E_NOT_READY: "RC_E_NOT_READY",
                RC_E_UNSUPPORTED: "RC_E_UNSUPPORTED"}
RC_OP_CONST, RC_OP_TID, RC_OP_BID, RC_OP_PARAM, RC_OP_ITER, RC_OP_ADD, RC_OP_MUL, RC_OP_FDIV, \
    RC_OP_MOD, RC_OP_LOAD = range(10)
RC_SCOPE_GLOBAL, RC_SCOPE_SHARED = 0, 1
RC_READ, RC_WRITE, RC_ATOMIC = 0, 1, 2
RC_PATH_AUTO, RC_PATH_SORT, RC_PATH_HASH = 0, 1, 2
RC_TEST_STALL_LOOKBACK = 1
RC_TEST_FEW_SCAN_WARPS = 2
RC_OPT_STAGE_TIMES = 1
RC_OPT_GRAPH = 2
RC_OPT_CHUNKED = 4
RC_OPT_LSD = 8

# every entry point declared in include/rc.h
EXPORTS = ["rc_status_str", "rc_get_limits", "rc_model_create", "rc_model_destroy", "rc_model_layout",
           "rc_workspace_size", "rc_check", "rc_batch_workspace_size", "rc_check_batch", "rc_report",
           "rc_expand_keys", "rc_sort_workspace_size", "rc_sort_keys", "rc_ticket_stage_times",
           "rc_sort_keys_static", "rc_sort_status", "rc_kernel_source", "rc_tune", "rc_server_create",
           "rc_server_submit", "rc_server_poll", "rc_server_stats", "rc_server_destroy"]
RC_SORT_STATIC_MAX_KEYS = 1 << 20


class RcError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)}")


# ---------------------------------------------------------------------------
# C structures
# ---------------------------------------------------------------------------
class rc_insn(Structure):
    _fields_ = [("op", c_int32), ("arg", c_int32), ("imm", c_int64)]


class rc_expr(Structure):
    _fields_ = [("code", POINTER(rc_insn)), ("len", c_uint32)]


class rc_loop(Structure):
    _fields_ = [("lower", rc_expr), ("upper", rc_expr), ("step", c_int64)]


class rc_access(Structure):
    _fields_ = [("array", c_uint32), ("kind", c_uint32), ("index", POINTER(rc_expr))]


class rc_stmt(Structure):
    _fields_ = [("phase", rc_expr),
                ("loops", POINTER(rc_loop)), ("n_loops", c_uint32),
                ("guards", POINTER(rc_expr)), ("n_guards", c_uint32),
                ("accesses", POINTER(rc_access)), ("n_accesses", c_uint32),
                ("warp_phase", rc_expr)]


class rc_array(Structure):
    _fields_ = [("name", c_char_p), ("scope", c_uint32), ("ndims", c_uint32), ("extent", c_int64 * 4)]


class rc_table(Structure):
    _fields_ = [("data", POINTER(c_int64)), ("len", c_uint64), ("superset", c_uint32), ("lo", c_int64),
                ("hi", c_int64)]


class rc_model_desc(Structure):
    _fields_ = [("grid", c_uint32 * 3), ("block", c_uint32 * 3),
                ("params", POINTER(c_int64)), ("n_params", c_uint32),
                ("n_phases", c_uint32),
                ("arrays", POINTER(rc_array)), ("n_arrays", c_uint32),
                ("stmts", POINTER(rc_stmt)), ("n_stmts", c_uint32),
                ("tables", POINTER(rc_table)), ("n_tables", c_uint32),
                ("n_warp_phases", c_uint32), ("grid_phase", POINTER(c_uint32))]


class rc_limits(Structure):
    _fields_ = [("max_loops", c_uint32), ("max_terms", c_uint32), ("max_stmts", c_uint32),
                ("max_accesses", c_uint32), ("max_phase_bits", c_uint32), ("key_bits", c_uint32)]


class rc_layout(Structure):
    _fields_ = [("kind_shift", c_uint32), ("thread_shift", c_uint32), ("block_shift", c_uint32),
                ("phase_shift", c_uint32), ("cell_shift", c_uint32),
                ("thread_bits", c_uint32), ("block_bits", c_uint32), ("phase_bits", c_uint32),
                ("cell_bits", c_uint32), ("sort_lo", c_uint32), ("sort_hi", c_uint32),
                ("key_slots", c_uint64), ("total_cells", c_uint64), ("n_arrays", c_uint32),
                ("n_threads_per_block", c_uint32), ("n_blocks", c_uint64),
                ("program_bytes", c_uint64), ("expand_jit", c_uint32), ("wide", c_uint32), ("array_base", c_uint64 * 64), ("array_cells", c_uint64 * 64)]


class rc_check_opts(Structure):
    _fields_ = [("path", c_uint32), ("digit_bits", c_uint32), ("early_exit", c_uint32),
                ("test_flags", c_uint32), ("flags", c_uint32), ("reserved", c_uint32),
                ("spin_limit", c_uint64), ("cell_lo", c_uint64), ("cell_hi", c_uint64),
                ("part_count", c_uint32), ("part_index", c_uint32)]


class rc_stage_times(Structure):
    _fields_ = [("expand_ms", ctypes.c_float), ("histogram_ms", ctypes.c_float),
                ("sort_ms", ctypes.c_float * 16), ("n_sort_passes", c_uint32), ("scan_ms", ctypes.c_float),
                ("witness_ms", ctypes.c_float), ("total_ms", ctypes.c_float), ("n_keys", c_uint64),
                ("histogram2_ms", ctypes.c_float), ("bucketed", c_uint32), ("histogram_fused", c_uint32)]


class rc_inst(Structure):
    _fields_ = [("block", c_uint64), ("thread", c_uint32), ("kind", c_uint32), ("phase", c_int64),
                ("gtid", c_uint64), ("warp_phase", c_uint32), ("reserved", c_uint32)]


class rc_result(Structure):
    _fields_ = [("status", c_int32), ("verdict", c_int32), ("racy_cells", c_uint64),
                ("instances", c_uint64), ("w_array", c_uint32), ("w_reserved", c_uint32),
                ("w_scope", c_uint64), ("w_addr", c_uint64), ("x", rc_inst), ("y", rc_inst),
                ("oob_stmt", c_uint32), ("oob_access", c_uint32), ("oob_gtid", c_uint64),
                ("oob_dim", c_int32), ("reserved2", c_int32)]


class rc_server_opts(Structure):
    _fields_ = [("memory_bytes", c_uint64), ("slots", c_uint32), ("max_batch", c_uint32),
                ("digit_bits", c_uint32), ("reserved", c_uint32)]


class rc_server_done(Structure):
    _fields_ = [("request", c_uint64), ("result", rc_result), ("submit_s", ctypes.c_double),
                ("start_s", ctypes.c_double), ("done_s", ctypes.c_double), ("batch_size", c_uint32),
                ("pad", c_uint32)]


# ---------------------------------------------------------------------------
# library loading (no fallback)
# ---------------------------------------------------------------------------
_lib = None
_lock = threading.Lock()


def load():
    """Load ``_build/librc.so``; raise if it is missing (build it with
    ``paper_2503_08946_gb300.build.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"race-checker CUDA library not built: {LIB_PATH} is missing")
        lib = ctypes.CDLL(LIB_PATH)
        lib.rc_status_str.argtypes = [c_int]
        lib.rc_status_str.restype = c_char_p
        lib.rc_get_limits.argtypes = [POINTER(rc_limits)]
        lib.rc_get_limits.restype = None
        lib.rc_model_create.argtypes = [POINTER(rc_model_desc), POINTER(c_void_p)]
        lib.rc_model_create.restype = c_int
        lib.rc_model_destroy.argtypes = [c_void_p]
        lib.rc_model_destroy.restype = None
        lib.rc_model_layout.argtypes = [c_void_p, POINTER(rc_layout)]
        lib.rc_model_layout.restype = c_int
        lib.rc_workspace_size.argtypes = [c_void_p, POINTER(rc_check_opts), POINTER(c_size_t)]
        lib.rc_workspace_size.restype = c_int
        lib.rc_check.argtypes = [c_void_p, POINTER(rc_check_opts), c_void_p, c_size_t, c_void_p,
                                 POINTER(c_void_p)]
        lib.rc_check.restype = c_int
        lib.rc_batch_workspace_size.argtypes = [POINTER(c_void_p), c_size_t, POINTER(rc_check_opts),
                                                POINTER(c_size_t)]
        lib.rc_batch_workspace_size.restype = c_int
        lib.rc_check_batch.argtypes = [POINTER(c_void_p), c_size_t, POINTER(rc_check_opts), c_void_p,
                                       c_size_t, c_void_p, POINTER(c_void_p)]
        lib.rc_check_batch.restype = c_int
        lib.rc_tune.argtypes = [POINTER(c_void_p), c_size_t, POINTER(rc_check_opts), c_void_p, c_size_t,
                                c_void_p, POINTER(rc_check_opts)]
        lib.rc_tune.restype = c_int
        lib.rc_server_create.argtypes = [POINTER(rc_server_opts), POINTER(c_void_p)]
        lib.rc_server_create.restype = c_int
        lib.rc_server_submit.argtypes = [c_void_p, c_void_p, POINTER(c_uint64)]
        lib.rc_server_submit.restype = c_int
        lib.rc_server_poll.argtypes = [c_void_p, POINTER(rc_server_done), c_size_t, POINTER(c_size_t), c_int]
        lib.rc_server_poll.restype = c_int
        lib.rc_server_stats.argtypes = [c_void_p, POINTER(c_uint64), POINTER(c_uint64)]
        lib.rc_server_stats.restype = c_int
        lib.rc_server_destroy.argtypes = [c_void_p]
        lib.rc_server_destroy.restype = c_int
        lib.rc_report.argtypes = [c_void_p, POINTER(rc_result), c_int]
        lib.rc_report.restype = c_int
        lib.rc_expand_keys.argtypes = [c_void_p, c_void_p, c_size_t, c_void_p, c_void_p, c_void_p]
        lib.rc_expand_keys.restype = c_int
        lib.rc_sort_workspace_size.argtypes = [c_uint64, c_uint32, POINTER(c_size_t)]
        lib.rc_sort_workspace_size.restype = c_int
        lib.rc_sort_keys.argtypes = [c_void_p, c_void_p, c_uint64, c_uint32, c_uint32, c_uint32, c_void_p,
                                     c_size_t, c_void_p]
        lib.rc_sort_keys.restype = c_int
        lib.rc_kernel_source.argtypes = [POINTER(rc_model_desc), ctypes.c_char_p, c_size_t, POINTER(c_size_t)]
        lib.rc_kernel_source.restype = c_int
        lib.rc_sort_keys_static.argtypes = [c_void_p, c_void_p, c_uint64, c_uint32, c_uint32, c_uint32, c_void_p]
        lib.rc_sort_keys_static.restype = c_int
        lib.rc_sort_status.argtypes = [c_void_p, c_void_p]
        lib.rc_sort_status.restype = c_int
        lib.rc_ticket_stage_times.argtypes = [c_void_p, POINTER(rc_stage_times)]
        lib.rc_ticket_stage_times.restype = c_int
        _lib = lib
        return lib


def rc_status_str(s: int) -> str:
    return load().rc_status_str(int(s)).decode()


def rc_get_limits() -> dict:
    lim = rc_limits()
    load().rc_get_limits(ctypes.byref(lim))
    return {f: getattr(lim, f) for f, _ in rc_limits._fields_}


# ---------------------------------------------------------------------------
# marshalling of workloads.spec.Model into rc_model_desc
# ---------------------------------------------------------------------------
_OPS = {"const": RC_OP_CONST, "tid": RC_OP_TID, "bid": RC_OP_BID, "param": RC_OP_PARAM,
        "iter": RC_OP_ITER}


def _postfix(e, out: list):
    op, a = e.op, e.args
    if op == "const":
        out.append((RC_OP_CONST, 0, int(a[0])))
    elif op in ("tid", "bid", "param", "iter"):
        out.append((_OPS[op], int(a[0]), 0))
    elif op == "add":
        _postfix(a[0], out)
        _postfix(a[1], out)
        out.append((RC_OP_ADD, 0, 0))
    elif op == "mul":
        _postfix(a[1], out)
        out.append((RC_OP_MUL, 0, int(a[0])))
    elif op == "fdiv":
        _postfix(a[0], out)
        out.append((RC_OP_FDIV, 0, int(a[1])))
    elif op == "mod":
        _postfix(a[0], out)
        out.append((RC_OP_MOD, 0, int(a[1])))
    elif op == "load":
        _postfix(a[1], out)
        out.append((RC_OP_LOAD, int(a[0]), 0))
    else:
        raise ValueError(f"unknown expression node {op}")


class _Desc:
    """Owns the ctypes arrays behind one rc_model_desc."""

    def __init__(self, model):
        self.keep = []
        d = rc_model_desc()
        for i in range(3):
            d.grid[i] = int(model.grid[i])
            d.block[i] = int(model.block[i])
        if model.params:
            pa = (c_int64 * len(model.params))(*[int(p) for p in model.params])
            self.keep.append(pa)
            d.params = ctypes.cast(pa, POINTER(c_int64))
        d.n_params = len(model.params)
        d.n_phases = int(model.n_phases)
        arrs = (rc_array * max(1, len(model.arrays)))()
        for i, a in enumerate(model.arrays):
            nm = a.name.encode()
            self.keep.append(nm)
            arrs[i].name = nm
            arrs[i].scope = RC_SCOPE_SHARED if a.scope == "shared" else RC_SCOPE_GLOBAL
            arrs[i].ndims = len(a.extents)
            for k, e in enumerate(a.extents[:4]):
                arrs[i].extent[k] = int(e)
        self.keep.append(arrs)
        d.arrays = arrs
        d.n_arrays = len(model.arrays)
        stmts = (rc_stmt * max(1, len(model.stmts)))()
        for i, s in enumerate(model.stmts):
            st = stmts[i]
            st.phase = self.expr(s.phase)
            loops = (rc_loop * max(1, len(s.loops)))()
            for l, lp in enumerate(s.loops):
                loops[l].lower = self.expr(lp.lower)
                loops[l].upper = self.expr(lp.upper)
                loops[l].step = int(lp.step)
            self.keep.append(loops)
            st.loops = loops
            st.n_loops = len(s.loops)
            guards = (rc_expr * max(1, len(s.guards)))()
            for g, ge in enumerate(s.guards):
                guards[g] = self.expr(ge)
            self.keep.append(guards)
            st.guards = guards
            st.n_guards = len(s.guards)
            accs = (rc_access * max(1, len(s.accesses)))()
            for k, ac in enumerate(s.accesses):
                idx = (rc_expr * max(1, len(ac.index)))()
                for j, ie in enumerate(ac.index):
                    idx[j] = self.expr(ie)
                self.keep.append(idx)
                accs[k].array = int(ac.array)
                accs[k].kind = {"W": RC_WRITE, "A": RC_ATOMIC}.get(ac.kind, RC_READ)
                accs[k].index = idx
            self.keep.append(accs)
            st.accesses = accs
            st.n_accesses = len(s.accesses)
            wp = getattr(s, "warp_phase", None)
            if wp is not None and not (wp.op == "const" and wp.args[0] == 0):
                st.warp_phase = self.expr(wp)
        self.keep.append(stmts)
        d.stmts = stmts
        d.n_stmts = len(model.stmts)
        tables = list(getattr(model, "tables", None) or [])
        superset = dict(getattr(model, "superset", None) or {})
        n_tab = max([len(tables)] + [int(t) + 1 for t in superset])
        if n_tab:
            tabs = (rc_table * n_tab)()
            for i in range(n_tab):
                t = tables[i] if i < len(tables) else []
                data = (c_int64 * max(1, len(t)))(*[int(v) for v in t])
                self.keep.append(data)
                tabs[i].data = ctypes.cast(data, POINTER(c_int64))
                tabs[i].len = len(t)
                if i in superset:
                    tabs[i].superset = 1
                    tabs[i].lo, tabs[i].hi = (int(v) for v in superset[i])
            self.keep.append(tabs)
            d.tables = tabs
        d.n_tables = n_tab
        d.n_warp_phases = int(getattr(model, "n_warp_phases", 1))
        gp = list(getattr(model, "grid_phase", None) or [])
        if gp:
            ga = (c_uint32 * len(gp))(*[int(v) for v in gp])
            self.keep.append(ga)
            d.grid_phase = ctypes.cast(ga, POINTER(c_uint32))
        self.desc = d

    def expr(self, e) -> rc_expr:
        code = []
        _postfix(e, code)
        arr = (rc_insn * len(code))(*[rc_insn(o, a, i) for o, a, i in code])
        self.keep.append(arr)
        x = rc_expr()
        x.code = arr
        x.len = len(code)
        return x


def _opts(opts) -> Optional[rc_check_opts]:
    if opts is None:
        return None
    if isinstance(opts, rc_check_opts):
        return opts
    o = rc_check_opts()
    for k, v in dict(opts).items():
        setattr(o, k, int(v))
    return o


def _ptr(x) -> int:
    """Device address of a torch tensor, or an int address."""
    if x is None:
        return 0
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    return int(x)


def _stream(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


# ---------------------------------------------------------------------------
# entry points
# ---------------------------------------------------------------------------
class RcModel:
    """Owning handle of an rc_model; destroyed with the object."""

    def __init__(self, ptr: int, name: str = ""):
        self.ptr = ptr
        self.name = name

    def close(self):
        if self.ptr:
            load().rc_model_destroy(c_void_p(self.ptr))
            self.ptr = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rc_model_create(model) -> RcModel:
    """Lower a :class:`workloads.spec.Model` (or any object with the same
    fields) and upload it to the current CUDA device."""
    lib = load()
    d = _Desc(model)
    out = c_void_p()
    st = lib.rc_model_create(ctypes.byref(d.desc), ctypes.byref(out))
    if st != RC_OK:
        raise RcError(st, "rc_model_create")
    return RcModel(out.value, getattr(model, "name", ""))


def rc_model_create_status(model) -> int:
    """Status of rc_model_create for a model (the model is destroyed again)."""
    lib = load()
    d = _Desc(model)
    out = c_void_p()
    st = lib.rc_model_create(ctypes.byref(d.desc), ctypes.byref(out))
    if st == RC_OK:
        lib.rc_model_destroy(out)
    return st


def rc_model_destroy(m: RcModel):
    m.close()


def rc_kernel_source(model) -> str:
    """Source of the expansion kernel generated for a model (host lowering only)."""
    lib = load()
    d = _Desc(model)
    n = c_size_t()
    st = lib.rc_kernel_source(ctypes.byref(d.desc), None, 0, ctypes.byref(n))
    if st != RC_OK:
        raise RcError(st, "rc_kernel_source")
    buf = ctypes.create_string_buffer(n.value + 1)
    lib.rc_kernel_source(ctypes.byref(d.desc), buf, n.value + 1, ctypes.byref(n))
    return buf.value.decode()


def rc_model_layout(m: RcModel) -> dict:
    lay = rc_layout()
    st = load().rc_model_layout(c_void_p(m.ptr), ctypes.byref(lay))
    if st != RC_OK:
        raise RcError(st, "rc_model_layout")
    d = {f: getattr(lay, f) for f, _ in rc_layout._fields_ if not f.startswith("array_")}
    d["array_base"] = [lay.array_base[i] for i in range(min(64, lay.n_arrays))]
    d["array_cells"] = [lay.array_cells[i] for i in range(min(64, lay.n_arrays))]
    return d


def rc_workspace_size(m: RcModel, opts=None) -> int:
    n = c_size_t()
    o = _opts(opts)
    st = load().rc_workspace_size(c_void_p(m.ptr), ctypes.byref(o) if o else None, ctypes.byref(n))
    if st != RC_OK:
        raise RcError(st, "rc_workspace_size")
    return n.value


def rc_check(m: RcModel, opts, workspace, stream=None):
    """Enqueue a check; returns a ticket (opaque int) for :func:`rc_report`."""
    o = _opts(opts)
    t = c_void_p()
    ws_bytes = workspace.numel() * workspace.element_size() if hasattr(workspace, "numel") else 0
    st = load().rc_check(c_void_p(m.ptr), ctypes.byref(o) if o else None, c_void_p(_ptr(workspace)),
                         c_size_t(ws_bytes), c_void_p(_stream(stream)), ctypes.byref(t))
    if st != RC_OK:
        raise RcError(st, "rc_check")
    return (t.value, 1)


def rc_batch_workspace_size(models: Sequence[RcModel], opts=None) -> int:
    arr = (c_void_p * max(1, len(models)))(*[m.ptr for m in models])
    n = c_size_t()
    o = _opts(opts)
    st = load().rc_batch_workspace_size(arr, len(models), ctypes.byref(o) if o else None, ctypes.byref(n))
    if st != RC_OK:
        raise RcError(st, "rc_batch_workspace_size")
    return n.value


def rc_check_batch(models: Sequence[RcModel], opts, workspace, stream=None):
    arr = (c_void_p * max(1, len(models)))(*[m.ptr for m in models])
    o = _opts(opts)
    t = c_void_p()
    ws_bytes = workspace.numel() * workspace.element_size()
    st = load().rc_check_batch(arr, len(models), ctypes.byref(o) if o else None, c_void_p(_ptr(workspace)),
                               c_size_t(ws_bytes), c_void_p(_stream(stream)), ctypes.byref(t))
    if st != RC_OK:
        raise RcError(st, "rc_check_batch")
    return (t.value, len(models))


def rc_tune(models: Sequence[RcModel], opts, workspace, stream=None) -> dict:
    """Time the candidate configurations for these models, record the fastest
    for their shape class (used by path=RC_PATH_AUTO) and return it."""
    arr = (c_void_p * max(1, len(models)))(*[m.ptr for m in models])
    o = _opts(opts)
    best = rc_check_opts()
    ws_bytes = workspace.numel() * workspace.element_size() if hasattr(workspace, "numel") else 0
    st = load().rc_tune(arr, len(models), ctypes.byref(o) if o else None, c_void_p(_ptr(workspace)),
                        c_size_t(ws_bytes), c_void_p(_stream(stream)), ctypes.byref(best))
    if st != RC_OK:
        raise RcError(st, "rc_tune")
    return {f: getattr(best, f) for f, _ in rc_check_opts._fields_}


@dataclass
class Result:
    status: int
    verdict: int
    racy_cells: int
    instances: int
    w_array: int
    w_scope: int
    w_addr: int
    x: tuple      # (block, phase, thread, kind)
    y: tuple
    oob_stmt: int
    oob_access: int
    oob_gtid: int
    oob_dim: int
    x_wphase: int = 0     # warp phases of the witness pair (models with warp barriers)
    y_wphase: int = 0

    @property
    def witness(self):
        """(array, scope instance, element, x=(b, p, t, k), y=(b, p, t, k)) or None."""
        if not self.verdict:
            return None
        return (self.w_array, self.w_scope, self.w_addr, self.x, self.y)


def _result(r: rc_result) -> Result:
    return Result(r.status, r.verdict, r.racy_cells, r.instances, r.w_array, r.w_scope, r.w_addr,
                  (r.x.block, r.x.phase, r.x.thread, r.x.kind), (r.y.block, r.y.phase, r.y.thread, r.y.kind),
                  r.oob_stmt, r.oob_access, r.oob_gtid, r.oob_dim, r.x.warp_phase, r.y.warp_phase)


class NotReady(Exception):
    pass


@dataclass
class Done:
    request: int
    result: "Result"
    submit_s: float
    start_s: float
    done_s: float
    batch_size: int


class RcServer:
    """Continuous-batching request server (rc_server_* of include/rc.h) on the
    current device.  Models passed to :meth:`submit` must stay alive until
    their results are polled."""

    def __init__(self, memory_bytes: int, slots: int = 4, max_batch: int = 0, digit_bits: int = 0):
        o = rc_server_opts(int(memory_bytes), int(slots), int(max_batch), int(digit_bits), 0)
        h = c_void_p()
        st = load().rc_server_create(ctypes.byref(o), ctypes.byref(h))
        if st != RC_OK:
            raise RcError(st, "rc_server_create")
        self.ptr = h.value
        self._hold = {}

    def submit(self, model: "RcModel") -> int:
        rid = c_uint64()
        st = load().rc_server_submit(c_void_p(self.ptr), c_void_p(model.ptr), ctypes.byref(rid))
        if st != RC_OK:
            raise RcError(st, "rc_server_submit")
        self._hold[rid.value] = model
        return rid.value

    def poll(self, cap: int = 1024, wait_ms: int = 0) -> List[Done]:
        out = (rc_server_done * max(1, cap))()
        n = c_size_t()
        st = load().rc_server_poll(c_void_p(self.ptr), out, cap, ctypes.byref(n), int(wait_ms))
        if st != RC_OK:
            raise RcError(st, "rc_server_poll")
        res = []
        for i in range(n.value):
            d = out[i]
            self._hold.pop(d.request, None)
            res.append(Done(d.request, _result(d.result), d.submit_s, d.start_s, d.done_s, d.batch_size))
        return res

    def stats(self):
        p, f = c_uint64(), c_uint64()
        load().rc_server_stats(c_void_p(self.ptr), ctypes.byref(p), ctypes.byref(f))
        return p.value, f.value

    def close(self):
        if self.ptr:
            st = load().rc_server_destroy(c_void_p(self.ptr))
            self.ptr = None
            self._hold.clear()
            if st != RC_OK:
                raise RcError(st, "rc_server_destroy")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rc_report_array(ticket, wait: bool = True):
    """The results of a ticket as one numpy record array, one record per
    model with the fields of ``rc_result`` (``x``/``y`` are records of the
    fields of ``rc_inst``).  No Python object is made per result: a batch of
    10,000 models decodes in about a millisecond instead of tens."""
    import numpy as np
    t, n = ticket
    out = (rc_result * max(1, n))()
    st = load().rc_report(c_void_p(t), out, 1 if wait else 0)
    if st == RC_E_NOT_READY:
        raise NotReady()
    if st != RC_OK:
        raise RcError(st, "rc_report")
    return np.ctypeslib.as_array(out)[:n]


def results_of(arr) -> List[Result]:
    """``Result`` objects of the records that :func:`rc_report_array` returns."""
    res = []
    for (s, v, rc_, ins, wa, _r, ws, wad, x, y, os_, oa, og, od, _r2) in arr.tolist():
        # rc_inst fields: block, thread, kind, phase, gtid, warp_phase, reserved
        res.append(Result(s, v, rc_, ins, wa, ws, wad, (x[0], x[3], x[1], x[2]), (y[0], y[3], y[1], y[2]),
                          os_, oa, og, od, x[5], y[5]))
    return res


def rc_report(ticket, wait: bool = True) -> List[Result]:
    return results_of(rc_report_array(ticket, wait))


def rc_ticket_stage_times(ticket) -> dict:
    """Per-stage device milliseconds of a check enqueued with RC_OPT_STAGE_TIMES
    (call before rc_report)."""
    t, _ = ticket
    st_ = rc_stage_times()
    st = load().rc_ticket_stage_times(c_void_p(t), ctypes.byref(st_))
    if st != RC_OK:
        raise RcError(st, "rc_ticket_stage_times")
    return {"expand_ms": st_.expand_ms, "histogram_ms": st_.histogram_ms,
            "sort_ms": [st_.sort_ms[i] for i in range(st_.n_sort_passes)], "scan_ms": st_.scan_ms,
            "witness_ms": st_.witness_ms, "total_ms": st_.total_ms, "n_keys": st_.n_keys,
            "histogram2_ms": st_.histogram2_ms, "bucketed": bool(st_.bucketed),
            "histogram_fused": bool(st_.histogram_fused)}


def rc_expand_keys(m: RcModel, workspace, keys, count, stream=None):
    ws_bytes = workspace.numel() * workspace.element_size()
    st = load().rc_expand_keys(c_void_p(m.ptr), c_void_p(_ptr(workspace)), c_size_t(ws_bytes),
                               c_void_p(_ptr(keys)), c_void_p(_ptr(count)), c_void_p(_stream(stream)))
    if st != RC_OK:
        raise RcError(st, "rc_expand_keys")


def rc_sort_workspace_size(n: int, digit_bits: int = 0) -> int:
    b = c_size_t()
    st = load().rc_sort_workspace_size(c_uint64(n), c_uint32(digit_bits), ctypes.byref(b))
    if st != RC_OK:
        raise RcError(st, "rc_sort_workspace_size")
    return b.value


def rc_sort_keys(keys_in, keys_out, n: int, lo_bit: int, hi_bit: int, digit_bits: int, workspace, stream=None):
    ws_bytes = workspace.numel() * workspace.element_size()
    st = load().rc_sort_keys(c_void_p(_ptr(keys_in)), c_void_p(_ptr(keys_out)), c_uint64(n), c_uint32(lo_bit),
                             c_uint32(hi_bit), c_uint32(digit_bits), c_void_p(_ptr(workspace)),
                             c_size_t(ws_bytes), c_void_p(_stream(stream)))
    if st != RC_OK:
        raise RcError(st, "rc_sort_keys")


def rc_sort_keys_static(keys_in, keys_out, n: int, lo_bit: int, hi_bit: int, digit_bits: int, stream=None):
    """rc_sort_keys without a workspace: the scratch is the library's static device
    array (at most RC_SORT_STATIC_MAX_KEYS keys), for callers that cannot allocate
    device memory when they sort.  Calls that overlap on the GPU race."""
    st = load().rc_sort_keys_static(c_void_p(_ptr(keys_in)), c_void_p(_ptr(keys_out)), c_uint64(n),
                                    c_uint32(lo_bit), c_uint32(hi_bit), c_uint32(digit_bits),
                                    c_void_p(_stream(stream)))
    if st != RC_OK:
        raise RcError(st, "rc_sort_keys_static")


def rc_sort_status(workspace=None, stream=None) -> int:
    """Status of the device work of the last sort on ``workspace`` (None: the
    last rc_sort_keys_static call on the current device); waits for ``stream``.
    Returns RC_OK, RC_E_TIMEOUT or RC_E_INVALID; raises on RC_E_CUDA."""
    st = load().rc_sort_status(c_void_p(_ptr(workspace) if workspace is not None else None),
                               c_void_p(_stream(stream)))
    if st == RC_E_CUDA:
        raise RcError(st, "rc_sort_status")
    return st


# ---------------------------------------------------------------------------
# convenience
# ---------------------------------------------------------------------------
def workspace(nbytes: int, device=None):
    import torch
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device or "cuda")


def check(model, opts=None, device=None, stream=None) -> Result:
    """Create, check and report one model (allocates its own workspace)."""
    m = model if isinstance(model, RcModel) else rc_model_create(model)
    ws = workspace(rc_workspace_size(m, opts), device)
    t = rc_check(m, opts, ws, stream)
    return rc_report(t, wait=True)[0]
