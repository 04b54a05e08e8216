"""Boundary tests that need no GPU: the CUDA library builds, loads and exports
every entry point declared in include/rc.h; the ctypes structures match the C
layout of rc.h as compiled by gcc; descriptor validation rejects malformed
models before touching the device."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

import workloads as w
from workloads.spec import Access, Array, Loop, Model, Stmt, bid, const, it, tid, R, W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rc.h")


@pytest.fixture(scope="module")
def rc():
    from paper_2503_08946_gb300 import build as b
    b.build()
    import paper_2503_08946_gb300 as pkg
    pkg.load()
    return pkg


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(rc_[a-z_]+)\s*\(", text)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(rc):
    lib = ctypes.CDLL(rc.binding.LIB_PATH)
    declared = header_functions()
    assert set(declared) == set(rc.EXPORTS), (declared, rc.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", rc.binding.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (rc_[a-z_]+)\b", out))
    assert set(declared) <= exported


def test_struct_layout_matches_c(rc):
    b = rc.binding
    structs = ["rc_insn", "rc_expr", "rc_loop", "rc_access", "rc_stmt", "rc_array", "rc_table", "rc_model_desc",
               "rc_limits", "rc_layout", "rc_check_opts", "rc_inst", "rc_result", "rc_server_opts",
               "rc_server_done"]
    fields = {s: [f for f, _ in getattr(b, s)._fields_] for s in structs}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){"]
    for s in structs:
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f in fields[s]:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(src, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-std=c11", "-o", exe, src], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    c_vals = dict(l.split() for l in out.strip().splitlines())
    for s in structs:
        cls = getattr(b, s)
        assert int(c_vals[s]) == ctypes.sizeof(cls), s
        for f in fields[s]:
            assert int(c_vals[f"{s}.{f}"]) == getattr(cls, f).offset, f"{s}.{f}"


def test_status_strings(rc):
    for s in range(9):
        assert rc.rc_status_str(s)
    lim = rc.rc_get_limits()
    assert lim["key_bits"] == 63 and lim["max_loops"] >= 2


def _status(rc, m):
    return rc.rc_model_create_status(m)


def test_validation_rejects_malformed(rc):
    ok_arr = [Array("a", "shared", (8,))]
    # phase that names tid: a barrier interval must be block-uniform
    m = Model((1, 1, 1), (8, 1, 1), ok_arr, [Stmt([Access(0, W, (tid.x,))], phase=tid.x % 2)], n_phases=2)
    assert _status(rc, m) == rc.RC_E_INVALID
    # phase through the iterator of a loop whose bounds depend on tid
    m = Model((1, 1, 1), (8, 1, 1), ok_arr,
              [Stmt([Access(0, W, (tid.x,))], loops=[Loop(0, tid.x)], phase=it(0) % 2)], n_phases=2)
    assert _status(rc, m) == rc.RC_E_INVALID
    # iterator outside the loop nest
    m = Model((1, 1, 1), (8, 1, 1), ok_arr, [Stmt([Access(0, W, (it(0),))])])
    assert _status(rc, m) == rc.RC_E_INVALID
    # parameter that does not exist
    m = Model((1, 1, 1), (8, 1, 1), ok_arr, [Stmt([Access(0, W, (w.param(3),))])], params=[1])
    assert _status(rc, m) == rc.RC_E_INVALID
    # zero-sized grid / zero phases / bad extent / non-positive step
    assert _status(rc, Model((0, 1, 1), (8, 1, 1), ok_arr, [])) == rc.RC_E_INVALID
    assert _status(rc, Model((1, 1, 1), (8, 1, 1), ok_arr, [], n_phases=0)) == rc.RC_E_INVALID
    assert _status(rc, Model((1, 1, 1), (8, 1, 1), [Array("a", "global", (0,))], [])) == rc.RC_E_INVALID
    m = Model((1, 1, 1), (8, 1, 1), ok_arr, [Stmt([Access(0, R, (it(0),))], loops=[Loop(0, 4, 0)])])
    assert _status(rc, m) == rc.RC_E_INVALID
    # too deep a loop nest
    deep = [Loop(0, 2) for _ in range(9)]
    m = Model((1, 1, 1), (8, 1, 1), ok_arr, [Stmt([Access(0, R, (tid.x,))], loops=deep)])
    assert _status(rc, m) == rc.RC_E_UNSUPPORTED


def test_validation_superset_tables(rc):
    """Superset tables: an empty range is invalid, and each free parameter
    takes a loop level (7 loops + 2 free parameters exceed 8)."""
    from workloads.spec import load
    arr = [Array("a", "shared", (64,))]
    one = Stmt([Access(0, W, (load(0, tid.x) % 64,))])
    assert _status(rc, Model((1, 1, 1), (8, 1, 1), arr, [one], tables=[[]], superset={0: (3, 2)})) == rc.RC_E_INVALID
    assert "rc_expand_jit" in rc.rc_kernel_source(Model((1, 1, 1), (8, 1, 1), arr, [one], superset={0: (0, 7)}))
    deep = Stmt([Access(0, W, ((load(0, tid.x) + load(0, tid.x + 1)) % 64,))], loops=[Loop(0, 2) for _ in range(7)])
    m = Model((1, 1, 1), (8, 1, 1), arr, [deep], superset={0: (0, 3)})
    assert _status(rc, m) == rc.RC_E_UNSUPPORTED
    deep.loops = deep.loops[:6]
    assert "rc_expand_jit" in rc.rc_kernel_source(m)


def test_validation_key_overflow(rc):
    # 2^20 blocks x 1024 threads x 2^40 cells need 74 key bits: the model lowers
    # as a wide model (checked in cell-range chunks)
    big = [Array("g", "global", (1 << 20, 1 << 20))]
    m = Model((1 << 20, 1, 1), (1024, 1, 1), big, [Stmt([Access(0, W, (tid.x, bid.x))])], n_phases=4)
    assert "rc_chunk_jit" in rc.rc_kernel_source(m)   # host lowering succeeds: the chunked kernel
    assert _status(rc, m) not in (rc.RC_E_KEY_OVERFLOW, rc.RC_E_INVALID, rc.RC_E_UNSUPPORTED)
    # a cell space of 2^62 cells cannot be addressed at all
    huge = [Array("g", "global", (1 << 31, 1 << 31))]
    m2 = Model((1, 1, 1), (32, 1, 1), huge, [Stmt([Access(0, W, (tid.x, tid.x))])])
    assert _status(rc, m2) == rc.RC_E_KEY_OVERFLOW


def test_generated_kernels_compile(rc, tmp_path):
    """The expansion kernels generated for a few models compile for sm_103a."""
    import shutil
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    deep = Model((2, 1, 1), (8, 1, 1), [Array("a", "shared", (64,))],
                 [Stmt([Access(0, W, ((tid.x + it(0) + it(1) + it(2) + it(3) + it(4)) % 64,))],
                       loops=[Loop(0, 2)] * 5)])
    csr = w.ge_spmm_csr(w.csr_row_lengths(1, 8), N=64, K=2)
    wide = w.random_affine(1, n_blocks=8, block=64, n_stmts=12, row_global=1 << 44)
    sup = w.ge_spmm_csr([3, 20, 7, 10], N=32, K=1, superset=True)
    for i, m in enumerate([w.random_affine(0), w.tiny_random(5), w.ge_spmm_uniform(), deep, csr,
                           w.tiny_random_tables(3), wide, w.tiny_random_sync(2), w.warp_reduction(2), sup]):
        src = rc.rc_kernel_source(m)
        assert ("rc_chunk_jit" if m is wide else "rc_expand_jit") in src
        f = tmp_path / f"k{i}.cu"
        f.write_text(src)
        r = subprocess.run([nvcc, "-c", str(f), "-o", str(tmp_path / f"k{i}.o"), "-std=c++17",
                            "-gencode", "arch=compute_103a,code=sm_103a"], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[:2000]


def test_record_array_decoding(rc):
    """rc_report_array's records decode to the same Result objects as the
    per-record decoder (field order of rc_result / rc_inst, witness tuples
    ordered (block, phase, thread, kind))."""
    import numpy as np
    b = rc.binding
    n = 5
    out = (b.rc_result * n)()
    for i in range(n):
        r = out[i]
        r.status, r.verdict, r.racy_cells, r.instances = i % 2, 1, 10 * i + 1, 1000 + i
        r.w_array, r.w_scope, r.w_addr = i, 7 * i, (1 << 40) + i
        r.x.block, r.x.thread, r.x.kind, r.x.phase, r.x.gtid, r.x.warp_phase = 3 + i, 17, 1, 2, 99, 1
        r.y.block, r.y.thread, r.y.kind, r.y.phase, r.y.gtid, r.y.warp_phase = 4 + i, 18, 2, 3, 100, 0
        r.oob_stmt, r.oob_access, r.oob_gtid, r.oob_dim = i, i + 1, (1 << 41) + i, -1 if i else 2
    arr = np.ctypeslib.as_array(out)[:n]
    got = b.results_of(arr)
    exp = [b._result(out[i]) for i in range(n)]
    assert got == exp
    assert got[2].witness == (2, 14, (1 << 40) + 2, (5, 2, 17, 1), (6, 3, 18, 2))
    assert (got[3].x_wphase, got[3].y_wphase) == (1, 0)
    assert b.results_of(arr[:0]) == []
