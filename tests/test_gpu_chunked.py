"""Chunked checks: models wider than one 63-bit key (their cells rebased per
chunk), and ordinary models checked in a workspace smaller than their keys
(RC_OPT_CHUNKED).  The CUDA path against the oracle: status, instance count,
racy-cell count and witness bit-exact."""
import pytest
import torch

import oracle
import workloads as w
from workloads.spec import Access, Array, Loop, Model, Stmt, bid, const, it, tid, R, W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rc():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2503_08946_gb300 import build as b
    b.build()
    oracle.build()
    import paper_2503_08946_gb300 as pkg
    pkg.load()
    return pkg


def same(got, exp):
    assert got.status == exp.status, (got, exp)
    assert got.instances == exp.instances
    if exp.status == oracle.STATUS_OOB:
        assert (got.oob_stmt, got.oob_access, got.oob_gtid, got.oob_dim) == \
               (exp.oob_stmt, exp.oob_access, exp.oob_gtid, exp.oob_dim)
        return
    assert (got.verdict, got.racy_cells) == (exp.verdict, exp.racy_cells), (got, exp)
    assert got.witness == exp.witness, (got.witness, exp.witness)


def check_ws(rc, model, opts, ws_bytes):
    """One check in a workspace of exactly ws_bytes (rounded up to 256)."""
    b = rc.binding
    m = b.rc_model_create(model)
    ws = b.workspace(ws_bytes)
    t = b.rc_check(m, opts, ws)
    return b.rc_report(t, wait=True)[0]


def wide_model(seed, plant=None, row_bits=44):
    return w.random_affine(seed, n_blocks=8, block=64, n_stmts=24, plant=plant, row_global=1 << row_bits)


# ---------------------------------------------------------------------------
# wide models
# ---------------------------------------------------------------------------

def test_wide_layout(rc):
    b = rc.binding
    m = b.rc_model_create(wide_model(0))
    lay = b.rc_model_layout(m)
    assert lay["wide"] == 1
    assert lay["cell_shift"] + lay["cell_bits"] == 63
    assert lay["total_cells"].bit_length() + lay["cell_shift"] > 63
    narrow = b.rc_model_layout(b.rc_model_create(w.random_affine(0, n_blocks=8, block=64, n_stmts=24)))
    assert narrow["wide"] == 0


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("jit", ["0", "1"])
def test_wide_random(rc, seed, jit, monkeypatch):
    monkeypatch.setenv("RC_JIT", jit)   # interpreted / generated count and route passes
    m = wide_model(seed)
    same(rc.check(m), oracle.check(m))


@pytest.mark.parametrize("seed", [0, 3])
@pytest.mark.parametrize("jit", ["0", "1"])
def test_wide_planted(rc, seed, jit, monkeypatch):
    monkeypatch.setenv("RC_JIT", jit)
    m = wide_model(seed, plant=True)
    h = rc.binding.rc_model_create(m)
    assert rc.binding.rc_model_layout(h)["expand_jit"] == int(jit)
    g = rc.check(h)
    same(g, oracle.check(m))
    assert g.racy_cells == 8 * 64


@pytest.mark.parametrize("row_bits", [41, 48, 51])
def test_wide_row_lengths(rc, row_bits):
    m = wide_model(5, plant=True, row_bits=row_bits)
    same(rc.check(m), oracle.check(m))


@pytest.mark.parametrize("frac", [0.6, 0.3])   # the shared array (one bucket) holds ~1/4 of the keys
@pytest.mark.parametrize("jit", ["0", "1"])
def test_wide_small_workspace(rc, frac, jit, monkeypatch):
    """Span-limited chunks grouped into several waves by a small workspace."""
    monkeypatch.setenv("RC_JIT", jit)
    model = wide_model(6, plant=True)
    b = rc.binding
    m = b.rc_model_create(model)
    full = b.rc_workspace_size(m)
    keys = b.rc_model_layout(m)["key_slots"]
    same(check_ws(rc, model, None, int(full - 16 * keys * (1 - frac))), oracle.check(model))


def test_cell_space_beyond_2_62(rc):
    # 3 arrays x 512 rows x 2^56 cells: the cells cannot be numbered in 62 bits
    assert rc.binding.rc_model_create_status(wide_model(5, row_bits=56)) == rc.binding.RC_E_KEY_OVERFLOW


def test_wide_shared_and_phases(rc):
    # a wide model with shared arrays, many barrier intervals (phase bits sorted)
    big = Array("G", "global", (1 << 30, 1 << 22))
    sh = Array("S", "shared", (64,))
    n = 40
    stmts = [Stmt([Access(0, W, (bid.x * 4 + tid.x % 4, (tid.x * 977 + k * 131) % (1 << 22)))], phase=const(k))
             for k in range(n)]
    stmts += [Stmt([Access(1, W, ((tid.x + k) % 64,)), Access(1, R, ((tid.x + k + 1) % 64,))], phase=const(k))
              for k in range(0, n, 7)]
    m = Model((16, 1, 1), (64, 1, 1), [big, sh], stmts, n_phases=n, name="wide_phases")
    same(rc.check(m), oracle.check(m))
    m2 = Model((16, 1, 1), (64, 1, 1), [big, sh], stmts, n_phases=n, name="wide_phases_jit")
    import os
    old = os.environ.get("RC_JIT")
    os.environ["RC_JIT"] = "1"
    try:
        same(rc.check(m2), oracle.check(m2))
    finally:
        if old is None:
            del os.environ["RC_JIT"]
        else:
            os.environ["RC_JIT"] = old


@pytest.mark.parametrize("jit", ["0", "1"])
def test_wide_out_of_bounds(rc, jit, monkeypatch):
    monkeypatch.setenv("RC_JIT", jit)
    big = Array("G", "global", (1 << 30, 1 << 30))
    m = Model((4, 1, 1), (32, 1, 1), [big],
              [Stmt([Access(0, W, (tid.x, it(0)))], loops=[Loop(0, 4)]),
               Stmt([Access(0, R, (tid.x + 1, (1 << 30) - 1 + bid.x))])], name="wide_oob")
    same(rc.check(m), oracle.check(m))


def test_wide_rejected_where_one_key_per_instance(rc):
    b = rc.binding
    m = b.rc_model_create(wide_model(1))
    with pytest.raises(b.RcError) as e:
        b.rc_batch_workspace_size([m])
    assert e.value.status == b.RC_E_KEY_OVERFLOW
    ws = b.workspace(b.rc_workspace_size(m))
    with pytest.raises(b.RcError) as e:
        b.rc_check(m, {"path": b.RC_PATH_HASH}, ws)
    assert e.value.status == b.RC_E_KEY_OVERFLOW


# ---------------------------------------------------------------------------
# RC_OPT_CHUNKED on ordinary models
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(12))
def test_chunked_equals_whole(rc, seed):
    m = w.tiny_random(seed)
    same(rc.check(m, {"flags": rc.binding.RC_OPT_CHUNKED}), oracle.check(m))


@pytest.mark.parametrize("seed,plant", [(0, False), (1, True), (7, True)])
@pytest.mark.parametrize("frac", [1.0, 0.3, 0.07])
def test_chunked_small_workspace(rc, seed, plant, frac):
    """A workspace holding a fraction of the keys: many chunks, same result."""
    model = w.random_affine(seed, n_blocks=16, block=64, n_stmts=24, plant=plant)
    b = rc.binding
    m = b.rc_model_create(model)
    opts = {"flags": b.RC_OPT_CHUNKED}
    full = b.rc_workspace_size(m, opts)
    keys = b.rc_model_layout(m)["key_slots"]
    # the chunk region for frac * keys keys plus the fixed parts
    ws = int(full - 16 * keys * (1 - frac))
    same(check_ws(rc, model, opts, ws), oracle.check(model))


def test_chunked_workspace_too_small(rc):
    b = rc.binding
    opts = {"flags": b.RC_OPT_CHUNKED}
    # not even the bucket counts fit
    model = w.random_affine(2, n_blocks=16, block=64, n_stmts=24)
    with pytest.raises(b.RcError) as e:
        check_ws(rc, model, opts, 4096)
    assert e.value.status == b.RC_E_NOMEM
    # one cell holds 64 x 64 x 8 keys, more than the workspace holds
    hot = Model((64, 1, 1), (64, 1, 1), [Array("g", "global", (16,))],
                [Stmt([Access(0, W, (const(3),))], loops=[Loop(0, 8)])], name="hot_cell")
    m = b.rc_model_create(hot)
    full = b.rc_workspace_size(m, opts)
    keys = b.rc_model_layout(m)["key_slots"]
    with pytest.raises(b.RcError) as e:
        check_ws(rc, hot, opts, int(full - 16 * (keys - 1000)))
    assert e.value.status == b.RC_E_NOMEM
    # with room for it, the hot cell is one racy cell
    same(check_ws(rc, hot, opts, full), oracle.check(hot))


@pytest.mark.parametrize("k", [2, 5])
def test_chunked_cell_ranges_merge(rc, k):
    """Cell-range partial checks with compaction merge to the whole check."""
    from paper_2503_08946_gb300 import distributed as dist
    model = w.random_affine(4, n_blocks=8, block=64, n_stmts=24, plant=True)
    b = rc.binding
    m = b.rc_model_create(model)
    total = b.rc_model_layout(m)["total_cells"]
    parts = []
    for lo, hi in dist.cell_ranges(total, k):
        if hi == lo:
            continue
        opts = {"flags": b.RC_OPT_CHUNKED, "cell_lo": lo, "cell_hi": hi}
        ws = b.workspace(b.rc_workspace_size(m, opts))
        parts.append(b.rc_report(b.rc_check(m, opts, ws), wait=True)[0])
    same(dist.merge_results(parts), oracle.check(model))


@pytest.mark.parametrize("ranges", [[(0, 1)], [(5, 5)]])
def test_chunked_degenerate_ranges(rc, ranges):
    model = w.neighbor_write_read(32)
    b = rc.binding
    m = b.rc_model_create(model)
    for lo, hi in ranges:
        opts = {"flags": b.RC_OPT_CHUNKED, "cell_lo": lo, "cell_hi": hi if hi > lo else lo + 1}
        r = b.rc_report(b.rc_check(m, opts, b.workspace(b.rc_workspace_size(m, opts))), wait=True)[0]
        exp = oracle.check_cells(model, opts["cell_lo"], opts["cell_hi"])
        same(r, exp)
