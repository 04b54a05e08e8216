"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by
element on the same seeded models: verdict, racy-cell count, instance count and
witness bit-exact; out-of-bounds reports identical; per-kernel parity of the
expansion (key multiset) and of the radix sort (stable order)."""
import numpy as np
import pytest
import torch

import oracle
import workloads as w
from workloads.spec import Access, Array, Loop, Model, Stmt, bid, const, it, tid, R, W

from . import pyref

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


def compare(rc, model, opts=None, exp=None):
    got = rc.check(model, opts)
    exp = exp or oracle.check(model)
    assert got.status == exp.status, (model.name, got, exp)
    assert got.instances == exp.instances, (model.name, got.instances, exp.instances)
    if exp.status == oracle.STATUS_OOB:
        assert (got.oob_stmt, got.oob_access, got.oob_gtid, got.oob_dim) == \
               (exp.oob_stmt, exp.oob_access, exp.oob_gtid, exp.oob_dim)
        return got
    assert (got.verdict, got.racy_cells) == (exp.verdict, exp.racy_cells), (model.name, got, exp)
    assert got.witness == exp.witness, (model.name, got.witness, exp.witness)
    return got


# ---------------------------------------------------------------------------
# whole-path parity
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("T", [1, 2, 3, 31, 32, 33, 256, 1024])
def test_neighbor(rc, T):
    compare(rc, w.neighbor_write_read(T))
    compare(rc, w.neighbor_write_read(T, n_blocks=3))


@pytest.mark.parametrize("bar,load", [(True, False), (False, False), (False, True), (True, True)])
def test_reduction_tree(rc, bar, load):
    g = compare(rc, w.reduction_tree(bar, load_phase=load))
    assert g.racy_cells == (0 if bar else (255 if load else 127))


@pytest.mark.parametrize("n", [2, 3, 5, 12, 64, 300])
def test_polyhedral_product(rc, n):
    g = compare(rc, w.polyhedral_product(n))
    assert g.racy_cells == 2 * n - 3
    compare(rc, w.polyhedral_product(n, init_stmt=True))


@pytest.mark.parametrize("pad", [False, True])
@pytest.mark.parametrize("bar", [False, True])
def test_transpose_small(rc, pad, bar):
    compare(rc, w.transpose(pad=pad, barrier=bar, n=256))


@pytest.mark.parametrize("pad", [False, True])
def test_transpose_full_size(rc, pad):
    g = compare(rc, w.transpose(pad=pad, barrier=False))
    assert g.racy_cells == 4063232 and g.instances == 16777216
    g = compare(rc, w.transpose(pad=pad, barrier=True))
    assert g.racy_cells == 0


@pytest.mark.parametrize("L", [1, 32, 33, 70])
@pytest.mark.parametrize("bar", [True, False])
def test_ge_spmm(rc, L, bar):
    compare(rc, w.ge_spmm_uniform(3, 64, 4, L, trailing_barrier=bar))


@pytest.mark.parametrize("seed", range(6))
def test_random_affine_reduced(rc, seed):
    for plant in (False, True):
        m = w.random_affine(seed, n_blocks=16, block=256, plant=plant)
        g = compare(rc, m)
        assert g.racy_cells == (m.n_threads if plant else 0)


@pytest.mark.parametrize("seed", range(300))
def test_tiny_random(rc, seed):
    compare(rc, w.tiny_random(seed))


@pytest.mark.parametrize("digit_bits", [4, 5, 7, 8])
def test_digit_widths(rc, digit_bits):
    opts = {"digit_bits": digit_bits}
    for m in (w.transpose(barrier=False, n=128), w.random_affine(3, n_blocks=4, block=128, plant=True),
              w.tiny_random(11)):
        compare(rc, m, opts)


def test_empty_and_degenerate(rc):
    arr = [Array("a", "global", (4,))]
    # no statements at all
    compare(rc, Model((1, 1, 1), (4, 1, 1), arr, []))
    # every guard false
    compare(rc, Model((2, 1, 1), (4, 1, 1), arr, [Stmt([Access(0, W, (tid.x,))], guards=[const(-1)])]))
    # zero-trip loop
    compare(rc, Model((2, 1, 1), (4, 1, 1), arr, [Stmt([Access(0, W, (tid.x,))], loops=[Loop(3, 3)])]))
    # one thread, one instance
    compare(rc, Model((1, 1, 1), (1, 1, 1), arr, [Stmt([Access(0, W, (const(2),))])]))
    # every thread of every block writes one global cell: one racy cell with all threads in it
    g = compare(rc, Model((64, 1, 1), (256, 1, 1), [Array("x", "global", (1,))],
                          [Stmt([Access(0, R, (const(0),))], loops=[Loop(0, 8)]),
                           Stmt([Access(0, W, (const(0),))])]))
    assert g.racy_cells == 1
    # a write by one thread among many readers of one shared cell, in one phase
    g = compare(rc, Model((3, 1, 1), (128, 1, 1), [Array("s", "shared", (2,))],
                          [Stmt([Access(0, R, (const(1),))]),
                           Stmt([Access(0, W, (const(1),))], guards=[const(0) - tid.x + 77])]))
    assert g.racy_cells == 3


@pytest.mark.parametrize("scope", ["shared", "global"])
@pytest.mark.parametrize("block", [60, 64, 65, 100, 512])
@pytest.mark.parametrize("writer", [None, (0, 5), (1, 0), (3, 7)])
def test_long_cells(rc, scope, block, writer):
    """Cells read by every thread of a block in phases 0 and 1 (2 x block keys
    per cell and block, many above the scan's long-cell cap), plus one writer
    thread in some phase: racy iff the writer shares a phase with readers or
    (global) another block reads the cell."""
    stmts = [Stmt([Access(0, R, (tid.x % 2,))], loops=[Loop(0, 2)], phase=it(0)),
             Stmt([Access(0, R, (const(1),))], loops=[Loop(0, 2)], phase=it(0))]
    if writer is not None:
        ph, t = writer
        stmts.append(Stmt([Access(0, W, (const(1),))], guards=[const(t) - tid.x, tid.x - t], phase=const(ph)))
    m = Model((3, 1, 1), (block, 1, 1), [Array("x", scope, (2,))], stmts, n_phases=4)
    compare(rc, m)


def test_out_of_bounds(rc):
    arr = [Array("a", "global", (10,))]
    m = Model((2, 1, 1), (8, 1, 1), arr, [Stmt([Access(0, R, (tid.x,))]), Stmt([Access(0, W, (tid.x + 3,))])])
    g = compare(rc, m)
    assert g.status == rc.RC_E_OOB
    m2 = Model((1, 1, 1), (4, 1, 1), [Array("a", "shared", (4,))],
               [Stmt([Access(0, W, (tid.x,))], phase=const(2))], n_phases=2)
    compare(rc, m2)
    m3 = Model((1, 1, 1), (4, 1, 1), [Array("a", "shared", (4, 4))],
               [Stmt([Access(0, W, (tid.x, tid.x - 2))])])
    compare(rc, m3)


def test_batch_matches_single(rc):
    models = [w.tiny_random(s) for s in range(20)] + [w.reduction_tree(False), w.neighbor_write_read(64)]
    handles = [rc.rc_model_create(m) for m in models]
    ws = rc.workspace(rc.rc_batch_workspace_size(handles))
    res = rc.rc_report(rc.rc_check_batch(handles, None, ws))
    for m, g in zip(models, res):
        exp = oracle.check(m)
        assert (g.status, g.verdict, g.racy_cells, g.instances) == (exp.status, exp.verdict, exp.racy_cells,
                                                                   exp.instances)
        if exp.status == 0:
            assert g.witness == exp.witness


def test_report_not_ready_then_ready(rc):
    m = rc.rc_model_create(w.random_affine(1, n_blocks=64, block=256))
    ws = rc.workspace(rc.rc_workspace_size(m))
    t = rc.rc_check(m, None, ws)
    got = None
    try:
        got = rc.rc_report(t, wait=False)[0]
    except rc.NotReady:
        got = rc.rc_report(t, wait=True)[0]
    assert got.status == 0


def test_workspace_too_small(rc):
    m = rc.rc_model_create(w.neighbor_write_read(32))
    ws = rc.workspace(rc.rc_workspace_size(m) - 512)
    with pytest.raises(rc.RcError) as e:
        rc.rc_check(m, None, ws)
    assert e.value.status == rc.RC_E_NOMEM


def test_lookback_timeout_is_reported_and_context_survives(rc):
    m = w.random_affine(5, n_blocks=16, block=256)
    opts = {"test_flags": rc.binding.RC_TEST_STALL_LOOKBACK, "spin_limit": 2000}
    g = rc.check(m, opts)
    assert g.status == rc.RC_E_TIMEOUT
    # the context is still usable and the next check is exact
    compare(rc, m)


# ---------------------------------------------------------------------------
# per-kernel parity
# ---------------------------------------------------------------------------

def decode_keys(keys: np.ndarray, lay: dict, model) -> list:
    keys = keys[keys != np.uint64(0xFFFFFFFFFFFFFFFF)]
    k = keys.astype(np.uint64)

    def field(shift, bits):
        return ((k >> np.uint64(shift)) & np.uint64((1 << bits) - 1)).astype(np.int64)

    kind = (k & np.uint64(1)).astype(np.int64)
    t = field(lay["thread_shift"], lay["thread_bits"])
    b = field(lay["block_shift"], lay["block_bits"])
    p = field(lay["phase_shift"], lay["phase_bits"])
    cell = (k >> np.uint64(lay["cell_shift"])).astype(np.int64)
    base = np.array(lay["array_base"], dtype=np.int64)
    cells = np.array(lay["array_cells"], dtype=np.int64)
    a = np.searchsorted(base, cell, side="right") - 1
    rem = cell - base[a]
    shared = np.array([1 if arr.scope == "shared" else 0 for arr in model.arrays], dtype=np.int64)[a]
    s = np.where(shared == 1, rem // cells[a], 0)
    e = np.where(shared == 1, rem % cells[a], rem)
    tup = np.stack([a, s, e, b, p, t, kind], axis=1)
    order = np.lexsort(tup.T[::-1])
    return tup[order]


def keyed_rows(exp: np.ndarray, model) -> np.ndarray:
    """The oracle's instances that get a key: those of arrays some statement
    writes.  A cell that is never written has no conflicting pair (a race needs
    a write, Introduction), so the expansion bounds-checks and counts the other
    instances but emits none."""
    written = {acc.array for st in model.stmts for acc in st.accesses if acc.kind == W}
    if len(exp) == 0:
        return exp
    return exp[np.isin(exp[:, 0], sorted(written))]


@pytest.mark.parametrize("which", ["tiny", "reduction", "transpose", "affine", "gespmm"])
def test_expand_key_multiset(rc, which):
    models = {
        "tiny": [w.tiny_random(s) for s in range(40)],
        "reduction": [w.reduction_tree(False, load_phase=True)],
        "transpose": [w.transpose(pad=True, barrier=True, n=128)],
        "affine": [w.random_affine(2, n_blocks=8, block=128, plant=True)],
        "gespmm": [w.ge_spmm_uniform(2, 64, 3, 45)],
    }[which]
    for model in models:
        m = rc.rc_model_create(model)
        lay = rc.rc_model_layout(m)
        n = lay["key_slots"]
        ws = rc.workspace(rc.rc_workspace_size(m))
        keys = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        rc.rc_expand_keys(m, ws, keys, cnt)
        torch.cuda.synchronize()
        got = decode_keys(keys[:n].cpu().numpy().view(np.uint64), lay, model)
        exp = oracle.expand(model)
        assert int(cnt.item()) == len(exp)
        exp = keyed_rows(exp, model)
        assert got.shape == exp.shape and np.array_equal(got, exp), model.name


@pytest.mark.parametrize("n", [0, 1, 2, 33, 4095, 4096, 4097, 100_000, 3_000_001])
@pytest.mark.parametrize("bits", [(0, 64), (5, 37), (21, 54), (60, 63)])
def test_sort_stable(rc, n, bits):
    lo, hi = bits
    g = torch.Generator().manual_seed(n * 131 + lo)
    x = torch.randint(-(1 << 62), 1 << 62, (max(n, 1),), generator=g, dtype=torch.int64)[:n]
    if n > 10:
        x[: n // 3] = x[: n // 3] & 0xFFFF    # heavy digit collisions
    keys = x.numpy().view(np.uint64)
    mask = np.uint64((1 << (hi - lo)) - 1) if hi - lo < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    digit = (keys >> np.uint64(lo)) & mask
    exp = keys[np.argsort(digit, kind="stable")]
    din = x.cuda()
    dout = torch.empty_like(din)
    for db in (8, 6):
        ws = rc.workspace(rc.rc_sort_workspace_size(n, db))
        rc.rc_sort_keys(din, dout, n, lo, hi, db, ws)
        torch.cuda.synchronize()
        got = dout.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, exp), (n, bits, db)
        assert rc.rc_sort_status(ws) == rc.RC_OK


def test_sort_timeout_is_reported_and_context_survives(rc, monkeypatch):
    """A look-back wait of the sort entry point that runs out (the test hook
    makes every wait look for a status epoch nothing publishes) is reported by
    rc_sort_status; the next sort is exact."""
    n = 300_000
    g = torch.Generator().manual_seed(77)
    x = torch.randint(-(1 << 62), 1 << 62, (n,), generator=g, dtype=torch.int64)
    keys = x.numpy().view(np.uint64)
    exp = keys[np.argsort((keys >> np.uint64(4)) & np.uint64((1 << 24) - 1), kind="stable")]
    din = x.cuda()
    dout = torch.empty_like(din)
    ws = rc.workspace(rc.rc_sort_workspace_size(n, 8))
    monkeypatch.setenv("RC_TEST_SORT_STALL", "1")
    rc.rc_sort_keys(din, dout, n, 4, 28, 8, ws)
    assert rc.rc_sort_status(ws) == rc.RC_E_TIMEOUT
    monkeypatch.delenv("RC_TEST_SORT_STALL")
    rc.rc_sort_keys(din, dout, n, 4, 28, 8, ws)
    assert rc.rc_sort_status(ws) == rc.RC_OK
    assert np.array_equal(dout.cpu().numpy().view(np.uint64), exp)


# ---------------------------------------------------------------------------
# hash path
# ---------------------------------------------------------------------------

HASH = {"path": 2}
HASH_EARLY = {"path": 2, "early_exit": 1}


def _hash_models():
    return ([w.tiny_random(s) for s in range(60)] +
            [w.neighbor_write_read(64, n_blocks=3), w.reduction_tree(False), w.reduction_tree(True),
             w.polyhedral_product(40), w.transpose(pad=True, barrier=False, n=128),
             w.transpose(pad=False, barrier=True, n=128), w.ge_spmm_uniform(2, 64, 3, 70, False),
             w.random_affine(4, n_blocks=8, block=128, plant=True),
             w.random_affine(4, n_blocks=8, block=128, plant=False)])


@pytest.mark.parametrize("i", range(69))
def test_hash_path_matches_oracle(rc, i):
    """Without early exit the hash path gives the sort path's full result."""
    compare(rc, _hash_models()[i], HASH)


def _is_racing_witness(model, wit):
    a, s, e, x, y = wit
    inst = {tuple(int(v) for v in row) for row in oracle.expand(model)}
    bs = model.block_size
    xt = (a, s, e, x[0], x[1], x[2], x[3])
    yt = (a, s, e, y[0], y[1], y[2], y[3])
    return xt in inst and yt in inst and pyref.race(xt, yt, bs)


@pytest.mark.parametrize("i", range(69))
def test_hash_early_exit_verdict(rc, i):
    """With early exit the verdict is exact, the count a lower bound, and the
    witness a racing pair of the model."""
    m = _hash_models()[i]
    exp = oracle.check(m)
    got = rc.check(m, HASH_EARLY)
    assert got.status == exp.status and got.instances == exp.instances
    assert got.verdict == exp.verdict
    if exp.verdict:
        assert 1 <= got.racy_cells <= exp.racy_cells
        assert _is_racing_witness(m, got.witness)


def test_hash_path_out_of_bounds(rc):
    m = Model((2, 1, 1), (8, 1, 1), [Array("a", "global", (10,))],
              [Stmt([Access(0, R, (tid.x,))]), Stmt([Access(0, W, (tid.x + 3,))])])
    compare(rc, m, HASH)


@pytest.mark.parametrize("i", range(40))
def test_scan_long_warp_ranges(rc, i):
    """Few scan warps, so each warp carries cells across many segments."""
    models = ([w.tiny_random(s) for s in range(25)] +
              [w.reduction_tree(False, load_phase=True), w.neighbor_write_read(300, n_blocks=5),
               w.polyhedral_product(120), w.transpose(pad=False, barrier=False, n=128),
               w.transpose(pad=True, barrier=True, n=128), w.ge_spmm_uniform(2, 64, 5, 90, False),
               w.random_affine(9, n_blocks=8, block=128, plant=True),
               w.random_affine(9, n_blocks=8, block=128, plant=False)] +
              [Model((3, 1, 1), (blk, 1, 1), [Array("x", sc, (2,))],
                     [Stmt([Access(0, R, (tid.x % 2,))], loops=[Loop(0, 2)], phase=it(0)),
                      Stmt([Access(0, R, (const(1),))], loops=[Loop(0, 2)], phase=it(0)),
                      Stmt([Access(0, W, (const(1),))], guards=[const(5) - tid.x, tid.x - 5], phase=const(ph))],
                     n_phases=4)
               for sc, blk, ph in [("shared", 700, 1), ("global", 700, 3), ("shared", 1024, 3),
                                   ("global", 33, 0), ("shared", 65, 2), ("global", 1000, 1), ("shared", 999, 0)]])
    compare(rc, models[i], {"test_flags": rc.binding.RC_TEST_FEW_SCAN_WARPS})


@pytest.mark.parametrize("n_phases", [2, 16, 17, 40, 300])
@pytest.mark.parametrize("seed", range(3))
def test_phase_counts(rc, n_phases, seed):
    """Models with at most 16 barrier intervals are sorted by cell only and the
    scan groups phases with tables; more intervals keep the phase bits in the
    sort.  Both give the oracle's result (also with long per-warp ranges)."""
    for plant in (False, True):
        m = w.random_affine(seed, n_blocks=8, block=128, n_stmts=14, n_phases=n_phases, plant=plant)
        compare(rc, m)
        compare(rc, m, {"test_flags": 2})   # RC_TEST_FEW_SCAN_WARPS


@pytest.mark.parametrize("n", [1000, 100_003])
def test_sort_unaligned_buffers(rc, n):
    """Key buffers that start 8 bytes past a 16-byte boundary (the histogram
    then takes its unvectorised path)."""
    g = torch.Generator().manual_seed(n)
    x = torch.randint(-(1 << 62), 1 << 62, (n + 1,), generator=g, dtype=torch.int64)
    keys = x[1:].numpy().view(np.uint64)
    exp = keys[np.argsort((keys >> np.uint64(3)) & np.uint64((1 << 20) - 1), kind="stable")]
    din = x.cuda()[1:]
    dbuf = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    dout = dbuf[1:]
    assert din.data_ptr() % 16 == 8 and dout.data_ptr() % 16 == 8
    ws = rc.workspace(rc.rc_sort_workspace_size(n, 8))
    rc.rc_sort_keys(din, dout, n, 3, 23, 8, ws)
    torch.cuda.synchronize()
    assert np.array_equal(dout.cpu().numpy().view(np.uint64), exp)
