"""The bucket path of the grouping step (partition passes on a bijective hash
of the cell, then a counting sort of every bucket in shared memory, then the
ordered cell scan with the first racy cell kept by value) against the CPU
oracle, bit-exact: verdict, racy-cell count, instance
count and witness.  Covers the partition plans (no pass, one pass, two
passes), bins holding several cells (cell spaces wider than the bucket and bin
bits), buckets larger than shared memory (grouped in the other key buffer),
cells longer than one thread's share (folded by the whole block), atomics,
warp and grid barriers, batches, and equality with the LSD radix-sort path."""
import pytest
import torch

import oracle
import workloads as w
from workloads.spec import A, Access, Array, Model, Stmt, bid, const, tid, R, W

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


def full(r):
    return (r.status, r.instances, r.verdict, r.racy_cells, r.witness)


def compare(rc, model, opts=None, exp=None):
    got = rc.check(model, opts)
    exp = exp or oracle.check(model)
    assert got.status == exp.status, (model.name, got, exp)
    assert got.instances == exp.instances, model.name
    if exp.status == oracle.STATUS_OOB:
        return got
    assert (got.verdict, got.racy_cells) == (exp.verdict, exp.racy_cells), (model.name, got, exp)
    assert got.witness == exp.witness, (model.name, got.witness, exp.witness)
    if exp.verdict:
        assert (got.x_wphase, got.y_wphase) == (exp.x_wphase, exp.y_wphase), model.name
    return got


def plan_of(rc, model, opts=None):
    """Whether the check ran on the bucket path, and its partition passes."""
    b = rc.binding
    h = b.rc_model_create(model)
    o = dict(opts or {})
    o["flags"] = o.get("flags", 0) | b.RC_OPT_STAGE_TIMES
    ws = b.workspace(b.rc_workspace_size(h, o))
    t = b.rc_check(h, o, ws)
    st = b.rc_ticket_stage_times(t)
    b.rc_report(t, wait=True)
    return st["bucketed"], len(st["sort_ms"])


def test_path_selection(rc):
    b = rc.binding
    m = w.random_affine(3, n_blocks=64, block=256)
    # passes: the partition passes, then the local sort of every bucket
    assert plan_of(rc, m) == (True, 3)                         # ~17M keys: two partition passes
    assert plan_of(rc, w.random_affine(3, n_blocks=1, block=256))[0]   # small: one pass or none
    assert plan_of(rc, w.neighbor_write_read(64)) == (True, 1)  # 128 key slots: one bucket, no pass
    assert plan_of(rc, w.reduction_tree(False)) == (True, 2)   # 6,144 key slots: one pass
    assert plan_of(rc, m, {"flags": b.RC_OPT_LSD})[0] is False
    assert plan_of(rc, m, {"digit_bits": 8})[0] is False
    many = Model((2, 1, 1), (64, 1, 1), [Array("s", "shared", (64,))],
                 [Stmt([Access(0, W, ((tid.x + k) % 64,))], phase=const(k)) for k in range(20)], n_phases=20)
    assert plan_of(rc, many)[0] is False                        # more than 16 intervals: LSD and ordered scan


@pytest.mark.parametrize("blocks", [1, 2, 5, 16, 64])
@pytest.mark.parametrize("plant", [False, True])
def test_random_affine_sizes(rc, blocks, plant):
    """No pass (tiny), one pass and two passes; planted races (T racy cells)."""
    m = w.random_affine(11 + blocks, n_blocks=blocks, block=256, plant=plant)
    g = compare(rc, m)
    assert g.racy_cells == (blocks * 256 if plant else 0)


@pytest.mark.parametrize("seed", range(6))
def test_random_affine_odd_threads(rc, seed):
    """Tail threads guarded off (padding keys dropped by pass A)."""
    m = w.random_affine(seed, n_blocks=7, block=256, n_threads=7 * 256 - 37 * (seed + 1), plant=seed % 2 == 0)
    compare(rc, m)


@pytest.mark.parametrize("row", [1 << 16, 1 << 24, 1 << 30])
def test_wide_cell_space_multi_cell_bins(rc, row):
    """Rows of 2^16..2^30 cells: far more cell bits than bucket and bin bits, so
    bins hold several cells (ordered by cell inside the bin)."""
    for seed in range(3):
        m = w.random_affine(seed, n_blocks=8, block=128, row_global=row, plant=seed == 1)
        compare(rc, m)


@pytest.mark.parametrize("T,nb,bar", [(1 << 10, 1, False), (1 << 10, 64, True), (256, 4096, True),
                                      (1024, 1024, False)])
def test_hot_cell(rc, T, nb, bar):
    """One counter cell of up to a million keys: a bucket larger than shared
    memory and a cell folded by the whole block."""
    compare(rc, w.atomic_counter(T, n_blocks=nb, barrier=bar))


def test_hot_cells_among_many(rc):
    """Several hot cells next to many ordinary ones, in a wide cell space (hot
    cells share bins with other cells)."""
    big = Array("g", "global", (1 << 33,))
    sh = Array("s", "shared", (256,))
    stmts = [Stmt([Access(0, W, (tid.x * 1021 + bid.x * 7919,))], name="spread"),
             Stmt([Access(0, A, (const(12345),))], name="hot_a"),
             Stmt([Access(0, R, (const(12345),))], guards=[-1 * tid.x], phase=const(1), name="hot_r"),
             Stmt([Access(0, W, (const(77) + bid.x % 3,))], guards=[-1 * tid.x], phase=const(1), name="hot_w"),
             Stmt([Access(1, W, (tid.x,)), Access(1, R, ((tid.x + 1) % 256,))], phase=const(1), name="sh")]
    m = Model((600, 1, 1), (256, 1, 1), [big, sh], stmts, n_phases=2, name="hot_among_many")
    compare(rc, m)
    compare(rc, m, {"flags": rc.binding.RC_OPT_LSD})


@pytest.mark.parametrize("seed", range(0, 300, 2))
def test_tiny_random_both_paths(rc, seed):
    m = w.tiny_random(seed)
    exp = oracle.check(m)
    compare(rc, m, exp=exp)
    compare(rc, m, {"flags": rc.binding.RC_OPT_LSD}, exp=exp)


@pytest.mark.parametrize("seed", range(60))
def test_tiny_random_atomic_both_paths(rc, seed):
    m = w.tiny_random(seed, atomic=0.4)
    exp = oracle.check(m)
    compare(rc, m, exp=exp)
    compare(rc, m, {"flags": rc.binding.RC_OPT_LSD}, exp=exp)


@pytest.mark.parametrize("seed", range(80))
def test_tiny_random_sync_both_paths(rc, seed):
    for m in (w.tiny_random_sync(seed), w.tiny_random_sync(seed, block_guards=True)):
        exp = oracle.check(m)
        compare(rc, m, exp=exp)
        compare(rc, m, {"flags": rc.binding.RC_OPT_LSD}, exp=exp)


@pytest.mark.parametrize("pad,bar", [(False, False), (True, True)])
def test_transpose_full_both_paths(rc, pad, bar):
    m = w.transpose(pad=pad, barrier=bar)
    a = rc.check(m)
    b = rc.check(m, {"flags": rc.binding.RC_OPT_LSD})
    assert full(a) == full(b)
    assert a.racy_cells == (0 if bar else 4063232)


def test_grid_sync_models_in_buckets(rc):
    """Warp and grid barriers at a size that takes partition passes."""
    for gp in ([0, 0, 0], [0, 0, 1], [0, 1, 2]):
        c = Array("c", "global", (1 << 20,))
        lane0 = [-1 * (tid.x % 32)]
        stmts = [Stmt([Access(0, R, ((bid.x * 131 + tid.x) % (1 << 20),))], phase=const(0),
                      warp_phase=(tid.x // 32) % 2),
                 Stmt([Access(0, A, (const(0),))], guards=lane0, phase=const(0), warp_phase=const(1)),
                 Stmt([Access(0, W, ((bid.x * 131 + tid.x + 1) % (1 << 20),))], phase=const(1),
                      warp_phase=const(0)),
                 Stmt([Access(0, R, (const(1),))], phase=const(2))]
        m = Model((300, 1, 1), (128, 1, 1), [c], stmts, n_phases=3, n_warp_phases=2, grid_phase=gp,
                  name=f"sync_buckets_{gp}")
        compare(rc, m)


# ---------------------------------------------------------------------------
# batches
# ---------------------------------------------------------------------------

def check_batch(rc, models, opts=None):
    b = rc.binding
    hs = [b.rc_model_create(m) for m in models]
    ws = b.workspace(b.rc_batch_workspace_size(hs, opts))
    got = b.rc_report(b.rc_check_batch(hs, opts, ws), wait=True)
    for m, g in zip(models, got):
        exp = oracle.check(m)
        assert full(g) == full(exp), (m.name, g, exp)
    return got


@pytest.mark.parametrize("graph", [False, True])
def test_batch_bucket_path(rc, graph):
    opts = {"flags": rc.binding.RC_OPT_GRAPH} if graph else None
    models = (w.batch_models(300, seed0=4242) + [w.tiny_random(s) for s in range(40)] +
              [w.tiny_random(s, atomic=0.4) for s in range(20)] + [w.tiny_random_sync(s) for s in range(40)] +
              [w.atomic_counter(1024, n_blocks=16, barrier=False), w.reduction_tree(False)])
    got = check_batch(rc, models, opts)
    b = rc.binding
    hs = [b.rc_model_create(m) for m in models]
    lo = {"flags": b.RC_OPT_LSD}
    lsd = b.rc_report(b.rc_check_batch(hs, lo, b.workspace(b.rc_batch_workspace_size(hs, lo))), wait=True)
    assert [full(a) for a in got] == [full(x) for x in lsd]


def test_padding_with_reused_workspace(rc):
    """Models with guard-false padding slots checked one after another in one
    workspace: the bucket's dropped padding must not leave earlier keys in the
    scanned range (the single unpartitioned bucket, one partition pass)."""
    b = rc.binding
    models = [w.atomic_counter(256, 1, True), w.reduction_tree(True), w.atomic_counter(256, 1, False),
              w.random_affine(3, n_blocks=2, block=256, n_threads=300), w.neighbor_write_read(64),
              w.atomic_counter(1024, 4, True)]
    hs = [b.rc_model_create(m) for m in models]
    ws = b.workspace(max(b.rc_workspace_size(h, None) for h in hs))
    ws.fill_(0x5A)   # stale contents
    for rep in range(2):
        for m, h in zip(models, hs):
            g = b.rc_report(b.rc_check(h, None, ws), wait=True)[0]
            exp = oracle.check(m)
            assert full(g) == full(exp), (rep, m.name, g, exp)


def _stages(rc, model, opts=None):
    b = rc.binding
    h = b.rc_model_create(model)
    o = dict(opts or {})
    o["flags"] = o.get("flags", 0) | b.RC_OPT_STAGE_TIMES
    ws = b.workspace(b.rc_workspace_size(h, o))
    t = b.rc_check(h, o, ws)
    st = b.rc_ticket_stage_times(t)
    return st, b.rc_report(t, wait=True)[0]


@pytest.mark.parametrize("seed,blocks,plant", [(3, 64, False), (5, 64, True), (9, 16, True)])
def test_histogram_counted_by_expansion(rc, seed, blocks, plant, monkeypatch):
    """The generated expansion counts the pass-A histogram as it writes the
    keys; the interpreted expansion leaves it to the histogram kernel.  Both
    give the oracle's result (a wrong count would misplace keys in pass A)."""
    m = w.random_affine(seed, n_blocks=blocks, block=256, plant=plant)
    monkeypatch.setenv("RC_JIT", "1")
    st1, r1 = _stages(rc, m)
    monkeypatch.setenv("RC_JIT", "0")
    st0, r0 = _stages(rc, m)
    assert st1["bucketed"] and st1["histogram_fused"] and not st0["histogram_fused"]
    assert full(r1) == full(r0)
    compare(rc, m)
    # a cell range: only the kept keys are counted
    lo = rc.binding.rc_model_layout(rc.binding.rc_model_create(m))["total_cells"] // 3
    monkeypatch.setenv("RC_JIT", "1")
    g = rc.check(m, {"cell_lo": lo, "cell_hi": 2 * lo})
    exp = oracle.check_cells(m, lo, 2 * lo)
    assert full(g) == full(exp)
