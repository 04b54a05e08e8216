"""Warp-scope (__syncwarp) and grid-wide barriers on the CUDA path: blocks are
ordered only by grid barriers, two warps of one block only by block barriers,
the threads of one warp also by warp barriers.  Parity with the oracle (count,
instance count, witness and the witness's warp phases bit-exact) on the sort
path with interpreted and generated expansion, in chunked checks and in
batches (one interval table per model; a pack with such a model holds only
models of at most 16 intervals), and on the hash path (three groups per
instance)."""
import pytest
import torch

import oracle
import workloads as w
from workloads.spec import A, Access, Array, Loop, Model, Stmt, bid, const, it, tid, R, W

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


def compare(rc, model, opts=None):
    got = rc.check(model, opts)
    exp = oracle.check(model)
    assert got.status == exp.status, (model.name, got, exp)
    assert got.instances == exp.instances
    if exp.status == oracle.STATUS_OOB:
        assert (got.oob_stmt, got.oob_access, got.oob_gtid, got.oob_dim) == \
               (exp.oob_stmt, exp.oob_access, exp.oob_gtid, exp.oob_dim)
        return got
    assert (got.verdict, got.racy_cells) == (exp.verdict, exp.racy_cells), (model.name, got, exp)
    assert got.witness == exp.witness, (model.name, got.witness, exp.witness)
    if exp.verdict:
        assert (got.x_wphase, got.y_wphase) == (exp.x_wphase, exp.y_wphase)
    return got


@pytest.mark.parametrize("nw,bar,shared,exp", [(2, True, False, 0), (2, False, False, 30), (1, False, False, 15),
                                               (2, True, True, 16), (3, False, True, 16), (1, True, True, 0),
                                               (16, True, False, 0), (16, False, False, 240)])
def test_warp_reduction(rc, nw, bar, shared, exp):
    g = compare(rc, w.warp_reduction(n_warps=nw, warp_barriers=bar, shared_half=shared))
    assert g.racy_cells == exp


@pytest.mark.parametrize("nb,bs,grid,exp", [(4, 8, True, 0), (4, 8, False, 4), (1, 8, False, 0), (3, 33, False, 3),
                                            (256, 256, False, 256), (256, 256, True, 0)])
def test_grid_neighbor(rc, nb, bs, grid, exp):
    g = compare(rc, w.grid_neighbor(nb, bs, grid_barrier=grid))
    assert g.racy_cells == exp


@pytest.mark.parametrize("seed", range(150))
@pytest.mark.parametrize("jit", ["0", "1"])
def test_tiny_random_sync(rc, seed, jit, monkeypatch):
    monkeypatch.setenv("RC_JIT", jit)   # interpreted / generated expansion
    compare(rc, w.tiny_random_sync(seed))


@pytest.mark.parametrize("seed", range(30))
def test_tiny_random_sync_chunked(rc, seed):
    compare(rc, w.tiny_random_sync(seed), {"flags": rc.binding.RC_OPT_CHUNKED})


@pytest.mark.parametrize("gp", [[0, 0, 0], [0, 0, 1], [0, 1, 2]])
def test_long_cells(rc, gp):
    """Cells of tens of thousands of keys (the long-cell pass and the witness on them)."""
    c = Array("c", "global", (2,))
    lane0 = [-1 * (tid.x % 32)]
    stmts = [Stmt([Access(0, R, (const(0),))], phase=const(0), warp_phase=(tid.x // 32) % 2),
             Stmt([Access(0, A, (const(0),))], guards=lane0, phase=const(0), warp_phase=const(1)),
             Stmt([Access(0, W, (const(1),))], guards=lane0, phase=const(1), warp_phase=const(0)),
             Stmt([Access(0, R, (const(1),))], phase=const(2))]
    m = Model((200, 1, 1), (128, 1, 1), [c], stmts, n_phases=3, n_warp_phases=2, grid_phase=gp, name="sync_long")
    compare(rc, m)


def test_out_of_range_warp_phase(rc):
    m = Model((1, 1, 1), (64, 1, 1), [Array("s", "shared", (64,))],
              [Stmt([Access(0, W, (tid.x,))], warp_phase=tid.x // 32 + 1)], n_warp_phases=2, name="wp_oob")
    compare(rc, m)


def test_sync_models_beyond_phase_tables(rc):
    """20 fine intervals with warp barriers: the phase-order scan; the hash
    path is refused for them."""
    b = rc.binding
    many = Model((1, 1, 1), (64, 1, 1), [Array("s", "shared", (64,))],
                 [Stmt([Access(0, W, (tid.x,))], phase=const(0)),
                  Stmt([Access(0, R, ((tid.x + 32) % 64,))], phase=const(4), warp_phase=const(3))],
                 n_phases=5, n_warp_phases=4)
    assert b.rc_model_create_status(many) == b.RC_OK
    compare(rc, many)
    with pytest.raises(rc.RcError) as e:
        rc.check(many, {"path": 2})
    assert e.value.status == b.RC_E_UNSUPPORTED


# ---------------------------------------------------------------------------
# batches
# ---------------------------------------------------------------------------

def check_batch(rc, models, opts=None):
    b = rc.binding
    hs = [b.rc_model_create(m) for m in models]
    ws = b.workspace(b.rc_batch_workspace_size(hs, opts))
    got = b.rc_report(b.rc_check_batch(hs, opts, ws), wait=True)
    assert len(got) == len(models)
    for m, g in zip(models, got):
        exp = oracle.check(m)
        assert g.status == exp.status, (m.name, g, exp)
        assert g.instances == exp.instances, m.name
        if exp.status == oracle.STATUS_OOB:
            continue
        assert (g.verdict, g.racy_cells) == (exp.verdict, exp.racy_cells), (m.name, g, exp)
        assert g.witness == exp.witness, (m.name, g.witness, exp.witness)
        if exp.verdict:
            assert (g.x_wphase, g.y_wphase) == (exp.x_wphase, exp.y_wphase), m.name
    return got


def _interleave(*groups):
    out = []
    for i in range(max(len(g) for g in groups)):
        out += [g[i] for g in groups if i < len(g)]
    return out


@pytest.mark.parametrize("graph", [False, True])
def test_batch_mixed_sync_and_plain(rc, graph):
    """Models with warp / grid barriers, plain models and atomic models in one
    batch: every result equals the oracle's, warp phases of the witness included."""
    opts = {"flags": rc.binding.RC_OPT_GRAPH} if graph else None
    sync = [w.tiny_random_sync(s) for s in range(80)]
    plain = [w.tiny_random(s) for s in range(50)]
    atomic = [w.tiny_random(s, atomic=0.4) for s in range(20)]
    named = [w.warp_reduction(2, warp_barriers=False), w.warp_reduction(16, warp_barriers=True),
             w.warp_reduction(3, warp_barriers=False, shared_half=True), w.grid_neighbor(4, 8, grid_barrier=False),
             w.grid_neighbor(256, 256, grid_barrier=True), w.grid_neighbor(3, 33, grid_barrier=False),
             w.neighbor_write_read(64), w.reduction_tree(False)]
    models = _interleave(sync, plain, atomic, named)
    got = check_batch(rc, models, opts)
    assert sum(g.verdict for g in got) > 10


def test_batch_sync_with_many_phase_models(rc):
    """Models of more than 16 barrier intervals go to packs of their own."""
    many = [Model((2, 1, 1), (64, 1, 1), [Array("s", "shared", (64,))],
                  [Stmt([Access(0, W, ((tid.x + k + j) % 64,)), Access(0, R, ((tid.x + k + 1) % 64,))],
                        phase=const(k)) for k in range(20)], n_phases=20, name=f"many_phases_{j}")
            for j in range(4)]
    sync = [w.tiny_random_sync(s) for s in range(200, 212)]
    check_batch(rc, _interleave(sync, many))


def test_batch_sync_long_cells(rc):
    """Cells of tens of thousands of keys in a batch (the long-cell pass reads
    the tables of the cell's model)."""
    c = Array("c", "global", (2,))
    lane0 = [-1 * (tid.x % 32)]
    out = []
    for gp in ([0, 0, 0], [0, 0, 1], [0, 1, 2]):
        stmts = [Stmt([Access(0, R, (const(0),))], phase=const(0), warp_phase=(tid.x // 32) % 2),
                 Stmt([Access(0, A, (const(0),))], guards=lane0, phase=const(0), warp_phase=const(1)),
                 Stmt([Access(0, W, (const(1),))], guards=lane0, phase=const(1), warp_phase=const(0)),
                 Stmt([Access(0, R, (const(1),))], phase=const(2))]
        out.append(Model((200, 1, 1), (128, 1, 1), [c], stmts, n_phases=3, n_warp_phases=2, grid_phase=gp,
                         name=f"sync_long_{gp}"))
    check_batch(rc, _interleave(out, [w.tiny_random(s) for s in range(6)]))


def test_batch_sync_equals_single(rc):
    models = [w.tiny_random_sync(s) for s in range(300, 340)]
    got = check_batch(rc, models)
    for m, g in zip(models, got):
        assert g == rc.check(m), m.name


# ---------------------------------------------------------------------------
# hash path
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(120))
def test_tiny_random_sync_hash(rc, seed):
    """Count, instances and witness bit-exact without early exit."""
    compare(rc, w.tiny_random_sync(seed), {"path": rc.RC_PATH_HASH, "early_exit": 0})


@pytest.mark.parametrize("seed", range(40))
def test_tiny_random_sync_hash_early_exit(rc, seed):
    m = w.tiny_random_sync(seed)
    got = rc.check(m, {"path": rc.RC_PATH_HASH, "early_exit": 1})
    exp = oracle.check(m)
    assert got.status == exp.status, (m.name, got, exp)
    if exp.status == oracle.STATUS_OK:
        assert got.verdict == exp.verdict, m.name


@pytest.mark.parametrize("nw,bar,shared,exp", [(2, True, False, 0), (2, False, False, 30), (3, False, True, 16),
                                               (16, False, False, 240)])
def test_warp_reduction_hash(rc, nw, bar, shared, exp):
    g = compare(rc, w.warp_reduction(n_warps=nw, warp_barriers=bar, shared_half=shared),
                {"path": rc.RC_PATH_HASH, "early_exit": 0})
    assert g.racy_cells == exp


@pytest.mark.parametrize("nb,bs,grid,exp", [(4, 8, True, 0), (4, 8, False, 4), (256, 256, False, 256),
                                            (256, 256, True, 0)])
def test_grid_neighbor_hash(rc, nb, bs, grid, exp):
    g = compare(rc, w.grid_neighbor(nb, bs, grid_barrier=grid), {"path": rc.RC_PATH_HASH, "early_exit": 0})
    assert g.racy_cells == exp


@pytest.mark.parametrize("gp", [[0, 0, 0], [0, 0, 1], [0, 1, 2], [3, 3, 9]])
def test_long_cells_hash(rc, gp):
    """Hot cells (the hash words of one cell take every update) and grid
    intervals numbered sparsely by the descriptor."""
    c = Array("c", "global", (2,))
    lane0 = [-1 * (tid.x % 32)]
    stmts = [Stmt([Access(0, R, (const(0),))], phase=const(0), warp_phase=(tid.x // 32) % 2),
             Stmt([Access(0, A, (const(0),))], guards=lane0, phase=const(0), warp_phase=const(1)),
             Stmt([Access(0, W, (const(1),))], guards=lane0, phase=const(1), warp_phase=const(0)),
             Stmt([Access(0, R, (const(1),))], phase=const(2))]
    m = Model((200, 1, 1), (128, 1, 1), [c], stmts, n_phases=3, n_warp_phases=2, grid_phase=gp, name="sync_long_h")
    compare(rc, m, {"path": rc.RC_PATH_HASH, "early_exit": 0})
    compare(rc, m)


def test_batch_sync_hash_path(rc):
    """A batch on the hash path checks its models one by one."""
    models = [w.tiny_random_sync(s) for s in range(400, 430)] + [w.tiny_random(s) for s in range(10)]
    check_batch(rc, models, {"path": rc.RC_PATH_HASH, "early_exit": 0})


# ---------------------------------------------------------------------------
# witnesses above the cell's lowest block (several grid intervals)
# ---------------------------------------------------------------------------

LATE = [(3, 1), (5, 1), (2, 1), (2, 2), (3, 2), (4, 3), (7, 33), (64, 64)]


@pytest.mark.parametrize("nb,bs", LATE)
@pytest.mark.parametrize("path", ["sort", "hash", "chunked"])
def test_grid_late_partner(rc, nb, bs, path):
    """Block 0 reads before the grid barrier, the later blocks write after it:
    the smallest racing instance is block 1's write, not an instance of the
    cell's lowest block."""
    opts = {"sort": None, "hash": {"path": rc.RC_PATH_HASH, "early_exit": 0},
            "chunked": {"flags": rc.binding.RC_OPT_CHUNKED}}[path]
    g = compare(rc, w.grid_late_partner(nb, bs), opts)
    if (nb - 1) * bs >= 2:
        assert g.witness[3][0] == 1   # x in block 1


@pytest.mark.parametrize("seed", range(600))
def test_tiny_random_sync_block_guards(rc, seed):
    compare(rc, w.tiny_random_sync(seed, block_guards=True))


@pytest.mark.parametrize("seed", range(0, 600, 3))
def test_tiny_random_sync_block_guards_hash(rc, seed):
    compare(rc, w.tiny_random_sync(seed, block_guards=True), {"path": rc.RC_PATH_HASH, "early_exit": 0})


@pytest.mark.parametrize("graph", [False, True])
def test_batch_block_guards(rc, graph):
    """Models with several grid intervals (per-block witness records) share
    packs only with each other; mixed with other models in one batch."""
    opts = {"flags": rc.binding.RC_OPT_GRAPH} if graph else None
    guarded = [w.tiny_random_sync(s, block_guards=True) for s in range(200)]
    late = [w.grid_late_partner(nb, bs) for nb, bs in LATE]
    other = [w.tiny_random_sync(s) for s in range(40)] + [w.tiny_random(s) for s in range(40)]
    got = check_batch(rc, _interleave(guarded, late, other), opts)
    assert sum(g.verdict for g in got) > 100


# ---------------------------------------------------------------------------
# more than 16 fine intervals: keys sorted by (cell, fine interval), the
# phase-order scan (short cells per thread, long cells per block)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(200))
def test_many_intervals(rc, seed):
    compare(rc, w.tiny_random_sync(seed, many=True))


@pytest.mark.parametrize("seed", range(200))
def test_many_intervals_block_guards(rc, seed):
    compare(rc, w.tiny_random_sync(seed, block_guards=True, many=True))


@pytest.mark.parametrize("seed", range(100))
def test_many_intervals_atomics_without_scopes(rc, seed):
    compare(rc, w.tiny_random_sync(seed, many=True, scopes=False))


def test_many_intervals_generated_kernel(rc, monkeypatch):
    monkeypatch.setenv("RC_JIT", "1")
    for seed in range(0, 200, 7):
        compare(rc, w.tiny_random_sync(seed, many=True))
        compare(rc, w.tiny_random_sync(seed, block_guards=True, many=True))


def _interval_model(n_phases, n_wp, gp, blocks=64, racy=True):
    """A hot counter cell and a spread array over n_phases x n_wp fine
    intervals: every thread adds to c[0] in each barrier interval (warp
    interval = its warp mod n_wp), lane 0 of each warp reads c[0] (racy with
    the atomics of other warps in its block interval) unless `racy` is off,
    and every thread writes then reads its neighbour's cell of d."""
    c = Array("c", "global", (2,))
    d = Array("d", "global", (blocks * 128 + 1,))
    lane0 = [-1 * (tid.x % 32)]
    gtid = bid.x * 128 + tid.x
    stmts = [Stmt([Access(0, A, (const(0),))], loops=[Loop(0, n_phases)], phase=it(0),
                  warp_phase=(tid.x // 32) % n_wp),
             Stmt([Access(1, W, (gtid,))], phase=const(0), warp_phase=const(0)),
             Stmt([Access(1, R, (gtid + 1,))], phase=const(n_phases - 1), warp_phase=const(n_wp - 1))]
    if racy:
        stmts.append(Stmt([Access(0, R, (const(0),))], guards=lane0, loops=[Loop(0, n_phases)], phase=it(0),
                          warp_phase=const(0)))
    return Model((blocks, 1, 1), (128, 1, 1), [c, d], stmts, n_phases=n_phases, n_warp_phases=n_wp,
                 grid_phase=gp, name=f"intervals_{n_phases}x{n_wp}_{'racy' if racy else 'free'}")


@pytest.mark.parametrize("n_phases,n_wp", [(10, 2), (10, 4), (5, 8)])
@pytest.mark.parametrize("grid", ["none", "pairs", "each"])
@pytest.mark.parametrize("racy", [True, False])
def test_20_and_40_fine_intervals(rc, n_phases, n_wp, grid, racy):
    """20 and 40 fine intervals; the hot cell has 64 x 128 x n_phases keys
    (far above one thread's share: the long-cell pass)."""
    gp = {"none": [0] * n_phases, "pairs": [p // 2 for p in range(n_phases)], "each": list(range(n_phases))}[grid]
    compare(rc, _interval_model(n_phases, n_wp, gp, racy=racy))


def test_many_intervals_chunked(rc):
    for seed in range(0, 60, 3):
        m = w.tiny_random_sync(seed, many=True)
        compare(rc, m, {"flags": rc.binding.RC_OPT_CHUNKED})


def test_many_intervals_in_batches(rc):
    """Each model beyond 16 intervals holds its pack alone, beside packs of
    ordinary and phase-table models."""
    models = [w.tiny_random_sync(s, many=True) for s in range(30)] + [w.tiny_random_sync(s) for s in range(20)] + \
             [w.tiny_random_sync(s, many=True, scopes=False) for s in range(15)] + \
             [w.tiny_random(s) for s in range(10)] + [_interval_model(10, 4, [p // 2 for p in range(10)], blocks=8)]
    for graph in (False, True):
        check_batch(rc, models, {"flags": rc.binding.RC_OPT_GRAPH} if graph else None)
