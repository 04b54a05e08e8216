"""Pins of the CPU oracle against facts that do not come from the oracle itself:
closed forms derived by hand (tests/golden/closed_forms.md), the verdict the
paper states for Ge-SpMM (tests/golden/paper_verdicts.json), an independent
pure-Python pairwise brute force on tiny random models, and invariances of the
race definition (thread relabelling, statement order, array padding)."""
import copy
import json
import os

import pytest

import oracle
import workloads as w
from workloads.spec import Expr

from . import pyref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def wit(r):
    return r.witness


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------

@pytest.mark.parametrize("T", [2, 3, 8, 33, 256])
def test_neighbor_write_read(T):
    r = oracle.check(w.neighbor_write_read(T))
    assert r.status == 0 and r.verdict == 1
    assert r.racy_cells == T - 1
    # first racy cell s[1]: thread 0 reads it, thread 1 writes it
    assert wit(r) == (0, 0, 1, (0, 0, 0, 0), (0, 0, 1, 1))


def test_neighbor_write_read_multi_block():
    r = oracle.check(w.neighbor_write_read(16, n_blocks=5))
    assert r.racy_cells == 5 * 15


def test_reduction_tree():
    bar = oracle.check(w.reduction_tree(True))
    assert (bar.status, bar.verdict, bar.racy_cells, bar.instances) == (0, 0, 0, 765)
    nob = oracle.check(w.reduction_tree(False))
    assert (nob.verdict, nob.racy_cells, nob.instances) == (1, 127, 765)
    assert wit(nob) == (0, 0, 1, (0, 0, 0, 0), (0, 0, 1, 1))
    ld = oracle.check(w.reduction_tree(False, load_phase=True))
    assert (ld.verdict, ld.racy_cells, ld.instances) == (1, 255, 1277)
    assert wit(ld) == (0, 0, 1, (0, 0, 0, 0), (0, 0, 1, 1))
    ldb = oracle.check(w.reduction_tree(True, load_phase=True))
    assert ldb.racy_cells == 0


@pytest.mark.parametrize("n", [2, 3, 4, 7, 12])
def test_polyhedral_product(n):
    r = oracle.check(w.polyhedral_product(n))
    assert r.racy_cells == 2 * n - 3
    assert r.verdict == 1
    # first racy cell C[1]: (thread 0, R) then its first partner (thread 1, W)
    assert wit(r) == (2, 0, 1, (0, 0, 0, 0), (0, 0, 1, 1))
    r2 = oracle.check(w.polyhedral_product(n, init_stmt=True))
    assert r2.racy_cells == 2 * n - 3


@pytest.mark.parametrize("pad", [False, True])
def test_transpose_small(pad):
    m_bar = w.transpose(pad=pad, barrier=True, n=256)
    m_nob = w.transpose(pad=pad, barrier=False, n=256)
    blocks = (256 // 32) ** 2
    rb = oracle.check(m_bar)
    assert (rb.verdict, rb.racy_cells, rb.instances) == (0, 0, 2 * 2 * 4 * 256 * blocks)
    rn = oracle.check(m_nob)
    assert rn.racy_cells == 992 * blocks
    # tile (array 2) of block 0, element 1: written by t1, read by t32
    assert wit(rn) == (2, 0, 1, (0, 0, 1, 1), (0, 0, 32, 0))


def test_transpose_full_size():
    r = oracle.check(w.transpose(pad=False, barrier=False))
    assert r.instances == 16777216
    assert r.racy_cells == 4063232
    assert wit(r) == (2, 0, 1, (0, 0, 1, 1), (0, 0, 32, 0))


@pytest.mark.parametrize("L", [1, 31, 32, 33, 70, 100])
def test_ge_spmm(L):
    golden = json.load(open(os.path.join(GOLDEN, "paper_verdicts.json")))
    assert golden["ge_spmm_algorithm2"]["expected_race_free"] is True
    M, N, K = 3, 64, 4
    r = oracle.check(w.ge_spmm_uniform(M, N, K, L, trailing_barrier=True))
    assert r.status == 0 and r.verdict == 0 and r.racy_cells == 0
    r2 = oracle.check(w.ge_spmm_uniform(M, N, K, L, trailing_barrier=False))
    assert r2.racy_cells == 2 * min(32, max(0, L - 32)) * M * (N // 32)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_affine_construction(seed):
    clean = w.random_affine(seed, n_blocks=8, block=64, n_stmts=20, plant=False)
    r = oracle.check(clean)
    assert r.status == 0 and r.racy_cells == 0
    planted = w.random_affine(seed, n_blocks=8, block=64, n_stmts=20, plant=True)
    rp = oracle.check(planted)
    assert rp.racy_cells == 8 * 64


# --------------------------------------------------------------------------
# independent brute force on tiny random models
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(150))
def test_tiny_random_vs_python_bruteforce(seed):
    m = w.tiny_random(seed)
    st, cnt, best = pyref.check(m)
    r = oracle.check(m)
    rb = oracle.brute(m)
    assert st == "ok"
    assert r.status == 0 and rb.status == 0
    assert r.racy_cells == cnt == rb.racy_cells
    assert r.verdict == (cnt > 0)
    inst, _ = pyref.instances(m)
    assert r.instances == len(inst) and r.distinct == len(set(inst))
    if best is None:
        assert r.witness is None
    else:
        x, y = best
        exp = (x[0], x[1], x[2], (x[3], x[4], x[5], x[6]), (y[3], y[4], y[5], y[6]))
        assert r.witness == exp
        assert rb.witness == exp


def test_oracle_expand_matches_python():
    for seed in range(20):
        m = w.tiny_random(seed)
        inst, _ = pyref.instances(m)
        got = [tuple(int(v) for v in row) for row in oracle.expand(m)]
        assert got == sorted(inst)


def test_out_of_bounds_reported():
    from workloads.spec import Access, Array, Model, Stmt, tid, R, W
    m = Model((2, 1, 1), (8, 1, 1), [Array("a", "global", (10,))],
              [Stmt([Access(0, R, (tid.x,))]), Stmt([Access(0, W, (tid.x + 3,))])])
    st, rec, _ = pyref.check(m)
    r = oracle.check(m)
    assert st == "oob" and r.status == oracle.STATUS_OOB
    assert (r.oob_stmt, r.oob_access, r.oob_gtid, r.oob_dim) == rec == (1, 0, 7, 1)
    # an interval outside [0, n_phases)
    m2 = Model((1, 1, 1), (4, 1, 1), [Array("a", "shared", (4,))],
               [Stmt([Access(0, W, (tid.x,))], phase=w.const(2))], n_phases=2)
    r2 = oracle.check(m2)
    assert r2.status == oracle.STATUS_OOB and (r2.oob_stmt, r2.oob_access, r2.oob_gtid, r2.oob_dim) == (0, 0, 0, 0)


def test_invalid_text():
    r = oracle.check_text("rcmodel 1 grid 1 1")
    assert r.status == oracle.STATUS_INVALID


# --------------------------------------------------------------------------
# invariances
# --------------------------------------------------------------------------

def _subst_tid_x(e: Expr, f):
    if e.op == "tid" and e.args[0] == 0:
        return f
    if e.op in ("add",):
        return Expr("add", _subst_tid_x(e.args[0], f), _subst_tid_x(e.args[1], f))
    if e.op == "mul":
        return Expr("mul", e.args[0], _subst_tid_x(e.args[1], f))
    if e.op in ("fdiv", "mod"):
        return Expr(e.op, _subst_tid_x(e.args[0], f), e.args[1])
    return e


def _relabel(m, a, c):
    """Model whose thread x behaves like thread (a*x + c) mod blockDim.x of m
    (a coprime to blockDim.x, so this is a permutation of each block's threads)."""
    import copy
    m2 = copy.deepcopy(m)
    f = (a * w.tid.x + c) % m.block[0]
    for st in m2.stmts:
        st.phase = _subst_tid_x(st.phase, f)
        st.guards = [_subst_tid_x(g, f) for g in st.guards]
        for lp in st.loops:
            lp.lower = _subst_tid_x(lp.lower, f)
            lp.upper = _subst_tid_x(lp.upper, f)
        for ac in st.accesses:
            ac.index = tuple(_subst_tid_x(e, f) for e in ac.index)
    return m2


@pytest.mark.parametrize("seed", range(3))
def test_thread_relabelling_keeps_verdict_and_count(seed):
    for m in [w.random_affine(seed, n_blocks=4, block=64, n_stmts=12, plant=(seed == 1)),
              w.reduction_tree(False), w.neighbor_write_read(32), w.tiny_random(seed)]:
        r = oracle.check(m)
        for a in (1, 3, 5, 7):
            if m.block[0] % a == 0 and a != 1:
                continue
            import math
            if math.gcd(a, m.block[0]) != 1:
                continue
            r2 = oracle.check(_relabel(m, a, 1))
            assert (r2.verdict, r2.racy_cells, r2.instances) == (r.verdict, r.racy_cells, r.instances)


@pytest.mark.parametrize("seed", range(5))
def test_statement_order_keeps_everything(seed):
    import copy
    for m in [w.random_affine(seed, n_blocks=4, block=32, n_stmts=10, plant=True), w.tiny_random(seed + 40)]:
        r = oracle.check(m)
        m2 = copy.deepcopy(m)
        m2.stmts = list(reversed(m2.stmts))
        r2 = oracle.check(m2)
        assert (r2.verdict, r2.racy_cells, r2.instances, r2.distinct, r2.witness) == \
               (r.verdict, r.racy_cells, r.instances, r.distinct, r.witness)


def test_padding_keeps_count():
    for bar in (True, False):
        a = oracle.check(w.transpose(pad=False, barrier=bar, n=128))
        b = oracle.check(w.transpose(pad=True, barrier=bar, n=128))
        assert a.racy_cells == b.racy_cells


# --------------------------------------------------------------------------
# planted mistakes must be caught by the pins above (run on the CPU only)
# --------------------------------------------------------------------------

def test_pins_detect_planted_mistake():
    """A model whose race definition drops the 'different threads' clause (as a
    buggy checker would) must disagree with the pairwise brute force."""
    m = w.reduction_tree(True)
    inst, _ = pyref.instances(m)
    u = sorted(set(inst))
    # buggy predicate: same cell, a write, same interval -- forgets gtid_x != gtid_y
    buggy = set()
    for i in range(len(u)):
        for j in range(i + 1, len(u)):
            x, y = u[i], u[j]
            if x[:3] == y[:3] and (x[6] or y[6]) and x[4] == y[4]:
                buggy.add(x[:3])
    assert len(buggy) > 0 and oracle.check(m).racy_cells == 0


# --------------------------------------------------------------------------
# data-dependent values: table loads (CSR row bounds of Ge-SpMM)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(120))
def test_tiny_tables_vs_python_bruteforce(seed):
    """Tiny models whose bounds, guards and indices read integer tables."""
    m = w.tiny_random_tables(seed)
    st, cnt, best = pyref.check(m)
    r = oracle.check(m)
    rb = oracle.brute(m)
    assert st == "ok" and r.status == 0 and rb.status == 0
    assert r.racy_cells == cnt == rb.racy_cells
    inst, _ = pyref.instances(m)
    assert r.instances == len(inst) and r.distinct == len(set(inst))
    if best is None:
        assert r.witness is None
    else:
        x, y = best
        assert r.witness == (x[0], x[1], x[2], (x[3], x[4], x[5], x[6]), (y[3], y[4], y[5], y[6]))


def test_table_reads_zero_outside():
    """for i < T[t]: W s[i] with T = [3, 1, 4] and 8 threads: threads 3..7 read
    0 (outside the table) and run no iteration; 8 instances; cells 0, 1, 2 are
    written by >= 2 threads, cell 3 by one."""
    from workloads.spec import Access, Array, Loop, Model, Stmt, W, it, load, tid
    m = Model((1, 1, 1), (8, 1, 1), [Array("s", "shared", (8,))],
              [Stmt([Access(0, W, (it(0),))], loops=[Loop(0, load(0, tid.x))])], tables=[[3, 1, 4]])
    r = oracle.check(m)
    assert (r.status, r.instances, r.racy_cells) == (0, 8, 3)
    assert r.witness == (0, 0, 0, (0, 0, 0, 1), (0, 0, 1, 1))


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("bar", [True, False])
def test_gespmm_csr_closed_form(seed, bar):
    """Ge-SpMM on a skewed CSR (row bounds loaded from rowPtr): race-free with
    the barrier after T (the paper's expected verdict for Ge-SpMM); without it
    2 * min(32, max(0, L_i - 32)) racy shared cells per block row and slab."""
    lens = w.csr_row_lengths(seed, 12, max_len=150)
    m = w.ge_spmm_csr(lens, N=64, K=3, trailing_barrier=bar)
    r = oracle.check(m)
    exp = 0 if bar else (64 // 32) * sum(2 * min(32, max(0, L - 32)) for L in lens)
    assert r.status == 0 and r.racy_cells == exp


@pytest.mark.parametrize("L", [1, 32, 33, 70])
def test_gespmm_csr_uniform_rows_equal_uniform_model(L):
    for bar in (True, False):
        a = oracle.check(w.ge_spmm_uniform(3, 64, 4, L, trailing_barrier=bar))
        b = oracle.check(w.ge_spmm_csr([L] * 3, 64, 4, trailing_barrier=bar))
        assert (a.status, a.instances, a.racy_cells, a.witness) == (b.status, b.instances, b.racy_cells, b.witness)


# --------------------------------------------------------------------------
# atomics: an atomic conflicts with plain reads and writes, not with atomics
# --------------------------------------------------------------------------

@pytest.mark.parametrize("T,B,nb,bar,rb,plain,exp", [
    (8, 4, 1, False, True, False, 4),     # two threads per bin: update vs read-back
    (8, 4, 3, False, True, False, 12),
    (8, 4, 1, True, True, False, 0),      # the barrier orders update and read-back
    (4, 4, 1, False, True, False, 0),     # one thread per bin
    (8, 4, 1, False, False, False, 0),    # atomics alone never race
    (64, 8, 2, False, False, False, 0),
    (8, 4, 1, True, True, True, 4),       # plain read-modify-write updates race
])
def test_atomic_histogram_closed_form(T, B, nb, bar, rb, plain, exp):
    m = w.atomic_histogram(T, B, n_blocks=nb, barrier=bar, read_back=rb, plain=plain)
    r = oracle.check(m)
    assert r.racy_cells == exp
    assert pyref.check(m)[1] == exp
    assert oracle.brute(m).racy_cells == exp


@pytest.mark.parametrize("T,nb,bar,exp", [(4, 1, True, 0), (4, 1, False, 1), (4, 2, True, 1), (1, 1, False, 0),
                                          (1, 3, True, 1)])
def test_atomic_counter_closed_form(T, nb, bar, exp):
    m = w.atomic_counter(T, n_blocks=nb, barrier=bar)
    assert oracle.check(m).racy_cells == exp
    assert pyref.check(m)[1] == exp


def test_atomic_counter_witness():
    # one block, no barrier: thread 0's read (R) races with thread 1's increment (A)
    r = oracle.check(w.atomic_counter(4, n_blocks=1, barrier=False))
    assert r.witness == (0, 0, 0, (0, 0, 0, 0), (0, 0, 1, 2))


@pytest.mark.parametrize("seed", range(120))
def test_tiny_random_atomic_vs_python_bruteforce(seed):
    m = w.tiny_random(seed, atomic=0.4)
    st, cnt, best = pyref.check(m)
    r = oracle.check(m)
    rb = oracle.brute(m)
    assert st == "ok" and r.status == 0
    assert r.racy_cells == cnt == rb.racy_cells
    if best is None:
        assert r.witness is None
    else:
        x, y = best
        exp = (x[0], x[1], x[2], (x[3], x[4], x[5], x[6]), (y[3], y[4], y[5], y[6]))
        assert r.witness == exp == rb.witness


def test_atomic_large_cell_witness():
    """The oracle's summary witness path (cells of more than 4096 instances)
    agrees with the pair-by-pair definition."""
    for m, exp in [(w.atomic_counter(1024, n_blocks=6, barrier=True), 1),
                   (w.atomic_counter(1024, n_blocks=1, barrier=False), 1),
                   (w.atomic_histogram(1024, 1, n_blocks=5, barrier=False), 5)]:   # one shared bin per block
        r, rb = oracle.check(m), oracle.brute(m)
        assert r.racy_cells == rb.racy_cells == exp
        assert r.witness == rb.witness


# --------------------------------------------------------------------------
# warp and grid barriers: blocks are ordered only by grid barriers, two warps
# of one block only by block barriers, the threads of one warp also by warp
# barriers
# --------------------------------------------------------------------------

@pytest.mark.parametrize("nw,bar,shared,exp", [
    (2, True, False, 0),      # warp barriers order the stages inside each warp
    (2, False, False, 30),    # 15 cells per warp without them
    (1, False, False, 15),
    (2, True, True, 16),      # warps meet on cells 0..15: warp barriers do not order warps
    (3, False, True, 16),
    (1, True, True, 0),
])
def test_warp_reduction_closed_form(nw, bar, shared, exp):
    m = w.warp_reduction(n_warps=nw, warp_barriers=bar, shared_half=shared)
    assert oracle.check(m).racy_cells == exp
    assert pyref.check(m)[1] == exp
    assert oracle.brute(m).racy_cells == exp


@pytest.mark.parametrize("nb,bs,grid,exp", [(4, 8, True, 0), (4, 8, False, 4), (1, 8, False, 0), (3, 33, False, 3),
                                            (3, 33, True, 0)])
def test_grid_neighbor_closed_form(nb, bs, grid, exp):
    m = w.grid_neighbor(nb, bs, grid_barrier=grid)
    assert oracle.check(m).racy_cells == exp
    assert pyref.check(m)[1] == exp


def test_grid_neighbor_witness():
    # cell 0: written by block 0's thread 0 in interval 0, read by block 1's last
    # thread (gtid 15, (15 + 1) mod 16 = 0) in interval 1 -- one grid interval
    r = oracle.check(w.grid_neighbor(2, 8, grid_barrier=False))
    assert r.witness == (0, 0, 0, (0, 0, 0, 1), (1, 1, 7, 0))


@pytest.mark.parametrize("nb,bs", [(3, 1), (5, 1), (2, 1), (2, 2), (3, 2), (4, 3), (7, 33)])
def test_grid_late_partner_closed_form(nb, bs):
    """The smallest racing instance lies outside the cell's lowest block: block
    0 reads before the grid barrier, the later blocks write after it
    (tests/golden/closed_forms.md)."""
    m = w.grid_late_partner(nb, bs)
    r, rb = oracle.check(m), oracle.brute(m)
    racy = (nb - 1) * bs >= 2
    assert r.racy_cells == rb.racy_cells == (1 if racy else 0)
    if not racy:
        assert r.witness is None and rb.witness is None
        return
    y = (1, 1, 1, 1) if bs >= 2 else (2, 1, 0, 1)
    assert r.witness == rb.witness == (0, 0, 0, (1, 1, 0, 1), y)
    st, cnt, best = pyref.check(m)
    assert cnt == 1 and best[0][3:7] == (1, 1, 0, 1) and best[1][3:7] == y


def _x_outside_lowest_block(m, best):
    """The pairwise reference's smallest racing instance lies in a block above
    the lowest block of its cell."""
    if best is None:
        return False
    x = best[0]
    insts, _ = pyref.instances(m)
    return x[3] != min(i[3] for i in insts if i[:3] == x[:3])


@pytest.mark.parametrize("seed", range(600))
def test_tiny_random_sync_block_guards_vs_python_bruteforce(seed):
    """Statements limited to some blocks (and threads), mostly global cells and
    grid barriers: the witness may lie above the cell's lowest block."""
    m = w.tiny_random_sync(seed, block_guards=True)
    st, cnt, best = pyref.check(m)
    r, rb = oracle.check(m), oracle.brute(m)
    assert st == "ok" and r.status == 0
    assert r.racy_cells == cnt == rb.racy_cells
    if best is None:
        assert r.witness is None
    else:
        x, y = best
        assert r.witness == (x[0], x[1], x[2], x[3:7], y[3:7]) == rb.witness
        if len(x) == 8:   # (the reference adds warp phases only to models with such barriers)
            assert (r.x_wphase, r.y_wphase) == (x[7], y[7]) == (rb.x_wphase, rb.y_wphase)


def test_block_guard_models_reach_the_late_witness():
    """The block-guarded generator produces the shape above often enough for
    the GPU tests over the same seeds to exercise it."""
    hits = [s for s in range(600) if _x_outside_lowest_block(w.tiny_random_sync(s, block_guards=True),
                                                              pyref.check(w.tiny_random_sync(s, block_guards=True))[2])]
    assert len(hits) >= 6, hits


@pytest.mark.parametrize("seed", range(150))
def test_tiny_random_sync_vs_python_bruteforce(seed):
    m = w.tiny_random_sync(seed)
    st, cnt, best = pyref.check(m)
    r, rb = oracle.check(m), oracle.brute(m)
    assert st == "ok" and r.status == 0
    assert r.racy_cells == cnt == rb.racy_cells
    if best is None:
        assert r.witness is None
    else:
        x, y = best
        assert r.witness == (x[0], x[1], x[2], x[3:7], y[3:7]) == rb.witness
        if len(x) == 8:
            assert (r.x_wphase, r.y_wphase) == (x[7], y[7]) == (rb.x_wphase, rb.y_wphase)


def test_sync_large_cell_witness():
    """The summary witness path (more than 4096 instances in the cell) with
    warp and grid barriers agrees with the pair-by-pair definition."""
    from workloads.spec import Access, Array, Model, Stmt, const, tid, R, W, A
    c = Array("c", "global", (2,))
    lane0 = [-1 * (tid.x % 32)]
    stmts = [Stmt([Access(0, R, (const(0),))], phase=const(0), warp_phase=(tid.x // 32) % 2),
             Stmt([Access(0, A, (const(0),))], guards=lane0, phase=const(0), warp_phase=const(1)),
             Stmt([Access(0, W, (const(1),))], guards=lane0, phase=const(1), warp_phase=const(0)),
             Stmt([Access(0, R, (const(1),))], phase=const(2))]
    for gp in ([0, 0, 0], [0, 0, 1], [0, 1, 2]):
        m = Model((40, 1, 1), (128, 1, 1), [c], stmts, n_phases=3, n_warp_phases=2, grid_phase=gp)
        r, rb = oracle.check(m), oracle.brute(m)
        assert r.racy_cells == rb.racy_cells
        assert r.witness == rb.witness and (r.x_wphase, r.y_wphase) == (rb.x_wphase, rb.y_wphase)


@pytest.mark.parametrize("seed", range(40))
def test_grid_interval_numbering_is_immaterial(seed):
    """Grid intervals matter only through equality: renumbering them with
    gaps (order kept) changes no result, in the oracle or the pairwise
    reference (the CUDA lowering numbers them densely)."""
    import dataclasses
    m = w.tiny_random_sync(seed)
    if m.grid_phase is None:
        pytest.skip("no grid barriers")
    sparse = [3 * g + 2 for g in m.grid_phase]
    m2 = dataclasses.replace(m, grid_phase=sparse, name=m.name + "_sparse")
    r, r2 = oracle.check(m), oracle.check(m2)
    assert (r.status, r.racy_cells, r.witness, r.x_wphase, r.y_wphase) == \
           (r2.status, r2.racy_cells, r2.witness, r2.x_wphase, r2.y_wphase)
    # (the reference adds a warp-phase field to its pairs when a model has grid
    # or warp barriers, and an all-zero grid list has none: compare 7 fields)
    (st, cnt, best), (st2, cnt2, best2) = pyref.check(m), pyref.check(m2)
    assert (st, cnt) == (st2, cnt2)
    assert (best is None) == (best2 is None)
    if best is not None:
        if len(best[0]) == len(best2[0]):
            assert best == best2
        else:   # one warp interval: the added field is warp phase 0
            assert (best[0][:7], best[1][:7]) == (best2[0][:7], best2[1][:7])
            assert best2[0][7:] == best2[1][7:] == (0,)


# --------------------------------------------------------------------------
# the superset domain: tables whose values are unknown (free parameters)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(4))
def test_superset_gespmm_race_free(seed):
    """The paper's verdict for Ge-SpMM holds on its superset domain: with rs,
    re free over [0, nnz] and the barriers after F and after T, no race."""
    golden = json.load(open(os.path.join(GOLDEN, "paper_verdicts.json")))["ge_spmm_superset"]
    lens = w.csr_row_lengths(seed, 3, max_len=24)
    r = oracle.check(w.ge_spmm_csr(lens, N=32, K=2, trailing_barrier=True, superset=True))
    assert r.status == 0
    assert (r.verdict == 0) == golden["expected_race_free"]


@pytest.mark.parametrize("lens", [[3, 20, 7, 10], [32, 1, 0], [12, 12, 12]])
def test_superset_gespmm_false_positive_closed_form(lens):
    """Without the trailing barrier and with every row at most 32 long, the
    concrete model is race-free (one chunk per row), but on the superset
    domain re - rs may exceed 32: F of chunk 1 writes sm_k[c] / sm_v[c] (c <
    nnz - 32) in the interval where T of chunk 0 reads them, so every block
    has 2 * min(32, nnz - 32) racy shared cells.  The first: sm_k[0] of block
    0, written by thread 0 (F, chunk 1) and read by thread 1 (T, chunk 0) in
    interval 1."""
    nnz, M = sum(lens), len(lens)
    conc = oracle.check(w.ge_spmm_csr(lens, N=32, K=1, trailing_barrier=False))
    sup = oracle.check(w.ge_spmm_csr(lens, N=32, K=1, trailing_barrier=False, superset=True))
    assert (conc.status, conc.racy_cells) == (0, 0)
    assert sup.status == 0 and sup.racy_cells == 2 * min(32, max(0, nnz - 32)) * M
    assert sup.witness == (5, 0, 0, (0, 1, 0, 1), (0, 1, 1, 0))


@pytest.mark.parametrize("n", [2, 3, 17, 64])
def test_superset_permutation_scatter_closed_form(n):
    """out[perm[t]] = ... is race-free for a permutation; with perm's values
    unknown in [0, n-1] every thread may write every cell: n racy cells, n^2
    instances, witness cell 0 written by threads 0 and 1."""
    conc = oracle.check(w.permutation_scatter(n, seed=n))
    sup = oracle.check(w.permutation_scatter(n, seed=n, superset=True))
    assert (conc.status, conc.racy_cells, conc.instances) == (0, 0, n)
    assert (sup.status, sup.racy_cells, sup.instances) == (0, n, n * n)
    assert sup.witness == (0, 0, 0, (0, 0, 0, 1), (0, 0, 1, 1))


@pytest.mark.parametrize("seed", range(80))
def test_superset_of_one_value_is_the_concrete_model(seed):
    """A free parameter whose range is the single value 0 is a load that reads
    0: the superset model with range [0, 0] equals the concrete model with
    empty tables (every load reads 0 outside its table), field for field."""
    base = w.tiny_random_tables(seed)
    zero = copy.deepcopy(base)
    zero.tables = [[] for _ in base.tables]
    one = copy.deepcopy(base)
    one.superset = {t: (0, 0) for t in range(len(base.tables))}
    a, b = oracle.check(zero), oracle.check(one)
    assert a == b


@pytest.mark.parametrize("seed", range(150))
def test_superset_contains_the_concrete_model(seed):
    """Table 0's range holds every value it gives (and 0), so the concrete
    instances are a subset of the superset's: at least as many instances and
    racy cells, and a concrete race is a superset race."""
    c = oracle.check(w.tiny_random_tables(seed))
    s = oracle.check(w.tiny_random_tables(seed, superset=True))
    if c.status == 0 and s.status == 0:
        assert s.instances >= c.instances and s.racy_cells >= c.racy_cells
        assert s.verdict >= c.verdict
    if c.status == oracle.STATUS_OOB:
        assert s.status == oracle.STATUS_OOB


@pytest.mark.parametrize("seed", range(200))
def test_superset_tiny_tables_vs_python_bruteforce(seed):
    m = w.tiny_random_tables(seed, superset=True)
    r = oracle.check(m)
    if r.instances > 4000:
        pytest.skip("too large for the pairwise check")
    st, cnt, best = pyref.check(m)
    if st == "oob":
        assert r.status == oracle.STATUS_OOB
        assert (r.oob_stmt, r.oob_access, r.oob_gtid, r.oob_dim) == cnt
        return
    assert r.status == 0 and r.racy_cells == cnt
    inst, _ = pyref.instances(m)
    assert r.instances == len(inst) and r.distinct == len(set(inst))
    if best is None:
        assert r.witness is None
    else:
        x, y = best
        assert r.witness == (x[0], x[1], x[2], (x[3], x[4], x[5], x[6]), (y[3], y[4], y[5], y[6]))


# --------------------------------------------------------------------------
# more than 16 fine intervals with warp / grid barriers or atomics
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(120))
@pytest.mark.parametrize("kind", ["many", "many_bg", "noscopes"])
def test_tiny_random_sync_many_intervals_vs_python_bruteforce(seed, kind):
    m = w.tiny_random_sync(seed, block_guards=kind == "many_bg", many=True, scopes=kind != "noscopes")
    assert m.n_phases * m.n_warp_phases > 16
    r = oracle.check(m)
    if r.instances > 6000:
        pytest.skip("too large for the pairwise check")
    st, cnt, best = pyref.check(m)
    rb = oracle.brute(m)
    assert st == "ok" and r.status == 0
    assert r.racy_cells == cnt == rb.racy_cells
    if best is None:
        assert r.witness is None
    else:
        x, y = best
        assert r.witness == (x[0], x[1], x[2], x[3:7], y[3:7]) == rb.witness
        if len(x) == 8:
            assert (r.x_wphase, r.y_wphase) == (x[7], y[7]) == (rb.x_wphase, rb.y_wphase)
