"""The multi-process decomposition, on CPU: a model split by cell range gives
partial results whose merge equals the whole check (racy-cell counts add up,
the witness is the lowest racy range's), pinned with the oracle's partial
checks; the merge and the weak-scaling reduction across a world of 2 gloo
ranks (127.0.0.1)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import oracle
import workloads as w
from paper_2503_08946_gb300 import distributed as D


def models():
    return ([w.tiny_random(s) for s in range(0, 40, 3)] +
            [w.neighbor_write_read(64, n_blocks=2), w.reduction_tree(False, load_phase=True),
             w.polyhedral_product(9), w.transpose(pad=False, barrier=False, n=64),
             w.random_affine(3, n_blocks=2, block=64, n_stmts=8, plant=True)])


def whole(m):
    r = oracle.check(m)
    return (r.status, r.instances, r.verdict, r.racy_cells, r.witness)


def merged(m, k):
    total = oracle.cell_count(m)
    parts = [oracle.check_cells(m, lo, hi) for lo, hi in D.cell_ranges(total, k)]
    r = D.merge_results(parts)
    return (r.status, r.instances, r.verdict, r.racy_cells, r.witness)


def test_cell_ranges():
    for total in (0, 1, 7, 64, 1000003):
        for k in (1, 2, 3, 8):
            rs = D.cell_ranges(total, k)
            assert len(rs) == k and rs[0][0] == 0 and rs[-1][1] == total
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            sizes = [hi - lo for lo, hi in rs]
            assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("k", [2, 3, 7])
def test_partial_checks_merge_to_whole(k):
    for m in models():
        assert merged(m, k) == whole(m), m.name


@pytest.mark.parametrize("k", [2, 4, 8])
def test_hash_parts_merge_to_whole(k):
    """The hash parts of the check options partition the cells: the parts'
    distinct instances and racy cells add up to the whole check's, and the
    merge (the racy part with the smallest witness cell) gives its witness."""
    for m in models():
        parts = [oracle.check_part(m, k, r) for r in range(k)]
        a = oracle.check(m)
        r = D.merge_results(parts)
        assert (r.status, r.instances, r.verdict, r.racy_cells, r.witness) == whole(m), m.name
        if a.status == 0:
            assert sum(p.distinct for p in parts) == a.distinct, m.name


def test_hash_parts_are_balanced():
    """Each of k parts holds about 1/k of the keys of a regular access pattern."""
    m = w.neighbor_write_read(4096, n_blocks=4)
    for k in (2, 4, 8):
        d = [oracle.check_part(m, k, r).distinct for r in range(k)]
        assert max(d) <= 1.1 * sum(d) / k, (k, d)


@pytest.mark.parametrize("k", [1, 2, 3, 7, 16])
def test_parallel_oracle_equals_whole_check(k):
    """The all-cores oracle (cell ranges on std::thread workers) gives the full
    result of the single-threaded check, witness and instance counts included."""
    extra = [w.tiny_random_sync(s, block_guards=True) for s in range(0, 60, 7)] + \
            [w.tiny_random(s, atomic=0.4) for s in range(5)] + [w.grid_late_partner(4, 3)]
    for m in models() + extra:
        a, b = oracle.check(m), oracle.check_parallel(m, k)
        assert (a.status, a.instances, a.distinct, a.verdict, a.racy_cells, a.witness, a.x_wphase, a.y_wphase) == \
               (b.status, b.instances, b.distinct, b.verdict, b.racy_cells, b.witness, b.x_wphase, b.y_wphase), m.name


def test_parallel_oracle_reports_out_of_bounds():
    from workloads.spec import Access, Array, Model, Stmt, tid, W
    m = Model((2, 1, 1), (8, 1, 1), [Array("s", "shared", (4,))], [Stmt([Access(0, W, (tid.x,))])])
    a, b = oracle.check(m), oracle.check_parallel(m, 3)
    assert a.status == b.status == oracle.STATUS_OOB
    assert (a.oob_stmt, a.oob_access, a.oob_gtid, a.oob_dim) == (b.oob_stmt, b.oob_access, b.oob_gtid, b.oob_dim)


def test_merge_keeps_errors():
    from paper_2503_08946_gb300 import binding as B
    ok = B.Result(0, 1, 3, 10, 0, 0, 5, (0, 0, 1, 0), (0, 0, 2, 1), 0, 0, 0, 0)
    bad = B.Result(B.RC_E_OOB, 0, 0, 10, 0, 0, 0, (0, 0, 0, 0), (0, 0, 0, 0), 1, 0, 7, 1)
    assert D.merge_results([ok, bad]).status == B.RC_E_OOB
    quiet = B.Result(0, 0, 0, 10, 0, 0, 0, (0, 0, 0, 0), (0, 0, 0, 0), 0, 0, 0, 0)
    r = D.merge_results([quiet, ok, ok])
    assert (r.racy_cells, r.verdict, r.witness) == (6, 1, ok.witness)


def test_partition_opts(monkeypatch):
    """A rank's split options: its hash part when the world is a power of two
    (the default), else its cell range; the caller's options are kept and not
    changed; an empty range keeps no cell."""
    from paper_2503_08946_gb300 import binding as B
    monkeypatch.setattr(B, "rc_model_layout", lambda model: {"total_cells": 10})
    base = {"early_exit": 0}
    for k in (1, 2, 4, 8):
        for r in range(k):
            assert D.partition_opts(None, r, k, base) == {"early_exit": 0, "part_count": k, "part_index": r}
    assert base == {"early_exit": 0}
    got = [D.partition_opts(None, r, 3) for r in range(3)]
    assert [(o["cell_lo"], o["cell_hi"]) for o in got] == [(0, 4), (4, 7), (7, 10)]
    assert D.partition_opts(None, 1, 2, by="range") == {"cell_lo": 5, "cell_hi": 10}
    # more ranks than cells: one cell each for the first ten, a range past the
    # last cell for the rest (cell_hi = 0 would mean every cell)
    rs = [D.partition_opts(None, r, 12, by="range") for r in range(12)]
    assert [(o["cell_lo"], o["cell_hi"]) for o in rs[:10]] == [(c, c + 1) for c in range(10)]
    assert all(o["cell_hi"] > o["cell_lo"] >= 10 for o in rs[10:])
    with pytest.raises(ValueError):
        D.partition_opts(None, 0, 3, by="hash")
    with pytest.raises(ValueError):
        D.partition_opts(None, 0, 2, by="cells")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        for m in models():
            lo, hi = D.cell_ranges(oracle.cell_count(m), world)[rank]
            part = oracle.check_cells(m, lo, hi)
            r = D.all_merge(part)
            assert (r.status, r.instances, r.verdict, r.racy_cells, r.witness) == whole(m), m.name
        total, ms, rate = D.weak_scaling_rate(1e9 * (rank + 1), 100.0 * (rank + 1))
        assert total == 3e9 and ms == 200.0 and abs(rate - 15.0) < 1e-9
    finally:
        dist.destroy_process_group()


def test_gloo_world_of_two():
    oracle.build()
    mp.spawn(_worker, args=(2, _free_port()), nprocs=2, join=True)
