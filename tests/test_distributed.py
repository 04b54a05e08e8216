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


def test_merge_keeps_errors():
    from paper_2503_08946_gb300 import binding as B
    ok = B.Result(0, 1, 3, 10, 0, 0, 5, (0, 0, 1, 0), (0, 0, 2, 1), 0, 0, 0, 0)
    bad = B.Result(B.RC_E_OOB, 0, 0, 10, 0, 0, 0, (0, 0, 0, 0), (0, 0, 0, 0), 1, 0, 7, 1)
    assert D.merge_results([ok, bad]).status == B.RC_E_OOB
    quiet = B.Result(0, 0, 0, 10, 0, 0, 0, (0, 0, 0, 0), (0, 0, 0, 0), 0, 0, 0, 0)
    r = D.merge_results([quiet, ok, ok])
    assert (r.racy_cells, r.verdict, r.witness) == (6, 1, ok.witness)


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
