"""One model checked as k cell-range partitions on one GPU (the per-rank work
of a multi-GPU split, emulated sequentially): the merged partial results equal
the whole check and the oracle, on the sort path (interpreted and generated
expansion) and the hash path."""
import pytest

import oracle
import workloads as w
from paper_2503_08946_gb300 import distributed as D

from .test_gpu_parity import rc  # noqa: F401  (module fixture)

pytestmark = pytest.mark.gpu


def models():
    return ([w.tiny_random(s) for s in range(900, 930)] +
            [w.neighbor_write_read(256, n_blocks=4), w.reduction_tree(False), w.polyhedral_product(50),
             w.transpose(pad=False, barrier=False, n=256), w.random_affine(6, n_blocks=16, block=256, plant=True),
             w.random_affine(7, n_blocks=8, block=128, n_phases=40, plant=True)])


def key(r):
    return (r.status, r.instances, r.verdict, r.racy_cells, r.witness)


@pytest.mark.parametrize("opts", [None, {"path": 2}])
@pytest.mark.parametrize("k", [2, 5])
def test_partitions_merge_to_whole(rc, opts, k):
    for m in models():
        h = rc.rc_model_create(m)
        ws = rc.workspace(rc.rc_workspace_size(h, opts))
        parts = [D.check_partition(h, r, k, ws, opts=opts, by="range") for r in range(k)]
        got = D.merge_results(parts)
        exp = oracle.check(m)
        assert key(got) == (exp.status, exp.instances, exp.verdict, exp.racy_cells, exp.witness), m.name
        assert key(got) == key(rc.check(m, opts)), m.name


def test_partitions_generated_kernel(rc, monkeypatch):
    monkeypatch.setenv("RC_JIT", "1")
    for m in models()[::4]:
        h = rc.rc_model_create(m)
        assert rc.rc_model_layout(h)["expand_jit"] == 1
        ws = rc.workspace(rc.rc_workspace_size(h))
        got = D.merge_results([D.check_partition(h, r, 3, ws, by="range") for r in range(3)])
        exp = oracle.check(m)
        assert key(got) == (exp.status, exp.instances, exp.verdict, exp.racy_cells, exp.witness), m.name


# ---------------------------------------------------------------------------
# hash parts (rc_check_opts.part_count / part_index)
# ---------------------------------------------------------------------------

def full(r):
    return (r.status, r.instances, r.verdict, r.racy_cells, r.witness)


@pytest.mark.parametrize("opts", [None, {"flags": 8}])
@pytest.mark.parametrize("k", [2, 4, 8])
def test_hash_parts_equal_oracle_parts(rc, opts, k):
    """Every part equals the oracle's check of that part, field for field, on
    the bucket and the LSD path; the merged parts equal the whole check."""
    for m in models():
        h = rc.rc_model_create(m)
        ws = rc.workspace(max(rc.rc_workspace_size(h, D.partition_opts(h, r, k, opts, by="hash")) for r in range(k)))
        parts = [D.check_partition(h, r, k, ws, opts=opts, by="hash") for r in range(k)]
        for r, p in enumerate(parts):
            assert full(p) == full(oracle.check_part(m, k, r)), (m.name, r)
        exp = oracle.check(m)
        assert key(D.merge_results(parts)) == (exp.status, exp.instances, exp.verdict, exp.racy_cells, exp.witness)


def test_hash_parts_generated_kernel(rc, monkeypatch):
    monkeypatch.setenv("RC_JIT", "1")
    for m in models()[::3] + [w.random_affine(8, n_blocks=64, block=256, plant=True)]:
        h = rc.rc_model_create(m)
        ws = rc.workspace(rc.rc_workspace_size(h, {"part_count": 4}))
        for r in range(4):
            got = D.check_partition(h, r, 4, ws, by="hash")
            assert full(got) == full(oracle.check_part(m, 4, r)), (m.name, r)


def test_hash_parts_rejected_where_unsupported(rc):
    b = rc.binding
    m = w.tiny_random(3)
    for o in ({"part_count": 4, "part_index": 4}, {"part_count": 3, "part_index": 1}):
        with pytest.raises(rc.RcError) as e:
            rc.check(m, o)
        assert e.value.status == b.RC_E_INVALID
    for o in ({"path": 2}, {"flags": b.RC_OPT_CHUNKED}):
        with pytest.raises(rc.RcError) as e:
            rc.check(m, dict(o, part_count=4, part_index=1))
        assert e.value.status == b.RC_E_UNSUPPORTED


def test_hash_parts_of_atomic_and_barrier_models(rc):
    """Hash parts of models with atomics, warp and grid barriers (the phase-
    table scan and its witness), each part equal to the oracle's."""
    models = ([w.tiny_random(s, atomic=0.4) for s in range(0, 40, 3)] +
              [w.tiny_random_sync(s) for s in range(0, 40, 3)] +
              [w.tiny_random_sync(s, block_guards=True) for s in range(0, 60, 7)] +
              [w.atomic_counter(1024, n_blocks=8, barrier=False), w.grid_late_partner(4, 3)])
    for m in models:
        h = rc.rc_model_create(m)
        ws = rc.workspace(max(rc.rc_workspace_size(h, D.partition_opts(h, r, 4, by="hash")) for r in range(4)))
        parts = [D.check_partition(h, r, 4, ws, by="hash") for r in range(4)]
        for r, p in enumerate(parts):
            exp = oracle.check_part(m, 4, r)
            assert full(p) == full(exp), (m.name, r, p, exp)
            if exp.verdict:
                assert (p.x_wphase, p.y_wphase) == (exp.x_wphase, exp.y_wphase), (m.name, r)
        exp = oracle.check(m)
        assert key(D.merge_results(parts)) == (exp.status, exp.instances, exp.verdict, exp.racy_cells, exp.witness)
