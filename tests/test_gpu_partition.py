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
        parts = [D.check_partition(h, r, k, ws, opts=opts) for r in range(k)]
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
        got = D.merge_results([D.check_partition(h, r, 3, ws) for r in range(3)])
        exp = oracle.check(m)
        assert key(got) == (exp.status, exp.instances, exp.verdict, exp.racy_cells, exp.witness), m.name
