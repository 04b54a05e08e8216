"""Parity of the batched check (rc_check_batch: one expansion over a work
queue, one sort and one scan for all models) with the CPU oracle, model by
model: status, instance count, out-of-bounds report, verdict, racy-cell count
and witness bit-exact, and equal to the single-model check of the same model."""
import pytest
import torch

import oracle
import workloads as w
from workloads.spec import Access, Array, Model, Stmt, const, tid, R, W

from .test_gpu_parity import rc  # noqa: F401  (module fixture)

pytestmark = pytest.mark.gpu


def check_batch(rc, models, opts=None):
    handles = [rc.rc_model_create(m) for m in models]
    ws = rc.workspace(rc.rc_batch_workspace_size(handles, opts))
    res = rc.rc_report(rc.rc_check_batch(handles, opts, ws))
    assert len(res) == len(models)
    return res


def assert_same(model, got, exp):
    assert got.status == exp.status, (model.name, got, exp)
    assert got.instances == exp.instances, (model.name, got.instances, exp.instances)
    if exp.status == oracle.STATUS_OOB:
        assert (got.oob_stmt, got.oob_access, got.oob_gtid, got.oob_dim) == \
               (exp.oob_stmt, exp.oob_access, exp.oob_gtid, exp.oob_dim), model.name
        return
    assert (got.verdict, got.racy_cells) == (exp.verdict, exp.racy_cells), (model.name, got, exp)
    assert got.witness == exp.witness, (model.name, got.witness, exp.witness)


def batch_compare(rc, models, opts=None):
    res = check_batch(rc, models, opts)
    for m, g in zip(models, res):
        assert_same(m, g, oracle.check(m))
    return res


def test_mixed_small_models(rc):
    models = [w.tiny_random(s) for s in range(60)]
    models += [w.reduction_tree(False), w.reduction_tree(True), w.neighbor_write_read(64),
               w.neighbor_write_read(33, n_blocks=3), w.polyhedral_product(12),
               w.transpose(pad=False, barrier=False, n=128), w.transpose(pad=True, barrier=True, n=128),
               w.ge_spmm_uniform(3, 64, 4, 33)]
    batch_compare(rc, models)


@pytest.mark.parametrize("seed0", [0, 1000])
def test_batch_generator(rc, seed0):
    """Many random models of uneven size (thread counts log-uniform), some
    with planted races of exactly T racy cells."""
    models = w.batch_models(300, seed0=seed0, t_max=4096)
    res = batch_compare(rc, models)
    for m, g in zip(models, res):
        assert g.racy_cells == (m.n_model_threads if m.planted else 0)


def test_planted_races_in_batch(rc):
    models = [w.random_affine(s, n_blocks=4, block=64, n_stmts=6, plant=(s % 3 == 0)) for s in range(24)]
    res = batch_compare(rc, models)
    for m, g in zip(models, res):
        assert g.racy_cells == (m.n_threads if m.planted else 0)


def test_batch_equals_single(rc):
    models = [w.tiny_random(s) for s in range(100, 140)] + [w.random_affine(7, n_blocks=8, block=128, plant=True)]
    res = check_batch(rc, models)
    for m, g in zip(models, res):
        s = rc.check(m)
        assert (g.status, g.instances, g.verdict, g.racy_cells, g.witness) == \
               (s.status, s.instances, s.verdict, s.racy_cells, s.witness), m.name


def test_out_of_bounds_in_batch(rc):
    arr = [Array("a", "shared", (8,))]
    oob = Model((2, 1, 1), (8, 1, 1), arr, [Stmt([Access(0, W, (tid.x + 3,))])], name="oob")
    ok = w.neighbor_write_read(16)
    batch_compare(rc, [ok, oob, ok, w.tiny_random(3), oob])


def test_read_only_and_empty_models(rc):
    ro = Model((2, 1, 1), (32, 1, 1), [Array("g", "global", (64,))],
               [Stmt([Access(0, R, (tid.x,))]), Stmt([Access(0, R, (tid.x + 1,))])], name="read_only")
    empty = Model((1, 1, 1), (4, 1, 1), [Array("a", "global", (4,))], [], name="empty")
    batch_compare(rc, [ro, empty, w.neighbor_write_read(8), empty, ro])


def test_same_model_twice(rc):
    m = w.random_affine(11, n_blocks=2, block=64, n_stmts=5, plant=True)
    h = rc.rc_model_create(m)
    ws = rc.workspace(rc.rc_batch_workspace_size([h, h]))
    a, b = rc.rc_report(rc.rc_check_batch([h, h], None, ws))
    exp = oracle.check(m)
    assert_same(m, a, exp)
    assert_same(m, b, exp)


def test_packs(rc):
    """Models whose combined key fields exceed 63 bits are checked in several
    packs: each model alone fits, any three together do not."""
    def big(k):
        arr = [Array("g", "global", (1 << 28, 1 << 27))]
        return Model((1, 1, 1), (32, 1, 1), arr,
                     [Stmt([Access(0, W, (const(k), tid.x % 4))]), Stmt([Access(0, R, (const(k), tid.x))])],
                     name=f"big{k}")
    models = [big(k) for k in range(5)] + [w.tiny_random(5)]
    batch_compare(rc, models)


@pytest.mark.parametrize("opts", [{"digit_bits": 5}, {"digit_bits": 11},
                                  {"test_flags": 2}])   # RC_TEST_FEW_SCAN_WARPS
def test_batch_options(rc, opts):
    models = [w.tiny_random(s) for s in range(200, 230)] + \
             [w.random_affine(4, n_blocks=8, block=256, plant=True), w.transpose(barrier=False, n=256)]
    batch_compare(rc, models, opts)


def test_hash_batch_is_per_model(rc):
    models = [w.tiny_random(s) for s in range(300, 320)]
    batch_compare(rc, models, {"path": 2})


def test_empty_batch(rc):
    ws = rc.workspace(max(rc.rc_batch_workspace_size([]), 256))
    assert rc.rc_report(rc.rc_check_batch([], None, ws)) == []


def test_batch_workspace_too_small(rc):
    handles = [rc.rc_model_create(w.tiny_random(s)) for s in range(5)]
    ws = rc.workspace(rc.rc_batch_workspace_size(handles) - 512)
    with pytest.raises(rc.RcError) as e:
        rc.rc_check_batch(handles, None, ws)
    assert e.value.status == rc.RC_E_NOMEM


def test_graph_replay(rc):
    """RC_OPT_GRAPH: the first call captures the batch as a CUDA graph, later
    calls relaunch it; every call gives the oracle's results."""
    models = [w.tiny_random(s) for s in range(400, 430)] + [w.random_affine(9, n_blocks=4, block=128, plant=True)]
    handles = [rc.rc_model_create(m) for m in models]
    opts = {"flags": rc.binding.RC_OPT_GRAPH}
    ws = rc.workspace(rc.rc_batch_workspace_size(handles, opts))
    exp = [oracle.check(m) for m in models]
    for _ in range(3):
        res = rc.rc_report(rc.rc_check_batch(handles, opts, ws))
        for m, g, e in zip(models, res, exp):
            assert_same(m, g, e)


def test_tuner_choice_is_used(rc):
    """rc_tune records a choice for the shape class; AUTO checks then give the
    oracle's results with it, for a single model and for a batch."""
    m = w.random_affine(5, n_blocks=8, block=256, plant=True)
    h = rc.rc_model_create(m)
    ws = rc.workspace(max(rc.rc_workspace_size(h, {"path": 1, "digit_bits": d}) for d in (6, 8, 11)) +
                      rc.rc_workspace_size(h, {"path": 2}))
    best = rc.rc_tune([h], None, ws)
    assert best["path"] in (1, 2)
    g = rc.rc_report(rc.rc_check(h, {"path": 0}, ws))[0]
    assert_same(m, g, oracle.check(m))

    models = [w.tiny_random(s) for s in range(500, 540)]
    hs = [rc.rc_model_create(x) for x in models]
    need = max(rc.rc_batch_workspace_size(hs, {"path": p, "digit_bits": d}) for p, d in ((1, 6), (1, 11), (2, 0)))
    wsb = rc.workspace(need)
    best = rc.rc_tune(hs, None, wsb)
    assert best["path"] in (1, 2)
    res = rc.rc_report(rc.rc_check_batch(hs, {"path": 0}, wsb))
    for x, g in zip(models, res):
        assert_same(x, g, oracle.check(x))


def test_batch_with_many_phases(rc):
    """A pack holding a model with more than 16 barrier intervals sorts on the
    phase bits too; the results do not change."""
    models = [w.tiny_random(s) for s in range(800, 820)] + \
             [w.random_affine(s, n_blocks=2, block=128, n_stmts=10, n_phases=40, plant=(s % 2 == 0))
              for s in range(4)]
    batch_compare(rc, models)
    batch_compare(rc, models, {"test_flags": 2})


def test_report_array(rc):
    """The record-array report holds the same results as the object report."""
    models = w.batch_models(200, seed0=77, t_max=2048) + \
        [w.neighbor_write_read(33, n_blocks=3), w.atomic_histogram(64, 8, n_blocks=2, barrier=False)]
    handles = [rc.rc_model_create(m) for m in models]
    ws = rc.workspace(rc.rc_batch_workspace_size(handles))
    arr = rc.rc_report_array(rc.rc_check_batch(handles, None, ws))
    assert arr.shape == (len(models),)
    got = rc.results_of(arr)
    again = rc.rc_report(rc.rc_check_batch(handles, None, ws))
    assert got == again
    for m, g, rec in zip(models, got, arr):
        assert_same(m, g, oracle.check(m))
        assert (int(rec["status"]), int(rec["racy_cells"]), int(rec["instances"])) == \
               (g.status, g.racy_cells, g.instances)
        if g.verdict:
            assert (int(rec["x"]["block"]), int(rec["x"]["phase"]), int(rec["x"]["thread"]),
                    int(rec["x"]["kind"])) == g.x


def test_full_batch_of_10000_models(rc):
    """The benchmarked batch at its full size: 10,000 generator models in one
    graph-replayed batch.  Every model's result has its generator's closed
    form (T racy cells when a race is planted, else none); the planted models
    and every 97th model are checked against the oracle field for field."""
    models = w.batch_models(10000, seed0=0)
    res = check_batch(rc, models, {"flags": rc.binding.RC_OPT_GRAPH})
    planted = 0
    for m, g in zip(models, res):
        assert g.status == rc.RC_OK, m.name
        assert g.racy_cells == (m.n_model_threads if m.planted else 0), m.name
        planted += m.planted
    assert planted > 0
    for k, (m, g) in enumerate(zip(models, res)):
        if m.planted or k % 97 == 0:
            assert_same(m, g, oracle.check(m))
