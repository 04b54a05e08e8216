"""The request server (rc_server_*): continuous batching of race-check
requests.  Every result equals the model's own single check (bit-exact) and
the oracle's, whether the request ran alone or in a mix with others, under
memory pressure and with concurrent submitters."""
import threading
import time

import pytest

import oracle
import workloads as w
from workloads.spec import Access, Array, Model, Stmt, tid, W

from .test_gpu_parity import rc  # noqa: F401  (module fixture)
from .test_gpu_batch import assert_same

pytestmark = pytest.mark.gpu


def key(r):
    return (r.status, r.instances, r.verdict, r.racy_cells, r.witness,
            (r.oob_stmt, r.oob_access, r.oob_gtid, r.oob_dim) if r.status == rc_oob() else None)


def rc_oob():
    return oracle.STATUS_OOB


def drain(srv, n, timeout=120.0):
    got = {}
    t0 = time.time()
    while len(got) < n:
        for d in srv.poll(wait_ms=50):
            got[d.request] = d
        assert time.time() - t0 < timeout, f"only {len(got)} of {n} requests finished"
    return got


def mix_models():
    ms = [w.tiny_random(s) for s in range(600, 680)]
    ms += w.batch_models(60, seed0=77, t_max=8192)
    ms += [w.random_affine(3, n_blocks=16, block=256, plant=True), w.transpose(barrier=False, n=256),
           w.reduction_tree(False)]
    return ms


def test_mix_equals_alone_and_oracle(rc):
    models = mix_models()
    handles = [rc.rc_model_create(m) for m in models]
    srv = rc.RcServer(memory_bytes=1 << 30, slots=4)
    try:
        # alone: one request at a time
        alone = {}
        for i, h in enumerate(handles):
            rid = srv.submit(h)
            alone[i] = drain(srv, 1)[rid].result
        # in a mix: everything at once
        ids = [srv.submit(h) for h in handles]
        got = drain(srv, len(ids))
        sizes = [got[r].batch_size for r in ids]
        assert max(sizes) > 1, "requests that wait together are batched"
        for i, (m, rid) in enumerate(zip(models, ids)):
            r = got[rid].result
            assert key(r) == key(alone[i]), m.name
            assert_same(m, r, oracle.check(m))
            assert got[rid].submit_s <= got[rid].start_s <= got[rid].done_s
    finally:
        srv.close()


def test_memory_pressure(rc):
    """A pool that holds about one of these models' workspaces at a time: the
    requests are admitted as memory frees up and all finish correctly."""
    models = [w.random_affine(s, n_blocks=32, block=256, plant=(s % 2 == 0)) for s in range(6)]
    handles = [rc.rc_model_create(m) for m in models]
    need = max(rc.rc_batch_workspace_size([h]) for h in handles)
    srv = rc.RcServer(memory_bytes=int(need * 1.5), slots=3)
    try:
        ids = [srv.submit(h) for h in handles]
        got = drain(srv, len(ids))
        assert max(got[r].batch_size for r in ids) < len(ids), "the pool cannot hold all of them at once"
        for m, rid in zip(models, ids):
            assert_same(m, got[rid].result, oracle.check(m))
    finally:
        srv.close()


def test_request_larger_than_pool(rc):
    big = rc.rc_model_create(w.random_affine(1, n_blocks=64, block=256))
    small = rc.rc_model_create(w.neighbor_write_read(32))
    srv = rc.RcServer(memory_bytes=1 << 20, slots=2)
    try:
        a = srv.submit(big)
        b = srv.submit(small)
        got = drain(srv, 2)
        assert got[a].result.status == rc.RC_E_NOMEM
        assert got[b].result.status == rc.RC_OK and got[b].result.racy_cells == 31
    finally:
        srv.close()


def test_concurrent_submitters(rc):
    models = [w.tiny_random(s) for s in range(700, 760)]
    handles = [rc.rc_model_create(m) for m in models]
    srv = rc.RcServer(memory_bytes=256 << 20, slots=2, max_batch=8)
    ids = [None] * len(handles)

    def worker(k):
        for i in range(k, len(handles), 3):
            ids[i] = srv.submit(handles[i])
            time.sleep(0.0005)

    try:
        ts = [threading.Thread(target=worker, args=(k,)) for k in range(3)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        got = drain(srv, len(ids))
        for m, rid in zip(models, ids):
            assert got[rid].batch_size <= 8
            assert_same(m, got[rid].result, oracle.check(m))
    finally:
        srv.close()


def test_out_of_bounds_request(rc):
    oob = Model((2, 1, 1), (8, 1, 1), [Array("a", "shared", (8,))], [Stmt([Access(0, W, (tid.x + 3,))])])
    h = rc.rc_model_create(oob)
    srv = rc.RcServer(memory_bytes=64 << 20, slots=1)
    try:
        rid = srv.submit(h)
        r = drain(srv, 1)[rid].result
        assert_same(oob, r, oracle.check(oob))
    finally:
        srv.close()
