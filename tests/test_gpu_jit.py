"""Parity of the generated (NVRTC-compiled) expansion kernel with the CPU
oracle: RC_JIT=1 makes rc_model_create generate the kernel for every model."""
import numpy as np
import pytest
import torch

import oracle
import workloads as w
from workloads.spec import Access, Array, Loop, Model, Stmt, const, it, tid, R, W

from .test_gpu_parity import compare, decode_keys, keyed_rows

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


@pytest.fixture()
def jit_on(monkeypatch):
    monkeypatch.setenv("RC_JIT", "1")


def _models():
    deep = Model((2, 1, 1), (8, 1, 1), [Array("a", "shared", (64,))],
                 [Stmt([Access(0, W, ((tid.x + it(0) + it(1) + it(2) + it(3) + it(4)) % 64,))],
                       loops=[Loop(0, 2)] * 5)])
    return ([w.tiny_random(s) for s in range(80)] +
            [w.reduction_tree(False, load_phase=True), w.reduction_tree(True), w.neighbor_write_read(100, 3),
             w.polyhedral_product(50), w.transpose(pad=True, barrier=False, n=256),
             w.ge_spmm_uniform(3, 64, 4, 70, True), w.ge_spmm_uniform(3, 64, 4, 70, False),
             w.random_affine(1, n_blocks=16, block=256, plant=True),
             w.random_affine(2, n_blocks=16, block=256, plant=False), deep])


@pytest.mark.parametrize("i", range(90))
def test_jit_matches_oracle(rc, jit_on, i):
    m = _models()[i]
    h = rc.rc_model_create(m)
    assert rc.rc_model_layout(h)["expand_jit"] == 1
    compare(rc, h if False else m)


@pytest.mark.parametrize("seed", range(10))
def test_jit_key_multiset(rc, jit_on, seed):
    model = w.tiny_random(seed + 200)
    m = rc.rc_model_create(model)
    assert rc.rc_model_layout(m)["expand_jit"] == 1
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
    assert np.array_equal(got, keyed_rows(exp, model))


def test_jit_out_of_bounds(rc, jit_on):
    m = Model((2, 1, 1), (8, 1, 1), [Array("a", "global", (10,))],
              [Stmt([Access(0, R, (tid.x,))]), Stmt([Access(0, W, (tid.x + 3,))])])
    compare(rc, m)
    m2 = Model((1, 1, 1), (4, 1, 1), [Array("a", "shared", (4,))],
               [Stmt([Access(0, W, (tid.x,))], phase=const(2))], n_phases=2)
    compare(rc, m2)
