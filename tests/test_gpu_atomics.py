"""Atomic accesses on the CUDA path: an atomic read-modify-write conflicts with
plain reads and writes of other threads, not with other atomics.  Parity with
the oracle (count, instance count and witness bit-exact) on the sort path
(interpreted and generated expansion, single checks, batches, chunked checks)
and the hash path."""
import pytest
import torch

import oracle
import workloads as w
from workloads.spec import A, Access, Array, Model, Stmt, const, tid, R

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


def compare(rc, model, opts=None, exp=None):
    got = rc.check(model, opts)
    exp = exp or oracle.check(model)
    assert got.status == exp.status, (model.name, got, exp)
    assert got.instances == exp.instances
    assert (got.verdict, got.racy_cells) == (exp.verdict, exp.racy_cells), (model.name, got, exp)
    assert got.witness == exp.witness, (model.name, got.witness, exp.witness)
    return got


@pytest.mark.parametrize("T,B,nb,bar,rb,plain,exp", [
    (8, 4, 1, False, True, False, 4),
    (8, 4, 3, False, True, False, 12),
    (8, 4, 1, True, True, False, 0),
    (4, 4, 1, False, True, False, 0),
    (8, 4, 1, False, False, False, 0),
    (256, 16, 64, False, True, False, 64 * 16),
    (256, 16, 64, True, True, False, 0),
    (256, 16, 64, True, True, True, 64 * 16),
])
def test_histogram(rc, T, B, nb, bar, rb, plain, exp):
    g = compare(rc, w.atomic_histogram(T, B, n_blocks=nb, barrier=bar, read_back=rb, plain=plain))
    assert g.racy_cells == exp


@pytest.mark.parametrize("T,nb,bar,exp", [(4, 1, True, 0), (4, 1, False, 1), (4, 2, True, 1), (1, 1, False, 0),
                                          (256, 4096, True, 1), (256, 1, True, 0)])
def test_counter(rc, T, nb, bar, exp):
    # (256, 4096): one cell of a million keys -- the long-cell scan and the witness on it
    g = compare(rc, w.atomic_counter(T, n_blocks=nb, barrier=bar))
    assert g.racy_cells == exp


@pytest.mark.parametrize("seed", range(100))
@pytest.mark.parametrize("jit", ["0", "1"])
def test_tiny_random_atomic(rc, seed, jit, monkeypatch):
    monkeypatch.setenv("RC_JIT", jit)
    compare(rc, w.tiny_random(seed, atomic=0.4))


@pytest.mark.parametrize("seed", range(40))
def test_tiny_random_atomic_hash(rc, seed):
    m = w.tiny_random(seed, atomic=0.4)
    compare(rc, m, {"path": rc.RC_PATH_HASH, "early_exit": 0})


@pytest.mark.parametrize("seed", range(20))
def test_tiny_random_atomic_chunked(rc, seed):
    compare(rc, w.tiny_random(seed, atomic=0.4), {"flags": rc.binding.RC_OPT_CHUNKED})


def test_batch_mixed_atomic(rc):
    """Atomic and plain models in one batch (the pack takes the 2-bit kind field)."""
    b = rc.binding
    models = [w.tiny_random(s, atomic=0.4 if s % 2 else 0.0) for s in range(60)]
    models += [w.atomic_histogram(64, 8, n_blocks=4, barrier=False), w.atomic_counter(32, n_blocks=3)]
    hs = [b.rc_model_create(m) for m in models]
    ws = b.workspace(b.rc_batch_workspace_size(hs))
    got = b.rc_report(b.rc_check_batch(hs, None, ws), wait=True)
    for m, g in zip(models, got):
        exp = oracle.check(m)
        assert (g.status, g.racy_cells, g.instances) == (exp.status, exp.racy_cells, exp.instances), m.name
        assert g.witness == exp.witness, m.name


def test_atomics_beyond_phase_tables(rc):
    """20 barrier intervals with atomics: keys sorted by (cell, interval) and
    the phase-order scan; the hash path is refused for them."""
    m = Model((1, 1, 1), (8, 1, 1), [Array("c", "global", (4,))],
              [Stmt([Access(0, A, (const(0),))], phase=const(19)),
               Stmt([Access(0, R, (const(0),))], guards=[-1 * tid.x], phase=const(19))], n_phases=20)
    exp = oracle.check(m)
    got = rc.check(m)
    assert (got.racy_cells, got.witness) == (exp.racy_cells, exp.witness) and exp.racy_cells == 1
    b = rc.binding
    lay = b.rc_model_layout(b.rc_model_create(m))
    assert lay["sort_lo"] == lay["phase_shift"]   # the sort takes the interval bits too
    with pytest.raises(rc.RcError) as e:
        rc.check(m, {"path": 2})
    assert e.value.status == b.RC_E_UNSUPPORTED
