"""The CUDA path against the relation-algebra form of the dependence test
(``oracle.relations``) on small models: racy-cell count and the smallest racing
pair, on the sort path (generated and interpreted expansion) and the hash path."""
import pytest
import torch

import workloads as w
from oracle import relations as rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rc():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2503_08946_gb300 import build as b
    b.build()
    import paper_2503_08946_gb300 as pkg
    pkg.load()
    return pkg


def _agree(rc, m, opts=None):
    st, cnt, best = rel.race_check(m)
    got = rc.check(m, opts)
    if st != "ok":
        assert got.status == rc.RC_E_OOB
        return
    assert got.status == rc.RC_OK
    assert got.racy_cells == cnt and got.verdict == (cnt > 0)
    if best is None:
        assert got.witness is None
    else:
        x, y = best
        assert got.witness == (x[0], x[1], x[2], x[3:], y[3:])


@pytest.mark.parametrize("seed", range(40))
@pytest.mark.parametrize("jit", ["0", "1"])
def test_tiny_random(rc, seed, jit, monkeypatch):
    monkeypatch.setenv("RC_JIT", jit)   # interpreted / generated expansion kernel
    _agree(rc, w.tiny_random(seed))


@pytest.mark.parametrize("seed", range(10))
def test_tiny_random_tables(rc, seed):
    _agree(rc, w.tiny_random_tables(seed))


@pytest.mark.parametrize("bar", [False, True])
def test_ge_spmm_csr(rc, bar):
    _agree(rc, w.ge_spmm_csr([0, 3, 40, 70, 1, 33], N=64, K=2, trailing_barrier=bar))


@pytest.mark.parametrize("n", [2, 5, 9])
def test_polynomial_product(rc, n):
    _agree(rc, w.polyhedral_product(n))
    _agree(rc, w.polyhedral_product(n, init_stmt=True))


@pytest.mark.parametrize("seed", range(12))
def test_hash_path_count(rc, seed):
    m = w.tiny_random(seed)
    st, cnt, _ = rel.race_check(m)
    got = rc.check(m, {"path": rc.RC_PATH_HASH, "early_exit": 0})
    if st == "ok":
        assert got.racy_cells == cnt
