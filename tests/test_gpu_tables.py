"""Data-dependent values (table loads) on the GPU: the CSR row bounds of the
paper's Ge-SpMM model and tiny random models whose bounds, guards and indices
read integer tables, against the oracle on the sort path (interpreted and
generated expansion), the hash path and in batches."""
import pytest

import oracle
import workloads as w

from .test_gpu_parity import rc, compare  # noqa: F401  (module fixture)
from .test_gpu_batch import batch_compare

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", range(150))
def test_tiny_tables(rc, seed):
    compare(rc, w.tiny_random_tables(seed))


@pytest.mark.parametrize("seed", range(0, 150, 7))
def test_tiny_tables_hash(rc, seed):
    compare(rc, w.tiny_random_tables(seed), {"path": 2})


def test_tiny_tables_generated_kernel(rc, monkeypatch):
    monkeypatch.setenv("RC_JIT", "1")
    for seed in range(0, 150, 5):
        m = w.tiny_random_tables(seed)
        assert rc.rc_model_layout(rc.rc_model_create(m))["expand_jit"] == 1
        compare(rc, m)


@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("bar", [True, False])
def test_gespmm_csr(rc, seed, bar):
    lens = w.csr_row_lengths(seed, 24, max_len=150)
    m = w.ge_spmm_csr(lens, N=128, K=4, trailing_barrier=bar)
    g = compare(rc, m)
    assert g.racy_cells == (0 if bar else (128 // 32) * sum(2 * min(32, max(0, L - 32)) for L in lens))


@pytest.mark.parametrize("bar", [True, False])
def test_gespmm_csr_large(rc, bar):
    """4096 rows x 512 columns (65,536 blocks), skewed row lengths: the
    closed form at a size the oracle is not run on."""
    lens = w.csr_row_lengths(7, 4096, max_len=200)
    m = w.ge_spmm_csr(lens, N=512, K=2, trailing_barrier=bar)
    r = rc.check(m)
    assert r.status == rc.RC_OK
    assert r.racy_cells == (0 if bar else (512 // 32) * sum(2 * min(32, max(0, L - 32)) for L in lens))


def test_tables_in_batches(rc):
    models = [w.tiny_random_tables(s) for s in range(300, 360)] + \
             [w.ge_spmm_csr(w.csr_row_lengths(s, 10), N=64, K=2, trailing_barrier=(s % 2 == 0)) for s in range(4)]
    batch_compare(rc, models)
