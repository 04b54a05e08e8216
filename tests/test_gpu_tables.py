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


# ---------------------------------------------------------------------------
# the superset domain: tables whose values are unknown (free parameters)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(150))
def test_superset_tiny_tables(rc, seed):
    compare(rc, w.tiny_random_tables(seed, superset=True))


@pytest.mark.parametrize("seed", range(0, 150, 5))
def test_superset_tiny_tables_lsd_and_hash(rc, seed):
    m = w.tiny_random_tables(seed, superset=True)
    exp = oracle.check(m)
    compare(rc, m, {"flags": rc.binding.RC_OPT_LSD}, exp=exp)
    compare(rc, m, {"path": 2}, exp=exp)


def test_superset_generated_kernel(rc, monkeypatch):
    monkeypatch.setenv("RC_JIT", "1")
    for seed in range(0, 150, 5):
        m = w.tiny_random_tables(seed, superset=True)
        assert rc.rc_model_layout(rc.rc_model_create(m))["expand_jit"] == 1
        compare(rc, m)


@pytest.mark.parametrize("lens", [[3, 20, 7, 10], [32, 1, 0], [5, 40, 2]])
@pytest.mark.parametrize("bar", [True, False])
def test_superset_gespmm(rc, lens, bar):
    """Race-free with the trailing barrier (the paper's verdict on the
    superset domain); without it 2 * min(32, nnz - 32) racy shared cells per
    block, also where the concrete model has none."""
    m = w.ge_spmm_csr(lens, N=32, K=1, trailing_barrier=bar, superset=True)
    g = compare(rc, m)
    assert g.racy_cells == (0 if bar else 2 * min(32, max(0, sum(lens) - 32)) * len(lens))


@pytest.mark.parametrize("bar", [True, False])
def test_superset_gespmm_larger(rc, bar):
    """8 rows x 64 columns with 64 non-zeros: rs, re over [0, 64] (4,225 pairs
    per statement instance), the closed form at a size the oracle is not run on."""
    lens = [9, 0, 16, 3, 11, 8, 7, 10]
    m = w.ge_spmm_csr(lens, N=64, K=2, trailing_barrier=bar, superset=True)
    r = rc.check(m, {"early_exit": 0})
    assert r.status == rc.RC_OK
    assert r.racy_cells == (0 if bar else 2 * min(32, max(0, sum(lens) - 32)) * len(lens) * 2)


@pytest.mark.parametrize("n", [2, 64, 256])
def test_superset_permutation_scatter(rc, n):
    g = compare(rc, w.permutation_scatter(n, seed=n, superset=True))
    assert (g.racy_cells, g.instances) == (n, n * n)
    assert compare(rc, w.permutation_scatter(n, seed=n)).racy_cells == 0


def test_superset_in_batches(rc):
    models = [w.tiny_random_tables(s, superset=True) for s in range(400, 440)] + \
             [w.ge_spmm_csr([3, 20, 7, 10], N=32, K=1, trailing_barrier=b, superset=True) for b in (True, False)] + \
             [w.permutation_scatter(32, superset=True), w.permutation_scatter(32)]
    batch_compare(rc, models)
