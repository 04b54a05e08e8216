"""The relation-algebra form of the dependence test (``oracle.relations``):
pins against closed forms, and the cross-check with the concrete oracle.

The paper's appendix listing runs its dependence test on the polynomial
product (statement S: ``C[k] = 0`` for ``0 <= k < 2n-1``; statement T:
``C[i+j] += A[i] * B[j]`` for ``0 <= i, j < n``; schedule S[k] -> (0, k, 0),
T[i, j] -> (1, i, j)).  Its RaW / WaW / WaR sets have sizes that follow from
counting: with ``n_c = min(c, 2n-2-c) + 1`` statement instances of T per cell
``C[c]``, all T instances of a cell are totally ordered (lexicographically in
i) and S[c] precedes them, so per cell the RaW pairs are sum_{m<n_c} (m + 1),
the WaW pairs are the ordered pairs of a chain of ``n_c + 1`` writers, and
the WaR pairs those of a chain of ``n_c`` instances.
"""
from __future__ import annotations

import pytest

import workloads as w
from oracle import relations as rel

from . import pyref


def _polyprod_relations(n):
    """Domain, Read, Write and Schedule of the appendix listing at parameter n."""
    S = [("S", (k,)) for k in range(2 * n - 1)]
    T = [("T", (i, j)) for i in range(n) for j in range(n)]
    read = rel.Relation([(t, ("C", t[1][0] + t[1][1])) for t in T] +
                        [(t, ("B", t[1][1])) for t in T] +
                        [(t, ("A", t[1][0])) for t in T])
    write = rel.Relation([(s, ("C", s[1][0])) for s in S] + [(t, ("C", t[1][0] + t[1][1])) for t in T])
    schedule = {s: (0, s[1][0], 0) for s in S}
    schedule.update({t: (1, t[1][0], t[1][1]) for t in T})
    return read, write, schedule


def _cell_sizes(n):
    return [min(c, 2 * n - 2 - c) + 1 for c in range(2 * n - 1)]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7])
def test_polynomial_product_dependence_counts(n):
    read, write, schedule = _polyprod_relations(n)
    raw, waw, war = rel.dependences(read, write, rel.lex_before(schedule))
    sizes = _cell_sizes(n)
    assert sum(sizes) == n * n
    assert len(raw) == sum(sum(m + 1 for m in range(nc)) for nc in sizes)
    assert len(waw) == sum((nc + 1) * nc // 2 for nc in sizes)
    assert len(war) == sum(nc * (nc - 1) // 2 for nc in sizes)
    before = rel.lex_before(schedule)
    assert raw <= before and waw <= before and war <= before


def test_polynomial_product_dependence_members():
    read, write, schedule = _polyprod_relations(3)
    raw, waw, war = rel.dependences(read, write, rel.lex_before(schedule))
    S = lambda k: ("S", (k,))
    T = lambda i, j: ("T", (i, j))
    # the initialisation of every cell flows into each of its updates
    for i in range(3):
        for j in range(3):
            assert (S(i + j), T(i, j)) in raw
            assert (T(i, j), S(i + j)) not in raw
    # C[1]: T[0,1] precedes T[1,0]; both read and write C[1]
    assert (T(0, 1), T(1, 0)) in raw and (T(0, 1), T(1, 0)) in waw and (T(0, 1), T(1, 0)) in war
    assert (T(1, 0), T(0, 1)) not in raw
    # different cells never depend; an instance never depends on itself
    assert (T(0, 0), T(0, 1)) not in raw
    assert all(x != y for x, y in raw)
    # A and B are never written
    assert all(c[0] == "C" for _, c in write)


def test_relation_operators():
    a = rel.Relation([(1, "p"), (2, "p"), (3, "q")])
    assert a.inverse().inverse().pairs == a.pairs
    assert set(a.compose(a.inverse())) == {(1, 1), (1, 2), (2, 1), (2, 2), (3, 3)}
    assert len(a * rel.Relation([(1, "p"), (9, "z")])) == 1
    assert len(a + rel.Relation([(9, "z")])) == 4
    assert a.domain() == {1, 2, 3} and a.range() == {"p", "q"}
    assert set(rel.lex_before({"x": (0, 1), "y": (0, 2), "z": (1, 0)})) == {("x", "y"), ("x", "z"), ("y", "z")}


# --------------------------------------------------------------------------
# SIMT races as relations: closed forms
# --------------------------------------------------------------------------

@pytest.mark.parametrize("T", [2, 5, 32])
def test_neighbor_closed_form(T):
    st, cnt, best = rel.race_check(w.neighbor_write_read(T))
    assert st == "ok" and cnt == T - 1
    # s[1]: thread 0 reads it, thread 1 writes it
    assert best == ((0, 0, 1, 0, 0, 0, 0), (0, 0, 1, 0, 0, 1, 1))


@pytest.mark.parametrize("n", [2, 3, 6])
def test_parallel_polynomial_product_closed_form(n):
    st, cnt, _ = rel.race_check(w.polyhedral_product(n))
    assert st == "ok" and cnt == 2 * n - 3


def test_reduction_closed_forms():
    assert rel.race_check(w.reduction_tree(barriers=True, T=64))[1] == 0
    assert rel.race_check(w.reduction_tree(barriers=False, T=64))[1] == 31
    assert rel.race_check(w.reduction_tree(barriers=False, load_phase=True, T=64))[1] == 63


def test_ge_spmm_csr_small_race_free_with_barrier():
    rows = [0, 3, 40, 70, 1]
    m = w.ge_spmm_csr(rows, N=32, K=2, trailing_barrier=True)
    assert rel.race_check(m)[1] == 0
    mb = w.ge_spmm_csr(rows, N=32, K=2, trailing_barrier=False)
    # per block row with L_i > 32: 2 * min(32, L_i - 32) shared cells race
    exp = sum(2 * min(32, max(0, L - 32)) for L in rows)
    assert rel.race_check(mb)[1] == exp


# --------------------------------------------------------------------------
# cross-check: relations == pairwise reference == oracle
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(60))
def test_tiny_random_relations_match(seed):
    from oracle import check
    m = w.tiny_random(seed)
    got = rel.race_check(m)
    exp = pyref.check(m)
    assert got[0] == exp[0] == "ok"
    assert got[1] == exp[1]
    assert got[2] == exp[2]
    r = check(m)
    assert r.racy_cells == got[1]
    if got[2] is None:
        assert r.witness is None
    else:
        x, y = got[2]
        assert r.witness == (x[0], x[1], x[2], x[3:], y[3:])


@pytest.mark.parametrize("seed", range(10))
def test_tiny_random_tables_relations_match(seed):
    m = w.tiny_random_tables(seed)
    got = rel.race_check(m)
    exp = pyref.check(m)
    assert got[0] == exp[0]
    if got[0] == "ok":
        assert got[1:] == exp[1:]


@pytest.mark.parametrize("seed", range(40))
def test_tiny_random_atomic_relations_match(seed):
    m = w.tiny_random(seed, atomic=0.4)
    assert rel.race_check(m) == pyref.check(m)


def test_atomic_closed_forms_as_relations():
    assert rel.race_check(w.atomic_histogram(8, 4, barrier=False))[1] == 4
    assert rel.race_check(w.atomic_histogram(8, 4, barrier=False, read_back=False))[1] == 0
    assert rel.race_check(w.atomic_counter(4, n_blocks=2))[1] == 1


@pytest.mark.parametrize("seed", range(40))
def test_tiny_random_sync_relations_match(seed):
    m = w.tiny_random_sync(seed)
    assert rel.race_check(m) == pyref.check(m)


def test_sync_closed_forms_as_relations():
    assert rel.race_check(w.warp_reduction(2, warp_barriers=True))[1] == 0
    assert rel.race_check(w.warp_reduction(2, warp_barriers=False))[1] == 30
    assert rel.race_check(w.grid_neighbor(4, 8, grid_barrier=False))[1] == 4
    assert rel.race_check(w.grid_neighbor(4, 8, grid_barrier=True))[1] == 0
