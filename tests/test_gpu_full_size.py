"""The benchmarked model at its full size, 4096 blocks x 256 threads of the
seeded random affine generator (1.1 G access instances, a 30-bit cell space,
two partition passes and the local sort of every bucket), checked against what
holds at any size and against the oracle on cell ranges it can finish:

* the generator's closed form: a race-free seed has no racy cell, a planted
  seed exactly T = 1,048,576 (one per thread row of the planted array);
* the first racy cell's witness equals the oracle's on that cell alone (no
  cell below it races, by the closed form);
* cell-range checks (the same model restricted to a range of linear cells)
  equal the oracle's check of the range bit for bit: count, instances and
  witness.

Linear cells are numbered array by array in the model's order, each array
row-major (the layout of the cell-range check)."""
import concurrent.futures as cf
import math
import os

import pytest
import torch

import oracle
import workloads as w

pytestmark = pytest.mark.gpu

BLOCKS, THREADS = 4096, 256
T = BLOCKS * THREADS


@pytest.fixture(scope="module")
def rc():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2503_08946_gb300 import build as b
    b.build()
    oracle.build()
    import paper_2503_08946_gb300 as pkg
    pkg.load()
    return pkg


def array_base(m, a):
    """First linear cell of array `a` (arrays in order, row-major; a shared
    array has one copy per block)."""
    return sum(array_cells(m, i) for i in range(a))


def array_cells(m, a):
    x = m.arrays[a]
    return math.prod(x.extents) * (m.grid[0] * m.grid[1] * m.grid[2] if x.scope == "shared" else 1)


def planted_cells(m):
    """The planted cells: row g, offset off0 of one owner-only array."""
    (st,) = [s for s in m.stmts if s.name == "plant_own"]
    acc = st.accesses[0]
    off0 = acc.index[1].args[0]
    row = m.arrays[acc.array].extents[1]
    return array_base(m, acc.array), row, off0


def full(r):
    return (r.status, r.instances, r.verdict, r.racy_cells, r.witness)


def planted_ranges(m):
    base, row, off0 = planted_cells(m)
    first = base + off0                       # row 0 of the planted array: the first racy cell
    # the first racy cell alone; whole rows; ranges starting and ending inside a row
    return [(first, first + 1), (base, base + row), (first, base + row + off0 + 1),
            (base, base + 64 * row), (first - 5, base + 64 * row + off0 + 1)]


def clean_ranges(m):
    """Sampled ranges of every array (rows of the read-only and owner-only
    global arrays, rows of the shared array in blocks 0 and 3)."""
    out = []
    for a in range(len(m.arrays)):
        base, size, row = array_base(m, a), array_cells(m, a), m.arrays[a].extents[-1]
        for lo_row in (0, 777):
            lo = base + lo_row * row
            out.append((lo, min(base + size, lo + 32 * row)))
    return out


@pytest.fixture(scope="module")
def models():
    return {"planted": w.random_affine(1, n_blocks=BLOCKS, block=THREADS, plant=True),
            "clean": w.random_affine(0, n_blocks=BLOCKS, block=THREADS)}


@pytest.fixture(scope="module")
def expected(models):
    """Every oracle range check of this file, run concurrently on the host's
    cores (each call enumerates the whole model and keeps its range)."""
    jobs = [("planted", r) for r in planted_ranges(models["planted"])] + \
           [("clean", r) for r in clean_ranges(models["clean"])]
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 1)) as ex:
        res = list(ex.map(lambda j: oracle.check_cells(models[j[0]], *j[1]), jobs))
    return dict(zip(jobs, res))


def test_race_free_seed_full_size(rc, models):
    g = rc.check(models["clean"], {"early_exit": 0})
    assert g.status == rc.RC_OK
    assert (g.verdict, g.racy_cells) == (0, 0)
    assert g.instances == 1_106_247_680


def test_planted_seed_full_size_count_and_witness(rc, models, expected):
    m = models["planted"]
    g = rc.check(m, {"early_exit": 0})
    assert g.status == rc.RC_OK
    assert (g.verdict, g.racy_cells) == (1, T)
    exp = expected[("planted", planted_ranges(m)[0])]
    assert (exp.verdict, exp.racy_cells) == (1, 1)
    assert g.witness == exp.witness
    assert (g.x_wphase, g.y_wphase) == (exp.x_wphase, exp.y_wphase)


def test_planted_cell_ranges(rc, models, expected):
    m = models["planted"]
    for k, (lo, hi) in enumerate(planted_ranges(m)):
        exp = expected[("planted", (lo, hi))]
        assert exp.racy_cells == [1, 1, 2, 64, 65][k]
        got = rc.check(m, {"cell_lo": lo, "cell_hi": hi, "early_exit": 0})
        assert full(got) == full(exp), (lo, hi, got, exp)


def test_race_free_cell_ranges(rc, models, expected):
    m = models["clean"]
    for lo, hi in clean_ranges(m):
        exp = expected[("clean", (lo, hi))]
        assert exp.distinct > 0 and exp.racy_cells == 0
        got = rc.check(m, {"cell_lo": lo, "cell_hi": hi, "early_exit": 0})
        assert full(got) == full(exp), (lo, hi, got, exp)
