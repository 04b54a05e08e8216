"""Seeded synthetic kernel models.

Each function returns a :class:`workloads.spec.Model` (or a list of them).  The
shapes follow the workloads the race check is measured on:

* :func:`reduction_tree` — shared-memory tree reduction, 1 block x 256 threads,
  ``s[256]``, 8 barrier intervals (stride 128 .. 1).
* :func:`transpose` — tiled matrix transpose, grid 64x64 of 32x8 threads,
  shared tile 32x32 or 32x33, global 2048x2048 in/out.
* :func:`random_affine` — seeded random affine / quasi-affine kernel models,
  default 4096 blocks x 256 threads, ~1e9 access instances, race-free by
  construction unless a race is planted.
* :func:`batch_models` — many small random models of uneven size.
* :func:`request_stream` — Poisson arrivals of such models for the serving loop.

and the small models whose race counts have closed forms:

* :func:`neighbor_write_read` — ``s[t] = W; s[t+1] = R``.
* :func:`polyhedral_product` — the paper's polynomial-product example
  (Section "Using ISCC in Formal Analysis", statements S and T) run with one
  thread per ``i``.
* :func:`ge_spmm_uniform` — the paper's Ge-SpMM Algorithm 2 model (Section
  "Doing this for Ge-SpMM": code sections I, F, T) on a CSR matrix whose rows
  all hold ``L`` non-zeros, so ``rs``/``re`` are affine in the row.
* :func:`tiny_random` — tiny random models for exhaustive pairwise checks.
"""
from __future__ import annotations

import math
from typing import List, Optional, Tuple

from .rng import SplitMix64
from .spec import (GLOBAL, SHARED, A, Access, Array, Expr, Loop, Model, R, Stmt, W,
                   bid, const, it, load, param, tid)

__all__ = [
    "reduction_tree", "transpose", "random_affine", "batch_models", "request_stream",
    "neighbor_write_read", "polyhedral_product", "ge_spmm_uniform", "ge_spmm_csr", "csr_row_lengths",
    "atomic_histogram", "atomic_counter", "warp_reduction", "grid_neighbor", "grid_late_partner", "tiny_random_sync",
    "tiny_random", "tiny_random_tables",
    "RANDOM_AFFINE_ROW_GLOBAL", "RANDOM_AFFINE_ROW_SHARED",
]


# ---------------------------------------------------------------------------
# closed-form models
# ---------------------------------------------------------------------------

def neighbor_write_read(T: int, n_blocks: int = 1) -> Model:
    """Each thread writes ``s[t]`` and reads ``s[t+1]`` in one barrier interval.

    Per block exactly ``T - 1`` cells (s[1] .. s[T-1]) are touched by two
    different threads with a write among them.
    """
    s = Array("s", SHARED, (T + 1,))
    st = Stmt([Access(0, W, (tid.x,)), Access(0, R, (tid.x + 1,))], name="S")
    return Model((n_blocks, 1, 1), (T, 1, 1), [s], [st], name=f"neighbor_T{T}")


def polyhedral_product(n: int, init_stmt: bool = False) -> Model:
    """The paper's polynomial product ``C[i+j] += A[i] * B[j]`` with one thread per ``i``.

    Statement T reads A[i], B[j], C[i+j] and writes C[i+j] for ``0 <= j < n``;
    statement S (``C[k] = 0``, optional) is executed by thread 0 in its own
    barrier interval before T.  Racy cells: ``C[k]`` for ``1 <= k <= 2n-3``,
    i.e. ``2n - 3`` cells for ``n >= 2``.
    """
    A = Array("A", GLOBAL, (n,))
    B = Array("B", GLOBAL, (n,))
    C = Array("C", GLOBAL, (2 * n - 1,))
    i = tid.x
    j = it(0)
    T = Stmt([Access(0, R, (i,)), Access(1, R, (j,)), Access(2, R, (i + j,)), Access(2, W, (i + j,))],
             loops=[Loop(0, n)], phase=const(1 if init_stmt else 0), name="T")
    stmts = [T]
    if init_stmt:
        S = Stmt([Access(2, W, (it(0),))], loops=[Loop(0, 2 * n - 1)], guards=[-1 * tid.x],
                 phase=const(0), name="S")
        stmts = [S, T]
    return Model((1, 1, 1), (n, 1, 1), [A, B, C], stmts, n_phases=2 if init_stmt else 1,
                 name=f"polyprod_n{n}")


def atomic_histogram(T: int, B: int, n_blocks: int = 1, barrier: bool = True, read_back: bool = True,
                     plain: bool = False) -> Model:
    """Per-block shared histogram: thread t adds to bin ``t mod B`` atomically
    (a plain read-modify-write ``R`` + ``W`` with ``plain``), then reads its bin
    back (``read_back``), after a barrier or in the same interval.

    Racy cells: none with the barrier, none without a read-back of atomics;
    otherwise ``n_blocks * B`` when ``T >= 2B`` (every bin has two threads, one
    update races with the other's read), else none (one thread per bin).  With
    ``plain`` updates and ``T >= 2B`` the bins race in any case (two writes)."""
    hist = Array("hist", SHARED, (B,))
    b_ = tid.x % B
    upd = [Access(0, R, (b_,)), Access(0, W, (b_,))] if plain else [Access(0, A, (b_,))]
    stmts = [Stmt(upd, phase=const(0), name="add")]
    if read_back:
        stmts.append(Stmt([Access(0, R, (b_,))], phase=const(1 if barrier else 0), name="read"))
    return Model((n_blocks, 1, 1), (T, 1, 1), [hist], stmts, n_phases=2 if barrier else 1,
                 name=f"hist_T{T}_B{B}_{'bar' if barrier else 'nobar'}{'_plain' if plain else ''}")


def atomic_counter(T: int, n_blocks: int = 1, barrier: bool = True) -> Model:
    """Every thread increments one global counter atomically; thread 0 of each
    block then reads it (after a barrier, or in the same interval).

    Racy cells: 1 if the read can meet another thread's increment -- always
    with two blocks or more (a barrier orders one block only), and in one
    block without the barrier when ``T >= 2`` -- else 0."""
    ctr = Array("counter", GLOBAL, (1,))
    stmts = [Stmt([Access(0, A, (const(0),))], phase=const(0), name="inc"),
             Stmt([Access(0, R, (const(0),))], guards=[-1 * tid.x], phase=const(1 if barrier else 0), name="read")]
    return Model((n_blocks, 1, 1), (T, 1, 1), [ctr], stmts, n_phases=2 if barrier else 1,
                 name=f"counter_T{T}_G{n_blocks}_{'bar' if barrier else 'nobar'}")


def warp_reduction(n_warps: int = 2, warp_barriers: bool = True, shared_half: bool = False) -> Model:
    """Warp-level tree reduction (the CWM style of Ge-SpMM: warps synchronise
    with ``__syncwarp`` only): in one block of ``32 * n_warps`` threads, stage k
    = 0..4 lets lane l < 16 >> k of every warp add ``s[base + l + (16 >> k)]``
    into ``s[base + l]``, with ``base = 32 * warp`` (``shared_half``: every warp
    uses base 0).  With ``warp_barriers`` stage k is warp interval k.

    Racy cells: 0 with warp barriers and private bases; without them 15 per
    warp (cells 1..15 of its slice: written at a stage by lane c, read at an
    earlier stage by a lane of the same warp); with a shared base and two warps
    or more, the warps write cells 0..15 in one barrier interval and warp
    barriers do not order warps, so those 16 cells race with or without them
    (cells 16..31 are only read)."""
    T = 32 * n_warps
    s_ = Array("s", SHARED, (T,))
    lane = tid.x % 32
    base = const(0) if shared_half else (tid.x // 32) * 32
    stmts = []
    for k in range(5):
        stride = 16 >> k
        stmts.append(Stmt([Access(0, R, (base + lane,)), Access(0, R, (base + lane + stride,)),
                           Access(0, W, (base + lane,))],
                          guards=[(stride - 1) - lane], phase=const(0),
                          warp_phase=const(k if warp_barriers else 0), name=f"stage{k}"))
    return Model((1, 1, 1), (T, 1, 1), [s_], stmts, n_phases=1, n_warp_phases=5 if warp_barriers else 1,
                 name=f"warpred_W{n_warps}_{'sync' if warp_barriers else 'nosync'}{'_shared' if shared_half else ''}")


def grid_neighbor(n_blocks: int, block: int, grid_barrier: bool = True) -> Model:
    """Thread g writes ``out[g]``; after a barrier it reads ``out[(g + 1) mod
    T]``.  With a grid-wide barrier (grid intervals 0, 1) the kernel is
    race-free; with a block barrier only, the read of the first cell of every
    block by the last thread of the previous block is unordered: ``n_blocks``
    racy cells (for two blocks or more)."""
    T = n_blocks * block
    out = Array("out", GLOBAL, (T,))
    g = bid.x * block + tid.x
    stmts = [Stmt([Access(0, W, (g,))], phase=const(0), name="write"),
             Stmt([Access(0, R, ((g + 1) % T,))], phase=const(1), name="read")]
    return Model((n_blocks, 1, 1), (block, 1, 1), [out], stmts, n_phases=2,
                 grid_phase=[0, 1] if grid_barrier else [0, 0],
                 name=f"gridnb_{n_blocks}x{block}_{'grid' if grid_barrier else 'block'}")


def grid_late_partner(n_blocks: int = 3, block: int = 1) -> Model:
    """Global ``c[1]``: block 0 reads ``c[0]`` in barrier interval 0 (grid
    interval 0); every later block writes it in interval 1 (grid interval 1).
    The grid barrier orders block 0's read before every write, so the read has
    no partner; the writes of two later blocks share grid interval 1 and race.
    For ``n_blocks >= 3``: one racy cell, whose smallest racing instance lies in
    block 1 (not in the cell's lowest block, 0); its partner is the write of
    block 2 by thread 0 (writes in one block by several threads also race, but
    the smallest partner is taken in tuple order: block 1's other threads come
    first when ``block > 1``)."""
    c = Array("c", GLOBAL, (1,))
    stmts = [Stmt([Access(0, R, (const(0),))], guards=[-1 * bid.x], phase=const(0), name="read0"),
             Stmt([Access(0, W, (const(0),))], guards=[bid.x - 1], phase=const(1), name="write")]
    return Model((n_blocks, 1, 1), (block, 1, 1), [c], stmts, n_phases=2, grid_phase=[0, 1],
                 name=f"gridlate_{n_blocks}x{block}")


def reduction_tree(barriers: bool = True, load_phase: bool = False, T: int = 256) -> Model:
    """Shared-memory tree reduction: for stride = T/2 .. 1: if t < stride: s[t] += s[t+stride].

    With ``barriers`` each stride is its own barrier interval (phase k); without
    them every statement is in interval 0.  ``load_phase`` adds the initial
    ``s[t] = in[gtid]`` statement.
    """
    s = Array("s", SHARED, (T,))
    arrays = [s]
    stmts = []
    k0 = 0
    if load_phase:
        arrays.append(Array("in", GLOBAL, (T,)))
        stmts.append(Stmt([Access(1, R, (tid.x,)), Access(0, W, (tid.x,))], phase=const(0), name="load"))
        k0 = 1
    levels = int(math.log2(T))
    for k in range(levels):
        stride = (T // 2) >> k
        stmts.append(Stmt(
            [Access(0, R, (tid.x,)), Access(0, R, (tid.x + stride,)), Access(0, W, (tid.x,))],
            guards=[stride - 1 - tid.x],  # t < stride
            phase=const(k0 + k if barriers else 0),
            name=f"stride{stride}"))
    n_phases = (k0 + levels) if barriers else 1
    return Model((1, 1, 1), (T, 1, 1), arrays, stmts, n_phases=n_phases,
                 name=f"reduction_{'bar' if barriers else 'nobar'}{'_load' if load_phase else ''}")


def transpose(pad: bool = False, barrier: bool = True, n: int = 2048, tile: int = 32,
              rows: int = 8) -> Model:
    """Tiled transpose ``out[x][y] = in[y][x]`` through a shared tile.

    Grid ``(n/tile, n/tile)``, block ``(tile, rows)``; each thread moves
    ``tile/rows`` elements per phase.  Phase 0: read ``in``, write the tile;
    phase 1 (or 0 when ``barrier`` is False): read the tile transposed, write
    ``out``.  ``pad`` gives the tile ``tile+1`` columns.
    """
    g = n // tile
    tin = Array("in", GLOBAL, (n, n))
    tout = Array("out", GLOBAL, (n, n))
    sh = Array("tile", SHARED, (tile, tile + 1 if pad else tile))
    j = it(0)
    loop = [Loop(0, tile, rows)]
    ld = Stmt([Access(0, R, (bid.y * tile + tid.y + j, bid.x * tile + tid.x)),
               Access(2, W, (tid.y + j, tid.x))], loops=loop, phase=const(0), name="load")
    stp = Stmt([Access(2, R, (tid.x, tid.y + j)),
                Access(1, W, (bid.x * tile + tid.y + j, bid.y * tile + tid.x))],
               loops=[Loop(0, tile, rows)], phase=const(1 if barrier else 0), name="store")
    return Model((g, g, 1), (tile, rows, 1), [tin, tout, sh], [ld, stp],
                 n_phases=2 if barrier else 1,
                 name=f"transpose_{n}_{'pad' if pad else 'nopad'}_{'bar' if barrier else 'nobar'}")


def ge_spmm_uniform(M: int = 4, N: int = 64, K: int = 8, L: int = 70,
                    trailing_barrier: bool = True) -> Model:
    """Ge-SpMM Algorithm 2 as modelled in the paper (code sections I, F, T).

    One block of 32 threads per (row ``i``, 32-column slab of ``j``); the CSR
    matrix has ``L`` non-zeros in every row, so ``rs = i*L`` and ``re = rs + L``.
    F (per 32-wide chunk ``m`` of the row) copies ``colInd``/``val`` into the
    shared ``sm_k``/``sm_v`` under the guard ``ptr + (j % 32) < re``; T reads
    them back for ``kk < 32`` with ``ptr + kk < re``, reads ``B[k, j]`` (``k``
    free, enumerated over ``[0, K)``) and updates ``C[i, j]``.  With the barrier
    after F and after T every chunk has its own two intervals and the model is
    race-free, the verdict the paper expects for Ge-SpMM.  Without the trailing
    barrier T of chunk m shares an interval with F of chunk m+1, giving
    ``2 * min(32, max(0, L - 32)) * M * N/32`` racy shared cells.
    """
    if N % 32:
        raise ValueError("N must be a multiple of 32")
    nch = (L + 31) // 32
    i = bid.x
    j = bid.y * 32 + tid.x
    m, kk, k = it(0), it(1), it(2)
    arrays = [
        Array("A_rowPtr", GLOBAL, (M + 1,)),
        Array("A_colInd", GLOBAL, (M * L,)),
        Array("A_val", GLOBAL, (M * L,)),
        Array("B", GLOBAL, (K, N)),
        Array("C", GLOBAL, (M, N)),
        Array("sm_k", SHARED, (32,)),
        Array("sm_v", SHARED, (32,)),
    ]
    ptr = i * L + 32 * m
    I = Stmt([Access(0, R, (i,)), Access(0, R, (i + 1,))], phase=const(0), name="I")
    F = Stmt([Access(1, R, (ptr + (j % 32),)), Access(2, R, (ptr + (j % 32),)),
              Access(5, W, (j % 32,)), Access(6, W, (j % 32,))],
             loops=[Loop(0, nch)],
             guards=[(i * L + L) - (ptr + (j % 32)) - 1],      # ptr + (j % 32) < re
             phase=(2 * m) if trailing_barrier else m, name="F")
    T = Stmt([Access(5, R, ((j - (j % 32)) % 32 + kk,)), Access(6, R, ((j - (j % 32)) % 32 + kk,)),
              Access(4, R, (i, j)), Access(4, W, (i, j))],
             loops=[Loop(0, nch), Loop(0, 32)],
             guards=[(i * L + L) - (ptr + kk) - 1],             # ptr + kk < re
             phase=(2 * m + 1) if trailing_barrier else (m + 1), name="T")
    TB = Stmt([Access(3, R, (k, j))],
              loops=[Loop(0, nch), Loop(0, 32), Loop(0, K)],
              guards=[(i * L + L) - (ptr + kk) - 1],
              phase=(2 * m + 1) if trailing_barrier else (m + 1), name="T_B")
    n_phases = 2 * nch if trailing_barrier else nch + 1
    return Model((M, N // 32, 1), (32, 1, 1), arrays, [I, F, T, TB], n_phases=max(n_phases, 1),
                 name=f"gespmm_M{M}_N{N}_K{K}_L{L}_{'bar' if trailing_barrier else 'nobar'}")


def ge_spmm_csr(row_lengths: List[int], N: int = 64, K: int = 8, trailing_barrier: bool = True,
                superset: bool = False) -> Model:
    """Ge-SpMM Algorithm 2 on a CSR matrix with the given row lengths.

    As :func:`ge_spmm_uniform`, but the row bounds are read from the row
    pointer array itself: ``rs = rowPtr[i]`` and ``re = rowPtr[i + 1]`` are table
    loads (table 0 holds rowPtr), so the number of 32-wide chunks of block row
    ``i`` is ``ceil((re - rs) / 32)`` and its barrier intervals depend on the
    row -- the data-dependent Domain that the paper's model over-approximates
    with a superset (Section "Problems to deal with").  Without the trailing
    barrier each block row ``i`` has ``2 * min(32, max(0, L_i - 32))`` racy
    shared cells per 32-column slab; with it the model is race-free.

    ``superset=True`` checks the paper's superset domain instead: the row
    pointer's values are unknown, ``rs`` and ``re`` are free parameters over
    ``[0, nnz]`` (the Domain's ``0 <= rs``, ``re <= A_S``), and the model has
    enough barrier intervals for any row of up to ``nnz`` non-zeros.  With the
    trailing barrier it stays race-free (the paper's verdict holds for every
    matrix of that many non-zeros); without it every block has
    ``2 * min(32, max(0, nnz - 32))`` racy shared cells, a false positive
    whenever all rows are at most 32 long.
    """
    if N % 32:
        raise ValueError("N must be a multiple of 32")
    M = len(row_lengths)
    lens = [int(v) for v in row_lengths]
    if M == 0 or min(lens) < 0:
        raise ValueError("need at least one row and non-negative lengths")
    row_ptr = [0]
    for v in lens:
        row_ptr.append(row_ptr[-1] + v)
    nnz = max(1, row_ptr[-1])
    max_ch = max(1, max((v + 31) // 32 for v in lens))
    i = bid.x
    j = bid.y * 32 + tid.x
    m, kk, k = it(0), it(1), it(2)
    rs, re = load(0, i), load(0, i + 1)
    n_ch = (re - rs + 31) // 32
    arrays = [
        Array("A_rowPtr", GLOBAL, (M + 1,)),
        Array("A_colInd", GLOBAL, (nnz,)),
        Array("A_val", GLOBAL, (nnz,)),
        Array("B", GLOBAL, (K, N)),
        Array("C", GLOBAL, (M, N)),
        Array("sm_k", SHARED, (32,)),
        Array("sm_v", SHARED, (32,)),
    ]
    ptr = rs + 32 * m
    I = Stmt([Access(0, R, (i,)), Access(0, R, (i + 1,))], phase=const(0), name="I")
    F = Stmt([Access(1, R, (ptr + (j % 32),)), Access(2, R, (ptr + (j % 32),)),
              Access(5, W, (j % 32,)), Access(6, W, (j % 32,))],
             loops=[Loop(0, n_ch)],
             guards=[re - (ptr + (j % 32)) - 1],                 # ptr + (j % 32) < re
             phase=(2 * m) if trailing_barrier else m, name="F")
    T = Stmt([Access(5, R, ((j - (j % 32)) % 32 + kk,)), Access(6, R, ((j - (j % 32)) % 32 + kk,)),
              Access(4, R, (i, j)), Access(4, W, (i, j))],
             loops=[Loop(0, n_ch), Loop(0, 32)],
             guards=[re - (ptr + kk) - 1],                        # ptr + kk < re
             phase=(2 * m + 1) if trailing_barrier else (m + 1), name="T")
    TB = Stmt([Access(3, R, (k, j))],
              loops=[Loop(0, n_ch), Loop(0, 32), Loop(0, K)],
              guards=[re - (ptr + kk) - 1],
              phase=(2 * m + 1) if trailing_barrier else (m + 1), name="T_B")
    if superset:
        max_ch = max(1, (row_ptr[-1] + 31) // 32)
    n_phases = 2 * max_ch if trailing_barrier else max_ch + 1
    return Model((M, N // 32, 1), (32, 1, 1), arrays, [I, F, T, TB], n_phases=n_phases,
                 name=f"gespmm_csr_M{M}_N{N}_K{K}_{'bar' if trailing_barrier else 'nobar'}"
                      f"{'_superset' if superset else ''}",
                 tables=[row_ptr], superset={0: (0, row_ptr[-1])} if superset else {})


def permutation_scatter(n: int, seed: int = 0, superset: bool = False) -> Model:
    """n threads of one block, thread t writes out[perm[t]] for a seeded
    permutation held in table 0: race-free.  With ``superset=True`` the
    table's values are unknown in [0, n-1] (the paper's superset domain), so
    every thread may write every cell: all n cells are racy (n >= 2), a false
    positive of the over-approximation; the witness is cell 0 with x = thread
    0 and y = thread 1, both writes."""
    rng = SplitMix64(0x5CA7 ^ seed)
    perm = list(range(n))
    for i in range(n - 1, 0, -1):
        j = rng.below(i + 1)
        perm[i], perm[j] = perm[j], perm[i]
    out = Array("out", GLOBAL, (n,))
    st = Stmt([Access(0, W, (load(0, tid.x),))], name="scatter")
    return Model((1, 1, 1), (n, 1, 1), [out], [st], tables=[perm],
                 superset={0: (0, n - 1)} if superset else {},
                 name=f"perm_scatter_{n}{'_superset' if superset else ''}")


def csr_row_lengths(seed: int, M: int, max_len: int = 150, empty: float = 0.1) -> List[int]:
    """Seeded skewed row lengths: log-uniform in [1, max_len], a fraction of
    empty rows."""
    rng = SplitMix64(0xC5A ^ seed)
    out = []
    for _ in range(M):
        if rng.chance(empty):
            out.append(0)
        else:
            out.append(max(1, min(max_len, int(math.exp(rng.random() * math.log(max_len))))))
    return out


# ---------------------------------------------------------------------------
# seeded random affine models
# ---------------------------------------------------------------------------

RANDOM_AFFINE_ROW_GLOBAL = 256   # cells per thread-owned row of a global array
RANDOM_AFFINE_ROW_SHARED = 16    # cells per thread-owned row of the shared array


def _offset_expr(rng: SplitMix64, depth: int, row_len: int) -> Expr:
    e = const(rng.uniform_int(-4, 4))
    if depth >= 1:
        e = e + rng.uniform_int(-4, 4) * it(0)
    if depth >= 2:
        e = e + rng.uniform_int(-4, 4) * it(1)
    e = e + rng.uniform_int(-4, 4) * tid.x
    if rng.chance(0.2):
        d = rng.uniform_int(2, 32)
        e = (e // d) if rng.below(2) == 0 else (e % d)
    return e % row_len


def random_affine(seed: int, n_blocks: int = 4096, block: int = 256, n_stmts: int = 36,
                  n_phases: int = 8, max_depth: int = 2, max_trip: int = 16,
                  plant: Optional[bool] = None, n_threads: Optional[int] = None,
                  row_global: int = RANDOM_AFFINE_ROW_GLOBAL) -> Model:
    """Seeded random affine kernel model, race-free unless a race is planted.

    Arrays (rows of ``RANDOM_AFFINE_ROW_GLOBAL`` cells, one row per thread):
    A0 global read-only, A1 and A2 global owner-only (thread g touches row g
    only); A3 shared, one row of ``RANDOM_AFFINE_ROW_SHARED`` cells per thread of
    a block, whose mode is drawn per barrier interval (read-only or
    owner-only).  Each statement has a uniform phase, a loop nest of uniform
    depth 0..``max_depth`` with trip counts uniform in 1..``max_trip``, and one
    access whose in-row offset is ``c0 + ci*i + cj*j + ct*t`` (coefficients
    uniform in [-4, 4]), wrapped with probability 0.2 in a floor division or
    modulo by a constant uniform in [2, 32], reduced modulo the row length.
    Reads of read-only arrays use row ``(a*gtid + b) mod T``.  30% of the
    accesses that may write are writes.

    A planted race (probability 1%, or forced with ``plant=True``) adds two
    writes in one interval to one owner-only global array: row ``(g+1) mod T``
    and row ``g``, both at offset ``off0``; this makes exactly ``T`` cells racy.

    ``n_threads`` (default ``n_blocks * block``) may be smaller than the grid;
    then threads with ``gtid >= n_threads`` are guarded off.  ``row_global``
    sets the row length of the global arrays (a long row makes a sparse cell
    space: with rows of 2^40 cells and more the packed key needs more than 63
    bits and the model is checked in cell-range chunks).
    """
    rng = SplitMix64(seed)
    T = n_blocks * block if n_threads is None else int(n_threads)
    RG, RS = int(row_global), RANDOM_AFFINE_ROW_SHARED
    arrays = [
        Array("A0", GLOBAL, (T, RG)),
        Array("A1", GLOBAL, (T, RG)),
        Array("A2", GLOBAL, (T, RG)),
        Array("A3", SHARED, (block, RS)),
    ]
    shared_owner = [rng.below(2) == 1 for _ in range(n_phases)]
    gtid = bid.x * block + tid.x
    tail_guard = [] if T == n_blocks * block else [(T - 1) - gtid]
    stmts: List[Stmt] = []
    for s in range(n_stmts):
        ph = rng.below(n_phases)
        depth = rng.below(max_depth + 1)
        loops = [Loop(0, rng.uniform_int(1, max_trip)) for _ in range(depth)]
        a = rng.below(4)
        writable = a in (1, 2) or (a == 3 and shared_owner[ph])
        kind = W if (writable and rng.chance(0.3)) else R
        if a == 0:
            ra, rb = rng.uniform_int(-4, 4), rng.below(T)
            row = (ra * gtid + rb) % T
            off = _offset_expr(rng, depth, RG)
        elif a in (1, 2):
            row = gtid
            off = _offset_expr(rng, depth, RG)
        else:
            if shared_owner[ph]:
                row = tid.x
            else:
                ra, rb = rng.uniform_int(-4, 4), rng.below(block)
                row = (ra * tid.x + rb) % block
            off = _offset_expr(rng, depth, RS)
        stmts.append(Stmt([Access(a, kind, (row, off))], loops=loops, guards=list(tail_guard),
                          phase=const(ph), name=f"s{s}"))
    do_plant = rng.chance(0.01) if plant is None else bool(plant)
    if do_plant:
        ph = rng.below(n_phases)
        a = 1 + rng.below(2)
        off0 = rng.below(RG)
        stmts.append(Stmt([Access(a, W, ((gtid + 1) % T, const(off0)))], guards=list(tail_guard),
                          phase=const(ph), name="plant_next"))
        stmts.append(Stmt([Access(a, W, (gtid, const(off0)))], guards=list(tail_guard),
                          phase=const(ph), name="plant_own"))
    grid_blocks = n_blocks
    m = Model((grid_blocks, 1, 1), (block, 1, 1), arrays, stmts, n_phases=n_phases,
              name=f"affine_s{seed}_B{n_blocks}x{block}{'_planted' if do_plant else ''}")
    m.planted = do_plant
    m.n_model_threads = T
    return m


def batch_models(n: int = 10000, seed0: int = 0, t_min: int = 32, t_max: int = 65536) -> List[Model]:
    """Many small random models: thread count log-uniform in [t_min, t_max]
    (rounded up to a multiple of 32), block ``min(T, 256)``, 1-8 loop-free
    access statements, 1% planted races; model ``k`` is seeded ``seed0 + k``."""
    out = []
    for k in range(n):
        rng = SplitMix64(0xB47C4 ^ (seed0 + k) * 0x9E3779B97F4A7C15)
        lt = math.log(t_min) + rng.random() * (math.log(t_max) - math.log(t_min))
        T = int(math.ceil(math.exp(lt) / 32.0)) * 32
        T = max(t_min, min(t_max, T))
        blk = min(T, 256)
        nb = (T + blk - 1) // blk
        n_st = rng.uniform_int(1, 8)
        out.append(random_affine(seed0 + k, n_blocks=nb, block=blk, n_stmts=n_st, max_depth=0,
                                 n_threads=T))
    return out


def request_stream(n: int, rate_hz: float = 2000.0, seed: int = 0,
                   t_min: int = 32, t_max: int = 65536) -> List[Tuple[float, Model]]:
    """Poisson arrivals (exponential gaps of mean ``1/rate_hz`` seconds) of
    models drawn like :func:`batch_models`."""
    rng = SplitMix64(0x5E4E ^ seed)
    models = batch_models(n, seed0=seed * 1000003, t_min=t_min, t_max=t_max)
    t = 0.0
    out = []
    for m in models:
        u = rng.random()
        t += -math.log(1.0 - u) / rate_hz
        out.append((t, m))
    return out


# ---------------------------------------------------------------------------
# tiny random models for exhaustive pairwise checks
# ---------------------------------------------------------------------------

def _tiny_expr(rng: SplitMix64, n_iter: int, allow_tid: bool = True, n_params: int = 2) -> Expr:
    e = const(rng.uniform_int(-3, 3))
    terms = []
    if allow_tid:
        terms += [tid.x, tid.y]
    terms += [bid.x, bid.y] + [param(p) for p in range(n_params)] + [it(l) for l in range(n_iter)]
    for v in terms:
        if rng.chance(0.45):
            e = e + rng.uniform_int(-3, 3) * v
    if rng.chance(0.35):
        d = rng.uniform_int(2, 5)
        e = (e // d) if rng.below(2) == 0 else (e % d)
        if rng.chance(0.5):
            e = e + rng.uniform_int(-2, 2) * (tid.x if allow_tid else bid.x)
    return e


def tiny_random(seed: int, atomic: float = 0.0) -> Model:
    """A tiny random model (a few hundred instances at most) that exercises
    2-D grids and blocks, shared and global arrays, multi-dimensional indices,
    loops whose bounds depend on tid / bid / outer iterators, steps > 1, guards,
    floor division and modulo, and phases that depend on bid and uniform loop
    iterators.  Every index is reduced modulo its extent, so it is in bounds.
    With ``atomic`` > 0 an access is atomic with that probability, a write
    with probability 0.2 and a read otherwise."""
    rng = SplitMix64(0x7111 ^ (seed * 0x9E3779B97F4A7C15))
    grid = (rng.uniform_int(1, 3), rng.uniform_int(1, 2), 1)
    block = (rng.uniform_int(1, 4), rng.uniform_int(1, 3), rng.uniform_int(1, 2))
    params = [rng.uniform_int(-3, 5), rng.uniform_int(0, 4)]
    n_arr = rng.uniform_int(1, 3)
    arrays = []
    for a in range(n_arr):
        nd = rng.uniform_int(1, 2)
        ext = tuple(rng.uniform_int(2, 6) for _ in range(nd))
        arrays.append(Array(f"a{a}", SHARED if rng.below(2) else GLOBAL, ext))
    n_phases = rng.uniform_int(1, 3)
    stmts = []
    for s in range(rng.uniform_int(1, 4)):
        depth = rng.below(3)
        loops = []
        uniform = True
        uniform_levels = []
        for l in range(depth):
            tid_dep = rng.chance(0.4)
            lo = _tiny_expr(rng, l, allow_tid=tid_dep)
            span = rng.uniform_int(0, 3)
            if rng.chance(0.5):
                hi = lo + span
            else:
                hi = _tiny_expr(rng, l, allow_tid=tid_dep) + span
            loops.append(Loop(lo, hi, rng.uniform_int(1, 2)))
            # the loop is thread-uniform if neither bound names tid nor a
            # non-uniform outer iterator
            lvl_uniform = uniform and not tid_dep
            uniform = lvl_uniform
            if lvl_uniform:
                uniform_levels.append(l)
        guards = [_tiny_expr(rng, depth) for _ in range(rng.below(3))]
        ph = const(rng.below(n_phases))
        if n_phases > 1 and rng.chance(0.4):
            pe = rng.uniform_int(0, 2) * bid.x
            for l in uniform_levels:
                pe = pe + rng.uniform_int(0, 1) * it(l)
            ph = (pe + rng.below(n_phases)) % n_phases
        accs = []
        for _ in range(rng.uniform_int(1, 3)):
            a = rng.below(n_arr)
            idx = tuple(_tiny_expr(rng, depth) % e for e in arrays[a].extents)
            if atomic > 0.0:
                u = rng.random()
                kind = A if u < atomic else (W if u < atomic + 0.2 else R)
            else:
                kind = W if rng.chance(0.4) else R
            accs.append(Access(a, kind, idx))
        stmts.append(Stmt(accs, loops=loops, guards=guards, phase=ph, name=f"t{s}"))
    return Model(grid, block, arrays, stmts, params=params, n_phases=n_phases, name=f"tiny{seed}")


def tiny_random_sync(seed: int, block_guards: bool = False, many: bool = False, scopes: bool = True) -> Model:
    """A small random model with warp and grid barriers: one to three blocks of
    33..80 threads (so two or three warps), up to three barrier intervals
    mapped to up to three grid intervals, up to three warp intervals per
    statement (a constant, a warp-uniform ``tid.x // 32`` term or a uniform
    loop iterator), shared and global arrays, R / W / A accesses.

    ``block_guards``: two to four blocks, and about half of the statements run
    in a subset of the blocks only (a guard ``bid.x - c >= 0`` or
    ``c - bid.x >= 0``), so that the lowest block of a cell may hold no racing
    instance while later blocks of one grid interval do.

    ``many``: more than 16 fine intervals (6 to 14 barrier intervals of 3 or 4
    warp intervals each, four to ten statements).  ``scopes=False`` (with
    ``many``): no warp or grid barriers but 17 to 24 barrier intervals, with
    atomics."""
    rng = SplitMix64(0x5C3A ^ (seed * 0x9E3779B97F4A7C15))
    n_blocks = rng.uniform_int(2, 4) if block_guards else rng.uniform_int(1, 3)
    T = rng.uniform_int(33, 80)
    if many:
        n_phases = rng.uniform_int(6, 14) if scopes else rng.uniform_int(17, 24)
    else:
        n_phases = rng.uniform_int(1, 3)
    gp, g = [], 0
    for _ in range(n_phases):
        gp.append(g)
        if rng.chance(0.8 if block_guards else 0.4) and scopes:
            g += 1
    if many:
        n_wp = rng.uniform_int(3, 4) if scopes else 1
    else:
        n_wp = rng.uniform_int(1, 3)
    arrays = [Array("sh", SHARED, (rng.uniform_int(4, 40),)), Array("gl", GLOBAL, (rng.uniform_int(4, 60),))]
    stmts = []
    for si in range(rng.uniform_int(4, 10) if many else rng.uniform_int(1, 5)):
        depth = rng.below(2)
        loops = [Loop(0, rng.uniform_int(1, 3))] if depth else []
        ph = const(rng.below(n_phases))
        u = rng.below(3)
        if u == 0 or n_wp == 1:
            wp = const(rng.below(n_wp))
        elif u == 1:
            wp = (tid.x // 32 + rng.below(n_wp)) % n_wp
        else:
            wp = (it(0) + rng.below(n_wp)) % n_wp if depth else const(rng.below(n_wp))
        accs = []
        for _ in range(rng.uniform_int(1, 3)):
            # (with block guards mostly the global array: a shared cell has one block)
            a = 1 if (block_guards and rng.chance(0.8)) else rng.below(2)
            ext = arrays[a].extents[0]
            e = rng.uniform_int(0, 5) + rng.uniform_int(0, 3) * tid.x + rng.uniform_int(0, 2) * bid.x
            if depth:
                e = e + rng.uniform_int(0, 3) * it(0)
            if rng.chance(0.3):
                e = e // rng.uniform_int(2, 8)
            u2 = rng.random()
            kind = A if u2 < 0.25 else (W if u2 < 0.55 else R)
            accs.append(Access(a, kind, (e % ext,)))
        guards = []
        if block_guards and rng.chance(0.9):
            c0 = rng.below(n_blocks)
            guards = [bid.x - c0] if rng.chance(0.5) else [c0 - bid.x]
            if rng.chance(0.7):
                guards.append(const(rng.below(2)) - tid.x)   # the first one or two threads only
        stmts.append(Stmt(accs, loops=loops, guards=guards, phase=ph, warp_phase=wp, name=f"y{si}"))
    return Model((n_blocks, 1, 1), (T, 1, 1), arrays, stmts, n_phases=n_phases, n_warp_phases=n_wp,
                 grid_phase=gp if scopes else [],
                 name=f"tinysync_{seed}{'_bg' if block_guards else ''}{'_many' if many else ''}"
                      f"{'' if scopes else '_noscopes'}")


def tiny_random_tables(seed: int, superset: bool = False) -> Model:
    """A tiny random model whose loop bounds, guards and indices read small
    integer tables (data-dependent values; indices outside a table read 0):
    loop bounds such as ``T0[tid.x + i0]``, scatter writes such as
    ``a[T1[tid.x] mod 4]``.  Indices of arrays are reduced modulo the extent.

    ``superset=True``: the same model with table 0's values unknown in the
    range of its values and 0 (the value read outside it), so the concrete
    model's instances are a subset of the superset model's."""
    rng = SplitMix64(0x7AB1E ^ (seed * 0x9E3779B97F4A7C15))
    tables = [[rng.uniform_int(-2, 6) for _ in range(rng.uniform_int(2, 8))]
              for _ in range(rng.uniform_int(1, 2))]

    def maybe_load(e):
        if rng.chance(0.5):
            return load(rng.below(len(tables)), e) + rng.uniform_int(-1, 1)
        return e

    grid = (rng.uniform_int(1, 3), 1, 1)
    block = (rng.uniform_int(1, 5), rng.uniform_int(1, 2), 1)
    params = [rng.uniform_int(-2, 4), rng.uniform_int(0, 3)]
    arrays = [Array(f"a{a}", SHARED if rng.below(2) else GLOBAL, (rng.uniform_int(2, 6),))
              for a in range(rng.uniform_int(1, 3))]
    n_phases = rng.uniform_int(1, 3)
    stmts = []
    for s_ in range(rng.uniform_int(1, 4)):
        depth = rng.below(3)
        loops = []
        for l in range(depth):
            lo = const(rng.uniform_int(-1, 1))
            hi = maybe_load(_tiny_expr(rng, l, allow_tid=True))
            loops.append(Loop(lo, hi, 1))
        guards = [maybe_load(_tiny_expr(rng, depth)) for _ in range(rng.below(2))]
        ph = const(rng.below(n_phases))
        accs = []
        for _ in range(rng.uniform_int(1, 3)):
            a = rng.below(len(arrays))
            idx = (maybe_load(_tiny_expr(rng, depth)) % arrays[a].extents[0],)
            accs.append(Access(a, W if rng.chance(0.45) else R, idx))
        stmts.append(Stmt(accs, loops=loops, guards=guards, phase=ph, name=f"t{s_}"))
    sup = {}
    if superset:
        vals = tables[0] + [0]
        sup = {0: (min(vals), max(vals))}
    return Model(grid, block, arrays, stmts, params=params, n_phases=n_phases,
                 name=f"tinytab{seed}{'_superset' if superset else ''}", tables=tables, superset=sup)

