"""Relation-algebra form of the dependence test, over explicit finite sets
(test infrastructure: the symbolic cross-check of the concrete checker).

The paper states its check with ISCC relations (Section "Using ISCC in Formal
Analysis/Verification" and the appendix listing of the full dependence test
for the polynomial product): a *Domain* of labelled statement instances, *Read*
and *Write* maps from statement instances to array cells, a *Schedule* map to
time tuples, ``Before := Schedule << Schedule`` (lexicographically earlier
time), and the three dependence relations

    RaW := (Write . Read^-1) * Before
    WaW := (Write . Write^-1) * Before
    WaR := (Read . Write^-1) * Before

where ``A . B`` is composition (x -> z whenever x -> y in A and y -> z in B),
``^-1`` the inverse and ``*`` intersection.  ISCC keeps the parameters symbolic;
here every set is enumerated at fixed small parameter values, so each relation
is a plain Python set of pairs and each operator is the textbook set operation.

For a SIMT kernel model the sequential ``Before`` is replaced by the
concurrency relation of the barrier rule (two statement instances of distinct
threads are concurrent iff they are in different blocks of the same grid
interval, or in the same block and barrier interval and in different warps or
the same warp interval; without warp and grid barriers: different blocks or the
same barrier interval), and a race is a conflicting pair that is concurrent:

    Race := ((Write . Read^-1) + (Write . Write^-1) + (Read . Write^-1)) * Concurrent

Atomic read-modify-write accesses form a third relation, *Atomic*, which
conflicts with plain reads and writes but not with itself (two atomics on one
cell are ordered by the memory system): the conflicting pairs gain
``(Atomic . Read^-1) + (Read . Atomic^-1) + (Atomic . Write^-1) + (Write . Atomic^-1)``.

Nothing here is shared with the CUDA path or with ``oracle.cpp``: the
statement instances are enumerated by this module's own expression evaluator.
Only ``tests/`` import it.  Cost is quadratic in the instances of one cell, so
it is meant for models of at most a few thousand instances.
"""
from __future__ import annotations

from itertools import product
from typing import Dict, Iterable, List, Optional, Set, Tuple

__all__ = [
    "Relation", "lex_before", "dependences", "SimtInstances", "simt_instances",
    "conflicts", "concurrent_pairs", "races", "race_check",
]


# ---------------------------------------------------------------------------
# finite binary relations
# ---------------------------------------------------------------------------
class Relation:
    """A finite binary relation: a set of (x, y) pairs."""

    __slots__ = ("pairs",)

    def __init__(self, pairs: Iterable[Tuple] = ()):
        self.pairs = frozenset(pairs)

    def inverse(self) -> "Relation":
        """R^-1 = {(y, x) : (x, y) in R}."""
        return Relation((y, x) for x, y in self.pairs)

    def compose(self, other: "Relation") -> "Relation":
        """ISCC's ``self . other``: {(x, z) : (x, y) in self and (y, z) in other}."""
        by_src: Dict = {}
        for y, z in other.pairs:
            by_src.setdefault(y, []).append(z)
        return Relation((x, z) for x, y in self.pairs for z in by_src.get(y, ()))

    def __mul__(self, other: "Relation") -> "Relation":
        """Intersection (ISCC ``*``)."""
        return Relation(self.pairs & other.pairs)

    def __add__(self, other: "Relation") -> "Relation":
        """Union (ISCC ``+``)."""
        return Relation(self.pairs | other.pairs)

    def __le__(self, other: "Relation") -> bool:
        """Subset (ISCC ``<=``)."""
        return self.pairs <= other.pairs

    def __len__(self) -> int:
        return len(self.pairs)

    def __contains__(self, pair) -> bool:
        return pair in self.pairs

    def __iter__(self):
        return iter(self.pairs)

    def domain(self) -> Set:
        return {x for x, _ in self.pairs}

    def range(self) -> Set:
        return {y for _, y in self.pairs}


def lex_before(schedule: Dict) -> Relation:
    """``Schedule << Schedule``: the pairs (x, y) of domain elements whose time
    tuple of x is lexicographically smaller than that of y (the appendix
    listing's ``Before``; tuples are compared as Python tuples)."""
    items = list(schedule.items())
    return Relation((x, y) for x, tx in items for y, ty in items if tx < ty)


def dependences(read: Relation, write: Relation, before: Relation):
    """(RaW, WaW, WaR) of the appendix listing's dependence test."""
    raw = write.compose(read.inverse()) * before
    waw = write.compose(write.inverse()) * before
    war = read.compose(write.inverse()) * before
    return raw, waw, war


# ---------------------------------------------------------------------------
# statement instances of a SIMT kernel model
# ---------------------------------------------------------------------------
def _ev(e, tid, bid, params, its, tables) -> int:
    """Value of a model expression (floor division and Euclidean modulo by a
    positive constant, as Python's ``//`` and ``%``; table reads 0 outside)."""
    op, a = e.op, e.args
    if op == "const":
        return a[0]
    if op == "tid":
        return tid[a[0]]
    if op == "bid":
        return bid[a[0]]
    if op == "param":
        return params[a[0]]
    if op == "iter":
        return its[a[0]]
    if op == "add":
        return _ev(a[0], tid, bid, params, its, tables) + _ev(a[1], tid, bid, params, its, tables)
    if op == "mul":
        return a[0] * _ev(a[1], tid, bid, params, its, tables)
    if op == "fdiv":
        return _ev(a[0], tid, bid, params, its, tables) // a[1]
    if op == "mod":
        return _ev(a[0], tid, bid, params, its, tables) % a[1]
    if op == "load":
        t = tables[a[0]]
        i = _ev(a[1], tid, bid, params, its, tables)
        return t[i] if 0 <= i < len(t) else 0
    raise ValueError(f"unknown expression op {op!r}")


class SimtInstances:
    """Domain, Read and Write of a kernel model at its parameter values.

    A statement instance is ``(stmt, iters, gtid)``; ``block``, ``thread`` and
    ``phase`` give its block, thread-in-block and barrier interval.  A cell is
    ``(array, scope instance, element)`` with the scope instance the block for
    shared arrays and 0 for global ones, and the element row-major.
    """

    def __init__(self):
        self.domain: List[Tuple] = []
        self.block: Dict[Tuple, int] = {}
        self.thread: Dict[Tuple, int] = {}
        self.phase: Dict[Tuple, int] = {}
        self.wphase: Dict[Tuple, int] = {}
        self.grid_phase: List[int] = []
        self.sync = False   # warp or grid barriers: witness tuples carry the warp interval
        self.read = Relation()
        self.write = Relation()
        self.atomic = Relation()
        self.out_of_bounds: List[Tuple] = []


def simt_instances(m) -> SimtInstances:
    """Enumerate the Domain and the Read / Write relations of a model."""
    gx, gy, gz = m.grid
    bx_, by_, bz_ = m.block
    bs = bx_ * by_ * bz_
    tables = getattr(m, "tables", [])
    out = SimtInstances()
    n_wp = getattr(m, "n_warp_phases", 1)
    out.grid_phase = list(getattr(m, "grid_phase", None) or []) or [0] * m.n_phases
    out.sync = n_wp > 1 or any(out.grid_phase)
    reads, writes, atomics = set(), set(), set()
    for bz, by, bx in product(range(gz), range(gy), range(gx)):
        b = bx + gx * (by + gy * bz)
        for tz, ty, tx in product(range(bz_), range(by_), range(bx_)):
            t = tx + bx_ * (ty + by_ * tz)
            gtid = b * bs + t
            tid, bid = (tx, ty, tz), (bx, by, bz)
            for si, st in enumerate(m.stmts):
                its: List[int] = []

                def visit(level: int):
                    if level < len(st.loops):
                        lp = st.loops[level]
                        lo = _ev(lp.lower, tid, bid, m.params, its, tables)
                        hi = _ev(lp.upper, tid, bid, m.params, its, tables)
                        v = lo
                        while v < hi:
                            its.append(v)
                            visit(level + 1)
                            its.pop()
                            v += lp.step
                        return
                    if any(_ev(g, tid, bid, m.params, its, tables) < 0 for g in st.guards):
                        return
                    x = (si, tuple(its), gtid)
                    out.domain.append(x)
                    out.block[x], out.thread[x] = b, t
                    out.phase[x] = _ev(st.phase, tid, bid, m.params, its, tables)
                    wp = getattr(st, "warp_phase", None)
                    out.wphase[x] = _ev(wp, tid, bid, m.params, its, tables) if wp is not None else 0
                    if not (0 <= out.phase[x] < m.n_phases) or not (0 <= out.wphase[x] < n_wp):
                        out.out_of_bounds.append((si, 0, gtid))
                    for ai, ac in enumerate(st.accesses):
                        arr = m.arrays[ac.array]
                        idx = [_ev(e, tid, bid, m.params, its, tables) for e in ac.index]
                        if len(idx) != len(arr.extents) or any(not 0 <= v < n for v, n in zip(idx, arr.extents)):
                            out.out_of_bounds.append((si, ai, gtid))
                            continue
                        e = 0
                        for v, n in zip(idx, arr.extents):
                            e = e * n + v
                        cell = (ac.array, b if arr.scope == "shared" else 0, e)
                        {"W": writes, "A": atomics}.get(ac.kind, reads).add((x, cell))

                visit(0)
    out.read, out.write, out.atomic = Relation(reads), Relation(writes), Relation(atomics)
    return out


# ---------------------------------------------------------------------------
# races as relations
# ---------------------------------------------------------------------------
def conflicts(inst: SimtInstances):
    """The conflicting pairs with the cell they meet at and their access kinds
    (R=0, W=1, A=2): a set of (x, kind_x, cell, y, kind_y) from ``Write .
    Read^-1`` (W, R), ``Write . Write^-1`` (W, W), ``Read . Write^-1`` (R, W)
    and the atomic compositions (A, R), (R, A), (A, W), (W, A).  The cell is
    kept (a composition through it) so that racy cells can be counted."""
    def through(a: Relation, b_inv: Relation, ka: int, kb: int):
        by_cell: Dict = {}
        for y, c in b_inv.inverse():
            by_cell.setdefault(c, []).append(y)
        for x, c in a:
            for y in by_cell.get(c, ()):
                yield (x, ka, c, y, kb)
    out = set()
    out.update(through(inst.write, inst.read.inverse(), 1, 0))
    out.update(through(inst.write, inst.write.inverse(), 1, 1))
    out.update(through(inst.read, inst.write.inverse(), 0, 1))
    out.update(through(inst.atomic, inst.read.inverse(), 2, 0))
    out.update(through(inst.read, inst.atomic.inverse(), 0, 2))
    out.update(through(inst.atomic, inst.write.inverse(), 2, 1))
    out.update(through(inst.write, inst.atomic.inverse(), 1, 2))
    return out


def concurrent_pairs(inst: SimtInstances, pairs: Iterable[Tuple]) -> Relation:
    """The part of ``pairs`` in the concurrency relation of the barrier rule:
    distinct threads, and either different blocks of the same grid interval,
    or the same block and barrier interval and (different warps or the same
    warp interval)."""
    keep = []
    g = inst.grid_phase
    for x, y in pairs:
        if x[2] == y[2]:
            continue
        if inst.block[x] != inst.block[y]:
            ok = g[inst.phase[x]] == g[inst.phase[y]]
        else:
            ok = inst.phase[x] == inst.phase[y] and (
                inst.thread[x] // 32 != inst.thread[y] // 32 or inst.wphase[x] == inst.wphase[y])
        if ok:
            keep.append((x, y))
    return Relation(keep)


def races(inst: SimtInstances):
    """The racing conflicts (x, kind_x, cell, y, kind_y)."""
    conf = conflicts(inst)
    conc = concurrent_pairs(inst, {(x, y) for x, _, _, y, _ in conf})
    return {r for r in conf if (r[0], r[3]) in conc}


def race_check(m) -> Tuple[str, object, Optional[Tuple]]:
    """(status, racy cell count, witness) from the relations, in the form of
    the pairwise reference: status "oob" with the smallest out-of-bounds
    (stmt, access, gtid) instead of a count; the witness is the smallest pair
    of access tuples (array, scope, element, block, phase, thread, kind)."""
    inst = simt_instances(m)
    if inst.out_of_bounds:
        return "oob", min(inst.out_of_bounds), None
    rs = races(inst)
    cells = {c for _, _, c, _, _ in rs}
    best = None
    for x, kx, c, y, ky in rs:
        X = c + (inst.block[x], inst.phase[x], inst.thread[x], kx)
        Y = c + (inst.block[y], inst.phase[y], inst.thread[y], ky)
        if inst.sync:
            X, Y = X + (inst.wphase[x],), Y + (inst.wphase[y],)
        pair = (X, Y) if X < Y else (Y, X)
        if best is None or pair < best:
            best = pair
    return "ok", len(cells), best
