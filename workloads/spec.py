"""Neutral description of a kernel model: threads, blocks, barrier phases, arrays and
access relations.

This module only *describes* a model; it evaluates nothing.  Both the CUDA path
(through its C-ABI marshalling) and the CPU oracle (through its own text format)
consume these objects, so neither side depends on the other.

The vocabulary follows the paper's statement of the problem (Introduction, list of
what a race model needs: thread and block ids, barriers/fences, shared-memory
arrays, input/output arrays) and its ISCC models (Section "Using ISCC in Formal
Analysis"): a *statement* is a labelled code section with an iteration *Domain*
(loop nest plus guards) and *Read*/*Write* access relations into arrays.  The
sequential ``Schedule`` of the paper is replaced by a barrier *phase* per
statement instance (the number of block barriers the thread passed before it).

Expressions are trees over thread index ``tid.{x,y,z}``, block index
``bid.{x,y,z}``, integer parameters, and the statement's loop iterators, closed
under ``+``, multiplication by an integer constant, floor division by a positive
constant and (Euclidean) modulo by a positive constant — the quasi-affine forms
the paper's Ge-SpMM model uses (``j % 32``).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Sequence, Tuple, Union

__all__ = [
    "Expr", "E", "tid", "bid", "param", "it", "const", "load",
    "Array", "Loop", "Access", "Stmt", "Model", "R", "W", "A", "GLOBAL", "SHARED",
]

R = "R"
W = "W"
A = "A"   # atomic read-modify-write: conflicts with plain reads and writes, not with atomics
GLOBAL = "global"
SHARED = "shared"


class Expr:
    """Immutable expression tree node.

    ``op`` is one of ``const, tid, bid, param, iter, add, mul, fdiv, mod, load``
    and ``args`` holds the operands: for leaves an ``int`` (the constant, the
    axis 0..2, the parameter number or the loop level), for ``add`` two
    ``Expr``, for ``mul`` ``(int c, Expr a)``, for ``fdiv``/``mod``
    ``(Expr a, int d)``, for ``load`` ``(int table, Expr index)`` -- the value
    of the model's integer table at the index, 0 outside the table.
    """

    __slots__ = ("op", "args")

    def __init__(self, op: str, *args):
        self.op = op
        self.args = args

    # -- construction helpers -------------------------------------------------
    @staticmethod
    def wrap(v: Union["Expr", int]) -> "Expr":
        if isinstance(v, Expr):
            return v
        if isinstance(v, bool) or not isinstance(v, int):
            raise TypeError(f"expression operand must be Expr or int, got {type(v)}")
        return Expr("const", int(v))

    def __add__(self, o):
        return Expr("add", self, Expr.wrap(o))

    def __radd__(self, o):
        return Expr("add", Expr.wrap(o), self)

    def __sub__(self, o):
        return Expr("add", self, Expr("mul", -1, Expr.wrap(o)))

    def __rsub__(self, o):
        return Expr("add", Expr.wrap(o), Expr("mul", -1, self))

    def __neg__(self):
        return Expr("mul", -1, self)

    def __mul__(self, c):
        if isinstance(c, Expr):
            if c.op == "const":
                c = c.args[0]
            else:
                raise TypeError("only multiplication by an integer constant is quasi-affine")
        if isinstance(c, bool) or not isinstance(c, int):
            raise TypeError("only multiplication by an integer constant is quasi-affine")
        return Expr("mul", int(c), self)

    __rmul__ = __mul__

    def __floordiv__(self, d):
        if isinstance(d, bool) or not isinstance(d, int) or d <= 0:
            raise ValueError("floor division only by a positive integer constant")
        return Expr("fdiv", self, int(d))

    def __mod__(self, d):
        if isinstance(d, bool) or not isinstance(d, int) or d <= 0:
            raise ValueError("modulo only by a positive integer constant")
        return Expr("mod", self, int(d))

    # -- inspection -------------------------------------------------------------
    def walk(self):
        yield self
        for a in self.args:
            if isinstance(a, Expr):
                yield from a.walk()

    def uses(self, op: str) -> bool:
        return any(n.op == op for n in self.walk())

    def max_iter(self) -> int:
        """Largest loop level referenced, or -1."""
        m = -1
        for n in self.walk():
            if n.op == "iter":
                m = max(m, n.args[0])
        return m

    def __repr__(self):
        op, a = self.op, self.args
        if op == "const":
            return str(a[0])
        if op in ("tid", "bid"):
            return f"{op}.{'xyz'[a[0]]}"
        if op == "param":
            return f"p{a[0]}"
        if op == "iter":
            return f"i{a[0]}"
        if op == "add":
            return f"({a[0]!r} + {a[1]!r})"
        if op == "mul":
            return f"{a[0]}*{a[1]!r}"
        if op == "fdiv":
            return f"floor({a[0]!r}/{a[1]})"
        if op == "mod":
            return f"({a[0]!r} mod {a[1]})"
        if op == "load":
            return f"T{a[0]}[{a[1]!r}]"
        raise ValueError(op)


class _Axis:
    def __init__(self, op):
        self.x = Expr(op, 0)
        self.y = Expr(op, 1)
        self.z = Expr(op, 2)


tid = _Axis("tid")
bid = _Axis("bid")


def param(i: int) -> Expr:
    return Expr("param", int(i))


def it(level: int) -> Expr:
    """Loop iterator of the enclosing statement, level 0 = outermost loop."""
    return Expr("iter", int(level))


def const(c: int) -> Expr:
    return Expr("const", int(c))


def load(table: int, index) -> Expr:
    """Value of the model's integer table `table` at `index` (0 outside it): a
    data-dependent bound such as a CSR row pointer."""
    return Expr("load", int(table), Expr.wrap(index))


E = Expr.wrap


@dataclass
class Array:
    """An array named in the access relations.

    ``scope`` is ``"shared"`` (one private copy per block, indexed block-locally)
    or ``"global"`` (one copy for the whole grid).  ``extents`` are the sizes of
    its dimensions (row-major, at most 4); one cell is one element.
    """
    name: str
    scope: str
    extents: Tuple[int, ...]

    def __post_init__(self):
        self.extents = tuple(int(e) for e in self.extents)


@dataclass
class Loop:
    """``for (v = lower; v < upper; v += step)``; bounds may use tid, bid,
    parameters and outer iterators."""
    lower: Expr
    upper: Expr
    step: int = 1

    def __post_init__(self):
        self.lower = Expr.wrap(self.lower)
        self.upper = Expr.wrap(self.upper)
        self.step = int(self.step)


@dataclass
class Access:
    """One access relation ``Stmt[iters] -> array[index]`` of kind R, W or A
    (atomic read-modify-write)."""
    array: int
    kind: str
    index: Tuple[Expr, ...]

    def __post_init__(self):
        self.index = tuple(Expr.wrap(e) for e in self.index)
        if self.kind not in (R, W, A):
            raise ValueError("kind must be 'R', 'W' or 'A'")


@dataclass
class Stmt:
    """A labelled code section: its loop nest, its guards (each ``>= 0``), its
    barrier phase (may use bid, parameters and iterators of thread-uniform
    loops, never tid), its warp interval (the number of warp barriers,
    ``__syncwarp``, its thread passed inside the current barrier phase; 0
    without warp barriers) and its accesses."""
    accesses: List[Access]
    loops: List[Loop] = field(default_factory=list)
    guards: List[Expr] = field(default_factory=list)
    phase: Expr = field(default_factory=lambda: const(0))
    name: str = ""
    warp_phase: Expr = field(default_factory=lambda: const(0))

    def __post_init__(self):
        self.phase = Expr.wrap(self.phase)
        self.warp_phase = Expr.wrap(self.warp_phase)
        self.guards = [Expr.wrap(g) for g in self.guards]


@dataclass
class Model:
    grid: Tuple[int, int, int]
    block: Tuple[int, int, int]
    arrays: List[Array]
    stmts: List[Stmt]
    params: List[int] = field(default_factory=list)
    n_phases: int = 1
    name: str = ""
    tables: List[List[int]] = field(default_factory=list)
    # warp intervals per barrier phase (statements' warp_phase in [0, n)), and
    # the grid interval of each barrier phase (grid-wide barriers; empty = none)
    n_warp_phases: int = 1
    grid_phase: List[int] = field(default_factory=list)
    # tables whose values are unknown, table -> (lo, hi): every distinct load
    # of such a table in a statement is a free parameter over [lo, hi] (the
    # paper's superset domain for data-dependent bounds)
    superset: Dict[int, Tuple[int, int]] = field(default_factory=dict)

    def __post_init__(self):
        self.grid = tuple(int(v) for v in (list(self.grid) + [1, 1, 1])[:3])
        self.block = tuple(int(v) for v in (list(self.block) + [1, 1, 1])[:3])
        self.params = [int(p) for p in self.params]
        self.tables = [[int(v) for v in t] for t in self.tables]
        self.grid_phase = [int(v) for v in self.grid_phase]
        self.superset = {int(t): (int(r[0]), int(r[1])) for t, r in self.superset.items()}
        if self.grid_phase and len(self.grid_phase) != self.n_phases:
            raise ValueError("grid_phase needs one entry per barrier phase")
        if any(b < a for a, b in zip(self.grid_phase, self.grid_phase[1:])):
            raise ValueError("grid phases must not decrease (a grid barrier also ends a block interval)")

    @property
    def n_blocks(self) -> int:
        return self.grid[0] * self.grid[1] * self.grid[2]

    @property
    def block_size(self) -> int:
        return self.block[0] * self.block[1] * self.block[2]

    @property
    def n_threads(self) -> int:
        return self.n_blocks * self.block_size
