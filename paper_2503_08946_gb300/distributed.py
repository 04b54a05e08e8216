"""Checks split across processes (one per GPU).

Two ways to use several GPUs, neither of which exchanges keys:

* independent models -- each rank checks its own models (a batch share, a
  request stream share); ranks only agree on timing (:func:`weak_scaling_rate`);
* one model split by cells -- every rank expands the whole model but keeps only
  the keys of its cells, either a contiguous cell range (``cell_lo`` /
  ``cell_hi`` of the check options) or a hash part (``part_count`` /
  ``part_index``: about equal key shares whatever the access pattern), so each
  cell is checked on exactly one rank.  A cell races or not on its own, so the
  racy-cell counts of disjoint cell sets add up, and the smallest racing pair of
  the model is the racy part's pair with the smallest cell (the pair order
  starts with the cell).  :func:`merge_results` combines the partial results;
  :func:`all_merge` does it across a ``torch.distributed`` group.

Instance counts and out-of-bounds reports cover the whole model on every rank.
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence, Tuple

from . import binding


def cell_ranges(total_cells: int, world: int) -> List[Tuple[int, int]]:
    """Split [0, total_cells) into `world` contiguous ranges of near-equal size."""
    if world < 1:
        raise ValueError("world must be >= 1")
    q, r = divmod(int(total_cells), world)
    out, lo = [], 0
    for k in range(world):
        hi = lo + q + (1 if k < r else 0)
        out.append((lo, hi))
        lo = hi
    return out


def rank_range(model: "binding.RcModel", rank: int, world: int) -> Tuple[int, int]:
    """The cell range of `rank` for a lowered model (its layout's cell count)."""
    return cell_ranges(binding.rc_model_layout(model)["total_cells"], world)[rank]


def partition_opts(model: "binding.RcModel", rank: int, world: int, opts=None, by: str = "auto") -> dict:
    """Check options of `rank`'s share of a model split over `world` ranks: its
    cell range (``by="range"``) or its hash part (``by="hash"``, a power-of-two
    `world`: about equal key shares).  ``"auto"``: the hash part when `world`
    is a power of two, else the cell range."""
    if by == "auto":
        by = "hash" if world & (world - 1) == 0 else "range"
    o = dict(opts or {})
    if by == "hash":
        if world & (world - 1):
            raise ValueError("a hash split takes a power-of-two number of ranks")
        o["part_count"], o["part_index"] = world, rank
        return o
    if by != "range":
        raise ValueError("by must be 'range' or 'hash'")
    lo, hi = rank_range(model, rank, world)
    o["cell_lo"], o["cell_hi"] = lo, hi
    if hi == lo:   # an empty range: no key is kept (cell_hi = 0 would mean "all cells")
        o["cell_lo"], o["cell_hi"] = 1 << 62, (1 << 62) + 1
    return o


def check_partition(model: "binding.RcModel", rank: int, world: int, workspace, stream=None, opts=None,
                    by: str = "auto"):
    """The partial check of `rank`: only the cells of its range or hash part.
    Size `workspace` with ``rc_workspace_size(model, partition_opts(...))``: a
    part's plan may differ from the whole check's (a small cell space takes the
    radix sort)."""
    o = partition_opts(model, rank, world, opts, by)
    return binding.rc_report(binding.rc_check(model, o, workspace, stream))[0]


def merge_results(parts: Sequence):
    """Merge partial results of disjoint cell sets (ranges or hash parts; an
    error of any part is the model's, the first one in the given order).  Works
    on any result records with the fields of :class:`binding.Result` (status,
    verdict, racy_cells, instances, witness fields)."""
    if not parts:
        raise ValueError("no partial results")
    for p in parts:
        if p.status != binding.RC_OK:
            return p   # an error (out-of-bounds, timeout, ...) is the model's
    insts = {p.instances for p in parts}
    if len(insts) != 1:
        raise ValueError(f"partial results disagree on the instance count: {sorted(insts)}")
    total = sum(p.racy_cells for p in parts)
    racy = [p for p in parts if p.verdict]
    # the racy part whose witness cell is the smallest (array, scope instance, element)
    first = min(racy, key=lambda p: (p.w_array, p.w_scope, p.w_addr)) if racy else None
    base = first if first is not None else parts[0]
    return dataclasses.replace(base, racy_cells=total, verdict=1 if total else 0)


def all_merge(result, group=None):
    """Merge the partial results of all ranks of a ``torch.distributed`` group
    (rank order = range order); every rank returns the merged result."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, result, group=group)
    return merge_results(parts)


def weak_scaling_rate(local_instances: float, local_ms: float, group=None, device=None):
    """Whole-job rate of independent per-rank work: the instances of all ranks
    over the slowest rank's time.  Returns (total instances, max ms, G inst/s)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_instances), float(local_ms)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    if dist.is_available() and dist.is_initialized():
        s = t.clone()
        dist.all_reduce(s, op=dist.ReduceOp.SUM, group=group)
        m = t.clone()
        dist.all_reduce(m, op=dist.ReduceOp.MAX, group=group)
        total, ms = float(s[0]), float(m[1])
    else:
        total, ms = float(t[0]), float(t[1])
    return total, ms, total / (ms / 1e3) / 1e9 if ms > 0 else float("nan")
