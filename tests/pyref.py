"""Independent pure-Python restatement of the race definition, for tiny models.

Used only to pin the oracle: it enumerates instances with Python loops and
Python integers (``//`` floors, ``%`` with a positive modulus is Euclidean) and
applies the pairwise race predicate directly, without the oracle's cell-level
shortcut.  Shares no code with ``oracle/`` or the CUDA path.
"""
from itertools import product


def ev(e, env):
    op, a = e.op, e.args
    if op == "const":
        return a[0]
    if op == "tid":
        return env["tid"][a[0]]
    if op == "bid":
        return env["bid"][a[0]]
    if op == "param":
        return env["params"][a[0]]
    if op == "iter":
        return env["iter"][a[0]]
    if op == "add":
        return ev(a[0], env) + ev(a[1], env)
    if op == "mul":
        return a[0] * ev(a[1], env)
    if op == "fdiv":
        return ev(a[0], env) // a[1]
    if op == "mod":
        return ev(a[0], env) % a[1]
    if op == "load":
        if a[0] in env.get("free", {}):
            return env["free"][a[0]][expr_key(e)]   # a free parameter of the superset domain
        t = env["tables"][a[0]]
        i = ev(a[1], env)
        return t[i] if 0 <= i < len(t) else 0
    raise ValueError(op)


def expr_key(e):
    """The expression as a nested tuple (equal expressions, equal keys)."""
    return (e.op,) + tuple(expr_key(x) if hasattr(x, "op") else x for x in e.args)


def free_loads(st, superset):
    """The superset domain: the distinct loads of tables with unknown values
    in a statement, as (table, key) pairs; a load inside such a load is part
    of it."""
    found = []

    def walk(e):
        if e.op == "load" and e.args[0] in superset:
            k = (e.args[0], expr_key(e))
            if k not in found:
                found.append(k)
            return
        for x in e.args:
            if hasattr(x, "op"):
                walk(x)
    exprs = [st.phase, getattr(st, "warp_phase", None)] + [x for lp in st.loops for x in (lp.lower, lp.upper)]
    exprs += list(st.guards) + [ie for ac in st.accesses for ie in ac.index]
    for e in exprs:
        if e is not None:
            walk(e)
    return found


def free_values(st, superset):
    """Every assignment of values to the statement's free parameters, as
    {table: {key: value}} (one empty assignment without superset tables)."""
    fl = free_loads(st, superset)
    for vals in product(*[range(superset[t][0], superset[t][1] + 1) for t, _ in fl]):
        out = {t: {} for t in superset}
        for (t, k), v in zip(fl, vals):
            out[t][k] = v
        yield out


def has_sync_scopes(m):
    return getattr(m, "n_warp_phases", 1) > 1 or any(getattr(m, "grid_phase", None) or [])


def instances(m):
    """List of (a, s, e, b, p, t, k) for every in-bounds access instance --
    with the warp interval w appended, (a, s, e, b, p, t, k, w), when the model
    has warp or grid barriers -- and the list of out-of-bounds records (stmt,
    access, gtid, dimcode)."""
    sync = has_sync_scopes(m)
    n_wp = getattr(m, "n_warp_phases", 1)
    gx, gy, gz = m.grid
    bx_, by_, bz_ = m.block
    bs = bx_ * by_ * bz_
    out, oob = [], []
    for bz, by, bx in product(range(gz), range(gy), range(gx)):
        b = bx + gx * (by + gy * bz)
        for tz, ty, tx in product(range(bz_), range(by_), range(bx_)):
            t = tx + bx_ * (ty + by_ * tz)
            env = {"tid": (tx, ty, tz), "bid": (bx, by, bz), "params": m.params, "iter": [0] * 8,
                   "tables": getattr(m, "tables", [])}
            superset = getattr(m, "superset", {}) or {}
            for si, st, free in ((si, st, free) for si, st in enumerate(m.stmts)
                                 for free in free_values(st, superset)):
                env["free"] = free
                def rec(level):
                    if level == len(st.loops):
                        if any(ev(g, env) < 0 for g in st.guards):
                            return
                        p = ev(st.phase, env)
                        wp = ev(st.warp_phase, env) if hasattr(st, "warp_phase") else 0
                        for ai, ac in enumerate(st.accesses):
                            arr = m.arrays[ac.array]
                            bad = False
                            if not (0 <= p < m.n_phases) or not (0 <= wp < n_wp):
                                oob.append((si, ai, b * bs + t, 0))
                                bad = True
                            e = 0
                            for d, (ie, ext) in enumerate(zip(ac.index, arr.extents)):
                                v = ev(ie, env)
                                if not (0 <= v < ext):
                                    oob.append((si, ai, b * bs + t, d + 1))
                                    bad = True
                                e = e * ext + v
                            if bad:
                                continue
                            s = b if arr.scope == "shared" else 0
                            x = (ac.array, s, e, b, p, t, {"W": 1, "A": 2}.get(ac.kind, 0))
                            out.append(x + (wp,) if sync else x)
                        return
                    lp = st.loops[level]
                    v = ev(lp.lower, env)
                    hi = ev(lp.upper, env)
                    while v < hi:
                        env["iter"][level] = v
                        rec(level + 1)
                        v += lp.step
                rec(0)
    return out, oob


def conflict(kx, ky):
    """Kinds R=0, W=1, A=2 (atomic): a W conflicts with everything, an A with
    an R; two atomics do not conflict."""
    return kx == 1 or ky == 1 or {kx, ky} == {0, 2}


def race(x, y, bs, grid_phase=None):
    """The pair predicate: same cell, different threads, conflicting kinds,
    and concurrent: different blocks in the same grid interval, or the same
    block and barrier interval and (different warps or the same warp
    interval).  Tuples without a warp interval (no warp or grid barriers):
    different blocks or the same barrier interval."""
    if x[:3] != y[:3]:
        return False
    if x[3] * bs + x[5] == y[3] * bs + y[5]:
        return False
    if not conflict(x[6], y[6]):
        return False
    if len(x) == 7:
        return x[3] != y[3] or x[4] == y[4]
    g = grid_phase or [0] * (max(x[4], y[4]) + 1)
    if x[3] != y[3]:
        return g[x[4]] == g[y[4]]
    return x[4] == y[4] and (x[5] // 32 != y[5] // 32 or x[7] == y[7])


def check(m):
    """(status, racy_cell_count, witness) with witness = (x, y) tuples or None;
    status 'oob' with the smallest out-of-bounds record instead of a count."""
    inst, oob = instances(m)
    if oob:
        return "oob", min(oob), None
    bs = m.block_size
    u = sorted(set(inst))
    by_cell = {}
    for x in u:
        by_cell.setdefault(x[:3], []).append(x)
    racy = set()
    best = None
    for cell, xs in by_cell.items():
        for i in range(len(xs)):
            for j in range(i + 1, len(xs)):
                if race(xs[i], xs[j], bs, getattr(m, "grid_phase", None)):
                    racy.add(cell)
                    if best is None or (xs[i], xs[j]) < best:
                        best = (xs[i], xs[j])
    return "ok", len(racy), best
