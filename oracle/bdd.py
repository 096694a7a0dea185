"""Reduced ordered BDDs for single constraints (TEST INFRASTRUCTURE ONLY).

Follows the paper's xBDD (Suppl. Note "Decision Diagrams", Def. xBDD): a DAG
whose decision nodes test a Boolean variable or a theory atom, with the atom
treated as a propositional variable and no LP pruning.  The paper builds its
diagrams with an off-the-shelf package (Results, Alg. 1 discussion); here the
diagram is built with the textbook apply/ITE construction (Bryant 1986): a
unique table gives reduction (no node with equal children, no duplicate
(var, hi, lo) triple) and a computed table memoises apply.

Variable order: the order of first occurrence in the constraint's literal list.

Pins: for every kind and random literal lists the diagram's function is checked
against ``semantics.kind_value`` on all assignments, and node counts against
closed forms (OR of l literals has l nodes, XOR has 2l-1, ...).
"""
from __future__ import annotations

from . import semantics as S

FALSE, TRUE = 0, 1


class Manager:
    """A ROBDD manager over levels 0..L-1 (terminals have level L)."""

    def __init__(self, n_levels: int):
        self.L = n_levels
        self.level = [n_levels, n_levels]  # node id -> level
        self.hi = [-1, -1]
        self.lo = [-1, -1]
        self.unique = {}
        self.memo = {}

    def mk(self, lev: int, hi: int, lo: int) -> int:
        if hi == lo:
            return hi
        key = (lev, hi, lo)
        u = self.unique.get(key)
        if u is None:
            u = len(self.level)
            self.level.append(lev)
            self.hi.append(hi)
            self.lo.append(lo)
            self.unique[key] = u
        return u

    def var(self, lev: int, neg: bool = False) -> int:
        return self.mk(lev, FALSE, TRUE) if neg else self.mk(lev, TRUE, FALSE)

    def apply(self, op: str, u: int, v: int) -> int:
        if u <= TRUE and v <= TRUE:
            a, b = u == TRUE, v == TRUE
            r = {"and": a and b, "or": a or b, "xor": a != b}[op]
            return TRUE if r else FALSE
        key = (op, u, v)
        r = self.memo.get(key)
        if r is not None:
            return r
        lu, lv = self.level[u], self.level[v]
        top = min(lu, lv)
        u1, u0 = (self.hi[u], self.lo[u]) if lu == top else (u, u)
        v1, v0 = (self.hi[v], self.lo[v]) if lv == top else (v, v)
        r = self.mk(top, self.apply(op, u1, v1), self.apply(op, u0, v0))
        self.memo[key] = r
        return r

    def neg(self, u: int) -> int:
        return self.apply("xor", u, TRUE)

    def ite(self, f: int, g: int, h: int) -> int:
        return self.apply("or", self.apply("and", f, g), self.apply("and", self.neg(f), h))


def build(kind: int, param: int, lits):
    """Builds the ROBDD of one constraint.  Returns (manager, root)."""
    L = len(lits)
    M = Manager(L)
    x = [M.var(t, bool(int(lits[t]) & 1)) for t in range(L)]  # the literals, level t
    if kind == S.OR:
        r = FALSE
        for u in x:
            r = M.apply("or", r, u)
    elif kind == S.XOR:
        r = FALSE
        for u in x:
            r = M.apply("xor", r, u)
    elif kind == S.NAE:
        some_true, some_false = FALSE, FALSE
        for u in x:
            some_true = M.apply("or", some_true, u)
            some_false = M.apply("or", some_false, M.neg(u))
        r = M.apply("and", some_true, some_false)
    elif kind == S.CARD_LE:
        # at most k of x[i:] true: ite(x_i, atmost(i+1, k-1), atmost(i+1, k))
        cache = {}

        def atmost(i, k):
            if k < 0:
                return FALSE
            if i == L:
                return TRUE
            if (i, k) not in cache:
                cache[(i, k)] = M.ite(x[i], atmost(i + 1, k - 1), atmost(i + 1, k))
            return cache[(i, k)]

        r = atmost(0, int(param))
    elif kind == S.MUX:
        b = int(param)
        assert L == b + (1 << b)

        def sel(i, base):
            if i == b:
                return x[b + base]
            return M.ite(x[i], sel(i + 1, base + (1 << i)), sel(i + 1, base))

        r = sel(0, 0)
    elif kind == S.NEQ_OR:
        P = int(param)
        r = FALSE
        for t in range(P):
            r = M.apply("or", r, M.apply("xor", x[2 * t], x[2 * t + 1]))
        for u in x[2 * P:]:
            r = M.apply("or", r, u)
    else:
        raise ValueError(kind)
    return M, r


def flatten(M: Manager, root: int, lits):
    """Decision nodes reachable from root in topological order (by level).

    Returns (var, hi, lo) where var[v] is the variable/atom id tested by node v
    and hi/lo index into the node list, with index V meaning the TRUE terminal
    and V+1 the FALSE terminal (V = number of decision nodes).
    """
    seen, stack = set(), [root]
    while stack:
        u = stack.pop()
        if u <= TRUE or u in seen:
            continue
        seen.add(u)
        stack += [M.hi[u], M.lo[u]]
    order = sorted(seen, key=lambda u: (M.level[u], u))
    V = len(order)
    pos = {u: i for i, u in enumerate(order)}
    pos[TRUE], pos[FALSE] = V, V + 1
    var = [int(lits[M.level[u]]) >> 1 for u in order]
    hi = [pos[M.hi[u]] for u in order]
    lo = [pos[M.lo[u]] for u in order]
    root_idx = pos[root]
    return var, hi, lo, root_idx


def constraint_diagram(inst, c):
    """(var, hi, lo, root) of constraint c of an instance."""
    lits = inst.lits(c)
    M, r = build(int(inst.con_kind[c]), int(inst.con_param[c]), lits)
    return flatten(M, r, lits)


def evaluate(diagram, truth_of_var) -> bool:
    """Follows the diagram from the root under a truth assignment of its variables."""
    var, hi, lo, root = diagram
    V = len(var)
    v = root
    while v < V:
        v = hi[v] if truth_of_var(var[v]) else lo[v]
    return v == V
