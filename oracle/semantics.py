"""Plain definitions of constraint kinds and atoms (TEST INFRASTRUCTURE ONLY).

A constraint c is a Boolean function of its literals' truth values (Results,
"Satisfiability Modulo Theories"; Methods, "Benchmark Problem Descriptions"
for cardinality, not-all-equal and parity).  An atom is the linear relation
sum_j q_ij y_j - q_i0 (rel) 0 (Results, "Walsh-Fourier Expansions"; rel one of
<=, <, >=, >, = as in Results, "Satisfiability Modulo Theories"); its indicator
delta_i(y) is -1 when it holds.

Pins: each kind is checked in the tests against hand-written truth tables and
the planted assignments of the input generators; atom truth is exact rational
arithmetic (Python Fractions), the textbook meaning of the relation.
"""
from fractions import Fraction

import numpy as np

OR, XOR, CARD_LE, NAE, MUX, NEQ_OR = 0, 1, 2, 3, 4, 5
LE, LT, GE, GT, EQ = 0, 1, 2, 3, 4


def kind_value(kind: int, param: int, t) -> bool:
    """The Boolean value of a constraint given its literals' truth values ``t`` (list of bool)."""
    if kind == OR:
        return any(t)
    if kind == XOR:
        return sum(t) % 2 == 1
    if kind == CARD_LE:
        return sum(t) <= param
    if kind == NAE:
        return any(t) and not all(t)
    if kind == MUX:
        b = param
        idx = sum((1 << i) for i in range(b) if t[i])
        return bool(t[b + idx])
    if kind == NEQ_OR:
        P = param
        return any(t[2 * i] != t[2 * i + 1] for i in range(P)) or any(t[2 * P:])
    raise ValueError(f"unknown constraint kind {kind}")


def atom_holds_exact(coef, var, q0, rel, y) -> bool:
    """Exact truth of sum_j coef_j y_var_j  rel  q0 for float y values (dyadic rationals)."""
    s = sum(Fraction(int(c)) * Fraction(float(y[int(v)])) for c, v in zip(coef, var)) - Fraction(int(q0))
    if rel == LE:
        return s <= 0
    if rel == LT:
        return s < 0
    if rel == GE:
        return s >= 0
    if rel == GT:
        return s > 0
    if rel == EQ:
        return s == 0
    raise ValueError(rel)


def normalized_atom(coef, q0, rel):
    """Rewrites GE/GT as LE/LT by negating both sides: returns (coef, q0, strict).
    An equality has no such form (its smoothed probability is 0: it may only be a
    projected unit constraint), so it raises."""
    if rel == EQ:
        raise ValueError("an equality atom has no relaxed (<=) form")
    if rel in (GE, GT):
        return [-int(c) for c in coef], -int(q0), rel == GT
    return [int(c) for c in coef], int(q0), rel == LT


def literal_truth(inst, l, x, y) -> bool:
    """Truth of literal l under a Boolean assignment x (+-1, -1 = TRUE) and reals y (exact)."""
    vid, neg = int(l) >> 1, int(l) & 1
    if vid < inst.n_bool:
        val = x[vid] == -1
    else:
        var, coef, q0, rel = inst.atom(vid - inst.n_bool)
        val = atom_holds_exact(coef, var, q0, rel, y)
    return val != bool(neg)


def constraint_holds(inst, c, x, y) -> bool:
    t = [literal_truth(inst, l, x, y) for l in inst.lits(c)]
    return kind_value(int(inst.con_kind[c]), int(inst.con_param[c]), t)


def unsat_constraints(inst, x, y):
    """Indices of the constraints violated by (x, y), all decided exactly."""
    return [c for c in range(inst.n_cons) if not constraint_holds(inst, c, x, y)]


def atom_truth_batch(inst, i, y):
    """Exact truth of atom i at each column of reals y [m][R] (float values).

    A float64 evaluation decides the sign when it is far from zero relative to
    a bound on its rounding error; otherwise the sign is computed in Fractions.
    """
    var, coef, q0, rel = inst.atom(i)
    yv = np.asarray(y, np.float64)[np.asarray(var, np.int64)]
    q = np.asarray(coef, np.float64)[:, None]
    s = (q * yv).sum(0) - float(q0)
    mag = (np.abs(q * yv)).sum(0) + abs(float(q0))
    unsure = np.abs(s) <= 1e-12 * mag
    for r in np.nonzero(unsure)[0]:
        fr = sum(Fraction(int(c)) * Fraction(float(v)) for c, v in zip(coef, yv[:, r])) - Fraction(int(q0))
        s[r] = float((fr > 0) - (fr < 0))  # the exact sign
    if rel == LE:
        return s <= 0
    if rel == LT:
        return s < 0
    if rel == GE:
        return s >= 0
    if rel == EQ:
        return s == 0
    return s > 0
