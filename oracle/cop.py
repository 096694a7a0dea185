"""Circuit-output probability of one constraint (TEST INFRASTRUCTURE ONLY), FP64.

Two independent evaluations, both vectorised over restarts only (every array
has shape [R]; restarts are independent copies of the same computation):

1. ``cop_definition`` -- the definition (Suppl. Note "Circuit-Output
   Probability", Remark COP): the sum over all truth assignments of the
   constraint's variables of [c holds] times the product of the literal
   probabilities.  Literal truth values are independent across Booleans and
   atoms, exactly as Alg. 3 treats every atom as its own propositional input.
   ``dcop_definition`` differentiates that sum term by term.  Exponential in
   the constraint width: used for widths up to ~16.

2. ``forward`` / ``backward`` -- the message passing of Alg. 3 and Alg. 4 on
   the constraint's ROBDD, in the paper's order: m_td pushed from the root in
   topological order, m_bu pulled from the TRUE terminal in reverse order.
   Alg. 4 prints Delta = m_td[v] (m_bu[v.F] - m_bu[v.T]); its proof of
   Thm. backward derives dCOP/dz_i = sum_v m_td[v] (m_bu[v.T] - m_bu[v.F]).
   ``backward`` returns that derivative of COP with respect to each variable's
   TRUE-probability; objective.py turns it into the gradient of
   C_sigma = sum_c w_c (1 - 2 COP_c).

Pins (tests/test_oracle_cop.py): definition == message passing on random
constraints of every kind; closed forms (OR: 1 - prod(1 - p); XOR: parity of
independent bits; unit literal: p); the worked arithmetic x1 v x2 v A with
p = (0.25, 0.6, 0.35) -> COP = 0.805; the xWFE identity (Cor. xWFE /
Thm. expectation: sum_{S,T} fhat(S,T) prod a prod d = 1 - 2 COP with fhat by
enumeration); Monte-Carlo rounding; m_td and m_bu invariants (Lemma forward /
Lemma backward).
"""
import itertools

import numpy as np

from . import semantics as S


def _lit_truth(l, var_true):
    return var_true != bool(int(l) & 1)


def cop_definition(kind, param, lits, ptrue):
    """COP_c = sum over assignments of [c] * prod P(literal variable values).

    ptrue maps a variable/atom id to its TRUE-probability (array [R]).
    """
    ids = [int(l) >> 1 for l in lits]
    tot = None
    for vals in itertools.product((True, False), repeat=len(ids)):
        t = [_lit_truth(l, v) for l, v in zip(lits, vals)]
        if not S.kind_value(kind, param, t):
            continue
        pr = 1.0
        for i, v in zip(ids, vals):
            pr = pr * (ptrue[i] if v else 1.0 - ptrue[i])
        tot = pr if tot is None else tot + pr
    if tot is None:
        any_p = next(iter(ptrue.values())) if ptrue else 0.0
        return np.zeros_like(np.asarray(any_p, np.float64))
    return np.asarray(tot, np.float64)


def dcop_definition(kind, param, lits, ptrue):
    """dCOP_c / dP[var true] for each variable of the constraint, from the definition."""
    ids = [int(l) >> 1 for l in lits]
    out = {i: 0.0 for i in ids}
    for vals in itertools.product((True, False), repeat=len(ids)):
        t = [_lit_truth(l, v) for l, v in zip(lits, vals)]
        if not S.kind_value(kind, param, t):
            continue
        for k, (i, v) in enumerate(zip(ids, vals)):
            pr = 1.0 if v else -1.0
            for k2, (i2, v2) in enumerate(zip(ids, vals)):
                if k2 != k:
                    pr = pr * (ptrue[i2] if v2 else 1.0 - ptrue[i2])
            out[i] = out[i] + pr
    return out


def forward(diagram, ptrue, R):
    """Alg. 3 on one diagram: returns (m_td [V+2][R], COP [R]).  Index V is TRUE, V+1 FALSE."""
    var, hi, lo, root = diagram
    V = len(var)
    m_td = np.zeros((V + 2, R))
    m_td[root] = 1.0
    for v in range(V):  # topological order
        p = ptrue[var[v]]
        m_td[hi[v]] += p * m_td[v]
        m_td[lo[v]] += (1.0 - p) * m_td[v]
    return m_td, m_td[V].copy()


def backward(diagram, ptrue, m_td, R):
    """Alg. 4 on one diagram: returns (m_bu [V+2][R], {var: dCOP/dP[var true]})."""
    var, hi, lo, root = diagram
    V = len(var)
    m_bu = np.zeros((V + 2, R))
    m_bu[V] = 1.0
    d = {}
    for v in reversed(range(V)):  # reverse topological order
        p = ptrue[var[v]]
        m_bu[v] = p * m_bu[hi[v]] + (1.0 - p) * m_bu[lo[v]]
        delta = m_td[v] * (m_bu[hi[v]] - m_bu[lo[v]])
        d[var[v]] = d[var[v]] + delta if var[v] in d else delta
    return m_bu, d
