"""The relaxed objective and its exact gradient (TEST INFRASTRUCTURE ONLY), FP64.

C_sigma(a, b) = sum_c w_c (1 - 2 COP_c)   (Alg. 3's fval; Results Eq. objective
with COP read as the probability that c holds, so that 1 - 2 COP_c is the
expectation of f_c in {-1 = TRUE, +1 = FALSE}).

Gradient (chain rule through p = (1 - a)/2 and p = (1 - d)/2, both with
dp/d(.) = -1/2, and d(1 - 2 COP)/dp = -2 dCOP/dp):
  dC/da_i = sum_c w_c dCOP_c/dp_i
  dC/db_j = sum_c w_c sum_{atoms i of c} dCOP_c/dp_i * dd_i/db_j
with dCOP/dp from Alg. 4 (cop.backward).  Check: c = (x_1) gives C = w a_1 and
dC/da_1 = +w; the printed Alg. 4 sign would give -w (an ascent direction).

Which constraints enter C: all of them, except that with the PROJECT policy a
unit atomic constraint (a single atom literal with no Boolean variable,
Prop. QP) is enforced by the projection instead (Methods, "Projected Gradient
Descent") and left out of the objective.

Pins: central finite differences in FP64; the multilinear identity
C(a_i = 1) - C(a_i = -1) = 2 dC/da_i (Lemma expectation: C is affine in each
a_i); definition-based COP on small widths (tests/test_oracle_objective.py).
"""
import numpy as np

from . import bdd, cop, relax

PROJECT, SOFT = 0, 1


def is_unit_atomic(inst, c) -> bool:
    ls = inst.lits(c)
    return int(inst.con_kind[c]) == 0 and len(ls) == 1 and (int(ls[0]) >> 1) >= inst.n_bool


def objective_constraints(inst, policy=PROJECT):
    return [c for c in range(inst.n_cons) if not (policy == PROJECT and is_unit_atomic(inst, c))]


class Diagrams:
    """Per-instance cache of constraint diagrams (built lazily)."""

    def __init__(self, inst):
        self.inst = inst
        self._d = {}

    def __getitem__(self, c):
        d = self._d.get(c)
        if d is None:
            d = self._d[c] = bdd.constraint_diagram(self.inst, c)
        return d


def constraint_probs(inst, c, a, b, sigma):
    """TRUE-probabilities of the constraint's variables and the atoms' dd/db terms."""
    ptrue, dd = {}, {}
    for l in inst.lits(c):
        vid = int(l) >> 1
        if vid < inst.n_bool:
            ptrue[vid] = relax.p_bool(a[vid])
        else:
            p, terms = relax.atom_terms(inst, vid - inst.n_bool, b, sigma)
            ptrue[vid], dd[vid] = p, terms
    return ptrue, dd


def constraint_cop(inst, diagrams, c, a, b, sigma):
    R = a.shape[1] if a.ndim == 2 else b.shape[1]
    ptrue, _ = constraint_probs(inst, c, a, b, sigma)
    _, value = cop.forward(diagrams[c], ptrue, R)
    return value


def constraint_contrib(inst, diagrams, c, a, b, w_c, sigma):
    """(w_c (1 - 2 COP_c), COP_c, {i: dC/da_i part}, {j: dC/db_j part}) for one constraint."""
    R = a.shape[1] if a.ndim == 2 else b.shape[1]
    ptrue, dd = constraint_probs(inst, c, a, b, sigma)
    D = diagrams[c]
    m_td, value = cop.forward(D, ptrue, R)
    _, dcop = cop.backward(D, ptrue, m_td, R)
    ga, gb = {}, {}
    for vid, g in dcop.items():
        if vid < inst.n_bool:
            ga[vid] = ga.get(vid, 0.0) + w_c * g
        else:
            for j, ddj in dd[vid]:
                gb[j] = gb.get(j, 0.0) + w_c * g * ddj
    return w_c * (1.0 - 2.0 * value), value, ga, gb


def evaluate(inst, a, b, w, sigma, policy=PROJECT, diagrams=None, with_grad=True):
    """Full objective over an instance.

    a: [n][R], b: [m][R], w: [C][R] (indexed by constraint id).
    Returns obj [R], cop [C][R] (NaN for constraints outside the objective),
    grad_a [n][R], grad_b [m][R].
    """
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    w = np.asarray(w, np.float64)
    R = w.shape[1]
    diagrams = diagrams or Diagrams(inst)
    obj = np.zeros(R)
    cops = np.full((inst.n_cons, R), np.nan)
    grad_a = np.zeros((inst.n_bool, R))
    grad_b = np.zeros((inst.n_real, R))
    for c in objective_constraints(inst, policy):
        if with_grad:
            o, value, ga, gb = constraint_contrib(inst, diagrams, c, a, b, w[c], sigma)
            for i, g in ga.items():
                grad_a[i] += g
            for j, g in gb.items():
                grad_b[j] += g
        else:
            value = constraint_cop(inst, diagrams, c, a, b, sigma)
            o = w[c] * (1.0 - 2.0 * value)
        obj += o
        cops[c] = value
    return obj, cops, grad_a, grad_b
