"""Relaxed literal probabilities (TEST INFRASTRUCTURE ONLY), FP64.

* Booleans, randomized rounding (Eq. rounding; Alg. 1 and Alg. 3 set
  p_i = (1 - a_i)/2): the probability that x_i rounds to -1, i.e. TRUE.
* Atoms, Gaussian smoothing (Eq. sampling; Suppl. Note "Expectation"): for the
  atom q.y - q0 <= 0 and y ~ N(b, sigma^2 I), with z = q.b - q0 and
  s = sigma ||q||_2 (q0 excluded from the norm),
      d(b)  = E[delta(y)] = erf(z / (sqrt(2) s)),
      p     = P[atom true] = (1 - d)/2 = erfc(z / (sqrt(2) s)) / 2,
      dd/db_j = sqrt(2) q_j / (sqrt(pi) s) * exp(-z^2 / (2 s^2)).
  The derivative follows the proof of Prop. Lipschitz (Suppl. Note
  "Smoothness"); the printed formula in Suppl. Note "Expectation" has a garbled
  exponent denominator.  GE/GT atoms are negated into LE/LT form first.
  sigma = 0 is the unsmoothed indicator (Thm. expectation, sigma^2 = 0 case):
  p = [z <= 0] (or [z < 0] for a strict atom), decided exactly, and dd/db = 0.
  p is evaluated with erfc rather than 1 - erf so that tails keep their
  relative accuracy (mathematically identical).

Pins: Monte-Carlo over y ~ N(b, sigma^2 I) and central finite differences of d
in the tests; the closed form of the Gaussian CDF through scipy's ndtr.
"""
import math

import numpy as np
from scipy.special import erfc

from . import semantics as S

SQRT2 = math.sqrt(2.0)
TWO_OVER_SQRTPI = 2.0 / math.sqrt(math.pi)


def p_bool(a):
    """P[x_i = TRUE] = (1 - a_i)/2 (Eq. rounding)."""
    return (1.0 - np.asarray(a, np.float64)) / 2.0


def atom_terms(inst, i, b, sigma):
    """(p_true, dd_db) for atom i at points b ([m][R] float64).

    Returns p (shape [R]) and a list of (j, dd/db_j) pairs, each dd/db_j of shape [R].
    """
    var, coef, q0, rel = inst.atom(i)
    coef, q0, strict = S.normalized_atom(coef, q0, rel)
    q = np.asarray(coef, np.float64)
    z = sum(q[t] * np.asarray(b[int(var[t])], np.float64) for t in range(len(q))) - float(q0)
    if sigma == 0.0:  # the indicator itself, decided exactly
        p = S.atom_truth_batch(inst, i, b).astype(np.float64)
        return p, [(int(var[t]), np.zeros_like(z)) for t in range(len(q))]
    s = sigma * math.sqrt(float((q * q).sum()))
    u = z / (SQRT2 * s)
    p = 0.5 * erfc(u)
    g = TWO_OVER_SQRTPI * np.exp(-u * u) / (SQRT2 * s)  # dd/dz
    return p, [(int(var[t]), g * q[t]) for t in range(len(q))]


def atom_d(inst, i, b, sigma):
    """d_i(b) = 1 - 2 p_i  (= erf(z / (sqrt 2 sigma ||q||)))."""
    p, _ = atom_terms(inst, i, b, sigma)
    return 1.0 - 2.0 * p
