"""Pins for the oracle's relaxation, objective and gradient (no GPU)."""
import math

import numpy as np
import pytest
from scipy.special import ndtr

from oracle import objective as OBJ, relax
from workloads import instances as W


def small_instance(seed=3):
    return W.tiny_random(seed, n_bool=8, n_real=4, n_cons=25)


def test_atom_probability_is_gaussian_cdf():
    """Eq. sampling: P[q.Y <= q0], Y ~ N(b, sigma^2 I) = Phi(-z / (sigma ||q||))."""
    B = W._Builder(0, 3)
    B.atom([0, 2], [3, -4], 7, W.LE)
    B.con(W.OR, [W.lit(0)])
    inst = B.freeze("t", np.zeros(3), np.ones(3), [], np.zeros(3), 1.0)
    rng = np.random.default_rng(0)
    b = rng.uniform(-3, 3, (3, 50))
    for sigma in (0.3, 1.0, 4.0):
        p, _ = relax.atom_terms(inst, 0, b, sigma)
        z = 3 * b[0] - 4 * b[2] - 7
        np.testing.assert_allclose(p, ndtr(-z / (sigma * 5.0)), rtol=1e-12, atol=1e-300)


def test_atom_probability_monte_carlo():
    B = W._Builder(0, 2)
    B.atom([0, 1], [2, 1], 3, W.GE)
    B.con(W.OR, [W.lit(0)])
    inst = B.freeze("t", np.zeros(2), np.ones(2), [], np.zeros(2), 1.0)
    b = np.array([[1.2], [0.4]])
    sigma = 0.7
    p, _ = relax.atom_terms(inst, 0, b, sigma)
    rng = np.random.default_rng(1)
    N = 1_000_000
    y = b[:, 0][:, None] + sigma * rng.standard_normal((2, N))
    est = ((2 * y[0] + y[1]) >= 3).mean()
    assert abs(est - p[0]) < 4 * math.sqrt(p[0] * (1 - p[0]) / N)


def _two_atom_or(shared):
    """OR(A1, A2): with shared reals the scheduling non-overlap pair A1: y0 - y1 >= 2,
    A2: y1 - y0 >= 3; without, the same atoms over disjoint reals (y0, y1) and (y2, y3)."""
    B = W._Builder(0, 4)
    A1 = B.atom([1, 0], [1, -1], -2, W.LE)               # y0 - y1 >= 2
    A2 = B.atom([0, 1] if shared else [2, 3], [1, -1], -3, W.LE)   # y1 - y0 >= 3 (or y3 - y2 >= 3)
    B.con(W.OR, [W.lit(A1), W.lit(A2)])
    return B.freeze("or2", np.full(4, -50.0), np.full(4, 50.0), [], np.zeros(4), 1.0)


def test_cop_equals_gaussian_sampling_when_atoms_are_independent():
    """Thm. expectation: with y ~ N(b, sigma^2 I) and atoms over disjoint reals, the
    probability that the constraint holds is exactly the COP of independent atom
    marginals -- checked by sampling y itself (10^6 draws, 4 standard errors)."""
    inst = _two_atom_or(shared=False)
    b = np.array([[0.4], [-1.1], [2.0], [4.2]])
    sigma = 1.3
    w = np.ones((1, 1))
    _, cop, _, _ = OBJ.evaluate(inst, np.zeros((0, 1)), b, w, sigma, with_grad=False)
    rng = np.random.default_rng(5)
    N = 1_000_000
    y = b[:, 0][:, None] + sigma * rng.standard_normal((4, N))
    est = ((y[0] - y[1] >= 2) | (y[3] - y[2] >= 3)).mean()
    assert abs(est - cop[0, 0]) < 4 * math.sqrt(cop[0, 0] * (1 - cop[0, 0]) / N)


def test_shared_reals_diverge_from_gaussian_sampling_as_documented():
    """Reading R4: atoms of one constraint that share reals are correlated under
    y ~ N(b, sigma^2 I), but Alg. 3 (and the oracle) multiplies their marginals.  For
    the non-overlap pair the two atoms exclude each other, so sampling y gives
    P[A1] + P[A2] while the COP is 1 - (1 - P[A1])(1 - P[A2]): the COP falls short by the
    product P[A1] P[A2], far outside the sampling error.  Not a gate on the CUDA path:
    it records what the method computes."""
    inst = _two_atom_or(shared=True)
    b = np.array([[0.3], [0.1], [0.0], [0.0]])
    sigma = 4.0
    w = np.ones((1, 1))
    _, cop, _, _ = OBJ.evaluate(inst, np.zeros((0, 1)), b, w, sigma, with_grad=False)
    p1, _ = relax.atom_terms(inst, 0, b, sigma)
    p2, _ = relax.atom_terms(inst, 1, b, sigma)
    np.testing.assert_allclose(cop[0, 0], 1 - (1 - p1[0]) * (1 - p2[0]), rtol=1e-12)
    rng = np.random.default_rng(6)
    N = 1_000_000
    y = b[:, 0][:, None] + sigma * rng.standard_normal((4, N))
    est = ((y[0] - y[1] >= 2) | (y[1] - y[0] >= 3)).mean()
    se = math.sqrt(est * (1 - est) / N)
    assert abs(est - (p1[0] + p2[0])) < 4 * se
    assert est - cop[0, 0] > 20 * se and abs((est - cop[0, 0]) - p1[0] * p2[0]) < 4 * se


def test_atom_derivative_finite_difference():
    """dd/db_j (Prop. Lipschitz proof form) against central differences of d = 1 - 2p."""
    inst = small_instance()
    rng = np.random.default_rng(2)
    b = rng.uniform(0, 100, (inst.n_real, 3))
    for i in range(min(inst.n_atoms, 12)):
        for sigma in (5.0, 30.0):
            _, terms = relax.atom_terms(inst, i, b, sigma)
            for j, g in terms:
                h = 1e-4
                bp, bm = b.copy(), b.copy()
                bp[j] += h
                bm[j] -= h
                fd = (relax.atom_d(inst, i, bp, sigma) - relax.atom_d(inst, i, bm, sigma)) / (2 * h)
                np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-10)


def test_sigma_zero_is_the_indicator():
    B = W._Builder(0, 1)
    B.atom([0], [1], 2, W.LE)
    B.atom([0], [1], 2, W.LT)
    B.con(W.OR, [W.lit(0)])
    inst = B.freeze("t", np.zeros(1), np.ones(1), [], np.zeros(1), 1.0)
    b = np.array([[1.0, 2.0, 3.0]])
    p_le, t_le = relax.atom_terms(inst, 0, b, 0.0)
    p_lt, _ = relax.atom_terms(inst, 1, b, 0.0)
    assert list(p_le) == [1.0, 1.0, 0.0] and list(p_lt) == [1.0, 0.0, 0.0]
    assert all((g == 0).all() for _, g in t_le)


def test_sigma_infinity_is_a_fair_coin():
    """1/sigma = 0 (the first point of the gradient-time grid): every atom holds with
    probability 1/2 whatever b, and the objective does not depend on b."""
    B = W._Builder(1, 2)
    a0 = B.atom([0, 1], [3, -2], 1, W.LE)
    a1 = B.atom([1], [5], 2, W.LT)
    B.con(W.NAE, [W.lit(0), W.lit(a0)])  # P(not all equal) = 1/2 when the atom is a fair coin
    B.con(W.XOR, [W.lit(0), W.lit(a0, True), W.lit(a1)])
    inst = B.freeze("t", np.zeros(2), np.ones(2), [1], np.zeros(2), 1.0)
    b = np.array([[0.0, 0.3, 1.0], [0.9, 0.2, 0.0]])
    for i in range(2):
        p, terms = relax.atom_terms(inst, i, b, math.inf)
        assert (p == 0.5).all() and all((g == 0).all() for _, g in terms)
    a = np.array([[-0.4, 0.0, 0.7]])
    w = np.ones((2, 3))
    obj, cop, ga, gb = OBJ.evaluate(inst, a, b, w, math.inf)
    assert np.allclose(cop[0], 0.5) and np.allclose(cop[1], 0.5)  # each has a fair literal
    assert (gb == 0).all() and np.allclose(obj, 0.0)


@pytest.mark.parametrize("n", [100, 300])
def test_random_hybrid_planted_assignment_satisfies_everything(n):
    """The random hybrid generator's plant satisfies every cardinality, NAE and
    parity constraint exactly, with the sizes of the paper's benchmark."""
    from oracle import semantics as Sm
    inst = W.random_hybrid(1006, n)
    assert inst.n_bool == n and inst.n_real == n and inst.n_atoms == n
    assert inst.n_cons == 2 * (n // 5) + max(1, n // 50)
    lengths = np.diff(inst.con_ptr)
    assert (lengths[: 2 * (n // 5)] == min(50, n // 5)).all() and (lengths[2 * (n // 5):] == 50).all()
    assert Sm.unsat_constraints(inst, inst.planted_x, inst.planted_y) == []


def test_gradient_central_differences():
    inst = small_instance()
    R = 3
    a, b = W.initial_point(inst, R, seed=4)
    a = a.astype(np.float64) * 0.9
    b = b.astype(np.float64)
    w = np.random.default_rng(5).uniform(0.5, 2.0, (inst.n_cons, R))
    sigma = 20.0
    obj, _, ga, gb = OBJ.evaluate(inst, a, b, w, sigma)
    h = 1e-6
    for i in range(inst.n_bool):
        ap, am = a.copy(), a.copy()
        ap[i] += h
        am[i] -= h
        fd = (OBJ.evaluate(inst, ap, b, w, sigma, with_grad=False)[0] -
              OBJ.evaluate(inst, am, b, w, sigma, with_grad=False)[0]) / (2 * h)
        np.testing.assert_allclose(ga[i], fd, rtol=1e-6, atol=1e-8)
    for j in range(inst.n_real):
        hb = 1e-5
        bp, bm = b.copy(), b.copy()
        bp[j] += hb
        bm[j] -= hb
        fd = (OBJ.evaluate(inst, a, bp, w, sigma, with_grad=False)[0] -
              OBJ.evaluate(inst, a, bm, w, sigma, with_grad=False)[0]) / (2 * hb)
        np.testing.assert_allclose(gb[j], fd, rtol=1e-5, atol=1e-9)


def test_multilinear_identity():
    """Lemma expectation: C is affine in each a_i, so C(a_i=1) - C(a_i=-1) = 2 dC/da_i."""
    inst = small_instance(9)
    R = 2
    a, b = W.initial_point(inst, R, seed=1)
    a = a.astype(np.float64)
    b = b.astype(np.float64)
    w = np.ones((inst.n_cons, R))
    _, _, ga, _ = OBJ.evaluate(inst, a, b, w, 15.0)
    for i in range(inst.n_bool):
        ap, am = a.copy(), a.copy()
        ap[i], am[i] = 1.0, -1.0
        diff = OBJ.evaluate(inst, ap, b, w, 15.0, with_grad=False)[0] - \
            OBJ.evaluate(inst, am, b, w, 15.0, with_grad=False)[0]
        np.testing.assert_allclose(diff, 2 * ga[i], atol=1e-12)


@pytest.mark.parametrize("make", [lambda: W.tiny_random(1001), lambda: W.jobshop(1002, 8, 4),
                                  lambda: W.placement2d(1003, 12), lambda: W.large_scheduling(1005, 16, 20, 6, 3, 5),
                                  lambda: W.large_scheduling(1005, 5, 20, 6, 3, 5),
                                  lambda: W.placement3d(1007, 4, 2)])
def test_soundness_at_planted_vertex(make):
    """Thm. Soundness / Cor. cop=wfe at sigma = 0: every COP is 1 and C = -sum w at a model."""
    inst = make()
    a = inst.planted_x.astype(np.float64)[:, None]
    b = inst.planted_y[:, None]
    w = np.ones((inst.n_cons, 1))
    obj, cops, _, _ = OBJ.evaluate(inst, a, b, w, 0.0, policy=OBJ.SOFT)
    assert np.all(cops == 1.0)
    assert obj[0] == -inst.n_cons


def test_optimality_sigma_zero_affine():
    """Thm. optimality: at sigma = 0, C is multilinear in a (no interior optimum): the
    second difference along each coordinate vanishes."""
    inst = small_instance(4)
    a, b = W.initial_point(inst, 2, seed=8)
    a = a.astype(np.float64) * 0.5
    b = b.astype(np.float64)
    w = np.ones((inst.n_cons, 2))
    for i in range(inst.n_bool):
        vals = []
        for t in (-0.2, 0.0, 0.2):
            ap = a.copy()
            ap[i] += t
            vals.append(OBJ.evaluate(inst, ap, b, w, 0.0, with_grad=False)[0])
        np.testing.assert_allclose(vals[0] - 2 * vals[1] + vals[2], 0.0, atol=1e-12)
