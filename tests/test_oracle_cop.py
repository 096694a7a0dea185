"""Pins for the oracle's diagrams and COP (no GPU).

Each check is fixed by something other than the code under test: truth tables
of the kinds, closed-form probabilities, the xWFE expansion by enumeration,
Monte-Carlo sampling, or the paper's own lemmas.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import bdd, cop, semantics as S
from workloads import instances as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
KINDS = [S.OR, S.XOR, S.CARD_LE, S.NAE, S.MUX, S.NEQ_OR]


def random_constraint(rng, kind):
    if kind == S.MUX:
        b = int(rng.integers(1, 3))
        L, param = b + (1 << b), b
    elif kind == S.NEQ_OR:
        P = int(rng.integers(1, 4))
        L, param = 2 * P + int(rng.integers(0, 3)), P
    else:
        L = int(rng.integers(1, 8))
        param = int(rng.integers(0, L + 1)) if kind == S.CARD_LE else 0
    ids = rng.choice(40, L, replace=False)
    lits = [2 * int(i) + int(rng.integers(2)) for i in ids]
    return kind, param, lits


@pytest.mark.parametrize("kind", KINDS)
def test_diagram_computes_the_kind(kind):
    rng = np.random.default_rng(kind)
    for _ in range(25):
        k, param, lits = random_constraint(rng, kind)
        M, root = bdd.build(k, param, lits)
        D = bdd.flatten(M, root, lits)
        ids = [l >> 1 for l in lits]
        for vals in itertools.product((True, False), repeat=len(ids)):
            truth = dict(zip(ids, vals))
            t = [truth[l >> 1] != bool(l & 1) for l in lits]
            assert bdd.evaluate(D, truth.__getitem__) == S.kind_value(k, param, t)
        # reduced: no node with equal children, no duplicate triple
        var, hi, lo, _ = D
        assert all(h != l for h, l in zip(hi, lo))
        assert len(set(zip(var, hi, lo))) == len(var)
        # topological: children come later
        assert all(h > v and l > v for v, (h, l) in enumerate(zip(hi, lo)))


def test_node_count_closed_forms():
    for L in range(1, 9):
        lits = [2 * i for i in range(L)]
        assert len(bdd.flatten(*bdd.build(S.OR, 0, lits), lits)[0]) == L
        assert len(bdd.flatten(*bdd.build(S.XOR, 0, lits), lits)[0]) == 2 * L - 1
    lits = [2 * i for i in range(6)]
    assert len(bdd.flatten(*bdd.build(S.MUX, 2, lits), lits)[0]) == 7
    for P in range(1, 9):
        for r in range(3):
            lits = [2 * i for i in range(2 * P + r)]
            assert len(bdd.flatten(*bdd.build(S.NEQ_OR, P, lits), lits)[0]) == 3 * P + r


def probs_for(lits, rng, R):
    return {l >> 1: rng.uniform(0.0, 1.0, R) for l in lits}


@pytest.mark.parametrize("kind", KINDS)
def test_message_passing_equals_definition(kind):
    """Alg. 3 / Alg. 4 on the diagram == the sum over assignments (Remark COP)."""
    rng = np.random.default_rng(100 + kind)
    R = 5
    for _ in range(20):
        k, param, lits = random_constraint(rng, kind)
        P = probs_for(lits, rng, R)
        D = bdd.flatten(*bdd.build(k, param, lits), lits)
        m_td, value = cop.forward(D, P, R)
        ref = cop.cop_definition(k, param, lits, P)
        np.testing.assert_allclose(value, ref, rtol=0, atol=1e-14)
        _, dd = cop.backward(D, P, m_td, R)
        dref = cop.dcop_definition(k, param, lits, P)
        for i in dref:
            np.testing.assert_allclose(dd.get(i, 0.0), dref[i], rtol=0, atol=1e-13)


def test_closed_forms():
    rng = np.random.default_rng(7)
    R = 6
    for L in range(1, 8):
        lits = [2 * i + int(rng.integers(2)) for i in range(L)]
        P = probs_for(lits, rng, R)
        pl = [P[l >> 1] if not (l & 1) else 1 - P[l >> 1] for l in lits]  # literal probabilities
        D = lambda k, prm: bdd.flatten(*bdd.build(k, prm, lits), lits)
        # OR: 1 - prod(1 - p_l)
        np.testing.assert_allclose(cop.forward(D(S.OR, 0), P, R)[1], 1 - np.prod([1 - p for p in pl], 0), atol=1e-14)
        # XOR: P[odd number true] = (1 - prod(1 - 2 p_l)) / 2
        np.testing.assert_allclose(cop.forward(D(S.XOR, 0), P, R)[1], (1 - np.prod([1 - 2 * p for p in pl], 0)) / 2, atol=1e-14)
        # CARD_LE: Poisson-binomial distribution by polynomial multiplication
        for k in range(L + 1):
            dist = np.ones((1, R))
            for p in pl:
                nd = np.zeros((dist.shape[0] + 1, R))
                nd[:-1] += dist * (1 - p)
                nd[1:] += dist * p
                dist = nd
            np.testing.assert_allclose(cop.forward(D(S.CARD_LE, k), P, R)[1], dist[:k + 1].sum(0), atol=1e-13)
        # NAE: 1 - P[all true] - P[all false]
        np.testing.assert_allclose(cop.forward(D(S.NAE, 0), P, R)[1],
                                   1 - np.prod(pl, 0) - np.prod([1 - p for p in pl], 0), atol=1e-14)
    # MUX with 2 selectors: sum over indices of P[index] * p_data
    lits = [0, 3, 4, 7, 8, 10]
    P = probs_for(lits, rng, R)
    pl = [P[l >> 1] if not (l & 1) else 1 - P[l >> 1] for l in lits]
    ref = sum((pl[0] if i & 1 else 1 - pl[0]) * (pl[1] if i & 2 else 1 - pl[1]) * pl[2 + i] for i in range(4))
    np.testing.assert_allclose(cop.forward(bdd.flatten(*bdd.build(S.MUX, 2, lits), lits), P, R)[1], ref, atol=1e-14)


def test_worked_clause_arithmetic():
    """x1 v x2 v A with a = (0.5, -0.2), d_A = 0.3: p = (0.25, 0.6, 0.35), COP = 0.805,
    C = 1 - 2 COP = -0.61, dC/da1 = dCOP/dp1 = 0.4 * 0.65 = 0.26."""
    lits = [0, 2, 4]
    P = {0: np.array([0.25]), 1: np.array([0.6]), 2: np.array([0.35])}
    D = bdd.flatten(*bdd.build(S.OR, 0, lits), lits)
    m_td, value = cop.forward(D, P, 1)
    assert abs(value[0] - 0.805) < 1e-15
    assert abs(1 - 2 * value[0] + 0.61) < 1e-15
    _, dd = cop.backward(D, P, m_td, 1)
    assert abs(dd[0][0] - 0.26) < 1e-15


@pytest.mark.parametrize("kind", KINDS)
def test_xwfe_identity(kind):
    """Cor. xWFE + Thm. expectation: sum_U fhat(U) prod_{i in U} E[z_i] = 1 - 2 COP,
    with fhat(U) = E_z[f(z) prod_U z_i] over the uniform cube and f = -1 when c holds."""
    rng = np.random.default_rng(300 + kind)
    for _ in range(10):
        k, param, lits = random_constraint(rng, kind)
        if len(lits) > 7:
            continue
        ids = [l >> 1 for l in lits]
        L = len(ids)
        zs = list(itertools.product((-1, 1), repeat=L))  # -1 = TRUE
        f = {}
        for z in zs:
            t = [(zi == -1) != bool(l & 1) for zi, l in zip(z, lits)]
            f[z] = -1.0 if S.kind_value(k, param, t) else 1.0
        fhat = {}
        for U in itertools.product((0, 1), repeat=L):
            fhat[U] = sum(f[z] * np.prod([zi for zi, u in zip(z, U) if u]) for z in zs) / len(zs)
        P = probs_for(lits, rng, 3)
        Ez = [1 - 2 * P[i] for i in ids]  # E[z_i] = (+1)(1-p) + (-1)p: a_i for Booleans, d_i for atoms
        expansion = sum(fhat[U] * np.prod([e for e, u in zip(Ez, U) if u], 0) for U in fhat)
        value = cop.cop_definition(k, param, lits, P)
        np.testing.assert_allclose(expansion, 1 - 2 * value, atol=1e-13)


def test_monte_carlo_rounding():
    """E over independent literal samples (Eq. rounding) matches COP within 4 standard errors."""
    rng = np.random.default_rng(11)
    N = 400_000
    for kind in KINDS:
        k, param, lits = random_constraint(rng, kind)
        ids = [l >> 1 for l in lits]
        P = {i: np.array([rng.uniform(0.1, 0.9)]) for i in ids}
        samples = {i: rng.random(N) < P[i][0] for i in ids}
        T = np.stack([samples[l >> 1] != bool(l & 1) for l in lits])
        from oracle.pgd import kind_value_vec
        hits = kind_value_vec(k, param, T)
        est = hits.mean()
        se = math.sqrt(max(est * (1 - est), 1e-12) / N)
        D = bdd.flatten(*bdd.build(k, param, lits), lits)
        value = cop.forward(D, P, 1)[1][0]
        assert abs(est - value) <= 4 * se + 1e-12, (kind, est, value, se)


def test_message_invariants():
    """Lemma forward: m_td[v] is a path probability (in [0,1], terminals sum to 1).
    Lemma backward: m_bu[v] is the COP of the sub-diagram at v (in [0,1]); m_bu[root] = COP."""
    rng = np.random.default_rng(5)
    for kind in KINDS:
        for _ in range(10):
            k, param, lits = random_constraint(rng, kind)
            P = probs_for(lits, rng, 4)
            D = bdd.flatten(*bdd.build(k, param, lits), lits)
            V = len(D[0])
            m_td, value = cop.forward(D, P, 4)
            m_bu, _ = cop.backward(D, P, m_td, 4)
            assert (m_td >= -1e-15).all() and (m_td <= 1 + 1e-15).all()
            assert (m_bu >= -1e-15).all() and (m_bu <= 1 + 1e-15).all()
            np.testing.assert_allclose(m_td[V] + m_td[V + 1], 1.0, atol=1e-14)
            root = D[3]
            np.testing.assert_allclose(m_bu[root], value, atol=1e-14)


def test_fig2_toy_vertices():
    """Fig. 2: (not x) xor A and x and A, A = (y > 0): F = -2 at the global, 0 at the local minimum."""
    gold = json.load(open(os.path.join(GOLD, "fig2_toy.json")))
    B = W._Builder(1, 1)
    A = B.atom([0], [1], 0, W.GT)
    B.con(W.XOR, [W.lit(0, True), W.lit(A)])
    B.con(W.CARD_LE, [W.lit(0, True), W.lit(A, True)], param=0)  # x and A: no negated literal true
    for v in gold["vertices"]:
        xt, at = v["x"] == -1, v["delta"] == -1
        F = 0
        for c in range(2):
            ls = B.lits[B.ptr[c]:B.ptr[c + 1]]
            t = [(xt if (l >> 1) == 0 else at) != bool(l & 1) for l in ls]
            F += -1 if S.kind_value(B.kind[c], B.param[c], t) else 1
        assert F == v["F"], v


def test_intro_example_models():
    gold = json.load(open(os.path.join(GOLD, "intro_example.json")))
    found = []
    for x1, x2, A in itertools.product((True, False), repeat=3):
        if S.kind_value(S.XOR, 0, [x1, x2]) and S.kind_value(S.OR, 0, [x1, A]):
            found.append([x1, x2, A])
    assert sorted(found) == sorted(gold["satisfying"])
