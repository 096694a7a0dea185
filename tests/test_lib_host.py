"""The C-ABI library on the host (no GPU): loading, exported symbols, the xBDD
compiler against the oracle's diagrams, projection bounds, the exact verifier
and argument validation."""
import ctypes as C
import math
from fractions import Fraction
import os
import re

import numpy as np
import pytest

from oracle import bdd, objective as OBJ, pgd, semantics as S
from paper_2603_22877_b300 import _lib as L
from paper_2603_22877_b300 import build as B
from paper_2603_22877_b300.engine import Problem
from workloads import instances as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    B.build()
    return L.load()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "fsmt.h")).read()
    declared = set(re.findall(r"\b(fsmt_[a-z_0-9]+)\s*\(", hdr))
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(lib, name), name
    assert set(L.PROTOTYPES) == declared


SMALL = {
    "tiny_random": lambda: W.tiny_random(1001),
    "jobshop": lambda: W.jobshop(1002, 8, 4),
    "placement2d": lambda: W.placement2d(1003, 14),
    "placement2d_nosel": lambda: W.placement2d(1003, 10, selectors=False),
    "large_scheduling": lambda: W.large_scheduling(1005, 16, 24, 6, 3, 5),
    "large_scheduling_5w": lambda: W.large_scheduling(1005, 5, 24, 6, 3, 5),
    "placement3d": lambda: W.placement3d(1007, 4, 4),
    "uneven_batch": lambda: W.concat(W.uneven_batch(1004, 3, (3, 6), (2, 4)), "b"),
}


@pytest.mark.parametrize("name", list(SMALL))
def test_compiler_matches_oracle_diagrams(name):
    inst = SMALL[name]()
    P = Problem.from_instance(inst)
    for policy in (L.UNIT_PROJECT, L.UNIT_SOFT):
        comp = P.compile(policy)
        D = comp.diagrams()
        obj_cons = OBJ.objective_constraints(inst, policy)
        assert comp.info["n_obj_cons"] == len(obj_cons)
        assert list(D["con_id"][:len(obj_cons)]) == obj_cons
        assert sorted(D["con_id"]) == list(range(inst.n_cons))
        total = 0
        for s in range(inst.n_cons):
            c = int(D["con_id"][s])
            ref = bdd.constraint_diagram(inst, c)
            b0, b1 = D["con_ptr"][s], D["con_ptr"][s + 1]
            V = b1 - b0
            assert V == len(ref[0]), (name, c)  # canonical ROBDD for the same order
            total += V
            mine = (list(D["label"][b0:b1]), list(D["hi"][b0:b1]), list(D["lo"][b0:b1]),
                    int(D["con_root"][s]))
            # topological order: every child lies after its node (terminals V, V + 1), so
            # the device's walk from the root always ends at a terminal
            for v in range(V):
                assert D["hi"][b0 + v] > v and D["lo"][b0 + v] > v and D["hi"][b0 + v] <= V + 1
                assert D["lo"][b0 + v] <= V + 1
            assert int(D["con_root"][s]) <= V + 1 and (V == 0 or int(D["con_root"][s]) == 0)
            ids = sorted({int(l) >> 1 for l in inst.lits(c)})
            rng = np.random.default_rng(c)
            for _ in range(8):
                vals = {i: bool(rng.integers(2)) for i in ids}
                assert bdd.evaluate(mine, vals.__getitem__) == bdd.evaluate(ref, vals.__getitem__)
        assert total == comp.info["n_nodes"]


def test_all_kinds_random_constraints():
    rng = np.random.default_rng(3)
    Bd = W._Builder(30, 2)
    for _ in range(200):
        kind = int(rng.integers(6))
        if kind == W.MUX:
            b = int(rng.integers(1, 3))
            L_, param = b + (1 << b), b
        elif kind == W.NEQ_OR:
            P_ = int(rng.integers(0, 4))
            L_, param = 2 * P_ + int(rng.integers(0, 3)), P_
        else:
            L_ = int(rng.integers(0, 9))
            param = int(rng.integers(0, L_ + 2)) if kind == W.CARD_LE else 0
        ids = rng.choice(30, L_, replace=False)
        Bd.con(kind, [2 * int(i) + int(rng.integers(2)) for i in ids], param)
    inst = Bd.freeze("k", np.zeros(2), np.ones(2), np.ones(30), np.zeros(2), 1.0)
    comp = Problem.from_instance(inst).compile()
    D = comp.diagrams()
    for s in range(inst.n_cons):
        c = int(D["con_id"][s])
        b0, b1 = D["con_ptr"][s], D["con_ptr"][s + 1]
        mine = (list(D["label"][b0:b1]), list(D["hi"][b0:b1]), list(D["lo"][b0:b1]), int(D["con_root"][s]))
        ref = bdd.constraint_diagram(inst, c)
        assert b1 - b0 == len(ref[0])
        ls = inst.lits(c)
        ids = [int(l) >> 1 for l in ls]
        for mask in range(1 << len(ids)) if len(ids) <= 6 else rng.integers(0, 1 << len(ids), 40):
            vals = {i: bool((int(mask) >> k) & 1) for k, i in enumerate(ids)}
            t = [vals[int(l) >> 1] != bool(int(l) & 1) for l in ls]
            assert bdd.evaluate(mine, vals.__getitem__) == S.kind_value(int(inst.con_kind[c]),
                                                                        int(inst.con_param[c]), t)


def test_repeated_shapes_are_relabelled_not_confused():
    """The compiler builds each (kind, parameter, length, negations) shape once and
    relabels it: constraints of one shape over different variables, and constraints that
    differ only in the parameter or in one negation, must each compute their own function
    (every assignment checked)."""
    rng = np.random.default_rng(11)
    Bd = W._Builder(64, 1)
    specs = []
    for kind, L_, params in ((W.OR, 4, [0]), (W.XOR, 5, [0]), (W.NAE, 4, [0]), (W.CARD_LE, 5, [0, 1, 2, 3, 5]),
                             (W.MUX, 6, [2]), (W.NEQ_OR, 6, [0, 1, 2, 3])):
        negs = rng.integers(0, 2, L_)
        for param in params:
            for flip in (None, 0, L_ - 1):
                n2 = negs.copy()
                if flip is not None:
                    n2[flip] ^= 1
                for _ in range(3):                       # the same shape on other variables
                    ids = rng.choice(64, L_, replace=False)
                    specs.append((kind, param, [2 * int(i) + int(n) for i, n in zip(ids, n2)]))
    for kind, param, lits in specs:
        Bd.con(kind, lits, param)
    inst = Bd.freeze("shapes", np.zeros(1), np.ones(1), np.ones(64), np.zeros(1), 1.0)
    D = Problem.from_instance(inst).compile().diagrams()
    for s in range(inst.n_cons):
        c = int(D["con_id"][s])
        b0, b1 = D["con_ptr"][s], D["con_ptr"][s + 1]
        mine = (list(D["label"][b0:b1]), list(D["hi"][b0:b1]), list(D["lo"][b0:b1]), int(D["con_root"][s]))
        ls = inst.lits(c)
        ids = [int(l) >> 1 for l in ls]
        assert sorted(set(int(x) for x in mine[0])) == sorted(set(ids)) or b1 == b0
        for mask in range(1 << len(ids)):
            vals = {i: bool((mask >> k) & 1) for k, i in enumerate(ids)}
            t = [vals[int(l) >> 1] != bool(int(l) & 1) for l in ls]
            assert bdd.evaluate(mine, vals.__getitem__) == S.kind_value(int(inst.con_kind[c]),
                                                                        int(inst.con_param[c]), t), (c, mask)


def test_bounds_rounded_inward_and_match_oracle():
    inst = W.jobshop(1002, 8, 4)
    comp = Problem.from_instance(inst).compile()
    lo, hi = comp.bounds()
    dom = pgd.Domain(inst)
    np.testing.assert_allclose(lo, dom.lo, rtol=1e-7)
    np.testing.assert_allclose(hi, dom.hi, rtol=1e-7)
    assert (lo.astype(np.float64) >= dom.lo).all() and (hi.astype(np.float64) <= dom.hi).all()
    assert comp.info["n_halfspaces"] == len(dom.halfspaces)
    # fractional bound: 3 y <= 7 -> hi = largest float <= 7/3
    Bd = W._Builder(0, 1)
    Bd.con(W.OR, [W.lit(Bd.atom([0], [3], 7, W.LE))])
    Bd.con(W.OR, [W.lit(Bd.atom([0], [-3], -1, W.LT))])  # -3y < -1 -> y > 1/3
    inst2 = Bd.freeze("f", np.array([-5.0]), np.array([5.0]), [], np.zeros(1), 1.0)
    lo2, hi2 = Problem.from_instance(inst2).compile().bounds()
    assert float(hi2[0]) * 3 <= 7 and float(np.nextafter(hi2[0], np.float32(9))) * 3 > 7
    assert float(lo2[0]) * -3 < -1 and float(np.nextafter(lo2[0], np.float32(-9))) * -3 >= -1


@pytest.mark.parametrize("seed", range(6))
def test_random_unit_atoms_give_the_tightest_exact_fp32_box(seed):
    """Single-variable unit atoms of every relation, coefficient sign and literal polarity
    (several per real, all true at a planted point): the compiled FP32 box is the
    tightest one whose every point satisfies every unit atom exactly -- the clamp of the
    projection never leaves a unit atom false -- and it agrees with the oracle's exact
    rational box to FP32 rounding.  Where the atoms pin a real to a value FP32 cannot
    represent, the box is empty (lo > hi), no float satisfies them, and the compiled
    information counts it."""
    from fractions import Fraction
    rng = np.random.default_rng(seed)
    m = 12
    ystar = [Fraction(int(rng.integers(-400, 400)), int(rng.integers(1, 9))) for _ in range(m)]
    Bd = W._Builder(0, m)
    atoms = []
    for _ in range(60):
        j = int(rng.integers(m))
        cj = int(rng.integers(1, 8)) * int(rng.choice([-1, 1]))
        rel = int(rng.integers(4))
        v = cj * ystar[j]
        q0 = round(v) + int(rng.integers(-2, 3))          # often right at the boundary
        z = v - q0
        truth = {W.LE: z <= 0, W.LT: z < 0, W.GE: z >= 0, W.GT: z > 0}[rel]
        neg = not truth                                    # the literal holds at y*
        Bd.con(W.OR, [W.lit(Bd.atom([j], [cj], q0, rel), neg)])
        atoms.append((j, cj, q0, rel, neg))
    inst = Bd.freeze("box", np.full(m, -1000.0), np.full(m, 1000.0), [], np.array([float(y) for y in ystar]), 1.0)
    # every unit literal holds at the plant (by construction), so the box is not empty
    def lit_holds(j, cj, q0, rel, neg, y):
        z = cj * Fraction(y) - q0
        t = {W.LE: z <= 0, W.LT: z < 0, W.GE: z >= 0, W.GT: z > 0}[rel]
        return t != neg
    assert all(lit_holds(*a, ystar[a[0]]) for a in atoms)
    comp = Problem.from_instance(inst).compile()
    lo, hi = comp.bounds()
    dom = pgd.Domain(inst)
    assert comp.info["empty_boxes"] == int((lo > hi).sum())
    for j in range(m):
        mine = [a for a in atoms if a[0] == j]
        if lo[j] > hi[j]:
            # the unit atoms pin y_j to a value FP32 cannot represent: no float between
            # the two bounds (inclusive) satisfies them all, and the exact box is a point
            assert dom.lo[j] == dom.hi[j]
            f = hi[j]
            while f <= lo[j]:
                assert not all(lit_holds(*a, float(f)) for a in mine), (j, f)
                f = np.nextafter(f, np.float32(np.inf))
            continue
        for y in (float(lo[j]), float(hi[j])):
            assert all(lit_holds(*a, y) for a in mine), (j, y)
            assert -1000.0 <= y <= 1000.0
        # tightest: one FP32 step outwards breaks an atom or leaves the original box
        out_lo, out_hi = float(np.nextafter(lo[j], np.float32(-np.inf))), float(np.nextafter(hi[j], np.float32(np.inf)))
        assert out_lo < -1000.0 or not all(lit_holds(*a, out_lo) for a in mine), j
        assert out_hi > 1000.0 or not all(lit_holds(*a, out_hi) for a in mine), j
        assert abs(float(lo[j]) - dom.lo[j]) <= 1e-6 * max(1.0, abs(dom.lo[j]))
        assert abs(float(hi[j]) - dom.hi[j]) <= 1e-6 * max(1.0, abs(dom.hi[j]))


@pytest.mark.parametrize("name", list(SMALL))
def test_verify_exact_matches_oracle(name):
    inst = SMALL[name]()
    P = Problem.from_instance(inst)
    sat, first = P.verify_exact(inst.planted_x, inst.planted_y)
    assert sat and first == -1
    rng = np.random.default_rng(1)
    for _ in range(6):
        x = inst.planted_x.copy()
        flip = rng.random(inst.n_bool) < 0.1
        x[flip] *= -1
        y = inst.planted_y + rng.normal(0, 2.0, inst.n_real) * (rng.random(inst.n_real) < 0.3)
        sat, first = P.verify_exact(x, y)
        bad = S.unsat_constraints(inst, x, y)
        assert sat == (not bad)
        assert first == (bad[0] if bad else -1)


def test_verify_exact_boundary_and_tiny_values():
    Bd = W._Builder(0, 2)
    Bd.con(W.OR, [W.lit(Bd.atom([0, 1], [3, -7], 0, W.LE))])
    Bd.con(W.OR, [W.lit(Bd.atom([0, 1], [3, -7], 0, W.LT))])
    inst = Bd.freeze("e", np.zeros(2), np.ones(2), [], np.zeros(2), 1.0)
    P = Problem.from_instance(inst)
    y = np.array([7.0 * 2.0 ** -1060, 3.0 * 2.0 ** -1060])  # 3*7e - 7*3e = 0 exactly, subnormal scale
    assert P.verify_exact(np.zeros(0, np.int8), y) == (False, 1)
    y2 = np.array([7.0 * 2.0 ** -1060, np.nextafter(3.0 * 2.0 ** -1060, 1.0)])
    assert P.verify_exact(np.zeros(0, np.int8), y2) == (True, -1)


@pytest.mark.parametrize("seed", range(3))
def test_verify_exact_on_random_boundaries(seed):
    """The host's exact atom test against rational arithmetic: sums of up to six terms
    with coefficients up to 2^24 - 1 and reals spread over 2^-80 .. 2^60 (so that the
    terms' magnitudes are far apart), right-hand sides on, just below and just above the
    exact value, every relation, and the reals nudged by one ulp across the boundary."""
    from fractions import Fraction
    rng = np.random.default_rng(100 + seed)
    for _ in range(120):
        nnz = int(rng.integers(1, 7))
        var = list(range(nnz))
        coef = [int(rng.integers(1, 1 << 24)) * int(rng.choice([-1, 1])) for _ in range(nnz)]
        y = np.array([float(rng.integers(1, 1 << 20)) * 2.0 ** int(rng.integers(-80, 40)) * float(rng.choice([-1, 1]))
                      for _ in range(nnz)])
        exact = sum(Fraction(c_) * Fraction(float(v)) for c_, v in zip(coef, y))
        if abs(exact) >= 2 ** 52:
            continue
        base = math.floor(exact)
        for q0 in (base - 1, base, base + 1):
            for rel in (W.LE, W.LT, W.GE, W.GT):
                Bd = W._Builder(0, nnz)
                Bd.con(W.OR, [W.lit(Bd.atom(var, coef, q0, rel))])
                inst = Bd.freeze("b", np.full(nnz, -np.inf), np.full(nnz, np.inf), [], y, 1.0)
                P = Problem.from_instance(inst)
                for yy in (y, np.nextafter(y, np.inf), np.nextafter(y, -np.inf)):
                    z = sum(Fraction(c_) * Fraction(float(v)) for c_, v in zip(coef, yy)) - q0
                    want = {W.LE: z <= 0, W.LT: z < 0, W.GE: z >= 0, W.GT: z > 0}[rel]
                    assert P.verify_exact(np.zeros(0, np.int8), yy)[0] == want, (coef, list(yy), q0, rel)


@pytest.mark.parametrize("seed", range(8))
def test_projection_blocks_match_the_coupling_graph(seed):
    """Multi-variable unit atoms couple reals into blocks that the projection handles
    one by one: the compiled half-space, block and free-real counts equal the connected
    components of the coupling graph (computed here by a plain graph search), under
    PROJECT only; SOFT keeps every unit atom in C_sigma."""
    rng = np.random.default_rng(seed)
    m = 90
    Bd = W._Builder(3, m)
    edges = []
    for _ in range(int(rng.integers(5, 30))):
        k = int(rng.integers(2, 4))
        vs = [int(v) for v in rng.choice(m, k, replace=False)]
        Bd.con(W.OR, [W.lit(Bd.atom(vs, [1] * (k - 1) + [-1], int(rng.integers(-5, 5)), W.LE))])
        edges.append(vs)
    for _ in range(10):                                   # single-variable ones only tighten the box
        Bd.con(W.OR, [W.lit(Bd.atom([int(rng.integers(m))], [1], 100, W.LE))])
    Bd.con(W.OR, [W.lit(0), W.lit(Bd.atom([0, 1], [1, 1], 50, W.LE))])   # not unit: has a Boolean
    inst = Bd.freeze("blocks", np.zeros(m), np.full(m, 100.0), np.ones(3), np.zeros(m), 1.0)
    adj = {v: set() for v in range(m)}
    for vs in edges:
        for v in vs:
            adj[v] |= set(vs) - {v}
    seen, blocks, largest = set(), 0, 0
    for v in range(m):
        if v in seen or not adj[v]:
            continue
        blocks += 1
        stack, size = [v], 0
        while stack:
            u = stack.pop()
            if u not in seen:
                seen.add(u)
                size += 1
                stack += list(adj[u])
        largest = max(largest, size)
    P = Problem.from_instance(inst)
    if largest > 32:                                      # the projection's per-block limit
        with pytest.raises(L.FsmtError):
            P.compile(L.UNIT_PROJECT)
        return
    info = P.compile(L.UNIT_PROJECT).info
    assert info["n_halfspaces"] == len(edges)
    assert info["n_components"] == blocks
    assert info["n_free_reals"] == m - len(seen)
    assert info["n_obj_cons"] == 1
    soft = P.compile(L.UNIT_SOFT).info
    assert soft["n_halfspaces"] == 0 and soft["n_obj_cons"] == inst.n_cons


def test_projection_block_limits():
    """A block of reals coupled by unit atoms is accepted while one warp's CTA of the
    projection kernel holds it in shared memory: per thread the block's iterate, box
    corrections and multipliers, 4 (2 nv + nh) 32 bytes, plus the staged block, within
    225 KB (227 KB less the kernel's static shared memory).  A chain of 500 reals (499 half-spaces) fits, one of 600 does not (EINVAL
    under PROJECT; SOFT, with no projection, accepts it); 65 half-spaces over 4 reals fit."""
    def chain(n):
        Bd = W._Builder(0, n)
        for j in range(n - 1):
            Bd.con(W.OR, [W.lit(Bd.atom([j, j + 1], [1, -1], 0, W.LE))])
        return Problem.from_instance(Bd.freeze("chain", np.zeros(n), np.ones(n), [], np.zeros(n), 1.0))
    for n in (33, 100, 500):
        assert chain(n).compile(L.UNIT_PROJECT).info["n_components"] == 1
    P = chain(600)
    with pytest.raises(L.FsmtError) as e:
        P.compile(L.UNIT_PROJECT)
    assert e.value.status == L.EINVAL and "shared memory" in str(e.value)
    P.compile(L.UNIT_SOFT)
    Bd = W._Builder(0, 4)
    for t in range(65):
        Bd.con(W.OR, [W.lit(Bd.atom([t % 4, (t + 1) % 4], [1, -1], t, W.LE))])
    P = Problem.from_instance(Bd.freeze("hs", np.zeros(4), np.ones(4), [], np.zeros(4), 1.0))
    assert P.compile(L.UNIT_PROJECT).info["n_halfspaces"] == 65


def test_diagram_size_limit():
    """A cardinality constraint 'at most k of L' has (k + 1)(L - k) decision nodes; the
    node indices of a diagram are 16-bit, so compile accepts 256 x 255 = 65,280 nodes
    and refuses 256 x 257 = 65,792 (EINVAL)."""
    for L_, k, ok in ((510, 255, True), (512, 255, False)):
        Bd = W._Builder(L_, 1)
        Bd.con(W.CARD_LE, [W.lit(i) for i in range(L_)], k)
        P = Problem.from_instance(Bd.freeze("card", np.zeros(1), np.ones(1), np.ones(L_), np.zeros(1), 1.0))
        if ok:
            info = P.compile().info
            assert info["n_nodes"] == (k + 1) * (L_ - k) and info["max_nodes"] == info["n_nodes"]
        else:
            with pytest.raises(L.FsmtError) as e:
                P.compile()
            assert e.value.status == L.EINVAL


def test_kernel_paths_chosen_by_size():
    """Which forward + adjoint kernel can take an instance, from its compiled information:
    the chunked kernel while every constraint fits a chunk (at most 2,048 nodes, and at
    most 192 distinct literals when it needs the generic pass); the warp-per-constraint
    kernel while the largest diagram's messages fit its shared memory; neither for a
    2,102-node diagram, where the fused solver refuses the instance up front (before any
    device work) and points to the plain form."""
    from paper_2603_22877_b300 import Solver

    def build(kind, L_, k=0):
        Bd = W._Builder(L_ + 3, 1)
        Bd.con(kind, [W.lit(i) for i in range(L_)], k)
        Bd.con(W.OR, [W.lit(L_), W.lit(L_ + 1)])
        P = Problem.from_instance(Bd.freeze("x", np.zeros(1), np.ones(1), np.ones(L_ + 3), np.zeros(1), 1.0))
        return P, P.compile()

    _, c = build(W.OR, 190)                               # fits a chunk of 192 literals
    assert c.info["n_chunks"] > 0 and c.info["fused_ok"] == 1
    _, c = build(W.OR, 300)                               # 300 literals: warp kernel only
    assert c.info["n_chunks"] == 0 and c.info["fused_ok"] == 1
    _, c = build(W.CARD_LE, 100, 19)                      # 1,620 nodes: chunked only
    assert c.info["n_chunks"] > 0 and c.info["fused_ok"] == 0
    P, c = build(W.CARD_LE, 120, 20)                      # 2,100 nodes: neither
    assert c.info["n_chunks"] == 0 and c.info["fused_ok"] == 0 and c.info["max_nodes"] == 2100
    with pytest.raises(ValueError, match="plain"):
        Solver(P, c, 32, eta=0.1, b_scale=1.0)
    assert not c.uploaded


def test_argument_validation():
    P = Problem(3, 2)
    bad = [
        lambda: P.add_atoms([0, 2], [0, 0], [1, 1], [0], [0]),   # repeated variable
        lambda: P.add_atoms([0, 1], [0], [0], [0], [0]),         # zero coefficient
        lambda: P.add_atoms([0, 1], [5], [1], [0], [0]),         # variable out of range
        lambda: P.add_atoms([0, 1], [0], [1 << 24], [0], [0]),   # coefficient too large
        lambda: P.add_atoms([0, 1], [0], [1], [1 << 53], [0]),   # q0 too large
        lambda: P.add_atoms([0, 1], [0], [1], [0], [7]),         # relation
        lambda: P.add_constraints([0], [0], [0, 2], [0, 1]),     # same variable twice
        lambda: P.add_constraints([4], [2], [0, 3], [0, 2, 4]),  # MUX arity
        lambda: P.add_constraints([9], [0], [0, 1], [0]),        # kind
        lambda: P.add_constraints([0], [0], [0, 1], [100]),      # unknown id
    ]
    for f in bad:
        with pytest.raises(L.FsmtError) as e:
            f()
        assert e.value.status == L.EINVAL
    assert P.n_cons == 0
    # nothing of a failed bulk call was kept: a bulk call mixing a good and a bad row
    # adds neither, and the next constraint added gets id 0 (verify_exact names it)
    with pytest.raises(L.FsmtError):
        P.add_constraints([0, 0], [0, 0], [0, 1, 2], [0, 100])
    with pytest.raises(L.FsmtError):
        P.add_atoms([0, 1, 2], [1, 0], [1, 0], [100, 0], [0, 0])   # y1 <= 100 (true), then coef 0
    P.add_constraints([0], [0], [0, 1], [2])                 # OR(x1): false at x1 = FALSE (+1)
    assert P.verify_exact(np.array([1, 1, 1], np.int8), np.zeros(2)) == (False, 0)
    P.add_atoms([0, 1], [0], [1], [5], [0])                  # atom 0: y0 <= 5, literal id 3
    P.add_constraints([0], [0], [0, 1], [2 * 3])
    assert P.verify_exact(np.array([1, -1, 1], np.int8), np.array([6.0, 0.0])) == (False, 1)
    with pytest.raises(L.FsmtError):
        P.verify_exact(np.array([0, 1, 1], np.int8), np.zeros(2))


def test_device_calls_need_upload():
    inst = W.tiny_random(5, n_bool=4, n_real=4, n_cons=5)
    comp = Problem.from_instance(inst).compile()
    st = L.load().fsmt_forward(comp.h, 4, C.c_float(1.0), None, None, None, None, None, None)
    assert st == L.ESTATE


def _header_params():
    """Parameter count of every function declared in include/fsmt.h."""
    import re
    text = open(os.path.join(ROOT, "include", "fsmt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(fsmt_\w+)\s*\(([^;{]*?)\)\s*;", text, flags=re.S):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_prototypes_match_the_header():
    """The ctypes prototypes have as many arguments as the C declarations (a missing or
    extra argument would shift every later one)."""
    declared = _header_params()
    assert set(declared) == set(L.PROTOTYPES)
    for name, n in declared.items():
        assert len(L.PROTOTYPES[name]) == n, name


def _header_structs():
    """Member names, in order, of every `typedef struct { ... } fsmt_x;` in include/fsmt.h."""
    import re
    text = open(os.path.join(ROOT, "include", "fsmt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for m in re.finditer(r"typedef struct \{(.*?)\}\s*(fsmt_\w+)\s*;", text, flags=re.S):
        names = []
        for decl in m.group(1).split(";"):
            decl = decl.strip()
            if not decl:
                continue
            # "int32_t a, b" / "float* a" -> the declarator names
            first, *rest = decl.split(",")
            names.append(first.replace("*", " ").split()[-1])
            names += [r.replace("*", " ").strip() for r in rest]
        out[m.group(2)] = names
    return out


def test_binding_structs_match_the_header():
    """The ctypes structures list the header's members in the header's order (a member
    added on one side only would shift every later one)."""
    declared = _header_structs()
    for cname, py in (("fsmt_info", L.Info), ("fsmt_launch_config", L.LaunchConfig), ("fsmt_state", L.State),
                      ("fsmt_stage_config", L.StageConfig)):
        assert [f for f, _ in py._fields_] == declared[cname], cname


DEVICE_CALLS = ["fsmt_forward", "fsmt_adjoint", "fsmt_launch_configs", "fsmt_select_config", "fsmt_autotune",
                "fsmt_forward_plain", "fsmt_adjoint_plain", "fsmt_plain_noalloc", "fsmt_weight_sum",
                "fsmt_pgd_step", "fsmt_round_check", "fsmt_solve_stage", "fsmt_solve_stage_host",
                "fsmt_stage_form"]


@pytest.mark.parametrize("name", DEVICE_CALLS)
def test_every_device_call_checks_upload_first(name):
    """Every entry point that runs on the device answers FSMT_ESTATE for a compiled
    object that was never uploaded, before touching any buffer or the CUDA runtime
    (here there is no GPU at all)."""
    inst = W.tiny_random(5, n_bool=4, n_real=4, n_cons=5)
    comp = Problem.from_instance(inst).compile()
    args = [comp.h]
    for t in L.PROTOTYPES[name][1:]:
        if t is C.c_int32:
            args.append(4)
        elif t is C.c_float:
            args.append(C.c_float(1.0))
        elif t is C.c_void_p:
            args.append(None)
        elif t == C.POINTER(L.State):
            args.append(C.byref(L.State(R=4)))
        elif t == C.POINTER(L.StageConfig):
            args.append(C.byref(L.StageConfig()))
        elif t == C.POINTER(L.LaunchConfig):
            args.append(C.byref(L.LaunchConfig()))
        elif t == C.POINTER(C.c_int32):
            args.append(C.byref(C.c_int32()))
        else:
            raise AssertionError(f"{name}: unhandled argument type {t}")
    assert getattr(L.load(), name)(*args) == L.ESTATE


# --------------------------------------------------------------------------- equalities
def _eq_problem(eqs, n=3, extra=None, policy=L.UNIT_PROJECT):
    B_ = W._Builder(1, n)
    for var, coef, q0, neg in eqs:
        B_.con(W.OR, [W.lit(B_.atom(var, coef, q0, W.EQ), neg)])
    if extra:
        extra(B_)
    inst = B_.freeze("eq", np.full(n, -9.0), np.full(n, 9.0), [1], np.zeros(n), 1.0)
    return inst, Problem.from_instance(inst)


def test_equalities_only_as_projected_unit_atoms():
    """An equality (probability 0 under Gaussian smoothing) compiles only as the positive
    literal of a unit constraint under FSMT_UNIT_PROJECT: negated, inside a clause, or
    under SOFT it is refused with EINVAL."""
    _, P = _eq_problem([([0, 1], [1, -1], 2, False)])
    assert P.compile(L.UNIT_PROJECT).info["n_halfspaces"] == 1
    for eqs, extra, pol in (([([0, 1], [1, -1], 2, True)], None, L.UNIT_PROJECT),
                            ([([0, 1], [1, -1], 2, False)], None, L.UNIT_SOFT),
                            ([], lambda B_: B_.con(W.OR, [W.lit(0), W.lit(B_.atom([0, 1], [1, 1], 1, W.EQ))]),
                             L.UNIT_PROJECT)):
        _, P = _eq_problem(eqs, extra=extra)
        with pytest.raises(L.FsmtError) as e:
            P.compile(pol)
        assert e.value.status == L.EINVAL and "equality" in str(e.value)


def test_single_variable_equality_pins_the_real():
    """3 y0 = 6 pins y0 at 2 exactly; 3 y1 = 7 has no FP32 value, so y1's box is empty
    (counted in empty_boxes)."""
    _, P = _eq_problem([([0], [3], 6, False), ([1], [3], 7, False)])
    comp = P.compile(L.UNIT_PROJECT)
    lo, hi = comp.bounds()
    assert lo[0] == hi[0] == 2.0
    assert lo[1] > hi[1] and comp.info["empty_boxes"] == 1


def test_repair_matches_the_oracle():
    """fsmt_repair_equalities against the oracle's repair_equalities, on no-wait job-shop
    chains from points off their hyperplanes by FP32-sized amounts and by large ones:
    where the library's doubles hold the result, they are the oracle's exact values;
    then every equality holds exactly and fsmt_verify_exact agrees with the oracle's
    exact check on the repaired point."""
    inst = W.jobshop(1002, 6, 5, no_wait=3)
    P = Problem.from_instance(inst)
    rng = np.random.default_rng(4)
    agreed = 0
    for trial in range(40):
        scale = 1e-4 if trial % 2 else 3.0
        y = (inst.planted_y + rng.normal(0, scale, inst.n_real)).astype(np.float32).astype(np.float64)
        ok, yr = P.repair_equalities(y)
        ref = pgd.repair_equalities(inst, y)
        assert ok == (ref is not None)
        if not ok:
            continue
        assert [Fraction(v) for v in yr] == ref
        sat, first = P.verify_exact(inst.planted_x, yr)
        assert sat == (S.unsat_constraints(inst, inst.planted_x, yr) == [])
        agreed += 1
    assert agreed >= 30


def test_repair_refuses_what_a_double_cannot_hold():
    """y1 = y0 + 1 with y0 = 2^60 + ... is exact in Fractions but a double cannot hold
    y0 + 1 next to 2^-40 parts: the library reports ok = 0 and the oracle's repair, exact,
    succeeds; an equality with no coefficient +-1 that does not hold gives ok = 0 in both."""
    inst, P = _eq_problem([([0, 1], [1, -1], -1, False)])
    y = [2.0 ** 52, 0.5, 0.0]               # y1 = y0 + 1 = 2^52 + 1: exact; fine
    ok, yr = P.repair_equalities(y)
    assert ok and yr[1] == 2.0 ** 52 + 1
    y = [2.0 ** 53 + 2.0, 0.0, 0.0]          # y1 = 2^53 + 3 needs 54 bits
    ok, yr = P.repair_equalities(y)
    assert not ok and pgd.repair_equalities(inst, y) is not None
    inst, P = _eq_problem([([0, 1], [2, 3], 5, False)])
    assert P.repair_equalities([1.0, 0.9, 0.0])[0] is False
    assert pgd.repair_equalities(inst, [1.0, 0.9, 0.0]) is None
