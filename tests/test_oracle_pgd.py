"""Pins for the oracle's projection, PGD step, exact check and ERWA (no GPU)."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import objective as OBJ, pgd, semantics as S
from workloads import instances as W


def exact_projection(y, lo, hi, A, c):
    """argmin ||x - y||^2 s.t. lo <= x <= hi, A x <= c, by enumerating active sets (KKT)."""
    n = len(y)
    rows = []
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1
        rows.append((e, hi[i]))
        rows.append((-e, -lo[i]))
    for k in range(len(c)):
        rows.append((A[k], c[k]))
    best, best_d = None, np.inf
    for r in range(0, n + 1):
        for act in itertools.combinations(range(len(rows)), r):
            G = np.array([rows[k][0] for k in act]).reshape(r, n)
            h = np.array([rows[k][1] for k in act])
            if r:
                M = G @ G.T
                if abs(np.linalg.det(M)) < 1e-12:
                    continue
                lam = np.linalg.solve(M, G @ y - h)
                if (lam < -1e-12).any():
                    continue
                x = y - G.T @ lam
            else:
                x = y.copy()
            ok = all(rows[k][0] @ x <= rows[k][1] + 1e-9 for k in range(len(rows)))
            if ok and np.linalg.norm(x - y) < best_d:
                best, best_d = x, np.linalg.norm(x - y)
    return best


def halfspace_instance(rng, n_real=3, n_half=3):
    B = W._Builder(0, n_real)
    A, c = [], []
    for _ in range(n_half):
        var = rng.choice(n_real, 2, replace=False)
        coef = rng.integers(1, 4, 2) * rng.choice([-1, 1], 2)
        q0 = int(rng.integers(-3, 4))
        B.con(W.OR, [W.lit(B.atom(var, coef, q0, W.LE))])
        row = np.zeros(n_real)
        row[var] = coef
        A.append(row)
        c.append(q0)
    lo, hi = np.full(n_real, -4.0), np.full(n_real, 4.0)
    return B.freeze("h", lo, hi, [], np.zeros(n_real), 1.0), lo, hi, np.array(A), np.array(c, float)


def test_dykstra_matches_exact_qp():
    rng = np.random.default_rng(0)
    checked = polished = 0
    for _ in range(40):
        inst, lo, hi, A, c = halfspace_instance(rng)
        dom = pgd.Domain(inst)
        assert len(dom.halfspaces) == 3
        y = rng.uniform(-6, 6, inst.n_real)
        x_ex = exact_projection(y, lo, hi, A, c)
        if x_ex is None:  # empty feasible set
            continue
        x = dom.project_b(y[:, None], sweeps=3000, polish=0)[:, 0]
        np.testing.assert_allclose(x, x_ex, atol=1e-7)
        # where the polish lands in D exactly, it stays within the margin scale of the projection
        xp = dom.project_b(y[:, None], sweeps=3000, polish=32)[:, 0]
        feasible = all(sum(Fraction(float(A[k, j])) * Fraction(float(xp[j])) for j in range(len(xp)))
                       <= Fraction(float(c[k])) for k in range(len(c)))
        assert (xp >= lo).all() and (xp <= hi).all()
        if feasible:
            assert np.abs(xp - x_ex).max() <= 1e-2
            polished += 1
        checked += 1
    assert checked > 20 and polished >= checked // 2


def test_polish_makes_precedence_chains_exactly_feasible():
    """Job-shop precedence chains with box bounds (the workloads' unit atoms): from
    points near a feasible one (the regime of a PGD step), the projected point
    satisfies every unit atom exactly; without the polish, Dykstra's does not."""
    inst = W.jobshop(1002, 8, 6)
    dom = pgd.Domain(inst)
    assert len(dom.halfspaces) == 8 * 5
    rng = np.random.default_rng(5)
    unit = [c for c in range(inst.n_cons) if OBJ.is_unit_atomic(inst, c)]
    for noise in (0.5, 2.0, 10.0):
        y = inst.planted_y[:, None] + rng.normal(0, noise, (inst.n_real, 64))
        x = dom.project_b(y, sweeps=20, polish=32)
        _, viol = pgd.round_check(inst, np.zeros((inst.n_bool, 64)), x, constraints=unit)
        assert not viol[unit].any()
        x0 = dom.project_b(y, sweeps=20, polish=0)
        _, viol0 = pgd.round_check(inst, np.zeros((inst.n_bool, 64)), x0, constraints=unit)
        assert viol0[unit].any()
        assert np.abs(x - x0).max() <= 0.05  # the polish moves the point by the margin scale


def test_projection_idempotent_and_nonexpansive():
    rng = np.random.default_rng(1)
    inst, lo, hi, A, c = halfspace_instance(rng, 4, 3)
    dom = pgd.Domain(inst)
    y = rng.uniform(-8, 8, (4, 50))
    x = dom.project_b(y, 3000, polish=0)
    if exact_projection(y[:, 0], lo, hi, A, c) is None:
        pytest.skip("empty feasible set for this draw")
    np.testing.assert_allclose(dom.project_b(x, 3000, polish=0), x, atol=1e-7)
    d_in = np.linalg.norm(y[:, :25] - y[:, 25:], axis=0)
    d_out = np.linalg.norm(x[:, :25] - x[:, 25:], axis=0)
    assert (d_out <= d_in + 1e-7).all()


def test_single_variable_unit_atoms_tighten_the_box():
    B = W._Builder(0, 2)
    B.con(W.OR, [W.lit(B.atom([0], [3], 7, W.LE))])  # y0 <= 7/3
    B.con(W.OR, [W.lit(B.atom([1], [2], 1, W.GE))])  # y1 >= 1/2
    B.con(W.OR, [W.lit(B.atom([1], [1], 5, W.GT), True)])  # not (y1 > 5): y1 <= 5
    inst = B.freeze("u", np.array([-10.0, -10.0]), np.array([10.0, 10.0]), [], np.zeros(2), 1.0)
    dom = pgd.Domain(inst)
    assert dom.hi[0] == 7 / 3 and dom.lo[1] == 0.5 and dom.hi[1] == 5.0
    assert OBJ.objective_constraints(inst, OBJ.PROJECT) == []
    assert OBJ.objective_constraints(inst, OBJ.SOFT) == [0, 1, 2]


def test_descent_lemma():
    """Lemma descent with eta = 1/L, L from Prop. Lipschitz (scale 1, box only)."""
    inst = W.tiny_random(21, n_bool=6, n_real=4, n_cons=12)
    inst.scale = 1.0
    R = 4
    a, b = W.initial_point(inst, R, seed=3)
    a, b = a.astype(np.float64), b.astype(np.float64)
    w = np.ones((inst.n_cons, R))
    sigma = 30.0
    n, m = inst.n_bool, inst.n_real
    alpha = float(inst.n_cons)
    beta = max(1, max(sum(1 for l in inst.lits(c) if (l >> 1) >= n and j in inst.atom((l >> 1) - n)[0])
                      for c in range(inst.n_cons) for j in range(m)))
    gam = math.sqrt(2) * beta / (math.sqrt(math.pi) * sigma)
    rho = alpha * math.sqrt(n + m) * max(1.0, gam)
    L = math.sqrt(n + m * gam * gam) * rho
    eta = 1.0 / L
    dom = pgd.Domain(inst)
    for _ in range(5):
        obj, _, ga, gb = OBJ.evaluate(inst, a, b, w, sigma)
        a2, b2, gn2 = pgd.pgd_step(a, b, ga, gb, eta, 1.0, dom, 20)
        obj2 = OBJ.evaluate(inst, a2, b2, w, sigma, with_grad=False)[0]
        assert (obj2 - obj <= -eta / 2 * gn2 + 1e-12).all()
        a, b = a2, b2


@pytest.mark.parametrize("make", [lambda: W.tiny_random(1001), lambda: W.jobshop(1002, 8, 4),
                                  lambda: W.placement2d(1003, 12), lambda: W.placement2d(1003, 12, selectors=False),
                                  lambda: W.large_scheduling(1005, 16, 20, 6, 3, 5),
                                  lambda: W.large_scheduling(1005, 5, 20, 6, 3, 5)])
def test_exact_check_planted_and_flip(make):
    inst = make()
    a = inst.planted_x.astype(np.float64)[:, None] * 0.5
    b = inst.planted_y[:, None]
    x, viol = pgd.round_check(inst, a, b)
    assert not viol.any()
    assert (x[:, 0] == inst.planted_x).all()
    # the scalar definition agrees
    assert S.unsat_constraints(inst, inst.planted_x, inst.planted_y) == []
    # flipping every Boolean still leaves unit atom constraints intact, but violates some clause
    if inst.n_bool:
        _, viol2 = pgd.round_check(inst, -a, b)
        assert viol2.any()


def test_exact_check_boundary():
    """An atom exactly on its boundary: y0 - y1 <= -3 at y = (1, 4) holds; LT does not."""
    B = W._Builder(0, 2)
    B.con(W.OR, [W.lit(B.atom([0, 1], [1, -1], -3, W.LE))])
    B.con(W.OR, [W.lit(B.atom([0, 1], [1, -1], -3, W.LT))])
    inst = B.freeze("b", np.zeros(2), np.ones(2) * 9, [], np.zeros(2), 1.0)
    y = np.array([[1.0, 1.0 + 2.0 ** -40], [4.0, 4.0]])
    _, viol = pgd.round_check(inst, np.zeros((0, 2)), y)
    assert list(viol[0]) == [False, True] and list(viol[1]) == [True, True]


def test_kind_value_vec_matches_definition():
    rng = np.random.default_rng(4)
    for kind, L, param in [(S.OR, 4, 0), (S.XOR, 5, 0), (S.CARD_LE, 5, 2), (S.NAE, 3, 0),
                           (S.MUX, 6, 2), (S.MUX, 3, 1), (S.NEQ_OR, 7, 3)]:
        T = rng.random((L, 200)) < 0.5
        v = pgd.kind_value_vec(kind, param, T)
        for r in range(200):
            assert v[r] == S.kind_value(kind, param, list(T[:, r]))


def test_erwa_two_stages():
    """Alg. 2 with rho = 0.5, gamma = 2, tau = 1: h0 = 0, u = 1 -> w = 2, h = 1;
    then u = 0 -> h = 0.5 -> w = 2 * sqrt(2), h = 1."""
    w, h = np.ones((1, 1)), np.zeros((1, 1))
    w, h, n = pgd.erwa(w, h, np.ones((1, 1)), 1, 0.5, 2.0, 1)
    assert w[0, 0] == 2.0 and h[0, 0] == 1.0 and n[0] == 1
    w, h, n = pgd.erwa(w, h, np.zeros((1, 1)), 2, 0.5, 2.0, 1)
    assert abs(w[0, 0] - 2 * math.sqrt(2)) < 1e-15 and h[0, 0] == 1.0 and n[0] == 0
    # tau = 2: no weight update at odd stages
    w, h, n = pgd.erwa(np.ones((1, 1)), np.zeros((1, 1)), np.ones((1, 1)), 1, 0.5, 2.0, 2)
    assert w[0, 0] == 1.0 and h[0, 0] == 1.0


def test_fig2_toy_annealing_reaches_global_minimum():
    """Fig. 2: annealing 1/sigma upwards from a point between the minima ends at x = -1, y > 0."""
    B = W._Builder(1, 1)
    A = B.atom([0], [1], 0, W.GT)
    B.con(W.XOR, [W.lit(0, True), W.lit(A)])
    B.con(W.CARD_LE, [W.lit(0, True), W.lit(A, True)], param=0)
    inst = B.freeze("fig2", np.array([-1.0]), np.array([1.0]), [-1], np.array([0.5]), 1.0)
    cfg = pgd.Config(eta=0.05, t_max=200)
    a = np.array([[0.3]])
    b = np.array([[-0.2]])
    sat, a_end, b_end = pgd.anneal(inst, a, b, cfg)
    assert sat[0] > 0 and a_end[0, 0] < 0 and b_end[0, 0] > 0


@pytest.mark.parametrize("n_workers", [3, 5, 6, 7, 12, 20])
def test_scheduling_worker_index_in_range(n_workers):
    """Generator sanity for a worker count that is not a power of two: at the plant,
    re-coding one job's worker index to each of the 2**bits codes leaves every
    constraint that does not involve another job's time satisfied exactly iff the code
    names a worker (< n_workers), checked by brute force over all codes."""
    inst = W.large_scheduling(1005, n_workers, 6, 6, 0, 5)
    bits = (n_workers - 1).bit_length()
    assert inst.n_bool == bits * 6
    assert S.unsat_constraints(inst, inst.planted_x, inst.planted_y) == []
    lits_of = [inst.lits(c) for c in range(inst.n_cons)]
    mine = [c for c in range(inst.n_cons)                 # only job 0's bits, no atom
            if all(l // 2 < bits for l in lits_of[c])]
    for code in range(1 << bits):
        x = inst.planted_x.copy()
        for i in range(bits):
            x[i] = -1 if (code >> i) & 1 else 1
        ok = all(S.constraint_holds(inst, c, x, inst.planted_y) for c in mine)
        assert ok == (code < n_workers), code


def test_common_weight_factor_leaves_the_normalised_step_unchanged():
    """The weight rescale relies on this: with eta_r = eta |C_sigma| / sum_c w_c (Thm.
    max_step with L proportional to the total weight), scaling every weight of a restart
    by 2^-32 leaves the PGD iterates bit for bit unchanged (the epsilon test is off)."""
    inst = W.jobshop(1002, 6, 3)
    R = 8
    a, b = W.initial_point(inst, R, seed=4)
    w = np.random.default_rng(5).uniform(1.0, 9.0, (inst.n_cons, R))
    cfg = pgd.Config(eta=0.05, eps=0.0, t_max=3)
    sigma = inst.scale / 0.7
    out1 = pgd.run_stage(inst, a, b, w, np.zeros_like(w), sigma, 2, cfg)
    out2 = pgd.run_stage(inst, a, b, w * 2.0 ** -32, np.zeros_like(w), sigma, 2, cfg)
    np.testing.assert_array_equal(out1[0], out2[0])
    np.testing.assert_array_equal(out1[1], out2[1])
    np.testing.assert_array_equal(out1[4], out2[4])         # the same rounding outcome
    np.testing.assert_array_equal(out1[2] * 2.0 ** -32, out2[2])


def test_erwa_weight_rescale_keeps_long_schedules_finite():
    """Alg. 2 as printed grows every weight by at least gamma^rho per stage (h_c is reset
    to 1): after 300 stages the weights of a constraint that keeps failing exceed the FP32
    range.  With the rescale of a restart whose mean weight passed 2^32 the largest stays
    within it, the ratios between weights are those of Alg. 2 (so the weights of the
    constraints that hold fall towards zero, as they do relative to the others in
    Alg. 2), and restarts below the threshold are untouched."""
    n_c, R, T = 3, 2, 300
    u = np.zeros((n_c, R))
    u[0, :] = 1                                           # one constraint fails every stage
    w0, h0 = np.ones((n_c, R)), np.zeros((n_c, R))
    w, h, wr, hr = w0, h0, w0, h0
    for t in range(1, T + 1):
        w, h, _ = pgd.erwa(w, h, u, t, 0.5, 2.0, 1)
        wr, hr, _ = pgd.erwa(wr, hr, u, t, 0.5, 2.0, 1, mean_w=wr.mean(0))
    f32_max = float(np.finfo(np.float32).max)
    assert w.max() > f32_max
    assert wr.max() < 2.0 ** 40 and wr.min() > 0
    np.testing.assert_allclose(wr / wr[1:2], w / w[1:2], rtol=1e-12)
    # below the threshold nothing changes
    wa, _, _ = pgd.erwa(w0 * 3, h0, u, 1, 0.5, 2.0, 1, mean_w=np.full(R, 2.0 ** 32))
    wb, _, _ = pgd.erwa(w0 * 3, h0, u, 1, 0.5, 2.0, 1)
    np.testing.assert_array_equal(wa, wb)
    wc, _, _ = pgd.erwa(w0 * 3, h0, u, 1, 0.5, 2.0, 1, mean_w=np.array([2.0 ** 33, 1.0]))
    np.testing.assert_array_equal(wc[:, 0], wb[:, 0] * 2.0 ** -32)
    np.testing.assert_array_equal(wc[:, 1], wb[:, 1])


@pytest.mark.parametrize("n_macros,n_layers", [(2, 2), (4, 2), (4, 4), (8, 2)])
def test_placement3d_structure_and_plant(n_macros, n_layers):
    """Generator sanity for the 3D placement encoding: module and constraint counts,
    the association (every small memory with two small processes, every small process
    and large module in exactly one pair), the plant satisfies every constraint
    exactly, and moving one module of a pair to another macro (one macro bit flipped)
    breaks that bit's equality clause with each of its partners, plus non-overlap
    constraints with the module now at the same place in the new macro, and nothing
    that does not involve it."""
    inst = W.placement3d(1007, n_macros, n_layers)
    N = 2 * n_macros + n_macros * n_layers + n_macros * n_layers // 2
    bm, bl = n_macros.bit_length() - 1, n_layers.bit_length() - 1
    assert inst.meta["n_modules"] == N
    assert inst.n_bool == N * (bm + bl) and inst.n_real == 2 * N
    n_pairs = n_macros + n_macros * n_layers
    assert inst.meta["n_pairs"] == n_pairs
    assert inst.n_cons == 4 * N + n_pairs * (bm + 4) + N * (N - 1) // 2
    kinds = inst.meta["kinds"]
    assert kinds.count("small_proc") == n_macros * n_layers and kinds.count("small_mem") == n_macros * n_layers // 2
    # pairs from the equality clauses of macro bit 0: (module of first literal, module of second)
    partners = {j: [] for j in range(N)}
    for c in range(inst.n_cons):
        if int(inst.con_kind[c]) == W.XOR:
            l1, l2 = inst.lits(c)
            j, k = (l1 // 2) // (bm + bl), (l2 // 2) // (bm + bl)
            if (l1 // 2) % (bm + bl) == 0:
                partners[j].append(k)
                partners[k].append(j)
    for j in range(N):
        want = {"small_mem": 2, "small_proc": 1, "large_proc": 1, "large_mem": 1}[kinds[j]]
        assert len(partners[j]) == want
        other = {"small_mem": "small_proc", "small_proc": "small_mem", "large_proc": "large_mem",
                 "large_mem": "large_proc"}[kinds[j]]
        assert all(kinds[k] == other for k in partners[j])
    assert S.unsat_constraints(inst, inst.planted_x, inst.planted_y) == []
    j = kinds.index("small_proc")
    x = inst.planted_x.copy()
    x[j * (bm + bl)] *= -1                                   # macro bit 0 of module j
    bad = S.unsat_constraints(inst, x, inst.planted_y)
    assert sum(int(inst.con_kind[c]) == W.XOR for c in bad) == len(partners[j])
    assert any(int(inst.con_kind[c]) == W.NEQ_OR for c in bad)      # it lands on a peer
    for c in bad:
        assert j * (bm + bl) in {int(l) // 2 for l in inst.lits(c)}


def test_scheduling_early_closing_windows():
    """The deadline side of the workers' availability windows: the plant (redone so that
    no job on an early-closing worker ends after its close) satisfies every constraint
    exactly; each window clause is (X_j != w) OR (y_j + t_j <= e_w), so re-coding a job
    to such a worker with its start just past e_w - t_j violates exactly that clause
    among the constraints that involve only this job; the default instance is unchanged
    by the option's existence (its own random stream)."""
    base = W.large_scheduling(1005, 16, 30, 6, 4, 5)
    inst = W.large_scheduling(1005, 16, 30, 6, 4, 5, n_early=5)
    bits = 4
    assert inst.n_cons == base.n_cons + 5 * 30
    assert S.unsat_constraints(inst, inst.planted_x, inst.planted_y) == []
    close = inst.meta["close"]
    # the window clauses are the last 5 * 30 constraints, worker by worker
    first = inst.n_cons - 5 * 30
    lits = inst.lits(first)                      # worker w_0, job 0
    w0 = sum(1 << i for i, l in enumerate(lits[:bits]) if l & 1)
    var, coef, q0, rel = inst.atom(int(lits[-1]) // 2 - inst.n_bool)
    assert list(var) == [0] and list(coef) == [1]
    t0 = close[0] - int(q0)                      # q0 = e_w - t_0
    assert 1 <= t0 <= 6
    x = inst.planted_x.copy()
    y = inst.planted_y.copy()
    for i in range(bits):
        x[i] = -1 if (w0 >> i) & 1 else 1
    y[0] = float(close[0] - t0 + 1)
    own = [c for c in range(inst.n_cons)
           if all(l // 2 < bits or (l // 2 >= inst.n_bool and list(inst.atom(l // 2 - inst.n_bool)[0]) == [0])
                  for l in inst.lits(c))]
    bad = [c for c in own if not S.constraint_holds(inst, c, x, y)]
    assert bad == [first]


def test_fig2_sigma_above_two_reaches_the_global_minimum():
    """Fig. 2's trajectories (tests/golden/fig2_sigma.json): from starts in the local
    minimum's basin, PGD at a fixed sigma above 2 ends at the global minimum (x = -1,
    y > 0) and takes more iterations than at sigma = 0.5, below 2 it ends at the local
    one (x = +1, y <= 0).  A sign error in the gradient, a wrong smoothing width or a
    dropped constraint moves these end points."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fig2_sigma.json")))
    B = W._Builder(1, 1)
    A = B.atom([0], [1], 0, W.GT)
    B.con(W.XOR, [W.lit(0, True), W.lit(A)])
    B.con(W.CARD_LE, [W.lit(0, True), W.lit(A, True)], param=0)
    inst = B.freeze("fig2", np.array([-1.0]), np.array([1.0]), [-1], np.array([0.5]), 1.0)
    cfg = pgd.Config(eta=0.05, t_max=3000, eps=1e-6)

    def run(sigma, a0, b0):
        w, h = np.ones((2, 1)), np.zeros((2, 1))
        a, b, _, _, _, its, _ = pgd.run_stage(inst, np.array([[a0]]), np.array([[b0]]), w, h, sigma, 1, cfg)
        return a[0, 0], b[0, 0], int(its[0])

    for a0, b0 in g["starts"]:
        slow = []
        for sigma in g["sigma_global"]:
            a, b, its = run(sigma, a0, b0)
            assert a == -1.0 and b > 0, (sigma, a0, b0, a, b)
            slow.append(its)
        for sigma in g["sigma_local"]:
            a, b, its = run(sigma, a0, b0)
            assert a == 1.0 and b <= 0, (sigma, a0, b0, a, b)
            if sigma == g["sigma_fast"]:
                assert min(slow) > its
