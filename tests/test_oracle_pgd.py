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


# --------------------------------------------------------------------------- scaled coordinates
def rescaled(inst, k):
    """The same instance with every real measured in units k times smaller: y' = k y.
    Atoms q.y rel q0 become q.y' rel k q0; boxes, the plant and the length scale
    scale by k.  k a power of two keeps every value exact."""
    import dataclasses
    return dataclasses.replace(inst, atom_q0=inst.atom_q0 * k, lo=inst.lo * k, hi=inst.hi * k,
                               planted_y=inst.planted_y * k, scale=inst.scale * k)


@pytest.mark.parametrize("make", [lambda: W.jobshop(1002, 8, 4), lambda: W.tiny_random(21, 6, 4, 12),
                                  lambda: W.placement2d(1003, 8)])
def test_pgd_step_is_covariant_under_a_change_of_units(make):
    """The reals' step is taken in the coordinates y/S (Eq. pg1, pg2 on the paper's
    [0, 1]-scaled reals, Methods "Benchmarks").  A step defined that way cannot depend
    on the unit the reals are written in: measuring every real in units 4 times
    smaller (atoms, boxes, sigma and S times 4) must give the same Booleans, the reals
    times 4, the same ||g||^2 (Eq. grad_map in scaled coordinates) and the same
    objective, bit for bit (powers of two are exact).  An S where S^2 belongs in the
    b-step, or S^2 where S belongs in ||g||^2, breaks this."""
    inst = make()
    k = 4
    ik = rescaled(inst, k)
    R = 6
    a, b = W.initial_point(inst, R, seed=11)
    a, b = a.astype(np.float64), b.astype(np.float64)
    w = np.random.default_rng(2).uniform(0.5, 3.0, (inst.n_cons, R))
    cfg = pgd.Config(eta=0.05)
    sigma = inst.scale / 0.9
    dom, domk = pgd.Domain(inst), pgd.Domain(ik)
    etas = pgd.step_sizes(inst, w, cfg)
    np.testing.assert_array_equal(etas, pgd.step_sizes(ik, w, cfg))
    A, Bk = a.copy(), b * k
    for _ in range(3):
        obj, _, ga, gb = OBJ.evaluate(inst, a, b, w, sigma)
        objk, _, gak, gbk = OBJ.evaluate(ik, A, Bk, w, sigma * k)
        np.testing.assert_array_equal(obj, objk)
        np.testing.assert_array_equal(ga, gak)
        a, b, gn2 = pgd.pgd_step(a, b, ga, gb, etas, inst.scale, dom, cfg.sweeps, cfg.polish)
        A, Bk, gn2k = pgd.pgd_step(A, Bk, gak, gbk, etas, ik.scale, domk, cfg.sweeps, cfg.polish)
        np.testing.assert_array_equal(a, A)
        np.testing.assert_array_equal(b * k, Bk)
        np.testing.assert_array_equal(gn2, gn2k)
        assert (gn2 > 0).all()


def test_descent_lemma_in_scaled_coordinates():
    """Lemma descent at S != 1.  In u = y/S the objective is F(a, u) = C(a, S u); an
    atom q.(S u) <= q0 has the same probability as q.y <= q0 with sigma/S in place of
    sigma, so Prop. Lipschitz gives L of F with sigma/S.  With eta = 1/L the step
    (b-step eta S^2 dC/db = S times the u-step eta dF/du) must satisfy
    F(new) <= F - eta/2 ||g||^2 with ||g|| measured in u.  A b-step S times too large
    (S^3) overshoots and fails; S = 100 here, the reals' native range [0, 100]."""
    inst = W.tiny_random(21, n_bool=6, n_real=4, n_cons=12)
    S_ = inst.scale
    assert S_ == 100.0
    R = 4
    a, b = W.initial_point(inst, R, seed=3)
    a, b = a.astype(np.float64), b.astype(np.float64)
    w = np.ones((inst.n_cons, R))
    sigma_u = 0.3
    sigma = sigma_u * S_
    n, m = inst.n_bool, inst.n_real
    alpha = float(inst.n_cons)
    beta = max(1, max(sum(1 for l in inst.lits(c) if (l >> 1) >= n and j in inst.atom((l >> 1) - n)[0])
                      for c in range(inst.n_cons) for j in range(m)))
    gam = math.sqrt(2) * beta / (math.sqrt(math.pi) * sigma_u)
    rho = alpha * math.sqrt(n + m) * max(1.0, gam)
    L = math.sqrt(n + m * gam * gam) * rho
    eta = 1.0 / L
    dom = pgd.Domain(inst)
    moved = 0.0
    for _ in range(5):
        obj, _, ga, gb = OBJ.evaluate(inst, a, b, w, sigma)
        a2, b2, gn2 = pgd.pgd_step(a, b, ga, gb, eta, S_, dom, 20)
        obj2 = OBJ.evaluate(inst, a2, b2, w, sigma, with_grad=False)[0]
        assert (obj2 - obj <= -eta / 2 * gn2 + 1e-12).all()
        moved = max(moved, np.abs(b2 - b).max())
        a, b = a2, b2
    assert moved > 0


# --------------------------------------------------------------------------- step normalisation
def three_constraint_instance():
    """x0 OR A, NOT x1 OR B (in C_sigma) and the unit atom y0 + y1 <= 5 (projected)."""
    B = W._Builder(2, 2)
    A_ = B.atom([0, 1], [1, -2], 3)
    B_ = B.atom([1], [3], 4)
    U = B.atom([0, 1], [1, 1], 5)
    B.con(W.OR, [W.lit(0), W.lit(A_)])
    B.con(W.OR, [W.lit(1, True), W.lit(B_)])
    B.con(W.OR, [W.lit(U)])
    return B.freeze("three", np.zeros(2), np.full(2, 9.0), [-1, 1], np.array([1.0, 1.0]), 1.0)


def test_step_sizes_hand_derived():
    """eta_r = eta |C_sigma| / sum_{c in C_sigma} w_c (Thm. max_step with L proportional to
    the total weight alpha of Prop. Lipschitz).  By hand for the three-constraint
    instance, C_sigma = {0, 1} (constraint 2 is a projected unit atom):
      restart 0, w = (2, 3, 100): 0.1 * 2 / 5 = 0.04
      restart 1, w = (5, 1, 7):   0.1 * 2 / 6 = 1/30
      restart 2, w = (1, 1, 1):   0.1 (unit weights give the configured step)
    Summing over every constraint gives 0.1*2/105, 0.1*2/13 and 0.1*2/3; dropping
    |C_sigma| gives 0.02, 1/60 and 0.05.  With the unit atom kept in the objective
    (SOFT), |C_sigma| = 3 and the sums include it."""
    inst = three_constraint_instance()
    assert OBJ.objective_constraints(inst, OBJ.PROJECT) == [0, 1]
    w = np.array([[2.0, 5.0, 1.0], [3.0, 1.0, 1.0], [100.0, 7.0, 1.0]])
    cfg = pgd.Config(eta=0.1)
    got = pgd.step_sizes(inst, w, cfg)
    np.testing.assert_allclose(got, [0.04, 1.0 / 30.0, 0.1], rtol=1e-15)
    soft = pgd.step_sizes(inst, w, cfg, policy=OBJ.SOFT)
    np.testing.assert_allclose(soft, [0.1 * 3 / 105, 0.1 * 3 / 13, 0.1], rtol=1e-15)
    off = pgd.step_sizes(inst, w, pgd.Config(eta=0.1, normalize_eta=False))
    np.testing.assert_array_equal(off, [0.1, 0.1, 0.1])


def test_step_sizes_ignore_the_weights_of_projected_atoms():
    """A projected unit atom is not part of C_sigma, so its ERWA weight cannot change L
    and must not change the step: the whole PGD trajectory is the same whatever its
    weight (fails if the normalisation sums over every constraint)."""
    inst = W.jobshop(1002, 6, 3)
    R = 4
    a, b = W.initial_point(inst, R, seed=6)
    unit = [c for c in range(inst.n_cons) if OBJ.is_unit_atomic(inst, c)]
    assert unit
    w = np.random.default_rng(8).uniform(1.0, 4.0, (inst.n_cons, R))
    w2 = w.copy()
    w2[unit] *= 1000.0
    cfg = pgd.Config(eta=0.05, eps=0.0, t_max=3)
    sigma = inst.scale / 0.5
    o1 = pgd.run_stage(inst, a, b, w, np.zeros_like(w), sigma, 1, cfg)
    o2 = pgd.run_stage(inst, a, b, w2, np.zeros_like(w), sigma, 1, cfg)
    np.testing.assert_array_equal(o1[0], o2[0])
    np.testing.assert_array_equal(o1[1], o2[1])


# --------------------------------------------------------------------------- polish at a converged point
def test_polish_stays_within_its_margin_of_the_exact_projection():
    """Prop. QP's projection, computed exactly by active-set enumeration, against
    Dykstra run to convergence (3,000 sweeps) followed by the polish.  The polish only
    moves a half-space whose value is within its margin m = 2^-16 (|q0| + sum |q_j y_j|)
    of the boundary, onto q.y <= q0 - 2m, so:
      * where the exact projection keeps every half-space more than 4 margins inside,
        the polished point is Dykstra's point bit for bit (nothing moves);
      * elsewhere, where the polish settles in D exactly, it stays within 8 margins
        (max over the half-spaces) of the exact projection in every coordinate.
    The bound is 2x the largest distance seen over 1,500 random blocks of 2-4 reals and
    1-3 half-spaces (4.1 margins, at narrow corners where two moves of 2m add up).  A
    polish that overshoots (a target 10 margins inside, a step not divided by ||q||^2)
    or that moves points which need no move fails it."""
    rng = np.random.default_rng(0)
    interior = near = 0
    for _ in range(30):
        inst, lo, hi, A, c = halfspace_instance(rng, n_real=int(rng.integers(2, 5)), n_half=int(rng.integers(1, 4)))
        dom = pgd.Domain(inst)
        Y = rng.uniform(-6, 6, (inst.n_real, 8))            # 8 points per block, one call
        XD = dom.project_b(Y, sweeps=3000, polish=0)
        XP = dom.project_b(Y, sweeps=3000, polish=32)
        for r in range(Y.shape[1]):
            x_ex = exact_projection(Y[:, r], lo, hi, A, c)
            if x_ex is None:
                break
            xd, xp = XD[:, r], XP[:, r]
            M = max(pgd.POLISH_MARGIN * (abs(q0) + np.abs(q * x_ex[var]).sum()) for var, q, q0 in dom.halfspaces)
            slack = min(q0 - (q * x_ex[var]).sum() for var, q, q0 in dom.halfspaces)
            if slack > 4 * M:
                np.testing.assert_array_equal(xp, xd)
                interior += 1
                continue
            feasible = all(sum(Fraction(float(A[k, j])) * Fraction(float(xp[j])) for j in range(len(xp)))
                           <= Fraction(float(c[k])) for k in range(len(c)))
            if feasible:
                assert np.abs(xp - x_ex).max() <= 8 * M, (np.abs(xp - x_ex).max() / M)
                near += 1
    assert interior > 20 and near > 60


# --------------------------------------------------------------------------- equalities
def exact_projection_eq(y, lo, hi, A, c, eq):
    """argmin ||x - y||^2 s.t. lo <= x <= hi, A_k x <= c_k, and A_k x = c_k where eq[k]:
    active-set enumeration (KKT) with the equality rows always active and their
    multipliers of either sign."""
    n = len(y)
    rows = []
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1
        rows.append((e, hi[i], False))
        rows.append((-e, -lo[i], False))
    for k in range(len(c)):
        rows.append((A[k], c[k], bool(eq[k])))
    always = [k for k, r in enumerate(rows) if r[2]]
    optional = [k for k, r in enumerate(rows) if not r[2]]
    best, best_d = None, np.inf
    for r in range(0, n + 1 - len(always)):
        for extra in itertools.combinations(optional, r):
            act = list(always) + list(extra)
            G = np.array([rows[k][0] for k in act]).reshape(len(act), n)
            h = np.array([rows[k][1] for k in act])
            M = G @ G.T
            if abs(np.linalg.det(M)) < 1e-12:
                continue
            lam = np.linalg.solve(M, G @ y - h)
            if any(lam[t] < -1e-12 for t in range(len(always), len(act))):
                continue
            x = y - G.T @ lam
            ok = all((abs(rows[k][0] @ x - rows[k][1]) <= 1e-9) if rows[k][2] else (rows[k][0] @ x <= rows[k][1] + 1e-9)
                     for k in range(len(rows)))
            if ok and np.linalg.norm(x - y) < best_d:
                best, best_d = x, np.linalg.norm(x - y)
    return best


def test_dykstra_with_hyperplanes_matches_exact_qp():
    """Prop. QP with equality unit atoms: Dykstra's sweeps treat an equality as a
    hyperplane (its multiplier not clamped at zero) and converge to the Euclidean
    projection onto box, half-spaces and hyperplanes, against an active-set
    enumeration in which the equality rows are always active."""
    rng = np.random.default_rng(3)
    checked = 0
    for _ in range(30):
        n = 4
        B = W._Builder(0, n)
        A, c, eq = [], [], []
        for k in range(3):
            var = rng.choice(n, 2, replace=False)
            coef = rng.integers(1, 3, 2) * rng.choice([-1, 1], 2)
            q0 = int(rng.integers(-2, 3))
            rel = W.EQ if k == 0 else W.LE
            B.con(W.OR, [W.lit(B.atom(var, coef, q0, rel))])
            row = np.zeros(n)
            row[var] = coef
            A.append(row)
            c.append(q0)
            eq.append(rel == W.EQ)
        lo, hi = np.full(n, -5.0), np.full(n, 5.0)
        inst = B.freeze("eq", lo, hi, [], np.zeros(n), 1.0)
        dom = pgd.Domain(inst)
        assert dom.eq == [True, False, False]
        Y = rng.uniform(-7, 7, (n, 4))
        X = dom.project_b(Y, sweeps=4000, polish=0)
        for r in range(Y.shape[1]):
            x_ex = exact_projection_eq(Y[:, r], lo, hi, np.array(A), np.array(c, float), eq)
            if x_ex is None:
                continue
            np.testing.assert_allclose(X[:, r], x_ex, atol=1e-7)
            checked += 1
    assert checked > 60


def test_polish_returns_points_to_the_hyperplanes():
    """No-wait jobs (each precedence an equality) from points near the plant: after the
    projection every equality's residual is within its FP32 band (eq_band), every
    inequality unit atom holds exactly, and the repair then makes the equalities hold
    exactly while moving no real by more than a few bands."""
    inst = W.jobshop(1002, 8, 5, no_wait=3)
    dom = pgd.Domain(inst)
    rng = np.random.default_rng(9)
    y = (inst.planted_y[:, None] + rng.normal(0, 0.5, (inst.n_real, 16))).astype(np.float32).astype(np.float64)
    x = dom.project_b(y, 20, 32).astype(np.float32).astype(np.float64)
    unit = [c for c in range(inst.n_cons) if OBJ.is_unit_atomic(inst, c)]
    for r in range(16):
        for (var, q, q0), e in zip(dom.halfspaces, dom.eq):
            v = float((q * x[var, r]).sum() - q0)
            mag = abs(q0) + float(np.abs(q * x[var, r]).sum())
            if e:
                assert abs(v) <= 4 * pgd.eq_band(len(var), mag), (r, v)
        ineq = [c for c in unit if inst.atom((int(inst.lits(c)[0]) >> 1) - inst.n_bool)[3] != W.EQ]
        _, viol = pgd.round_check(inst, np.zeros((inst.n_bool, 1)), x[:, r:r + 1], constraints=ineq)
        assert not viol[ineq].any()
        rep = pgd.repair_equalities(inst, x[:, r])
        assert rep is not None
        for c in unit:
            var, coef, q0, rel = inst.atom((int(inst.lits(c)[0]) >> 1) - inst.n_bool)
            if rel == W.EQ:
                assert sum(Fraction(int(q)) * rep[int(v)] for v, q in zip(var, coef)) == q0
        assert max(abs(float(a_) - b_) for a_, b_ in zip(rep, x[:, r])) <= 1e-3


def test_repair_equalities_cases():
    """The repair solves each equality that does not hold for its last real with
    coefficient +-1 not yet used: chains are solved in order; an equality with no such
    real, or a later pivot that breaks an earlier equality, gives None."""
    def inst_of(eqs, n=3):
        B = W._Builder(0, n)
        for var, coef, q0 in eqs:
            B.con(W.OR, [W.lit(B.atom(var, coef, q0, W.EQ))])
        return B.freeze("r", np.full(n, -9.0), np.full(n, 9.0), [], np.zeros(n), 1.0)
    chain = inst_of([([0, 1], [1, -1], -2), ([1, 2], [1, -1], -3)])     # y1 = y0 + 2, y2 = y1 + 3
    rep = pgd.repair_equalities(chain, [0.5, 2.4999999, 0.0])
    assert rep == [Fraction(1, 2), Fraction(5, 2), Fraction(11, 2)]
    assert pgd.repair_equalities(inst_of([([0, 1], [2, 3], 5)]), [1.0, 0.9, 0.0]) is None   # no +-1 real
    assert pgd.repair_equalities(inst_of([([0, 1], [2, 3], 5)]), [1.0, 1.0, 0.0]) == [1, 1, 0]  # holds: kept
    broken = inst_of([([0, 1], [1, 1], 1), ([1, 2], [1, 1], 2), ([0, 1], [-1, 1], 0)])
    assert pgd.repair_equalities(broken, [0.0, 0.3, 0.1]) is None
    one = inst_of([([0], [3], 7)])                                        # 3 y0 = 7: pinned, no float fits
    dom = pgd.Domain(one)
    assert dom.lo[0] == dom.hi[0] == 7 / 3


def test_equalities_only_as_projected_unit_atoms():
    """A negated equality (a disequality) is not a convex set and cannot be projected
    onto; an equality has no relaxed form for C_sigma (its smoothed probability is 0)."""
    B = W._Builder(0, 2)
    B.con(W.OR, [W.lit(B.atom([0, 1], [1, -1], 0, W.EQ), True)])
    inst = B.freeze("ne", np.zeros(2), np.ones(2), [], np.zeros(2), 1.0)
    with pytest.raises(ValueError):
        pgd.Domain(inst)
    with pytest.raises(ValueError):
        S.normalized_atom([1, -1], 0, S.EQ)
