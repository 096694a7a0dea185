"""PGD step with projection, rounding + exact check + ERWA, and whole annealing
stages: CUDA path vs the FP64 oracle."""
import numpy as np
import pytest

from oracle import objective as OBJ, pgd
from workloads import instances as W

from _gpu_common import setup, sigmas_for, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("make,R", [(lambda: W.jobshop(1002, 10, 5), 70), (lambda: W.tiny_random(1001), 45),
                                    (lambda: W.large_scheduling(1005, 16, 30, 6, 4, 5), 40),
                                    # two jobs through 100 machines: blocks of 100 coupled reals
                                    (lambda: W.jobshop(1002, 2, 100), 64),
                                    # no-wait jobs: equalities' hyperplanes in the projection
                                    (lambda: W.jobshop(1002, 10, 5, no_wait=4), 70)])
def test_pgd_step_parity(make, R):
    import torch
    inst = make()
    P, comp, a, b, w = setup(inst, R)
    sigma = sigmas_for(inst)[1]
    _, _, ga, gb = OBJ.evaluate(inst, a.astype(np.float64), b.astype(np.float64), w.astype(np.float64), sigma)
    ga32, gb32 = ga.astype(np.float32), gb.astype(np.float32)
    eta = 0.05
    dom = pgd.Domain(inst)
    # per-restart step normalised by the total weight of C_sigma (oracle: pgd.step_sizes)
    etas = pgd.step_sizes(inst, w.astype(np.float64), pgd.Config(eta=eta))
    a_ref, b_ref, gn_ref = pgd.pgd_step(a.astype(np.float64), b.astype(np.float64), ga32.astype(np.float64),
                                        gb32.astype(np.float64), etas, inst.scale, dom, 20, 32)
    da, db, dga, dgb, dw = to_dev(a, b, ga32, gb32, w)
    gn = torch.zeros(R, device="cuda")
    wsum = torch.zeros(R, device="cuda")
    comp.weight_sum(R, dw, wsum)
    oc = OBJ.objective_constraints(inst)
    np.testing.assert_allclose(wsum.cpu().numpy(), w[oc].astype(np.float64).sum(0), rtol=1e-5)
    active = torch.ones(R, dtype=torch.uint8, device="cuda")
    active[1::3] = 0
    comp.pgd_step(R, eta, inst.scale, 20, da, db, dga, dgb, gn, active, wsum=wsum, polish=32)
    act = active.cpu().numpy().astype(bool)
    a_out, b_out = da.cpu().numpy(), db.cpu().numpy()
    np.testing.assert_allclose(a_out[:, act], a_ref[:, act], atol=2e-6)
    np.testing.assert_array_equal(a_out[:, ~act], a[:, ~act])
    scale_b = max(1.0, float(np.abs(b_ref).max()))
    np.testing.assert_allclose(b_out[:, act], b_ref[:, act], atol=2e-5 * scale_b)
    np.testing.assert_array_equal(b_out[:, ~act], b[:, ~act])
    np.testing.assert_allclose(gn.cpu().numpy(), gn_ref, rtol=2e-4, atol=1e-6)


@pytest.mark.parametrize("make", [lambda: W.jobshop(1002, 10, 5), lambda: W.large_scheduling(1005, 16, 40, 6, 4, 5)])
def test_projection_lands_in_D_exactly(make):
    """From points near a feasible one (a PGD step's regime), the projection with
    the feasibility polish satisfies every projected unit atom exactly, on the GPU
    and in the oracle, and the two agree."""
    import torch
    inst = make()
    R = 64
    P, comp, a, b, w = setup(inst, R)
    rng = np.random.default_rng(2)
    b = (inst.planted_y[:, None] + rng.normal(0, 3.0, (inst.n_real, R))).astype(np.float32)
    zero_a, zero_b = np.zeros_like(a), np.zeros_like(b)
    da, db, dga, dgb = to_dev(a, b, zero_a, zero_b)
    gn = torch.zeros(R, device="cuda")
    comp.pgd_step(R, 0.05, inst.scale, 20, da, db, dga, dgb, gn, polish=32)
    b_out = db.cpu().numpy().astype(np.float64)
    unit = [c for c in range(inst.n_cons) if OBJ.is_unit_atomic(inst, c)]
    _, viol = pgd.round_check(inst, a.astype(np.float64), b_out, constraints=unit)
    assert not viol[unit].any()
    b_ref = pgd.Domain(inst).project_b(b.astype(np.float64), 20, 32)
    np.testing.assert_allclose(b_out, b_ref, atol=1e-3)


@pytest.mark.parametrize("make,R", [(lambda: W.tiny_random(1001), 45), (lambda: W.jobshop(1002, 10, 5), 64),
                                    (lambda: W.placement2d(1003, 20), 33),
                                    (lambda: W.large_scheduling(1005, 16, 30, 6, 4, 5), 37)])
def test_round_check_erwa_parity(make, R):
    import torch
    inst = make()
    P, comp, a, b, w = setup(inst, R)
    # a third of the restarts sit exactly on the planted assignment (every constraint
    # holds, many atoms exactly on their boundary), a third are planted with a few flips
    rng = np.random.default_rng(3)
    a, b = a.copy(), b.copy()
    a[:, ::3] = 0.5 * inst.planted_x[:, None]
    b[:, ::3] = inst.planted_y[:, None]
    a[:, 1::3] = 0.5 * inst.planted_x[:, None] * np.where(rng.random((inst.n_bool, 1)) < 0.05, -1, 1)
    b[:, 1::3] = inst.planted_y[:, None]
    h0 = rng.uniform(0, 2, (inst.n_cons, R)).astype(np.float32)
    x_ref, viol_ref = pgd.round_check(inst, a.astype(np.float64), b.astype(np.float64))
    for update_w in (True, False):
        w_ref, h_ref, nu_ref = pgd.erwa(w.astype(np.float64), h0.astype(np.float64), viol_ref.astype(np.float64),
                                        1, 0.5, 2.0, 1 if update_w else 2)
        da, db, dw, dh = to_dev(a, b, w, h0)
        x = torch.zeros((inst.n_bool, R), dtype=torch.int8, device="cuda")
        viol = torch.zeros((inst.n_cons, R), dtype=torch.uint8, device="cuda")
        nu = torch.zeros(R, dtype=torch.int32, device="cuda")
        comp.round_check(R, da, db, nu, x=x, violated=viol, w=dw, h=dh, rho=0.5, gamma=2.0, update_w=update_w)
        np.testing.assert_array_equal(x.cpu().numpy(), x_ref)
        np.testing.assert_array_equal(viol.cpu().numpy().astype(bool), viol_ref)
        np.testing.assert_array_equal(nu.cpu().numpy(), nu_ref.astype(np.int32))
        np.testing.assert_allclose(dw.cpu().numpy(), w_ref, rtol=2e-6)
        np.testing.assert_allclose(dh.cpu().numpy(), h_ref, rtol=1e-6, atol=1e-6)
    assert (nu_ref[::3] == 0).all()
    # the weight rescale: restarts whose mean weight over C_sigma passed 2^32 (every
    # fourth, weights times 2^33) get their updated weights times 2^-32, the rest not
    big = w.copy()
    big[:, ::4] *= 2.0 ** 33
    mean = pgd.mean_weight(inst, big.astype(np.float64), OBJ.PROJECT)
    assert mean is not None and (mean[::4] > pgd.W_RESCALE_AT).all() and (mean[1::4] < 2.0 ** 8).all()
    w_ref, h_ref, _ = pgd.erwa(big.astype(np.float64), h0.astype(np.float64), viol_ref.astype(np.float64),
                               1, 0.5, 2.0, 1, mean_w=mean)
    da, db, dw, dh = to_dev(a, b, big, h0)
    wsum = torch.zeros(R, dtype=torch.float32, device="cuda")
    comp.weight_sum(R, dw, wsum)
    nu = torch.zeros(R, dtype=torch.int32, device="cuda")
    comp.round_check(R, da, db, nu, w=dw, h=dh, rho=0.5, gamma=2.0, update_w=True, wsum=wsum)
    np.testing.assert_allclose(dw.cpu().numpy(), w_ref, rtol=2e-6)
    np.testing.assert_allclose(dh.cpu().numpy(), h_ref, rtol=1e-6, atol=1e-6)


def _solver(inst, R, comp, P, **kw):
    from paper_2603_22877_b300 import Solver
    return Solver(P, comp, R, **kw)


@pytest.mark.parametrize("use_graph,form", [(True, "fused"), (False, "fused"), (False, "plain")])
def test_stage_matches_oracle_first_iterations(use_graph, form):
    """A stage of 5 PGD iterations then round/check/ERWA: GPU vs oracle run_stage,
    for the fused stage (graph or not) and the plain form driven call by call."""
    inst = W.jobshop(1002, 10, 5)
    R = 40
    P, comp, a, b, _ = setup(inst, R)
    eta = 0.02
    cfg = pgd.Config(eta=eta, t_max=5, sweeps=20, polish=32)
    S = _solver(inst, R, comp, P, eta=eta, b_scale=inst.scale, t_max=5, sweeps=20, use_graph=use_graph, form=form)
    S.reset(a, b)
    sigma = sigmas_for(inst)[0]
    S.stage(sigma, 1)
    w0 = np.ones((inst.n_cons, R))
    h0 = np.zeros((inst.n_cons, R))
    a_ref, b_ref, w_ref, h_ref, nu_ref, its_ref, obj_ref = pgd.run_stage(inst, a, b, w0, h0, sigma, 1, cfg)
    np.testing.assert_allclose(S.a.cpu().numpy(), a_ref, atol=1e-4)
    np.testing.assert_allclose(S.b.cpu().numpy(), b_ref, atol=1e-4 * inst.meta["horizon"])
    np.testing.assert_array_equal(S.iters.cpu().numpy(), its_ref)
    np.testing.assert_allclose(S.obj.cpu().numpy(), obj_ref, rtol=1e-4, atol=1e-3)
    # the check and ERWA on the GPU's own final point are exact
    _, viol = pgd.round_check(inst, S.a.cpu().numpy().astype(np.float64), S.b.cpu().numpy().astype(np.float64))
    np.testing.assert_array_equal(S.n_unsat.cpu().numpy(), viol.sum(0))
    np.testing.assert_allclose(S.w.cpu().numpy(), np.power(2.0, viol.astype(np.float64)), rtol=1e-6)
    assert (S.h.cpu().numpy() == 1.0).all()


@pytest.mark.parametrize("form", ["fused", "plain"])
def test_stage_epsilon_rule_stops_restarts(form):
    """With eps large every restart stops after its first iteration (Eq. critical)."""
    inst = W.tiny_random(1001)
    R = 50
    P, comp, a, b, _ = setup(inst, R)
    S = _solver(inst, R, comp, P, eta=0.01, b_scale=inst.scale, t_max=7, eps=1e6, form=form)
    S.reset(a, b)
    S.stage(sigmas_for(inst)[0], 1)
    assert (S.iters.cpu().numpy() == 1).all()
    if form == "fused":
        assert int(S.ctl[0].item()) == 0 and int(S.ctl[1].item()) == 0


def test_stage_host_buffers_match_device():
    inst = W.jobshop(1002, 10, 5)
    R = 64
    P, comp, a, b, _ = setup(inst, R)
    S1 = _solver(inst, R, comp, P, eta=0.02, b_scale=inst.scale, t_max=4)
    S1.reset(a, b)
    S1.stage(sigmas_for(inst)[0], 1)
    S2 = _solver(inst, R, comp, P, eta=0.02, b_scale=inst.scale, t_max=4)
    S2.reset(a, b)
    nu = np.zeros(R, np.int32)
    ob = np.zeros(R, np.float32)
    S2.stage_host(sigmas_for(inst)[0], 1, np.ascontiguousarray(a), np.ascontiguousarray(b), nu, ob)
    np.testing.assert_allclose(S2.a.cpu().numpy(), S1.a.cpu().numpy(), atol=1e-5)
    np.testing.assert_allclose(ob, S1.obj.cpu().numpy(), rtol=1e-5, atol=1e-3)
    np.testing.assert_array_equal(nu, S2.n_unsat.cpu().numpy())


def test_anneal_finds_exactly_verified_sat():
    """Alg. 2 on a small instance of the scheduling family: some restart reaches
    #Unsat = 0, and both the library's exact verifier and the oracle's exact
    check confirm the assignment."""
    from oracle import semantics as Sm
    inst = W.large_scheduling(1005, 16, 30, 6, 4, 5)
    R = 64
    P, comp, a, b, _ = setup(inst, R)
    S = _solver(inst, R, comp, P, eta=0.05, b_scale=inst.scale, t_max=50)
    S.reset(a, b)
    sched = [inst.scale / (0.1 * t) for t in range(1, 21)]
    res = S.anneal(sched)
    assert res["sat"], res
    assert Sm.unsat_constraints(inst, res["x"], res["y"]) == []
    assert res["rejected_candidates"] == 0   # the device check and the host verifier agree


def test_checkpoint_resume_reproduces_the_run():
    """Alg. 2 stopped after two stages, checkpointed, and resumed in a fresh
    solver: the state round-trips exactly, and after the third stage it matches an
    uninterrupted run up to the order of floating-point atomic additions (the
    kernels' reductions are not ordered)."""
    inst = W.large_scheduling(1005, 16, 30, 6, 4, 5)
    R = 48
    P, comp, a, b, _ = setup(inst, R)
    sched = [inst.scale / (0.1 * t) for t in range(1, 4)]
    S = _solver(inst, R, comp, P, eta=0.05, b_scale=inst.scale, t_max=8)
    S.reset(a, b)
    for t in (1, 2):
        S.stage(sched[t - 1], t)
    ckpt = S.state_dict()
    S.stage(sched[2], 3)
    S2 = _solver(inst, R, comp, P, eta=0.05, b_scale=inst.scale, t_max=8)
    S2.load_state_dict(ckpt)
    again = S2.state_dict()
    for k, v in ckpt.items():
        assert (again[k] == v).all(), k
    S2.stage(sched[2], 3)
    np.testing.assert_allclose(S2.a.cpu().numpy(), S.a.cpu().numpy(), atol=1e-4)
    np.testing.assert_allclose(S2.b.cpu().numpy(), S.b.cpu().numpy(), atol=1e-4 * inst.scale)
    same = (S2.n_unsat.cpu().numpy() == S.n_unsat.cpu().numpy()).mean()
    assert same >= 0.95, same


@pytest.mark.parametrize("form", ["fused", "plain"])
def test_long_schedule_keeps_weights_finite(form):
    """200 stages of Alg. 2 on an unsatisfiable instance (x0 and not x0): as printed the
    weights of the failing clauses pass the FP32 range near stage 90; with the rescale
    of a restart whose mean weight passed 2^32 they stay finite, no step is non-finite
    and the largest weight stays far below the range."""
    import torch
    B = W._Builder(3, 1)
    A = B.atom([0], [1], 5, W.LE)
    B.con(W.OR, [W.lit(0)])
    B.con(W.OR, [W.lit(0, True)])
    B.con(W.OR, [W.lit(1), W.lit(2), W.lit(A)])
    inst = B.freeze("unsat", [0.0], [10.0], np.ones(3, np.int8), np.zeros(1), 10.0)
    R = 40
    P, comp, a, b, _ = setup(inst, R)
    S = _solver(inst, R, comp, P, eta=0.05, b_scale=inst.scale, t_max=2, form=form)
    S.reset(a, b)
    for t in range(1, 201):
        S.stage(inst.scale / (0.1 * t), t)
    w = S.w.cpu().numpy()
    assert np.isfinite(w).all() and (w >= 0).all()
    assert w.max() < 2.0 ** 64
    assert (S.n_unsat.cpu().numpy() >= 1).all()
    assert np.isfinite(S.gnorm2.cpu().numpy()).all() and np.isfinite(S.obj.cpu().numpy()).all()
    if form == "fused":
        assert int(S.ctl[1].item()) == 0


def test_round_matches_the_oracle_rounding():
    """fsmt_round (Alg. 1: x = TRUE (-1) iff a < 0) against the oracle's rounding, on
    points that include exact zeros of both signs and the box ends."""
    import torch
    inst = W.jobshop(1002, 10, 5)
    R = 70
    P, comp, a, b, _ = setup(inst, R)
    a = a.copy()
    a[0, :4] = [0.0, -0.0, -1.0, 1.0]
    a[1, :3] = [np.float32(-1e-30), np.float32(1e-30), np.float32(-np.finfo(np.float32).tiny)]
    da, = to_dev(a)
    x = torch.zeros((inst.n_bool, R), dtype=torch.int8, device="cuda")
    comp.round(R, da, x)
    x_ref, _ = pgd.round_check(inst, a.astype(np.float64), b.astype(np.float64), constraints=[])
    np.testing.assert_array_equal(x.cpu().numpy(), x_ref)


def test_converge_and_nonfinite_marks():
    """fsmt_converge applies Eq. critical to restarts still iterating (active 1):
    ||g||^2 <= eps^2 stops one (active 0), a non-finite ||g||^2 stops it with active 2
    and ctl[1] bit 0, the others keep iterating and are counted in ctl[0]; every
    iterating restart's iteration count grows by one.  fsmt_mark_nonfinite then sets
    bit 31 of #Unsat exactly for the restarts with active 2."""
    import torch
    inst = W.tiny_random(1001)
    R = 8
    P, comp, _, _, _ = setup(inst, R)
    eps = 0.01
    g = np.array([0.5, 1e-5, np.nan, np.inf, 2.0, 1e-4, -np.inf, 3e-4], np.float32)
    act = np.array([1, 1, 1, 1, 0, 1, 1, 1], np.uint8)
    dg = torch.from_numpy(g).cuda()
    da = torch.from_numpy(act).cuda()
    it = torch.full((R,), 3, dtype=torch.int32, device="cuda")
    ctl = torch.tensor([R, 0, 0, 0], dtype=torch.int32, device="cuda")
    comp.converge(R, eps, dg, da, it, ctl)
    assert da.cpu().numpy().tolist() == [1, 0, 2, 2, 0, 0, 2, 1]
    assert it.cpu().numpy().tolist() == [4, 4, 4, 4, 3, 4, 4, 4]
    assert ctl.cpu().numpy().tolist()[:2] == [2, 1]
    nu = torch.tensor([3, 0, 5, 1, 0, 0, 7, 2], dtype=torch.int32, device="cuda")
    comp.mark_nonfinite(R, da, nu)
    bit = np.int32(-2 ** 31)
    want = np.array([3, 0, 5 | bit, 1 | bit, 0, 0, 7 | bit, 2], np.int32)
    np.testing.assert_array_equal(nu.cpu().numpy(), want)


@pytest.mark.parametrize("make,R", [(lambda: W.jobshop(1002, 10, 5), 70),
                                    (lambda: W.concat(W.uneven_batch(1004, 6, (3, 12), (3, 9)), "b"), 32),
                                    (lambda: W.jobshop(1002, 10, 5, no_wait=4), 40)])
def test_generated_projection_matches_the_generic_loop(make, R, monkeypatch):
    """Blocks of coupled reals whose shape got a run-time generated projection routine
    (fsmt_info.proj_shapes > 0: the iterate in registers, the coefficients as
    constants) end at the same points with the same ||g||^2, bit for bit, as the
    generic loop that FSMT_NO_JIT leaves every block to: the routines repeat its
    operations in its order."""
    import ctypes as C
    import torch
    from paper_2603_22877_b300 import _lib as L
    from paper_2603_22877_b300.engine import Problem
    inst = make()
    P, comp, a, b, w = setup(inst, R)
    info = L.Info()
    L.call("fsmt_compiled_info", comp.h, C.byref(info))
    assert info.proj_shapes > 0
    monkeypatch.setenv("FSMT_NO_JIT", "1")
    comp2 = Problem.from_instance(inst).compile().upload()
    L.call("fsmt_compiled_info", comp2.h, C.byref(info))
    assert info.proj_shapes == 0
    sigma = sigmas_for(inst)[1]
    _, _, ga, gb = OBJ.evaluate(inst, a.astype(np.float64), b.astype(np.float64), w.astype(np.float64), sigma)
    wsum = torch.zeros(R, device="cuda")   # one set of weight sums (their float atomics order varies by run)
    comp.weight_sum(R, to_dev(w)[0], wsum)
    outs = []
    for c_ in (comp, comp2):
        da, db, dga, dgb = to_dev(a, b, ga.astype(np.float32), gb.astype(np.float32))
        gn = torch.zeros(R, device="cuda")
        c_.pgd_step(R, 0.05, inst.scale, 20, da, db, dga, dgb, gn, wsum=wsum, polish=32)
        outs.append((da.cpu().numpy(), db.cpu().numpy(), gn.cpu().numpy()))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    # ||g||^2 adds the blocks' shares with float atomics, in an order that varies by run
    np.testing.assert_allclose(outs[0][2], outs[1][2], rtol=1e-6)


def test_equalities_check_within_the_margin_and_anneal_to_exact_sat():
    """No-wait jobs (each precedence an equality q.y = q0, projected as a hyperplane): after
    a PGD step every equality is within a few FP32 bands of its hyperplane; the device check
    counts an equality as holding within the polish margin, every other constraint exactly
    -- the oracle's exact check with that rule for the equalities gives the same #Unsat.
    Alg. 2 then reaches a restart that the host repairs onto the hyperplanes exactly and
    verifies exactly (fsmt_repair_equalities, fsmt_verify_exact), and the oracle's exact
    check agrees on the certificate."""
    import torch
    from fractions import Fraction
    from oracle import semantics as Sm
    inst = W.jobshop(1002, 8, 4, no_wait=3)
    R = 64
    P, comp, a, b, w = setup(inst, R)
    sigma = sigmas_for(inst)[1]
    _, _, ga, gb = OBJ.evaluate(inst, a.astype(np.float64), b.astype(np.float64), w.astype(np.float64), sigma)
    da, db, dga, dgb = to_dev(a, b, ga.astype(np.float32), gb.astype(np.float32))
    gn = torch.zeros(R, device="cuda")
    comp.pgd_step(R, 0.05, inst.scale, 20, da, db, dga, dgb, gn, polish=32)
    nu = torch.zeros(R, dtype=torch.int32, device="cuda")
    comp.round_check(R, da, db, nu)
    a_out, b_out = da.cpu().numpy().astype(np.float64), db.cpu().numpy().astype(np.float64)
    _, viol = pgd.round_check(inst, a_out, b_out)
    eq_cons = []
    for c in range(inst.n_cons):
        if OBJ.is_unit_atomic(inst, c):
            var, coef, q0, rel = inst.atom((int(inst.lits(c)[0]) >> 1) - inst.n_bool)
            if rel == W.EQ:
                eq_cons.append(c)
                for r in range(R):
                    viol[c, r] = not pgd.eq_holds_on_device(var, coef, q0, b_out[:, r])
                    z = sum(Fraction(int(q)) * Fraction(float(b_out[int(v), r])) for v, q in zip(var, coef)) - q0
                    mag = abs(q0) + sum(abs(float(q) * b_out[int(v), r]) for v, q in zip(var, coef))
                    assert abs(float(z)) <= 4 * pgd.eq_band(len(var), mag)
    assert eq_cons and not viol[eq_cons].any()
    np.testing.assert_array_equal(nu.cpu().numpy(), viol.sum(0))
    S = _solver(inst, R, comp, P, eta=0.05, b_scale=inst.scale, t_max=50)
    S.reset(a, b)
    res = S.anneal([inst.scale / (0.1 * t) for t in range(1, 61)])
    assert res["sat"], res
    assert Sm.unsat_constraints(inst, res["x"], res["y"]) == []
    for c in eq_cons:  # the certificate holds every equality exactly
        assert Sm.constraint_holds(inst, c, res["x"], res["y"])


@pytest.mark.parametrize("R", [4, 100, 512, 1100, 70])
def test_weight_sum_over_column_passes(R):
    """wsum[r] = sum of w over C_sigma: the float4 row kernel (R a multiple of 4,
    one or several 512-restart passes, a ragged last pass) and the general one (R = 70)."""
    import torch
    inst = W.jobshop(1002, 10, 5)
    from paper_2603_22877_b300.engine import Problem
    comp = Problem.from_instance(inst).compile().upload()
    w = np.random.default_rng(R).uniform(0.5, 3.0, (inst.n_cons, R)).astype(np.float32)
    wsum = torch.full((R,), float("nan"), device="cuda")
    comp.weight_sum(R, to_dev(w)[0], wsum)
    oc = OBJ.objective_constraints(inst)
    np.testing.assert_allclose(wsum.cpu().numpy(), w[oc].astype(np.float64).sum(0), rtol=1e-5)
