"""Edge cases of the CUDA path against the oracle: constant diagrams, a diagram
too large for a chunk (served by the warp-per-constraint kernel), wide atoms,
ragged restart counts, sigma = 0 and an objective with no constraints."""
import numpy as np
import pytest

from oracle import objective as OBJ
from workloads import instances as W

from _gpu_common import COP_TOL, assert_grad_close, gpu_adjoint, setup

pytestmark = pytest.mark.gpu


def mixed_instance(big=False, seed=0):
    rng = np.random.default_rng(seed)
    n_bool, n_real = 240, 30
    B = W._Builder(n_bool, n_real)
    py = rng.uniform(0, 10, n_real)
    atoms = []
    for _ in range(40):
        nnz = int(rng.integers(1, 21))
        var = rng.choice(n_real, nnz, replace=False)
        coef = rng.integers(1, 6, nnz) * rng.choice([-1, 1], nnz)
        atoms.append(B.atom(var, coef, int(np.ceil(float(coef @ py[var]))), W.LE))
    B.con(W.OR, [])                                       # constant FALSE
    B.con(W.CARD_LE, [W.lit(0), W.lit(1)], param=5)       # constant TRUE
    B.con(W.OR, [W.lit(2, True)])                         # a single literal
    for _ in range(60):
        kind = int(rng.choice([W.OR, W.XOR, W.CARD_LE, W.NAE, W.NEQ_OR]))
        L = int(rng.integers(2, 9))
        ids = list(rng.choice(n_bool, L, replace=False)) + list(rng.choice(atoms, 2, replace=False))
        lits = [2 * int(i) + int(rng.integers(2)) for i in ids]
        param = int(rng.integers(0, len(lits))) if kind == W.CARD_LE else (2 if kind == W.NEQ_OR else 0)
        B.con(kind, lits, param)
    if big:  # 200 distinct literals: more slots than a chunk holds
        B.con(W.XOR, [2 * i + (i % 2) for i in range(200)])
        B.con(W.CARD_LE, [2 * i for i in range(30, 60)] + [2 * atoms[0]], param=6)
    return B.freeze("mixed", np.zeros(n_real), np.full(n_real, 10.0), np.ones(n_bool, np.int8), py, 10.0)


@pytest.mark.parametrize("big", [False, True])
@pytest.mark.parametrize("R", [1, 33, 65])
def test_mixed_kinds_against_oracle(big, R):
    inst = mixed_instance(big)
    P, comp, a, b, w = setup(inst, R)
    if big:
        assert comp.info["n_chunks"] == 0  # the warp-per-constraint kernel serves this instance
    else:
        assert comp.info["n_chunks"] > 0
    D = OBJ.Diagrams(inst)
    oc = OBJ.objective_constraints(inst)
    for sigma in (0.0, 0.7, 5.0):
        obj_ref, cop_ref, ga_ref, gb_ref = OBJ.evaluate(inst, a.astype(np.float64), b.astype(np.float64),
                                                        w.astype(np.float64), sigma, diagrams=D)
        obj, cop, ga, gb = gpu_adjoint(comp, R, np.float32(sigma), a, b, w)
        assert np.abs(cop[oc] - cop_ref[oc]).max() <= COP_TOL
        assert cop[0].max() == 0.0 and cop[1].min() == 1.0
        np.testing.assert_allclose(obj, obj_ref, rtol=1e-5, atol=1e-4)
        assert_grad_close(ga, ga_ref, f"grad_a sigma={sigma}")
        assert_grad_close(gb, gb_ref, f"grad_b sigma={sigma}")


def test_objective_without_constraints():
    """Every constraint is a unit atom handled by the projection: C = 0, gradients 0."""
    B = W._Builder(3, 2)
    B.con(W.OR, [W.lit(B.atom([0], [1], 5, W.LE))])
    B.con(W.OR, [W.lit(B.atom([0, 1], [1, -1], -1, W.LE))])
    inst = B.freeze("units", np.zeros(2), np.full(2, 9.0), np.ones(3, np.int8), np.array([1.0, 3.0]), 1.0)
    R = 40
    P, comp, a, b, w = setup(inst, R)
    assert comp.info["n_obj_cons"] == 0
    obj, cop, ga, gb = gpu_adjoint(comp, R, 1.0, a, b, w)
    assert (obj == 0).all() and (ga == 0).all() and (gb == 0).all()


def test_atom_probability_within_published_erfc_bound():
    """The kernel's atom probability p = erfc(u)/2 uses Abramowitz & Stegun 7.1.26,
    whose absolute error is at most 1.5e-7; with FP32 rounding the COP of a
    one-atom constraint stays within 5e-7 of the exact Gaussian CDF over u in [-6, 6]."""
    from scipy.special import erfc
    B = W._Builder(0, 1)
    B.con(W.OR, [W.lit(B.atom([0], [1], 0, W.LE))])
    inst = B.freeze("erfc", np.array([-100.0]), np.array([100.0]), [], np.zeros(1), 1.0)
    R = 1024
    P, comp, _, _, _ = setup(inst, R, policy=OBJ.SOFT)
    sigma = 1.0
    u = np.linspace(-6, 6, R)
    b = (u * np.sqrt(2.0) * sigma).astype(np.float32)[None, :]  # z = b, ||q|| = 1
    w = np.ones((1, R), np.float32)
    _, cop, _, gb = gpu_adjoint(comp, R, sigma, np.zeros((0, R), np.float32), b, w)
    uu = b[0].astype(np.float64) / (np.sqrt(2.0) * sigma)
    ref = 0.5 * erfc(uu)
    assert np.abs(cop[0] - ref).max() <= 5e-7
    # and the derivative is the exact one: dC/db = -2 dp/db = (2/sqrt(pi)) e^{-u^2} / (sqrt(2) sigma)
    dref = 2.0 / np.sqrt(np.pi) * np.exp(-uu * uu) / (np.sqrt(2.0) * sigma)
    assert np.abs(gb[0] - dref).max() <= 1e-6 * dref.max()


@pytest.mark.parametrize("make,R", [(lambda: W.large_scheduling(1005, 16, 30, 6, 4, 5), 70),
                                    (lambda: W.placement2d(1003, 20), 33), (lambda: W.tiny_random(1001), 64)])
def test_specialised_and_generic_kernels_agree(make, R, monkeypatch):
    """Diagram shapes get run-time generated routines at upload; with FSMT_NO_JIT the
    ahead-of-time kernel runs every constraint through the generic path.  Both agree
    with the oracle."""
    from paper_2603_22877_b300.engine import Problem
    inst = make()
    P, comp, a, b, w = setup(inst, R)
    assert comp.upload().info is not None
    from paper_2603_22877_b300 import _lib as L
    import ctypes as C
    info = L.Info()
    L.call("fsmt_compiled_info", comp.h, C.byref(info))
    assert info.jit_shapes > 0
    monkeypatch.setenv("FSMT_NO_JIT", "1")
    comp2 = Problem.from_instance(inst).compile().upload()
    L.call("fsmt_compiled_info", comp2.h, C.byref(info))
    assert info.jit_shapes == 0
    sigma = float(np.float32(inst.scale))
    ref = OBJ.evaluate(inst, a.astype(np.float64), b.astype(np.float64), w.astype(np.float64), sigma)
    oc = OBJ.objective_constraints(inst)
    for c_ in (comp, comp2):
        obj, cop, ga, gb = gpu_adjoint(c_, R, sigma, a, b, w)
        assert np.abs(cop[oc] - ref[1][oc]).max() <= COP_TOL
        assert_grad_close(ga, ref[2], "grad_a")
        assert_grad_close(gb, ref[3], "grad_b")


@pytest.mark.parametrize("no_jit,no_stage", [("0", "1"), ("1", "0"), ("1", "1")])
def test_unstaged_and_generic_paths_agree(no_jit, no_stage, monkeypatch):
    """The chunk's reals are normally staged in shared memory per restart tile
    (b in, dC/db out); FSMT_NO_STAGE reads b and writes dC/db in global memory
    instead.  Every combination with and without generated routines agrees with
    the oracle, on an instance whose atoms share reals across constraints."""
    inst = W.large_scheduling(1005, 16, 30, 6, 4, 5)
    R = 70  # two restart tiles and a ragged third
    monkeypatch.setenv("FSMT_NO_JIT", no_jit)
    monkeypatch.setenv("FSMT_NO_STAGE", no_stage)
    P, comp, a, b, w = setup(inst, R)  # compiled and uploaded under these settings
    sigma = float(np.float32(inst.scale))
    ref = OBJ.evaluate(inst, a.astype(np.float64), b.astype(np.float64), w.astype(np.float64), sigma)
    oc = OBJ.objective_constraints(inst)
    obj, cop, ga, gb = gpu_adjoint(comp, R, sigma, a, b, w)
    assert np.abs(cop[oc] - ref[1][oc]).max() <= COP_TOL
    np.testing.assert_allclose(obj, ref[0], rtol=1e-5, atol=1e-4)
    assert_grad_close(ga, ref[2], "grad_a")
    assert_grad_close(gb, ref[3], "grad_b")


@pytest.mark.parametrize("policy", [0, 1])  # unit atoms projected (one warp per constraint) or in C_sigma (chunks)
def test_round_check_filter_keeps_boundary_cases_exact(policy):
    """The check decides each atom with an FP32 filter and falls back to exact
    arithmetic inside the filter's error band.  Points on an atom's boundary
    (z = 0) and one float step to either side, with large integer coefficients,
    strict and non-strict: the GPU's #Unsat and violations equal the oracle's
    exact check restart by restart."""
    import torch
    from oracle import pgd
    from paper_2603_22877_b300.engine import Problem
    rng = np.random.default_rng(5)
    B = W._Builder(0, 3)
    # c0 y0 + c1 y1 + c2 y2 (rel) q0 with q0 the value at an integer point Y
    Y = np.array([1234567.0, 89.0, 4097.0])
    coefs = [[3, -7, 0], [1_000_003, 0, -2], [5, 11, -13], [-8_388_607, 1, 0]]
    for cf in coefs:
        var = [j for j in range(3) if cf[j] != 0]
        c = [cf[j] for j in var]
        q0 = int(sum(cf[j] * int(Y[j]) for j in var))
        for rel in (W.LE, W.LT):
            B.con(W.OR, [W.lit(B.atom(var, c, q0, rel))])
    inst = B.freeze("boundary", np.full(3, -1e8), np.full(3, 1e8), [], Y, 1.0)
    R = 96
    b = np.repeat(Y.astype(np.float32)[:, None], R, axis=1)
    for r in range(R):  # each restart moves some reals by -1, 0 or +1 float steps
        steps = rng.integers(-1, 2, 3) if r else np.zeros(3, int)
        for j in range(3):
            for _ in range(abs(int(steps[j]))):
                b[j, r] = np.nextafter(b[j, r], np.float32(np.inf) if steps[j] > 0 else np.float32(-np.inf))
    comp = Problem.from_instance(inst).compile(policy).upload()
    assert (comp.info["n_chunks"] > 0) == (policy == 1)
    nu = torch.zeros(R, dtype=torch.int32, device="cuda")
    viol = torch.zeros((inst.n_cons, R), dtype=torch.uint8, device="cuda")
    comp.round_check(R, torch.zeros((0, R), device="cuda"), torch.from_numpy(b).cuda(), nu, violated=viol)
    _, ref = pgd.round_check(inst, np.zeros((0, R)), b.astype(np.float64))
    np.testing.assert_array_equal(viol.cpu().numpy().astype(bool), ref)
    np.testing.assert_array_equal(nu.cpu().numpy(), ref.sum(0))
    assert ref[:, 0].sum() == len(coefs)  # at Y itself every strict atom fails and every non-strict holds


@pytest.mark.parametrize("make,R", [(lambda: W.large_scheduling(1005, 16, 30, 6, 4, 5), 70),
                                    (lambda: mixed_instance(False), 33),
                                    (lambda: W.placement2d(1003, 20), 40),   # 7-node diagrams: odd row counts
                                    (lambda: W.random_hybrid(1006, 300), 24)])  # diagrams of up to 650 nodes
def test_every_launch_configuration_and_the_autotuner(make, R):
    """Each kernel configuration the library offers for an instance (kernel
    variant, restarts per lane, staged reals) agrees with the oracle; the
    autotuner times them all and pins one of them."""
    import torch
    inst = make()
    P, comp, a, b, w = setup(inst, R)
    cfgs = comp.launch_configs(R)
    assert len(cfgs) >= 2
    keys = {(c.variant, c.restarts_per_lane, c.staged_reals) for c in cfgs}
    assert len(keys) == len(cfgs)
    sigma = float(np.float32(inst.scale))
    ref = OBJ.evaluate(inst, a.astype(np.float64), b.astype(np.float64), w.astype(np.float64), sigma)
    oc = OBJ.objective_constraints(inst)
    for cfg in cfgs:
        comp.select_config(R, cfg)
        obj, cop, ga, gb = gpu_adjoint(comp, R, sigma, a, b, w)
        what = cfg.as_dict()
        assert np.abs(cop[oc] - ref[1][oc]).max() <= COP_TOL, what
        assert_grad_close(ga, ref[2], f"grad_a {what}")
        assert_grad_close(gb, ref[3], f"grad_b {what}")
    comp.select_config(R, None)
    da, db, dw = (torch.from_numpy(x).cuda() for x in (a, b, w))
    ga, gb, ob = torch.ones_like(da), torch.ones_like(db), torch.ones(R, device="cuda")
    best = comp.autotune(R, sigma, dw, da, db, ga, gb, ob)
    assert best.ms > 0 and (best.variant, best.restarts_per_lane, best.staged_reals) in keys
    assert not ga.any() and not gb.any() and not ob.any()  # scratch left zero
    obj, cop, ga2, gb2 = gpu_adjoint(comp, R, sigma, a, b, w)
    assert_grad_close(ga2, ref[2], "grad_a after autotune")


@pytest.mark.parametrize("policy", [OBJ.PROJECT, OBJ.SOFT])
def test_nonfinite_points_are_marked(policy):
    """A restart whose point has a NaN or infinite coordinate that the check reads gets
    bit 31 of its #Unsat set (chunked check and warp-per-constraint check alike); the
    other restarts' counts are the oracle's.  In a stage the box clamp turns such a
    point finite after one step, so the restart is marked from its non-finite ||g||^2
    (active = 2), in the fused and the plain form; the host-buffer stage reports
    FSMT_ENAN."""
    import torch
    from oracle import pgd
    from paper_2603_22877_b300 import Solver, _lib as L
    inst = W.jobshop(1002, 10, 5)
    R = 40
    P, comp, a, b, _ = setup(inst, R, policy)
    a, b = a.copy(), b.copy()
    bad = {3, 5, 7, 33}
    a[0, 3] = np.nan
    b[0, 5] = np.inf
    b[1, 7] = np.nan
    a[:, 33] = -np.inf
    nu = torch.zeros(R, dtype=torch.int32, device="cuda")
    comp.round_check(R, torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), nu)
    nu = nu.cpu().numpy()
    good = [r for r in range(R) if r not in bad]
    _, viol = pgd.round_check(inst, a[:, good].astype(np.float64), b[:, good].astype(np.float64))
    np.testing.assert_array_equal(nu[good], viol.sum(0))
    assert (nu[sorted(bad)] < 0).all()
    # the fused stage from host buffers: FSMT_ENAN, the finite restarts still iterate
    S = Solver(P, comp, R, eta=0.02, b_scale=inst.scale, t_max=3)
    nuh = np.zeros(R, np.int32)
    ob = np.zeros(R, np.float32)
    with pytest.raises(L.FsmtError) as err:
        S.stage_host(inst.scale / 0.5, 1, np.ascontiguousarray(a), np.ascontiguousarray(b), nuh, ob)
    assert err.value.status == L.ENAN
    assert (nuh[sorted(bad)] < 0).all() and (nuh[good] >= 0).all()
    assert np.isfinite(ob[good]).all()
    assert (S.active.cpu().numpy()[sorted(bad)] == 2).all() and int(S.ctl[1].item()) == 1
    S2 = Solver(P, comp, R, eta=0.02, b_scale=inst.scale, t_max=3, form="plain")
    S2.reset(a, b)
    S2.stage(inst.scale / 0.5, 1)
    nu2 = S2.n_unsat.cpu().numpy()
    assert (nu2[sorted(bad)] < 0).all() and (nu2[good] >= 0).all()
