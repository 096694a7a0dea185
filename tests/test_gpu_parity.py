"""Forward COP, objective and adjoint gradient: CUDA path vs the FP64 oracle.

Element by element on every (constraint, restart) and every gradient entry, at
sizes the oracle finishes in seconds that still span several restart tiles and
a ragged tail (R not a multiple of 32)."""
import numpy as np
import pytest

from oracle import objective as OBJ
from workloads import instances as W

from _gpu_common import COP_TOL, assert_grad_close, gpu_adjoint, setup, sigmas_for, to_dev

pytestmark = pytest.mark.gpu

CASES = {
    "tiny_random_R64": (lambda: W.tiny_random(1001), 64),
    "tiny_random_R45": (lambda: W.tiny_random(1001), 45),
    "jobshop_small_R70": (lambda: W.jobshop(1002, 10, 5), 70),
    "placement_small_R33": (lambda: W.placement2d(1003, 20), 33),
    "placement_nosel_R40": (lambda: W.placement2d(1003, 16, selectors=False), 40),
    "sched_small_R37": (lambda: W.large_scheduling(1005, 16, 30, 6, 4, 5), 37),
    "sched_5w_R50": (lambda: W.large_scheduling(1005, 5, 30, 6, 4, 5), 50),
    "placement3d_R36": (lambda: W.placement3d(1007, 4, 2), 36),
    "batch_small_R32": (lambda: W.concat(W.uneven_batch(1004, 4, (3, 8), (2, 5)), "b"), 32),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("policy", [OBJ.PROJECT, OBJ.SOFT])
def test_cop_objective_gradient(name, policy):
    make, R = CASES[name]
    inst = make()
    P, comp, a, b, w = setup(inst, R, policy)
    a64, b64, w64 = a.astype(np.float64), b.astype(np.float64), w.astype(np.float64)
    diagrams = OBJ.Diagrams(inst)
    obj_cons = OBJ.objective_constraints(inst, policy)
    others = sorted(set(range(inst.n_cons)) - set(obj_cons))
    for sigma in sigmas_for(inst):
        obj_ref, cop_ref, ga_ref, gb_ref = OBJ.evaluate(inst, a64, b64, w64, sigma, policy, diagrams)
        for plain in (False, True):
            obj, cop, ga, gb = gpu_adjoint(comp, R, sigma, a, b, w, plain)
            err = np.abs(cop[obj_cons] - cop_ref[obj_cons]).max()
            assert err <= COP_TOL, (name, sigma, plain, err)
            assert np.isnan(cop[others]).all()
            np.testing.assert_allclose(obj, obj_ref, rtol=1e-5, atol=1e-5 * np.abs(w64).sum(0).max())
            assert_grad_close(ga, ga_ref, f"{name} grad_a sigma={sigma} plain={plain}")
            assert_grad_close(gb, gb_ref, f"{name} grad_b sigma={sigma} plain={plain}")


@pytest.mark.parametrize("name", ["tiny_random_R45", "sched_small_R37", "placement_small_R33"])
def test_sigma_zero_exact_indicator(name):
    """sigma = 0: atoms are decided exactly on both sides; COPs match, grad_b = 0."""
    make, R = CASES[name]
    inst = make()
    P, comp, a, b, w = setup(inst, R)
    # put reals exactly on atom boundaries: the planted point in half the restarts
    b = b.copy()
    b[:, ::2] = inst.planted_y[:, None].astype(np.float32)
    obj_ref, cop_ref, ga_ref, gb_ref = OBJ.evaluate(inst, a.astype(np.float64), b.astype(np.float64),
                                                    w.astype(np.float64), 0.0)
    obj, cop, ga, gb = gpu_adjoint(comp, R, 0.0, a, b, w)
    oc = OBJ.objective_constraints(inst)
    assert np.abs(cop[oc] - cop_ref[oc]).max() <= COP_TOL
    assert (gb == 0).all() and (gb_ref == 0).all()
    assert_grad_close(ga, ga_ref, "sigma=0 grad_a")


def test_forward_only_matches_adjoint_objective():
    import torch
    inst = W.jobshop(1002, 10, 5)
    R = 96
    P, comp, a, b, w = setup(inst, R)
    sigma = sigmas_for(inst)[1]
    obj_a, cop_a, _, _ = gpu_adjoint(comp, R, sigma, a, b, w)
    da, db, dw = to_dev(a, b, w)
    obj = torch.zeros(R, device="cuda")
    cop = torch.full((inst.n_cons, R), float("nan"), device="cuda")
    comp.forward(R, sigma, dw, da, db, cop=cop, obj=obj)
    np.testing.assert_allclose(obj.cpu().numpy(), obj_a, rtol=1e-6, atol=1e-4)
    np.testing.assert_array_equal(np.isnan(cop.cpu().numpy()), np.isnan(cop_a))
    np.testing.assert_allclose(cop.cpu().numpy(), cop_a, atol=1e-7)


def test_autograd_function_and_finite_differences():
    """The adjoint behind torch.autograd.Function: backward == oracle gradient, and
    central differences of the GPU objective agree with it (C is affine in each a_i,
    so the a-differences are exact up to FP32 rounding)."""
    import torch
    from paper_2603_22877_b300 import relaxed_objective
    inst = W.jobshop(1002, 10, 5)
    R = 64
    P, comp, a, b, w = setup(inst, R)
    sigma = sigmas_for(inst)[1]
    a64, b64, w64 = a.astype(np.float64), b.astype(np.float64), w.astype(np.float64)
    _, _, ga_ref, gb_ref = OBJ.evaluate(inst, a64, b64, w64, sigma)
    for plain in (False, True):
        da, db, dw = to_dev(a, b, w)
        da.requires_grad_(True)
        db.requires_grad_(True)
        v = torch.linspace(0.5, 1.5, R, device="cuda")
        obj = relaxed_objective(comp, sigma, dw, da, db, plain=plain)
        (obj * v).sum().backward()
        vv = v.cpu().numpy()[None, :].astype(np.float64)
        assert_grad_close(da.grad.cpu().numpy() / vv, ga_ref, f"autograd a plain={plain}")
        assert_grad_close(db.grad.cpu().numpy() / vv, gb_ref, f"autograd b plain={plain}")
    rng = np.random.default_rng(0)
    da, db, dw = to_dev(a, b, w)
    for i in rng.choice(inst.n_bool, 6, replace=False):
        h = 0.25
        ap, am = da.clone(), da.clone()
        ap[i] += h
        am[i] -= h
        fd = ((relaxed_objective(comp, sigma, dw, ap, db).double() -
               relaxed_objective(comp, sigma, dw, am, db).double()) / (2 * h)).cpu().numpy()
        scale = np.abs(w).sum(0).max() * 2e-7 / h + 1e-4 * np.abs(ga_ref[i]).max()
        assert np.abs(fd - ga_ref[i]).max() <= 10 * scale, (i, np.abs(fd - ga_ref[i]).max(), scale)
    for j in rng.choice(inst.n_real, 4, replace=False):
        h = np.float32(0.02 * sigma)
        bp32, bm32 = b.copy(), b.copy()
        bp32[j] = b[j] + h
        bm32[j] = b[j] - h
        denom = bp32[j].astype(np.float64) - bm32[j].astype(np.float64)  # the perturbation FP32 really made
        dbp, dbm = to_dev(bp32, bm32)
        fd = (relaxed_objective(comp, sigma, dw, da, dbp).double() -
              relaxed_objective(comp, sigma, dw, da, dbm).double()).cpu().numpy() / denom
        fd_ref = (OBJ.evaluate(inst, a64, bp32.astype(np.float64), w64, sigma, with_grad=False)[0] -
                  OBJ.evaluate(inst, a64, bm32.astype(np.float64), w64, sigma, with_grad=False)[0]) / denom
        noise = np.abs(w).sum(0).max() * 4e-7 / float(h)
        assert np.abs(fd - fd_ref).max() <= 10 * noise + 1e-3 * np.abs(fd_ref).max(), j
        # the oracle's own central difference is close to its adjoint gradient (O(h^2))
        assert np.abs(fd_ref - gb_ref[j]).max() <= 1e-2 * np.abs(gb_ref[j]).max() + 1e-6


@pytest.mark.parametrize("n,R,forms", [(100, 40, ("fused", "plain")), (300, 24, ("fused", "plain")),
                                       (1000, 100, ("fused",))])
def test_random_hybrid_against_oracle(n, R, forms):
    """The random hybrid benchmark (cardinality, NAE and parity constraints of up
    to 50 literals over Booleans and atoms; diagrams of up to 650 nodes) at the
    gradient-time grid's extremes and between: sigma = 0 (exact), 1/sigma = 0.5,
    1/sigma = 0 (every atom a fair coin).  At n = 300 and 1,000 the fused form is
    the chunked kernel that the gradient-time experiment times there (650-node
    diagrams through its generic pass, up to 128 staged reals); n = 1,000 at
    R = 100 is that experiment's own group size."""
    import math
    inst = W.random_hybrid(1006, n)
    P, comp, a, b, w = setup(inst, R)
    if "fused" in forms:
        assert comp.info["fused_ok"] or comp.info["n_chunks"] > 0
    if n >= 300:
        assert comp.info["n_chunks"] > 0 and comp.info["max_nodes"] > 48   # the chunked kernel, generic pass
    D = OBJ.Diagrams(inst)
    oc = OBJ.objective_constraints(inst)
    for sigma in (0.0, 2.0, math.inf):
        ref = OBJ.evaluate(inst, a.astype(np.float64), b.astype(np.float64), w.astype(np.float64), sigma,
                           diagrams=D)
        for form in forms:
            obj, cop, ga, gb = gpu_adjoint(comp, R, np.float32(sigma), a, b, w, plain=form == "plain")
            assert np.abs(cop[oc] - ref[1][oc]).max() <= COP_TOL, (form, sigma)
            np.testing.assert_allclose(obj, ref[0], rtol=1e-5, atol=1e-3)
            assert_grad_close(ga, ref[2], f"grad_a {form} sigma={sigma}")
            assert_grad_close(gb, ref[3], f"grad_b {form} sigma={sigma}")
