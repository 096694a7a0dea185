"""The persistent stage kernel: Alg. 1's loop body fused in one cooperative launch
(forward + adjoint over C_sigma, a grid barrier, the PGD step and projection, a grid
barrier whose last CTA applies the epsilon test of Eq. critical), run once for the
whole stage ("stage") or once per iteration ("iteration").  Checked against the
oracle's run_stage, against the same stage run as separate launches, and for its
bounded barrier wait."""
import numpy as np
import pytest

from oracle import pgd
from workloads import instances as W

from _gpu_common import setup, sigmas_for

pytestmark = pytest.mark.gpu


def _pick(comp, R, variant):
    """Pins the forward + adjoint configuration the stage kernel is built around:
    'chunk' (the generated-routine chunked kernel) or 'warp' (warp per constraint)."""
    names = ("wide", "jit") if variant == "chunk" else ("warp",)
    for c in comp.launch_configs(R):
        if c.as_dict()["variant"] in names:
            comp.select_config(R, c)
            return c
    pytest.skip(f"no {variant} configuration for this instance")


def _solver(P, comp, R, **kw):
    from paper_2603_22877_b300 import Solver
    return Solver(P, comp, R, **kw)


@pytest.mark.parametrize("variant", ["chunk", "warp"])
@pytest.mark.parametrize("use_graph,stage_form", [(True, "stage"), (False, "stage"), (True, "iteration")])
def test_persistent_stage_matches_oracle(variant, use_graph, stage_form):
    """Five PGD iterations and round/check/ERWA in one persistent kernel (under a
    CUDA graph or launched directly) against the oracle's run_stage: the same
    tolerances as the separate-launch stage."""
    inst = W.jobshop(1002, 10, 5)
    R = 40
    P, comp, a, b, _ = setup(inst, R)
    _pick(comp, R, variant)
    assert comp.stage_form(R)
    eta = 0.02
    cfg = pgd.Config(eta=eta, t_max=5, sweeps=20, polish=32)
    S = _solver(P, comp, R, eta=eta, b_scale=inst.scale, t_max=5, sweeps=20, use_graph=use_graph,
                stage_form=stage_form)
    S.reset(a, b)
    sigma = sigmas_for(inst)[0]
    S.stage(sigma, 1)
    S.check_stage_status()
    w0 = np.ones((inst.n_cons, R))
    h0 = np.zeros((inst.n_cons, R))
    a_ref, b_ref, w_ref, h_ref, nu_ref, its_ref, obj_ref = pgd.run_stage(inst, a, b, w0, h0, sigma, 1, cfg)
    np.testing.assert_allclose(S.a.cpu().numpy(), a_ref, atol=1e-4)
    np.testing.assert_allclose(S.b.cpu().numpy(), b_ref, atol=1e-4 * inst.meta["horizon"])
    np.testing.assert_array_equal(S.iters.cpu().numpy(), its_ref)
    np.testing.assert_allclose(S.obj.cpu().numpy(), obj_ref, rtol=1e-4, atol=1e-3)
    _, viol = pgd.round_check(inst, S.a.cpu().numpy().astype(np.float64), S.b.cpu().numpy().astype(np.float64))
    np.testing.assert_array_equal(S.n_unsat.cpu().numpy(), viol.sum(0))
    # the gradient buffers are left at zero, as the separate launches leave them
    assert not S.grad_a.any() and not S.grad_b.any()
    assert int(S.ctl[1].item()) == 0


@pytest.mark.parametrize("variant", ["chunk", "warp"])
@pytest.mark.parametrize("stage_form", ["stage", "iteration"])
def test_persistent_stage_matches_separate_launches(variant, stage_form):
    """A batch of uneven job-shop instances (blocks of coupled reals of many sizes),
    R = 32, two stages of 20 iterations: the persistent kernel and the separate
    launches of the same configuration agree up to the order of floating-point atomic
    additions, whose rounding differences the 40 projected steps carry along (about
    1e-5 relative on the reals; exactness against the oracle is the first test's)."""
    inst = W.concat(W.uneven_batch(1004, n_inst=8, jobs=(5, 30), machines=(3, 10)), "uneven8")
    R = 32
    P, comp, a, b, _ = setup(inst, R)
    _pick(comp, R, variant)
    assert comp.stage_form(R)
    out = {}
    for form in (stage_form, "launches"):
        S = _solver(P, comp, R, eta=0.02, b_scale=inst.scale, t_max=20, sweeps=20, stage_form=form)
        S.reset(a, b)
        for t, sigma in enumerate([inst.scale / (0.1 * k) for k in (1, 2)], start=1):
            S.stage(sigma, t)
        S.check_stage_status()
        out[form] = {k: getattr(S, k).cpu().numpy() for k in ("a", "b", "w", "obj", "iters", "n_unsat")}
    p, s = out[stage_form], out["launches"]
    np.testing.assert_allclose(p["a"], s["a"], atol=1e-3)
    np.testing.assert_allclose(p["b"], s["b"], rtol=1e-4, atol=1e-4 * inst.scale)
    np.testing.assert_allclose(p["obj"], s["obj"], rtol=1e-4, atol=1e-3)
    assert (p["iters"] == s["iters"]).mean() >= 0.95
    assert (p["n_unsat"] == s["n_unsat"]).mean() >= 0.95


def test_persistent_epsilon_rule_and_host_buffers():
    """With eps large every restart stops after its first iteration, inside the
    kernel (ctl[0] = 0 ends its loop); the host-buffer stage returns the same."""
    inst = W.tiny_random(1001)
    R = 50
    P, comp, a, b, _ = setup(inst, R)
    assert comp.stage_form(R)
    S = _solver(P, comp, R, eta=0.01, b_scale=inst.scale, t_max=7, eps=1e6, stage_form="stage")
    S.reset(a, b)
    S.stage(sigmas_for(inst)[0], 1)
    assert (S.iters.cpu().numpy() == 1).all()
    assert int(S.ctl[0].item()) == 0 and int(S.ctl[1].item()) == 0
    nu = np.zeros(R, np.int32)
    ob = np.zeros(R, np.float32)
    S2 = _solver(P, comp, R, eta=0.01, b_scale=inst.scale, t_max=7, eps=1e6, stage_form="stage")
    S2.reset(a, b)
    S2.stage_host(sigmas_for(inst)[0], 1, np.ascontiguousarray(a), np.ascontiguousarray(b), nu, ob)
    np.testing.assert_array_equal(nu, S.n_unsat.cpu().numpy())
    np.testing.assert_allclose(ob, S.obj.cpu().numpy(), rtol=1e-5, atol=1e-4)


def test_barrier_wait_is_bounded(monkeypatch):
    """A barrier limit of 1 us is far below the forward + adjoint phase of the
    slowest CTA, so CTAs give up waiting: the kernel sets bit 4 of ctl[1] and ends,
    the host-buffer stage returns ETIMEOUT, and the context stays usable -- the next
    stage with the default limit matches the separate-launch form."""
    from paper_2603_22877_b300 import _lib as L
    inst = W.jobshop(1002, 10, 5)
    R = 64
    P, comp, a, b, _ = setup(inst, R)
    assert comp.stage_form(R)
    sigma = sigmas_for(inst)[0]
    S = _solver(P, comp, R, eta=0.02, b_scale=inst.scale, t_max=4, use_graph=False,
                stage_form="stage")
    S.reset(a, b)
    monkeypatch.setenv("FSMT_STAGE_BARRIER_NS", "1000")
    nu = np.zeros(R, np.int32)
    ob = np.zeros(R, np.float32)
    with pytest.raises(L.FsmtError) as e:
        S.stage_host(sigma, 1, np.ascontiguousarray(a), np.ascontiguousarray(b), nu, ob)
    assert e.value.status == L.ETIMEOUT
    assert int(S.ctl[1].item()) & 4
    with pytest.raises(L.FsmtError):
        S.check_stage_status()
    monkeypatch.delenv("FSMT_STAGE_BARRIER_NS")
    S.reset(a, b)
    S.stage(sigma, 1)
    S.check_stage_status()
    ref = _solver(P, comp, R, eta=0.02, b_scale=inst.scale, t_max=4, use_graph=False,
                  stage_form="launches")
    ref.reset(a, b)
    ref.stage(sigma, 1)
    np.testing.assert_allclose(S.a.cpu().numpy(), ref.a.cpu().numpy(), atol=1e-4)
    np.testing.assert_array_equal(S.iters.cpu().numpy(), ref.iters.cpu().numpy())


@pytest.mark.parametrize("variant", ["chunk", "warp"])
def test_tune_times_every_stage_form_and_keeps_the_state(variant):
    """Solver.tune with stage_form "auto" (the kernel configuration pinned) times the
    three stage forms from the current state, pins the fastest, and leaves the state
    as it found it."""
    inst = W.jobshop(1002, 10, 5)
    R = 64
    P, comp, a, b, _ = setup(inst, R)
    _pick(comp, R, variant)
    S = _solver(P, comp, R, eta=0.02, b_scale=inst.scale, t_max=4)
    S.reset(a, b)
    S.tune(sigmas_for(inst)[0], kernels=False)
    assert set(S.stage_form_ms) == {"launches", "stage", "iteration"}
    assert S.chosen_stage_form == min(S.stage_form_ms, key=S.stage_form_ms.get)
    np.testing.assert_array_equal(S.a.cpu().numpy(), a)
    np.testing.assert_array_equal(S.b.cpu().numpy(), b)
    assert (S.w.cpu().numpy() == 1).all() and not S.h.cpu().numpy().any()
