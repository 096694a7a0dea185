"""Shared set-up for the GPU parity tests: the same seeded inputs go to the
oracle (FP64, CPU) and to the CUDA path (FP32, through the C ABI)."""
import numpy as np

from oracle import objective as OBJ
from workloads import instances as W

COP_TOL = 1e-5        # |dCOP| per (constraint, restart)
GRAD_REL_TOL = 1e-4   # ||g_gpu - g_64|| / ||g_64|| per restart
GRAD_ELEM_TOL = 1e-4  # |dg| <= 1e-4 * max(||g_64||_inf, 1e-6), per restart


def sigmas_for(inst):
    """Three points of the annealing schedule sigma_t = S / (0.1 t): t = 1, 10, 20."""
    return [float(np.float32(inst.scale / (0.1 * t))) for t in (1, 10, 20)]


def make_inputs(inst, R, seed=7):
    a, b = W.initial_point(inst, R, seed)
    rng = np.random.default_rng(seed + 1)
    w = rng.uniform(0.5, 2.0, (inst.n_cons, R)).astype(np.float32)
    return a, b, w


def to_dev(*arrs):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in arrs]


def setup(inst, R, policy=OBJ.PROJECT, seed=7):
    from paper_2603_22877_b300.engine import Problem
    P = Problem.from_instance(inst)
    comp = P.compile(policy).upload()
    a, b, w = make_inputs(inst, R, seed)
    return P, comp, a, b, w


def gpu_adjoint(comp, R, sigma, a, b, w, plain=False):
    import torch
    da, db, dw = to_dev(a, b, w)
    ga = torch.zeros_like(da)
    gb = torch.zeros_like(db)
    obj = torch.zeros(R, device="cuda")
    cop = torch.full((comp.n_cons, R), float("nan"), device="cuda")
    if plain:
        work = torch.empty(comp.plain_work(R), device="cuda")
        comp.forward_plain(R, sigma, dw, da, db, work, cop=cop, obj=obj)
        comp.adjoint_plain(R, sigma, dw, da, db, work, ga, gb)
    else:
        comp.adjoint(R, sigma, dw, da, db, ga, gb, obj=obj, cop=cop)
    torch.cuda.synchronize()
    return obj.cpu().numpy(), cop.cpu().numpy(), ga.cpu().numpy(), gb.cpu().numpy()


def assert_grad_close(g_gpu, g_ref, what=""):
    """Per-restart relative L2 error and elementwise error, both against FP64."""
    g_gpu = np.asarray(g_gpu, np.float64)
    if g_ref.size == 0:
        assert g_gpu.size == 0
        return
    num = np.linalg.norm(g_gpu - g_ref, axis=0)
    den = np.linalg.norm(g_ref, axis=0)
    rel = num / np.maximum(den, 1e-30)
    ok = (rel <= GRAD_REL_TOL) | ((den == 0) & (num <= 1e-6))
    assert ok.all(), f"{what}: worst relative gradient error {rel.max():.3e}"
    scale = np.maximum(np.abs(g_ref).max(axis=0), 1e-6)
    elem = (np.abs(g_gpu - g_ref) / scale[None, :]).max()
    assert elem <= GRAD_ELEM_TOL, f"{what}: worst elementwise gradient error {elem:.3e}"


def assert_sampled_entries_close(g_gpu_row, g_ref_row, g_gpu_all, what=""):
    """One gradient entry per restart, computed by the oracle one by one: the
    elementwise bound |dg| <= 1e-4 max(||g||_inf, 1e-6), with ||g||_inf taken from
    the full GPU vector of each restart (the oracle has only the sampled entry)."""
    scale = np.maximum(np.abs(g_gpu_all).max(axis=0), 1e-6)
    err = np.abs(np.asarray(g_gpu_row, np.float64) - g_ref_row)
    assert (err <= GRAD_ELEM_TOL * scale).all(), f"{what}: worst {(err / scale).max():.3e}"
