"""Parity at the full workload sizes, in the launch configuration the benchmark
times: every output of the job-shop instance, and sampled outputs (computed one
by one by the oracle) of the placement, uneven-batch and large scheduling
instances, plus properties that hold at any size."""
import numpy as np
import pytest

from oracle import objective as OBJ
from workloads import instances as W

from _gpu_common import COP_TOL, assert_grad_close, assert_sampled_entries_close, setup, sigmas_for, to_dev

pytestmark = pytest.mark.gpu


def incidence(inst):
    """(constraint of each literal, id of each literal, atom of each atom nonzero)."""
    lit_con = np.repeat(np.arange(inst.n_cons), np.diff(inst.con_ptr))
    ids = inst.con_lits >> 1
    atom_of_nnz = np.repeat(np.arange(inst.n_atoms), np.diff(inst.atom_ptr))
    return lit_con, ids, atom_of_nnz


def cons_with_bool(inc, v):
    lit_con, ids, _ = inc
    return np.unique(lit_con[ids == v])


def cons_with_real(inst, inc, j):
    lit_con, ids, atom_of_nnz = inc
    atoms = atom_of_nnz[inst.atom_var == j] + inst.n_bool
    return np.unique(lit_con[np.isin(ids, atoms)])


def run_gpu(comp, inst, R, sigma, a, b, w):
    import torch
    da, db, dw = to_dev(a, b, w)
    ga, gb = torch.zeros_like(da), torch.zeros_like(db)
    obj = torch.zeros(R, device="cuda")
    cop = torch.full((inst.n_cons, R), float("nan"), device="cuda")
    comp.adjoint(R, sigma, dw, da, db, ga, gb, obj=obj, cop=cop)
    torch.cuda.synchronize()
    return obj, cop, ga, gb, dw


def sampled_parity(inst, R, n_cons_sample, n_bool_sample, n_real_sample, seed=0):
    import torch
    P, comp, a, b, w = setup(inst, R)
    sigma = sigmas_for(inst)[1]
    obj, cop, ga, gb, dw = run_gpu(comp, inst, R, sigma, a, b, w)
    oc = np.array(OBJ.objective_constraints(inst))
    # properties at any size: C = sum_c w_c (1 - 2 COP_c) over the GPU's own COPs,
    # COP in [0, 1] up to FP32 rounding, finite gradients
    ocd = torch.from_numpy(oc).cuda()
    total = (dw[ocd].double() * (1 - 2 * cop[ocd].double())).sum(0)
    np.testing.assert_allclose(obj.cpu().numpy(), total.cpu().numpy(), rtol=1e-5,
                               atol=2e-6 * float(dw.double().abs().sum(0).max()))
    assert torch.isfinite(ga).all() and torch.isfinite(gb).all()
    assert float(cop[ocd].min()) >= -1e-6 and float(cop[ocd].max()) <= 1.0 + 1e-6
    rng = np.random.default_rng(seed)
    D = OBJ.Diagrams(inst)
    a64, b64, w64 = a.astype(np.float64), b.astype(np.float64), w.astype(np.float64)
    # sampled COPs, every restart
    cs = rng.choice(oc, min(n_cons_sample, len(oc)), replace=False)
    cop_s = cop[torch.from_numpy(cs).cuda()].cpu().numpy()
    for k, c in enumerate(cs):
        ref = OBJ.constraint_cop(inst, D, int(c), a64, b64, sigma)
        assert np.abs(cop_s[k] - ref).max() <= COP_TOL, (c, np.abs(cop_s[k] - ref).max())
    # sampled gradient entries: the oracle sums every constraint that touches the variable
    inc = incidence(inst)
    ocset = set(oc.tolist())
    ga_c, gb_c = ga.cpu().numpy(), gb.cpu().numpy()
    if inst.n_bool:
        for v in rng.choice(inst.n_bool, min(n_bool_sample, inst.n_bool), replace=False):
            ref = np.zeros(R)
            for c in cons_with_bool(inc, v):
                if int(c) in ocset:
                    ref += OBJ.constraint_contrib(inst, D, int(c), a64, b64, w64[c], sigma)[2].get(int(v), 0.0)
            assert_sampled_entries_close(ga_c[v], ref, ga_c, f"bool {v}")
    for j in rng.choice(inst.n_real, min(n_real_sample, inst.n_real), replace=False):
        ref = np.zeros(R)
        for c in cons_with_real(inst, inc, j):
            if int(c) in ocset:
                ref += OBJ.constraint_contrib(inst, D, int(c), a64, b64, w64[c], sigma)[3].get(int(j), 0.0)
        assert_sampled_entries_close(gb_c[j], ref, gb_c, f"real {j}")


def test_jobshop_full_every_output():
    inst = W.jobshop(1002)
    R = 256
    P, comp, a, b, w = setup(inst, R)
    sigma = sigmas_for(inst)[1]
    obj, cop, ga, gb, _ = run_gpu(comp, inst, R, sigma, a, b, w)
    obj_ref, cop_ref, ga_ref, gb_ref = OBJ.evaluate(inst, a.astype(np.float64), b.astype(np.float64),
                                                    w.astype(np.float64), sigma)
    oc = OBJ.objective_constraints(inst)
    assert np.abs(cop.cpu().numpy()[oc] - cop_ref[oc]).max() <= COP_TOL
    np.testing.assert_allclose(obj.cpu().numpy(), obj_ref, rtol=1e-5, atol=1e-5 * float(np.abs(w).sum(0).max()))
    assert_grad_close(ga.cpu().numpy(), ga_ref, "jobshop grad_a")
    assert_grad_close(gb.cpu().numpy(), gb_ref, "jobshop grad_b")


def test_placement_full_sampled():
    sampled_parity(W.placement2d(1003), 1024, 300, 8, 4)


def test_uneven_batch_full_sampled():
    sampled_parity(W.concat(W.uneven_batch(1004), "uneven_batch"), 32, 400, 8, 6)


def test_large_scheduling_full_sampled():
    sampled_parity(W.large_scheduling(1005), 512, 200, 3, 2)
