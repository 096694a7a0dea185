"""The allocation-free entry point, for callers that may not call cudaMalloc
(programs that reserve device memory once at start-up, or that share a device
with an allocator owning all of its memory).  Through the C ABI, two calls in a
row must give what the fused entry point gives on the same inputs, and a size
beyond the fixed work array must be refused with a clear error.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test; it builds everything it needs, so
it also passes alone in a fresh process."""
import ctypes as C

import numpy as np
import pytest

from oracle import objective as OBJ
from workloads import instances as W

from _gpu_common import COP_TOL, assert_grad_close, make_inputs, to_dev

pytestmark = pytest.mark.gpu


def _noalloc(comp, R, sigma, w, a, b):
    import torch
    from paper_2603_22877_b300 import _lib as L
    ga = torch.full((comp.n_bool, R), float("nan"), device="cuda")
    gb = torch.full((comp.n_real, R), float("nan"), device="cuda")
    cop = torch.full((comp.n_cons, R), float("nan"), device="cuda")
    obj = torch.full((R,), float("nan"), device="cuda")
    ptr = lambda t: C.c_void_p(t.data_ptr())
    L.call("fsmt_plain_noalloc", comp.h, int(R), float(sigma), ptr(w), ptr(a), ptr(b), ptr(ga), ptr(gb), ptr(cop),
           ptr(obj), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return obj.cpu().numpy(), cop.cpu().numpy(), ga.cpu().numpy(), gb.cpu().numpy()


def _fused(comp, R, sigma, w, a, b):
    import torch
    ga, gb = torch.zeros_like(a), torch.zeros_like(b)
    cop = torch.full((comp.n_cons, R), float("nan"), device="cuda")
    obj = torch.zeros(R, device="cuda")
    comp.adjoint(R, sigma, w, a, b, ga, gb, obj=obj, cop=cop)
    torch.cuda.synchronize()
    return obj.cpu().numpy(), cop.cpu().numpy(), ga.cpu().numpy(), gb.cpu().numpy()


def test_noalloc_matches_fused_on_two_calls():
    from paper_2603_22877_b300.engine import Problem
    inst = W.jobshop(1002, 12, 6)
    R = 96
    comp = Problem.from_instance(inst).compile().upload()
    oc = OBJ.objective_constraints(inst)
    for call, (seed, sigma) in enumerate([(7, inst.scale), (8, inst.scale / 2.0)]):
        a, b, w = to_dev(*make_inputs(inst, R, seed))
        ref = _fused(comp, R, sigma, w, a, b)
        got = _noalloc(comp, R, sigma, w, a, b)
        assert np.abs(got[1][oc] - ref[1][oc]).max() <= COP_TOL, call
        np.testing.assert_allclose(got[0], ref[0], rtol=1e-5, atol=1e-3)
        assert_grad_close(got[2], ref[2].astype(np.float64), f"grad_a call {call}")
        assert_grad_close(got[3], ref[3].astype(np.float64), f"grad_b call {call}")


def test_noalloc_refuses_sizes_beyond_its_array():
    import torch
    from paper_2603_22877_b300 import _lib as L
    from paper_2603_22877_b300.engine import Problem
    inst = W.jobshop(1002)
    R = 1024  # needs about 98 Mi work floats, more than the fixed 16 Mi
    comp = Problem.from_instance(inst).compile().upload()
    assert comp.plain_work(R) > (1 << 24)
    z = torch.zeros(1, device="cuda")
    p = C.c_void_p(z.data_ptr())
    st = L.load().fsmt_plain_noalloc(comp.h, R, C.c_float(1.0), p, p, p, p, p, None, None, None)
    assert st == L.EINVAL
    assert "fixed array" in L.last_error()


def test_noalloc_leaves_free_device_memory_unchanged():
    """What the entry point exists for: after a first call on the device (which looks up
    the fixed array's address), further calls take no device memory.  cudaMemGetInfo
    (torch.cuda.mem_get_info) reports the same free bytes before and after a call whose
    inputs and outputs were all allocated beforehand."""
    import torch
    from paper_2603_22877_b300 import _lib as L
    from paper_2603_22877_b300.engine import Problem
    inst = W.jobshop(1002, 12, 6)
    R = 64
    comp = Problem.from_instance(inst).compile().upload()
    a, b, w = to_dev(*make_inputs(inst, R, 9))
    ga = torch.zeros((comp.n_bool, R), device="cuda")
    gb = torch.zeros((comp.n_real, R), device="cuda")
    obj = torch.zeros((R,), device="cuda")
    ptr = lambda t: C.c_void_p(t.data_ptr())
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    args = (comp.h, int(R), float(inst.scale), ptr(w), ptr(a), ptr(b), ptr(ga), ptr(gb), None, ptr(obj), stream)
    L.call("fsmt_plain_noalloc", *args)           # the first call on this device
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        L.call("fsmt_plain_noalloc", *args)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert np.isfinite(obj.cpu().numpy()).all()
