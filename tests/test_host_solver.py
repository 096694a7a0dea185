"""Host logic of the solver that needs no device: checkpoint round trip and validation
(tensors on the CPU stand in for the device state)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _cpu_solver(R=4, n=3, m=2, nc=5):
    import torch
    from paper_2603_22877_b300 import Solver
    S = object.__new__(Solver)
    S.R = R
    for k, shape, dt in (("a", (n, R), torch.float32), ("b", (m, R), torch.float32), ("w", (nc, R), torch.float32),
                         ("h", (nc, R), torch.float32), ("n_unsat", (R,), torch.int32), ("iters", (R,), torch.int32),
                         ("obj", (R,), torch.float32), ("grad_a", (n, R), torch.float32),
                         ("grad_b", (m, R), torch.float32)):
        setattr(S, k, torch.zeros(shape, dtype=dt))
    return S


def test_checkpoint_round_trip_and_shape_check():
    """state_dict holds the search state (points, weights, histories, last outcome);
    load_state_dict restores it into a solver of the same instance and R, zeroes the
    gradient work buffers, and refuses a checkpoint of another shape."""
    import torch
    S = _cpu_solver()
    S.a.uniform_(-1, 1)
    S.w.fill_(3.0)
    S.n_unsat[2] = 7
    ck = S.state_dict()
    assert set(ck) == {"a", "b", "w", "h", "n_unsat", "iters", "obj"}
    T = _cpu_solver()
    T.grad_a.fill_(5.0)
    T.load_state_dict(ck)
    assert torch.equal(T.a, S.a) and torch.equal(T.w, S.w) and int(T.n_unsat[2]) == 7
    assert float(T.grad_a.abs().sum()) == 0.0
    U = _cpu_solver(R=8)
    with pytest.raises(ValueError, match="shape"):
        U.load_state_dict(ck)


def test_stage_status_reports_a_barrier_timeout():
    """check_stage_status raises ETIMEOUT exactly when a persistent stage form ran and
    the stage's control block carries bit 4 of ctl[1] (a grid barrier gave up);
    the other error bits and the separate-launch form leave it silent."""
    import torch
    from paper_2603_22877_b300 import _lib as L
    from paper_2603_22877_b300.engine import STAGE_FORMS
    S = _cpu_solver()
    S.form = "fused"
    S.ctl = torch.zeros(4, dtype=torch.int32)
    for name, code in STAGE_FORMS.items():
        S._form_code = code
        S.ctl[1] = 1  # a non-finite ||g||^2 only
        S.check_stage_status()
        S.ctl[1] = 4 | 1
        if code == 0:
            S.check_stage_status()
        else:
            with pytest.raises(L.FsmtError) as e:
                S.check_stage_status()
            assert e.value.status == L.ETIMEOUT
