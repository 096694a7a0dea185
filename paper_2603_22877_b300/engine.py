"""Python front end of the C ABI: problem building, device calls on torch tensors,
the autograd bridge, and the annealing driver of Alg. 2.

Only argument marshalling and host-side orchestration live here; every
numerical step of the hot path runs in libfsmt.so.  PyTorch provides device
memory and streams.
"""
import ctypes as C
import time

import numpy as np

from . import _lib as L


def _np_ptr(a):
    return C.c_void_p(a.ctypes.data) if a is not None and a.size else C.c_void_p(0)


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dptr(t, dtype=None, shape=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (or NULL for None)."""
    if t is None:
        return C.c_void_p(0)
    import torch
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return C.c_void_p(t.data_ptr())


class Problem:
    """An fsmt_problem (constraint set C of Alg. 1)."""

    def __init__(self, n_bool, n_real):
        self.n_bool, self.n_real = int(n_bool), int(n_real)
        h = C.c_void_p()
        L.call("fsmt_problem_create", self.n_bool, self.n_real, C.byref(h))
        self.h = h
        self.n_atoms = 0
        self.n_cons = 0

    def __del__(self):
        if getattr(self, "h", None) and L._lib is not None:
            L._lib.fsmt_free_problem(self.h)
            self.h = None

    def set_bounds(self, lo, hi):
        for j in range(self.n_real):
            L.call("fsmt_set_real_bounds", self.h, j, float(lo[j]), float(hi[j]))

    def add_atoms(self, ptr, var, coef, q0, rel):
        ptr = np.ascontiguousarray(ptr, np.int64)
        var = np.ascontiguousarray(var, np.int32)
        coef = np.ascontiguousarray(coef, np.int64)
        q0 = np.ascontiguousarray(q0, np.int64)
        rel = np.ascontiguousarray(rel, np.int8)
        n = len(q0)
        L.call("fsmt_add_atoms", self.h, n, _np_ptr(ptr), _np_ptr(var), _np_ptr(coef), _np_ptr(q0), _np_ptr(rel))
        self.n_atoms += n

    def add_constraints(self, kind, param, ptr, lits):
        kind = np.ascontiguousarray(kind, np.int8)
        param = np.ascontiguousarray(param, np.int32)
        ptr = np.ascontiguousarray(ptr, np.int64)
        lits = np.ascontiguousarray(lits, np.int32)
        n = len(kind)
        L.call("fsmt_add_constraints", self.h, n, _np_ptr(kind), _np_ptr(param), _np_ptr(ptr), _np_ptr(lits))
        self.n_cons += n

    @classmethod
    def from_instance(cls, inst):
        """Builds the problem from an object with the fields of a generated instance."""
        P = cls(inst.n_bool, inst.n_real)
        P.set_bounds(inst.lo, inst.hi)
        P.add_atoms(inst.atom_ptr, inst.atom_var, inst.atom_coef, inst.atom_q0, inst.atom_rel)
        P.add_constraints(inst.con_kind, inst.con_param, inst.con_ptr, inst.con_lits)
        return P

    def verify_exact(self, x, y):
        """Exact check of a rounded assignment (x in +-1, y reals).  Returns (sat, first_violated)."""
        x = np.ascontiguousarray(x, np.int8)
        y = np.ascontiguousarray(y, np.float64)
        sat, first = C.c_int32(), C.c_int32()
        L.call("fsmt_verify_exact", self.h, _np_ptr(x), _np_ptr(y), C.byref(sat), C.byref(first))
        return bool(sat.value), int(first.value)

    def repair_equalities(self, y):
        """Exact repair of reals y so that every projected equality holds exactly
        (fsmt_repair_equalities).  Returns (ok, repaired y as float64)."""
        y = np.array(y, np.float64)
        ok = C.c_int32()
        L.call("fsmt_repair_equalities", self.h, _np_ptr(y), C.byref(ok))
        return bool(ok.value), y

    def compile(self, policy=L.UNIT_PROJECT):
        return Compiled(self, policy)


class Compiled:
    """An fsmt_compiled: flattened xBDDs, atoms and projection data."""

    def __init__(self, problem, policy=L.UNIT_PROJECT):
        h = C.c_void_p()
        L.call("fsmt_compile", problem.h, int(policy), C.byref(h))
        self.h = h
        info = L.Info()
        L.call("fsmt_compiled_info", self.h, C.byref(info))
        self.info = {k: getattr(info, k) for k, _ in L.Info._fields_}
        self.n_bool, self.n_real, self.n_cons = info.n_bool, info.n_real, info.n_cons
        self.uploaded = False
        self._work = None

    def __del__(self):
        if getattr(self, "h", None) and L._lib is not None:
            L._lib.fsmt_free_compiled(self.h)
            self.h = None

    def diagrams(self):
        """Host copy of the flattened diagrams: dict of numpy arrays."""
        nc, nn = self.info["n_cons"], self.info["n_nodes"]
        out = dict(con_ptr=np.zeros(nc + 1, np.int32), con_id=np.zeros(nc, np.int32),
                   con_root=np.zeros(nc, np.uint8), label=np.zeros(nn, np.int32),
                   hi=np.zeros(nn, np.uint16), lo=np.zeros(nn, np.uint16))
        L.call("fsmt_get_diagrams", self.h, *[_np_ptr(out[k]) for k in
                                              ("con_ptr", "con_id", "con_root", "label", "hi", "lo")])
        return out

    def bounds(self):
        lo = np.zeros(self.n_real, np.float32)
        hi = np.zeros(self.n_real, np.float32)
        L.call("fsmt_get_bounds", self.h, _np_ptr(lo), _np_ptr(hi))
        return lo, hi

    def upload(self, stream=None):
        L.call("fsmt_upload", self.h, _stream(stream))
        self.uploaded = True
        return self

    # ------------------------------------------------------ device calls --
    def _shapes(self, R):
        return (self.n_bool, R), (self.n_real, R), (self.n_cons, R)

    def forward(self, R, sigma, w, a, b, cop=None, obj=None, stream=None):
        import torch
        sa, sb, sw = self._shapes(R)
        L.call("fsmt_forward", self.h, int(R), float(sigma), _dptr(w, torch.float32, sw, "w"),
               _dptr(a, torch.float32, sa, "a"), _dptr(b, torch.float32, sb, "b"),
               _dptr(cop, torch.float32, sw, "cop"), _dptr(obj, torch.float32, (R,), "obj"), _stream(stream))

    def adjoint(self, R, sigma, w, a, b, grad_a, grad_b, obj=None, cop=None, stream=None):
        import torch
        sa, sb, sw = self._shapes(R)
        L.call("fsmt_adjoint", self.h, int(R), float(sigma), _dptr(w, torch.float32, sw, "w"),
               _dptr(a, torch.float32, sa, "a"), _dptr(b, torch.float32, sb, "b"),
               _dptr(grad_a, torch.float32, sa, "grad_a"), _dptr(grad_b, torch.float32, sb, "grad_b"),
               _dptr(obj, torch.float32, (R,), "obj"), _dptr(cop, torch.float32, sw, "cop"), _stream(stream))

    def launch_configs(self, R):
        """The kernel configurations that can run this instance at R restarts, default first."""
        n = C.c_int32()
        L.call("fsmt_launch_configs", self.h, int(R), None, 0, C.byref(n))
        arr = (L.LaunchConfig * max(1, n.value))()
        L.call("fsmt_launch_configs", self.h, int(R), arr, n.value, C.byref(n))
        return [arr[i] for i in range(n.value)]

    def select_config(self, R, cfg=None):
        """Pins one of launch_configs(R) for later passes and stages (None: the default)."""
        L.call("fsmt_select_config", self.h, int(R), C.byref(cfg) if cfg is not None else None)

    def stage_form(self, R):
        """True when the persistent stage forms (one kernel per stage, one per
        iteration) run at R restarts under the configuration now chosen
        (fsmt_stage_form); else a stage falls back to separate launches."""
        v = C.c_int32()
        L.call("fsmt_stage_form", self.h, int(R), C.byref(v))
        return bool(v.value)

    def stage_trace(self, trace):
        """Records per-phase device timestamps of later persistent stages into `trace`
        (a device uint64 / int64 tensor of 1 + 2 t_max entries; fsmt_stage_trace), or
        stops recording (None).  The buffer must outlive the stages that use it."""
        import torch
        ptr = None
        if trace is not None:
            if not (trace.is_cuda and trace.dtype in (torch.int64, torch.uint64) and trace.is_contiguous()):
                raise ValueError("trace must be a contiguous device int64 tensor")
            ptr = C.c_void_p(trace.data_ptr())
        self._trace = trace
        L.call("fsmt_stage_trace", self.h, ptr)

    def autotune(self, R, sigma, w, a, b, grad_a, grad_b, obj=None, stream=None):
        """Times every configuration on these inputs and pins the fastest; returns it."""
        import torch
        sa, sb, sw = self._shapes(R)
        best = L.LaunchConfig()
        L.call("fsmt_autotune", self.h, int(R), float(sigma), _dptr(w, torch.float32, sw, "w"),
               _dptr(a, torch.float32, sa, "a"), _dptr(b, torch.float32, sb, "b"),
               _dptr(grad_a, torch.float32, sa, "grad_a"), _dptr(grad_b, torch.float32, sb, "grad_b"),
               _dptr(obj, torch.float32, (R,), "obj"), C.byref(best), _stream(stream))
        return best

    def plain_work(self, R):
        n = C.c_int64()
        L.call("fsmt_plain_work_floats", self.h, int(R), C.byref(n))
        return int(n.value)

    def forward_plain(self, R, sigma, w, a, b, work, cop=None, obj=None, stream=None):
        import torch
        sa, sb, sw = self._shapes(R)
        L.call("fsmt_forward_plain", self.h, int(R), float(sigma), _dptr(w, torch.float32, sw, "w"),
               _dptr(a, torch.float32, sa, "a"), _dptr(b, torch.float32, sb, "b"),
               _dptr(work, torch.float32, None, "work"), _dptr(cop, torch.float32, sw, "cop"),
               _dptr(obj, torch.float32, (R,), "obj"), _stream(stream))

    def adjoint_plain(self, R, sigma, w, a, b, work, grad_a, grad_b, stream=None):
        import torch
        sa, sb, sw = self._shapes(R)
        L.call("fsmt_adjoint_plain", self.h, int(R), float(sigma), _dptr(w, torch.float32, sw, "w"),
               _dptr(a, torch.float32, sa, "a"), _dptr(b, torch.float32, sb, "b"),
               _dptr(work, torch.float32, None, "work"), _dptr(grad_a, torch.float32, sa, "grad_a"),
               _dptr(grad_b, torch.float32, sb, "grad_b"), _stream(stream))

    def weight_sum(self, R, w, wsum, stream=None):
        import torch
        L.call("fsmt_weight_sum", self.h, int(R), _dptr(w, torch.float32, (self.n_cons, R), "w"),
               _dptr(wsum, torch.float32, (R,), "wsum"), _stream(stream))

    def pgd_step(self, R, eta, b_scale, sweeps, a, b, grad_a, grad_b, gnorm2, active=None, wsum=None, polish=32,
                 stream=None):
        import torch
        sa, sb, _ = self._shapes(R)
        L.call("fsmt_pgd_step", self.h, int(R), float(eta), float(b_scale), int(sweeps), int(polish),
               _dptr(a, torch.float32, sa, "a"), _dptr(b, torch.float32, sb, "b"),
               _dptr(grad_a, torch.float32, sa, "grad_a"), _dptr(grad_b, torch.float32, sb, "grad_b"),
               _dptr(wsum, torch.float32, (R,), "wsum"), _dptr(gnorm2, torch.float32, (R,), "gnorm2"),
               _dptr(active, torch.uint8, (R,), "active"), _stream(stream))

    def round_check(self, R, a, b, n_unsat, x=None, violated=None, w=None, h=None, rho=0.5, gamma=2.0,
                    update_w=True, wsum=None, stream=None):
        import torch
        sa, sb, sw = self._shapes(R)
        L.call("fsmt_round_check", self.h, int(R), _dptr(a, torch.float32, sa, "a"),
               _dptr(b, torch.float32, sb, "b"), _dptr(x, torch.int8, sa, "x"),
               _dptr(violated, torch.uint8, sw, "violated"), _dptr(n_unsat, torch.int32, (R,), "n_unsat"),
               _dptr(w, torch.float32, sw, "w"), _dptr(h, torch.float32, sw, "h"), float(rho), float(gamma),
               int(bool(update_w)), _dptr(wsum, torch.float32, (R,), "wsum"), _stream(stream))


    def round(self, R, a, x, stream=None):
        """Alg. 1's rounding of every Boolean and restart into x (int8 [n_bool][R])."""
        import torch
        sa, _, _ = self._shapes(R)
        L.call("fsmt_round", self.h, int(R), _dptr(a, torch.float32, sa, "a"), _dptr(x, torch.int8, sa, "x"),
               _stream(stream))

    def converge(self, R, eps, gnorm2, active, iters, ctl, stream=None):
        """Eq. critical after one iteration (fsmt_converge): updates active, iters and ctl."""
        import torch
        L.call("fsmt_converge", self.h, int(R), float(eps), _dptr(gnorm2, torch.float32, (R,), "gnorm2"),
               _dptr(active, torch.uint8, (R,), "active"), _dptr(iters, torch.int32, (R,), "iters"),
               _dptr(ctl, torch.int32, None, "ctl"), _stream(stream))

    def mark_nonfinite(self, R, active, n_unsat, stream=None):
        """Bit 31 of n_unsat for the restarts stopped on a non-finite ||g||^2."""
        import torch
        L.call("fsmt_mark_nonfinite", self.h, int(R), _dptr(active, torch.uint8, (R,), "active"),
               _dptr(n_unsat, torch.int32, (R,), "n_unsat"), _stream(stream))


def relaxed_objective(compiled, sigma, w, a, b, plain=False):
    """C_sigma per restart as a differentiable torch function of (a, b)."""
    return RelaxedObjective.apply(a, b, compiled, w, float(sigma), bool(plain))


def _autograd_function():
    import torch

    class _RelaxedObjective(torch.autograd.Function):
        """forward: C_sigma(a, b) per restart ([R]); backward: the adjoint sweep.

        Fused form: one kernel computes C and its gradient in forward (the
        gradient is kept for backward).  Plain form: the forward kernel stores the
        top-down messages in a work buffer and backward runs the adjoint kernel.
        """

        @staticmethod
        def forward(ctx, a, b, compiled, w, sigma, plain):
            R = w.shape[1]
            obj = torch.empty(R, device=w.device, dtype=torch.float32)
            ga = torch.empty_like(a)
            gb = torch.empty_like(b)
            a_c, b_c = a.detach().contiguous(), b.detach().contiguous()
            if plain:
                work = torch.empty(compiled.plain_work(R), device=w.device, dtype=torch.float32)
                compiled.forward_plain(R, sigma, w, a_c, b_c, work, obj=obj)
                ctx.save_for_backward(a_c, b_c, w, work)
            else:
                compiled.adjoint(R, sigma, w, a_c, b_c, ga, gb, obj=obj)
                ctx.save_for_backward(ga, gb)
            ctx.compiled, ctx.sigma, ctx.plain, ctx.R = compiled, sigma, plain, R
            return obj

        @staticmethod
        def backward(ctx, g):
            if ctx.plain:
                a, b, w, work = ctx.saved_tensors
                ga = torch.empty_like(a)
                gb = torch.empty_like(b)
                ctx.compiled.adjoint_plain(ctx.R, ctx.sigma, w, a, b, work, ga, gb)
            else:
                ga, gb = ctx.saved_tensors
            g = g.reshape(1, -1)
            return ga * g, gb * g, None, None, None, None

    return _RelaxedObjective


def jsonl_log(path):
    """A `log` function for Solver.anneal that appends each stage's record to a JSON-lines
    file (one object per line, flushed per stage)."""
    import json
    f = open(path, "a")

    def write(rec):
        f.write(json.dumps(rec) + "\n")
        f.flush()
    write.close = f.close
    return write


def max_over_replicas(device="cpu"):
    """The `share` function of Solver.anneal over the default torch.distributed process
    group: an elementwise max all-reduce of a few integer flags (the restart replicas'
    one exchange; put the tensor on "cuda" under NCCL).  The identity without a group."""
    import torch
    import torch.distributed as dist

    def share(flags):
        if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
            return list(flags)
        t = torch.tensor([int(f) for f in flags], dtype=torch.int32, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return [int(v) for v in t.tolist()]
    return share


def gather_replicas(record):
    """Every replica's `record` (any picklable object), in rank order, on every rank of
    the default torch.distributed process group (all_gather_object; [record] without a
    group).  The host-side exchange of the independent-replica protocol, run once after
    the replicas have finished: nothing on the data path waits on it."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [record]
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, record)
    return out


def replica_median(runs, limit):
    """The paper's replica protocol (Methods, experimental setup: independent replicas,
    the median reported) scored as PAR-2 (a replica that found no exactly verified SAT
    counts twice the time limit): runs are dicts with "sat" and "seconds"."""
    if not runs:
        raise ValueError("no replica runs")
    return float(np.median([r["seconds"] if r["sat"] else 2.0 * float(limit) for r in runs]))


class _Lazy:
    def __init__(self):
        self.fn = None

    def apply(self, *args):
        if self.fn is None:
            self.fn = _autograd_function()
        return self.fn.apply(*args)


RelaxedObjective = _Lazy()


# fsmt_stage_config.persistent: how a fused stage runs its PGD iterations
STAGE_FORMS = {"launches": 0, "stage": 1, "iteration": 2}


class Solver:
    """Alg. 2 (annealing + ERWA) over R restarts with device-resident state.

    Each sigma stage is one fsmt_solve_stage call (a CUDA graph when use_graph);
    restarts whose check reports #Unsat = 0 are re-verified exactly on the host
    before SAT is reported.

    stage_form: how the fused stage's PGD iterations run -- "launches" (separate
    launches per iteration: forward + adjoint, the PGD kernels, the epsilon test),
    "stage" (one persistent kernel runs them all, phases separated by grid
    barriers), "iteration" (that kernel once per iteration), or "auto": separate
    launches until tune() has timed the three forms on the current state and pinned
    the fastest.  The persistent forms need the library's run-time compiled kernels
    (Compiled.stage_form); without them a stage uses separate launches.

    form="plain" runs the same stage as separate library calls issued from
    Python per iteration (plain forward and adjoint kernels with the top-down
    messages in device memory, the PGD step, the convergence test), no graph:
    the unfused form, for comparison.
    """

    def __init__(self, problem, compiled, R, eta, b_scale, eps=1e-2, t_max=200, sweeps=20, rho=0.5, gamma=2.0,
                 tau=1, use_graph=True, polish=32, normalize_eta=True, device="cuda", form="fused",
                 stage_form="auto"):
        import torch
        if form not in ("fused", "plain"):
            raise ValueError("form is 'fused' or 'plain'")
        info = compiled.info
        if form == "fused" and info["n_obj_cons"] > 0 and info["n_chunks"] == 0 and not info["fused_ok"]:
            # neither the chunked kernel (a constraint exceeds a chunk) nor the warp kernel
            # (the largest diagram's messages exceed its shared memory) takes this instance
            raise ValueError(f"no fused kernel takes a diagram of {info['max_nodes']} nodes; use form='plain'")
        self.form = form
        self._work = None
        self._x = None  # rounded Booleans of the candidates verified on the host
        self.problem, self.comp, self.R = problem, compiled, int(R)
        if not compiled.uploaded:
            compiled.upload()
        n, m, nc = compiled.n_bool, compiled.n_real, compiled.n_cons
        f32 = dict(device=device, dtype=torch.float32)
        self.a = torch.zeros((n, R), **f32)
        self.b = torch.zeros((m, R), **f32)
        self.w = torch.ones((nc, R), **f32)
        self.h = torch.zeros((nc, R), **f32)
        self.grad_a = torch.zeros((n, R), **f32)
        self.grad_b = torch.zeros((m, R), **f32)
        self.obj = torch.zeros(R, **f32)
        self.gnorm2 = torch.zeros(R, **f32)
        self.active = torch.zeros(R, device=device, dtype=torch.uint8)
        self.iters = torch.zeros(R, device=device, dtype=torch.int32)
        self.n_unsat = torch.zeros(R, device=device, dtype=torch.int32)
        self.ctl = torch.zeros(4, device=device, dtype=torch.int32)
        self.params = torch.zeros(16, **f32)
        self.wsum = torch.zeros(R, **f32)
        self.polish, self.normalize_eta = polish, normalize_eta
        self.eta, self.b_scale, self.eps, self.t_max, self.sweeps = eta, b_scale, eps, t_max, sweeps
        self.rho, self.gamma, self.tau, self.use_graph = rho, gamma, tau, use_graph
        if stage_form not in ("auto",) + tuple(STAGE_FORMS):
            raise ValueError(f"stage_form is 'auto' or one of {tuple(STAGE_FORMS)}")
        self.stage_form = stage_form
        self._form_code = 0 if stage_form == "auto" else STAGE_FORMS[stage_form]
        self.stage_form_ms = None  # tune(): ms per stage of each form, when it timed them
        self._state = L.State(self.R, *[C.c_void_p(t.data_ptr()) for t in (
            self.a, self.b, self.w, self.h, self.grad_a, self.grad_b, self.obj, self.gnorm2, self.active,
            self.iters, self.n_unsat, self.ctl, self.params, self.wsum)])

    def reset(self, a0, b0):
        """Loads initial points ([n][R], [m][R] float32, host or device) and resets weights."""
        import torch
        self.a.copy_(torch.as_tensor(a0))
        self.b.copy_(torch.as_tensor(b0))
        self.w.fill_(1.0)
        self.h.zero_()

    def state_dict(self):
        """A checkpoint of the search: points, ERWA weights and histories, and the
        per-restart outcome of the last stage (host copies; Alg. 2 resumes from it)."""
        return {k: getattr(self, k).detach().cpu().clone()
                for k in ("a", "b", "w", "h", "n_unsat", "iters", "obj")}

    def load_state_dict(self, state):
        """Restores a checkpoint taken by state_dict (same instance and R)."""
        for k, v in state.items():
            t = getattr(self, k)
            if tuple(t.shape) != tuple(v.shape):
                raise ValueError(f"checkpoint {k} has shape {tuple(v.shape)}, expected {tuple(t.shape)}")
            t.copy_(v)
        self.grad_a.zero_()
        self.grad_b.zero_()

    def tune(self, sigma, stages=2, kernels=True):
        """Autotunes the forward + adjoint kernel configuration on the current state
        (fsmt_autotune; the gradient buffers are scratch and left zero; kernels=False
        keeps the configuration already chosen).  With stage_form "auto" it then times
        `stages` stages of each stage form (after one untimed stage that captures its
        graph) from the current state, puts the state back, and pins the fastest form;
        the times are in stage_form_ms (None when the configuration has no persistent
        form).  Returns the forward + adjoint configuration (None with kernels=False)."""
        import torch
        best = None
        if kernels:
            best = self.comp.autotune(self.R, sigma, self.w, self.a, self.b, self.grad_a, self.grad_b, self.obj)
        if self.stage_form != "auto" or self.form != "fused" or not self.comp.stage_form(self.R):
            return best
        keep = {k: getattr(self, k).clone() for k in ("a", "b", "w", "h")}
        ms = {}
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for name, code in STAGE_FORMS.items():
            self._form_code = code
            for k, v in keep.items():
                getattr(self, k).copy_(v)
            self.stage(sigma, 1)
            e0.record()
            for t in range(stages):
                self.stage(sigma, 2 + t)
            e1.record()
            torch.cuda.synchronize()
            self.check_stage_status()
            ms[name] = e0.elapsed_time(e1) / stages
        for k, v in keep.items():
            getattr(self, k).copy_(v)
        self._form_code = STAGE_FORMS[min(ms, key=ms.get)]
        self.stage_form_ms = ms
        return best

    def config(self, sigma, t):
        return L.StageConfig(float(sigma), float(self.eta), float(self.b_scale), float(self.eps), int(self.t_max),
                             int(self.sweeps), float(self.rho), float(self.gamma), int(t % self.tau == 0),
                             int(bool(self.use_graph)), int(self.polish), int(bool(self.normalize_eta)),
                             int(self._form_code))

    def stage(self, sigma, t, stream=None):
        if self.form == "plain":
            return self._stage_plain(sigma, t, stream)
        cfg = self.config(sigma, t)
        L.call("fsmt_solve_stage", self.comp.h, C.byref(cfg), C.byref(self._state), _stream(stream))

    def _stage_plain(self, sigma, t, stream=None):
        """One stage of Alg. 2 in the plain form; the same steps as fsmt_solve_stage,
        each a library call issued from here: weight sums, then per iteration the
        plain forward and adjoint passes, the PGD step and the epsilon test
        (fsmt_converge, which also counts the restarts still iterating into ctl[0]),
        then round + check + ERWA and the marking of non-finite restarts."""
        import torch
        comp, R = self.comp, self.R
        if self._work is None:
            self._work = torch.empty(comp.plain_work(R), device=self.a.device, dtype=torch.float32)
        comp.weight_sum(R, self.w, self.wsum, stream)
        self.active.fill_(1)
        self.iters.zero_()
        self.ctl.zero_()
        for _ in range(int(self.t_max)):
            comp.forward_plain(R, sigma, self.w, self.a, self.b, self._work, obj=self.obj, stream=stream)
            comp.adjoint_plain(R, sigma, self.w, self.a, self.b, self._work, self.grad_a, self.grad_b, stream=stream)
            self.gnorm2.zero_()
            comp.pgd_step(R, self.eta, self.b_scale, self.sweeps, self.a, self.b, self.grad_a, self.grad_b,
                          self.gnorm2, active=self.active, wsum=self.wsum if self.normalize_eta else None,
                          polish=self.polish, stream=stream)
            comp.converge(R, self.eps, self.gnorm2, self.active, self.iters, self.ctl, stream=stream)
            if int(self.ctl[0].item()) == 0:
                break
        comp.round_check(R, self.a, self.b, self.n_unsat, w=self.w, h=self.h, rho=self.rho, gamma=self.gamma,
                         update_w=(t % self.tau == 0), wsum=self.wsum if self.normalize_eta else None,
                         stream=stream)
        comp.mark_nonfinite(R, self.active, self.n_unsat, stream=stream)

    @property
    def persistent(self):
        """Whether fused stages now ask for a persistent form ("stage" or "iteration")."""
        return self._form_code > 0

    @property
    def chosen_stage_form(self):
        """The stage form fused stages now run: "launches", "stage" or "iteration"."""
        if self.form != "fused" or (self._form_code > 0 and not self.comp.stage_form(self.R)):
            return "launches"
        return {v: k for k, v in STAGE_FORMS.items()}[self._form_code]

    def check_stage_status(self):
        """Raises FsmtError(ETIMEOUT) when the last fused stage's persistent kernel gave
        up waiting at a grid barrier (bit 4 of ctl[1]); its outputs are then invalid."""
        if self.form == "fused" and self.persistent and int(self.ctl[1].item()) & 4:
            raise L.FsmtError(L.ETIMEOUT, "the persistent stage kernel gave up waiting at a grid barrier")

    def stage_host(self, sigma, t, a_host, b_host, n_unsat_host, obj_host, stream=None):
        """The same stage with host input/output buffers (copies inside the call)."""
        cfg = self.config(sigma, t)
        L.call("fsmt_solve_stage_host", self.comp.h, C.byref(cfg), C.byref(self._state), _np_ptr(a_host),
               _np_ptr(b_host), _np_ptr(n_unsat_host), _np_ptr(obj_host), _stream(stream))

    def verify_restart(self, r):
        """Restart r's rounded point (fsmt_round) checked exactly on the host: y is the
        restart's reals widened to float64 exactly, repaired exactly onto the projected
        equalities (fsmt_repair_equalities), then fsmt_verify_exact."""
        import torch
        if self._x is None:
            self._x = torch.empty((self.comp.n_bool, self.R), device=self.a.device, dtype=torch.int8)
        self.comp.round(self.R, self.a, self._x)
        # whole arrays to the host (one copy each), then restart r's column
        x = np.ascontiguousarray(self._x.cpu().numpy()[:, r])
        y = self.b.cpu().numpy()[:, r].astype(np.float64)
        ok, y = self.problem.repair_equalities(y)  # equalities held within FP32 rounding: made exact
        if not ok:
            return False, x, y
        sat, _ = self.problem.verify_exact(x, y)
        return sat, x, y

    def anneal(self, schedule, time_limit=None, share=None, log=None):
        """Runs the sigma schedule (Alg. 2); returns dict with the first exactly verified
        SAT restart (or None), the stages run, the fewest unsatisfied constraints any
        restart had at a rounding, and how many restarts ended on a non-finite point
        (n_unsat < 0; they are never SAT candidates).  Without `share` it stops early when
        every restart is non-finite.

        share: for restart replicas (one solver per rank, independent seeds), a function
        that takes this rank's flags [verified SAT, out of time] and returns their
        elementwise maximum over the ranks (max_over_replicas).  Every rank calls it once
        per stage and all stop after the same stage: the first at which some rank
        verified SAT (the others return stopped_by_peer = True) or ran out of time.

        log: called after every stage with one record (a dict: stage, sigma, seconds since
        the start, fewest and median #Unsat over the finite restarts, restarts at #Unsat
        0, non-finite restarts, mean PGD iterations, median ||g||^2 of the last iteration,
        best objective, and the stage's device time from CUDA events around it, gpu_ms);
        jsonl_log(path) writes them one JSON line each.

        The result also counts rejected_candidates: restarts whose device check reported
        #Unsat = 0 but whose rounded point failed the exact host verification (a
        disagreement between the two checks; 0 is expected)."""
        import torch
        t0 = time.perf_counter()
        best, t, nonfinite, rejected = None, 0, 0, 0
        ev = None
        if log is not None and self.n_unsat.is_cuda:
            ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        for t, sigma in enumerate(schedule, start=1):
            if ev is not None:
                ev[0].record()
            self.stage(sigma, t)
            if ev is not None:
                ev[1].record()
            # the stage's outcome reaches the host as one small copy; the statistics are
            # taken there (no device kernels beyond the library's own in the loop)
            nu = self.n_unsat.cpu().numpy()
            self.check_stage_status()
            nonfinite = int((nu < 0).sum())
            found = None
            lo = None
            if nonfinite < self.R:
                lo = int(nu[nu >= 0].min())
                best = lo if best is None else min(best, lo)
            if log is not None:
                fin = nu[nu >= 0]
                ob = self.obj.cpu().numpy()
                ob = ob[np.isfinite(ob)]
                gn = self.gnorm2.cpu().numpy().astype(np.float64)
                log(dict(stage=t, sigma=float(sigma), seconds=time.perf_counter() - t0, min_unsat=lo,
                         median_unsat=float(np.median(fin)) if fin.size else None,
                         at_zero=int((nu == 0).sum()), nonfinite=nonfinite,
                         mean_iters=float(self.iters.cpu().numpy().astype(np.float64).mean()),
                         median_gnorm2=float(np.nanmedian(gn)) if not np.isnan(gn).all() else None,
                         best_obj=float(ob.min()) if ob.size else None,
                         gpu_ms=(ev[1].synchronize(), ev[0].elapsed_time(ev[1]))[1] if ev is not None else None))
            if nonfinite < self.R:
                cand = np.nonzero(nu == 0)[0].tolist() if lo == 0 else []
                for r in cand:
                    sat, x, y = self.verify_restart(r)
                    if sat:
                        found = dict(sat=True, restart=r, stage=t, x=x, y=y)
                        break
                    rejected += 1
            elif share is None:
                break
            late = time_limit is not None and time.perf_counter() - t0 > time_limit
            flags = [int(found is not None), int(late)]
            if share is not None:
                flags = [int(v) for v in share(flags)]
            if found is not None:
                return dict(found, stages_run=t, best_unsat=0, nonfinite=nonfinite, stopped_by_peer=False,
                            seconds=time.perf_counter() - t0, rejected_candidates=rejected)
            if flags[0]:
                return dict(sat=False, restart=None, stage=None, stages_run=t, best_unsat=best,
                            nonfinite=nonfinite, stopped_by_peer=True, seconds=time.perf_counter() - t0,
                            rejected_candidates=rejected)
            if flags[1]:
                break
        if self.n_unsat.is_cuda:
            torch.cuda.synchronize()
        return dict(sat=False, restart=None, stage=None, stages_run=t, best_unsat=best, nonfinite=nonfinite,
                    stopped_by_peer=False, seconds=time.perf_counter() - t0, rejected_candidates=rejected)
