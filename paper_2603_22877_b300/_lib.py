"""ctypes binding of libfsmt.so (the C ABI declared in include/fsmt.h).

Argument marshalling only: every computation runs in the library.  Loading
fails loudly if the shared library is missing; there is no fallback.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfsmt.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENAN, ESTATE = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "ENAN", -6: "ESTATE"}
LE, LT, GE, GT, EQ = 0, 1, 2, 3, 4
OR, XOR, CARD_LE, NAE, MUX, NEQ_OR = 0, 1, 2, 3, 4, 5
UNIT_PROJECT, UNIT_SOFT = 0, 1


class FsmtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"fsmt {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Info(C.Structure):
    _fields_ = [("n_bool", C.c_int32), ("n_real", C.c_int32), ("n_atoms", C.c_int32), ("n_cons", C.c_int32),
                ("n_obj_cons", C.c_int32), ("n_nodes", C.c_int64), ("n_obj_nodes", C.c_int64),
                ("max_nodes", C.c_int32), ("n_halfspaces", C.c_int32), ("n_components", C.c_int32),
                ("n_free_reals", C.c_int32), ("atom_nnz", C.c_int64), ("fused_ok", C.c_int32),
                ("n_chunks", C.c_int32), ("jit_shapes", C.c_int32), ("empty_boxes", C.c_int32),
                ("proj_shapes", C.c_int32)]


class State(C.Structure):
    _fields_ = [("R", C.c_int32), ("a", C.c_void_p), ("b", C.c_void_p), ("w", C.c_void_p), ("h", C.c_void_p),
                ("grad_a", C.c_void_p), ("grad_b", C.c_void_p), ("obj", C.c_void_p), ("gnorm2", C.c_void_p),
                ("active", C.c_void_p), ("iters", C.c_void_p), ("n_unsat", C.c_void_p), ("ctl", C.c_void_p),
                ("params", C.c_void_p), ("wsum", C.c_void_p)]


class StageConfig(C.Structure):
    _fields_ = [("sigma", C.c_float), ("eta", C.c_float), ("b_scale", C.c_float), ("eps", C.c_float),
                ("t_max", C.c_int32), ("sweeps", C.c_int32), ("rho", C.c_float), ("gamma", C.c_float),
                ("update_w", C.c_int32), ("use_graph", C.c_int32), ("polish", C.c_int32),
                ("normalize_eta", C.c_int32), ("persistent", C.c_int32)]


P = C.c_void_p
i32, i64, f32, f64 = C.c_int32, C.c_int64, C.c_float, C.c_double

class LaunchConfig(C.Structure):
    _fields_ = [("variant", C.c_int32), ("restarts_per_lane", C.c_int32), ("staged_reals", C.c_int32),
                ("warps", C.c_int32), ("smem_bytes", C.c_int64), ("ms", C.c_float), ("reserved", C.c_int32)]

    VARIANTS = {0: "warp", 1: "chunked", 2: "jit", 3: "wide"}

    def as_dict(self):
        return {"variant": self.VARIANTS.get(self.variant, str(self.variant)),
                "restarts_per_lane": self.restarts_per_lane, "staged_reals": self.staged_reals,
                "warps": self.warps, "smem_bytes": self.smem_bytes, "ms": self.ms}


PROTOTYPES = {
    "fsmt_problem_create": [i32, i32, C.POINTER(P)],
    "fsmt_set_real_bounds": [P, i32, f64, f64],
    "fsmt_add_atom": [P, i32, P, P, i64, i32, C.POINTER(i32)],
    "fsmt_add_atoms": [P, i32, P, P, P, P, P],
    "fsmt_add_constraint": [P, i32, i32, P, i32],
    "fsmt_add_constraints": [P, i32, P, P, P, P],
    "fsmt_free_problem": [P],
    "fsmt_verify_exact": [P, P, P, C.POINTER(i32), C.POINTER(i32)],
    "fsmt_repair_equalities": [P, P, C.POINTER(i32)],
    "fsmt_compile": [P, i32, C.POINTER(P)],
    "fsmt_compiled_info": [P, C.POINTER(Info)],
    "fsmt_get_diagrams": [P, P, P, P, P, P, P],
    "fsmt_get_bounds": [P, P, P],
    "fsmt_upload": [P, P],
    "fsmt_free_compiled": [P],
    "fsmt_forward": [P, i32, f32, P, P, P, P, P, P],
    "fsmt_adjoint": [P, i32, f32, P, P, P, P, P, P, P, P],
    "fsmt_launch_configs": [P, i32, C.POINTER(LaunchConfig), i32, C.POINTER(i32)],
    "fsmt_select_config": [P, i32, C.POINTER(LaunchConfig)],
    "fsmt_autotune": [P, i32, f32, P, P, P, P, P, P, C.POINTER(LaunchConfig), P],
    "fsmt_plain_work_floats": [P, i32, C.POINTER(i64)],
    "fsmt_forward_plain": [P, i32, f32, P, P, P, P, P, P, P],
    "fsmt_adjoint_plain": [P, i32, f32, P, P, P, P, P, P, P],
    "fsmt_plain_noalloc": [P, i32, f32, P, P, P, P, P, P, P, P],
    "fsmt_weight_sum": [P, i32, P, P, P],
    "fsmt_pgd_step": [P, i32, f32, f32, i32, i32, P, P, P, P, P, P, P, P],
    "fsmt_round_check": [P, i32, P, P, P, P, P, P, P, f32, f32, i32, P, P],
    "fsmt_round": [P, i32, P, P, P],
    "fsmt_converge": [P, i32, f32, P, P, P, P, P],
    "fsmt_mark_nonfinite": [P, i32, P, P, P],
    "fsmt_solve_stage": [P, C.POINTER(StageConfig), C.POINTER(State), P],
    "fsmt_stage_form": [P, i32, C.POINTER(i32)],
    "fsmt_stage_trace": [P, P],
    "fsmt_solve_stage_host": [P, C.POINTER(StageConfig), C.POINTER(State), P, P, P, P, P],
    "fsmt_last_error": [],
    "fsmt_version": [],
}
VOID_FUNCS = {"fsmt_free_problem", "fsmt_free_compiled"}
STRING_FUNCS = {"fsmt_last_error", "fsmt_version"}

_lib = None


def load():
    """Loads libfsmt.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise FsmtError(ESTATE, f"{LIB_PATH} is missing: build it with paper_2603_22877_b300.build.build()")
    lib = C.CDLL(LIB_PATH)
    for name, args in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        if name in VOID_FUNCS:
            fn.restype = None
        elif name in STRING_FUNCS:
            fn.restype = C.c_char_p
        else:
            fn.restype = C.c_int
    _lib = lib
    return lib


def call(name, *args):
    """Calls an fsmt_* entry point and raises FsmtError on a non-OK status."""
    lib = load()
    st = getattr(lib, name)(*args)
    if st != OK:
        raise FsmtError(st, lib.fsmt_last_error().decode())
    return st


def last_error():
    return load().fsmt_last_error().decode()
