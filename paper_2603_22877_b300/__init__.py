"""B300-native (sm_103a) engine for the hot path of FourierSMT (arxiv 2603.22877).

The numerical work runs in libfsmt.so (C ABI, include/fsmt.h): compiled xBDDs,
the fused forward/adjoint kernel, PGD with projection, rounding with an exact
check, and graph-captured annealing stages.  This package only marshals
arguments; importing it does not touch the GPU, and every device entry point
fails loudly if the library is missing.
"""
from ._lib import FsmtError, load  # noqa: F401
from .engine import (Compiled, Problem, Solver, gather_replicas, jsonl_log, max_over_replicas,  # noqa: F401
                     relaxed_objective, replica_median)

__all__ = ["FsmtError", "load", "Problem", "Compiled", "Solver", "jsonl_log", "max_over_replicas",
           "gather_replicas", "replica_median", "relaxed_objective"]
