"""gradsolve-gb300: record-and-replay gradients of ODE ensembles on one GB300.

The hot path (adaptive record, reverse discrete-adjoint sweep) is hand-written
CUDA for sm_103a behind the C-ABI of include/gs.h; this package is its thin
Python face (argument marshalling, a torch.autograd.Function, the request
server) plus the seeded workload generator.
"""
from . import workloads
from .api import (GsFunction, Record, forward_grad, forward_record, odeint_ensemble, problem_info, replay_jvp,
                  reverse, solve, solve_grad)

__all__ = ["GsFunction", "Record", "forward_grad", "forward_record", "odeint_ensemble", "problem_info",
           "replay_jvp", "reverse", "solve", "solve_grad", "workloads"]
