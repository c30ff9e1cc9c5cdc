"""FP64 CPU oracle of the hybrid FEM/FDM method (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
reference legs may import this package; the GPU product path never does.
"""
from .hybrid import (BC_ABC, BC_NEUMANN0, Problem, cg_direction, cg_step, data_weights,  # noqa: F401
                     drop_blocked, element_stiffness, kuhn_tets, misfit, p1_element, problem_from_workload,
                     projected_gradient, pulse, quadratic_step, value_and_grad)
