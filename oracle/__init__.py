"""CPU FP64 oracle (test infrastructure; never imported by the library)."""
from .magnus import (  # noqa: F401
    gauss_legendre, interval_starts, node_times, drive_coefficients, first_order_term,
    second_order_term, expm_minus_i, interval_propagators, propagate_state,
    propagate_unitary, magnus_evolve, evolve_workload, unitarity_defect, norm_defect,
    interval_propagators_second_order, evolve_workload_second_order, evolve_workload_streamed,
)
