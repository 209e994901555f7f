"""CPU oracle (test infrastructure only; see the docstrings of lyap_oracle and projection)."""
from .lyap_oracle import (  # noqa: F401
    param_matrix,
    lyap_kron,
    lyap_exact,
    lyap_bartels_stewart,
    lyap_solve,
    trace_product,
    solve,
    trace_EX,
    gradient,
    check_solution,
    sweep,
)
