"""FP64 CPU oracle (test infrastructure only; see ``oracle/qp.py``)."""
from .qp import (backward, backward_batch, backward_sym, initial_point, kkt_matrix,  # noqa: F401
                 max_step, residuals, solve, solve_batch, STATUS_CONVERGED, STATUS_MAX_ITER)
