"""GB300-native batched differentiable QP solver (the OptNet layer hot path, arxiv 1703.00443).

Entry points mirror the C ABI in include/qp_gb300.h:
``qp_forward``, ``qp_backward``, ``workspace_bytes``, ``supported``, ``uses_global_path``,
``uses_tensor_cores``, plus ``QPFunction`` /
``qp_layer`` for autograd.  Import of the CUDA library is lazy; the first call loads it and
fails loudly if it cannot.
"""
from .qp import (QPError, ForwardResult, alloc_workspace, default_options, qp_backward,  # noqa: F401
                 qp_forward, supported, workspace_bytes, STATUS_CONVERGED, STATUS_MAX_ITER,
                 STATUS_NOT_PD, STATUS_NUMERICAL, STATUS_NO_FORWARD, STATUS_INFEASIBLE,
                 STATUS_TIMEOUT, FLAG_NEAR_DEGENERATE, FLAG_REGULARIZED_Q, uses_global_path,
                 uses_tensor_cores)
from .autograd import QPFunction, qp_layer  # noqa: F401
