"""GB300 (sm_103a) hierarchical ORAS solver for the impedance Helmholtz problem.

The compute path is libhh.so (hand-written CUDA, C-ABI in include/hh.h); this package
is its thin ctypes binding plus a small convenience wrapper.  PyTorch provides device
memory and streams only.
"""
from __future__ import annotations

from ._lib import (  # noqa: F401
    HH_EBREAKDOWN, HH_ECUDA, HH_EINVAL, HH_ENOCONV, HH_ENOMEM, HH_ENOTIMPL, HH_ETIMEOUT, HH_OK,
    HH_PREC_FP64, HH_PREC_MIXED, LIB, LIB_PATH, HHError, hh_apply_operator, hh_coarse_apply,
    hh_destroy, hh_footprint, hh_get_basis, hh_interface_map, hh_leaf_solve, hh_node_info,
    hh_params, hh_precondition, hh_residual, hh_set_allocator, hh_setup, hh_sketch_samples,
    hh_solve, hh_solve_host, hh_stats, make_params, status_string, use_torch_allocator,
)
from .solver import Solver  # noqa: F401
