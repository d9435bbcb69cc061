"""GB300 (sm_103a) hierarchical ORAS solver for the impedance Helmholtz problem.

The compute path is libhh.so (hand-written CUDA, C-ABI in include/hh.h); this package
is its thin ctypes binding plus a small convenience wrapper.  PyTorch provides device
memory and streams only.

The shared library is loaded on first use of any binding name (so that the ``build``
submodule can be imported before it exists); if it is missing, that first use raises
ImportError -- there is no fallback path.
"""
from __future__ import annotations

import importlib

_BINDING = {
    "HH_EBREAKDOWN", "HH_ECUDA", "HH_EINVAL", "HH_ENOCONV", "HH_ENOMEM", "HH_ENOTIMPL", "HH_ETIMEOUT",
    "HH_OK", "HH_PREC_FP64", "HH_PREC_MIXED", "LIB", "LIB_PATH", "HHError", "hh_apply_operator",
    "hh_coarse_apply", "hh_destroy", "hh_footprint", "hh_get_basis", "hh_interface_map", "hh_leaf_solve",
    "hh_node_info", "hh_params", "hh_precondition", "hh_residual", "hh_set_allocator", "hh_setup",
    "hh_sketch_samples", "hh_solve", "hh_solve_host", "hh_stats", "make_params", "status_string",
    "use_torch_allocator", "hh_profile_enable", "hh_profile_categories", "hh_profile_read", "hh_launch_count", "PROFILE_CATEGORIES",
    "HH_LEAF_EIGEN", "HH_LEAF_BLOCK", "HH_OUTER_ORAS", "HH_OUTER_GMRES",
    "hh_residual_noalloc", "HH_ETOOLARGE", "HH_NOALLOC_MAX_ROWS", "hh_setup_batch", "hh_solve_batch", "hh_server_create", "hh_server_submit",
    "hh_server_poll", "hh_server_destroy", "HH_EPENDING", "HH_FLAG_COARSE_FP32", "HH_FLAG_CUDA_CORE_SWEEPS", "HH_FLAG_TENSOR_CORE_SWEEPS", "HH_FLAG_BILINEAR",
    "hh_debug_set_wait_limit", "hh_autotune_report",
}


def __getattr__(name):
    if name in _BINDING:
        return getattr(importlib.import_module("._lib", __name__), name)
    if name == "Solver":
        return importlib.import_module(".solver", __name__).Solver
    raise AttributeError(name)


__all__ = sorted(_BINDING | {"Solver"})
