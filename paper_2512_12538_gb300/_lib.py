"""ctypes binding of libhh.so (the C-ABI declared in include/hh.h).

Argument marshalling only: every function forwards to the C entry point of the same
name.  Device arrays are passed as torch tensors (complex128, on the current CUDA
device) or as raw integer pointers; streams default to torch's current stream.  There
is no fallback: if the shared library is missing or cannot be loaded, import fails.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhh.so")

HH_OK, HH_EINVAL, HH_ENOMEM, HH_ENOCONV, HH_EBREAKDOWN, HH_ETIMEOUT, HH_ECUDA, HH_ENOTIMPL = (
    0, -1, -2, -3, -4, -5, -6, -7)
HH_ETOOLARGE = -8
HH_EPENDING = -9
HH_NOALLOC_MAX_ROWS = 16384
HH_PREC_FP64, HH_PREC_MIXED = 0, 1
HH_LEAF_EIGEN, HH_LEAF_BLOCK = 0, 1
HH_OUTER_ORAS, HH_OUTER_GMRES = 0, 1
HH_FLAG_COARSE_FP32 = 1
HH_FLAG_CUDA_CORE_SWEEPS = 2
HH_FLAG_TENSOR_CORE_SWEEPS = 4
HH_FLAG_BILINEAR = 8


class hh_params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("k", ctypes.c_double),
                ("levels", ctypes.c_int), ("overlap", ctypes.c_int), ("rank", ctypes.c_int),
                ("oversample", ctypes.c_int), ("n_inner", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("precision", ctypes.c_int),
                ("seed", ctypes.c_ulonglong), ("leaf_solver", ctypes.c_int), ("outer", ctypes.c_int),
                ("restart", ctypes.c_int), ("flags", ctypes.c_uint), ("k_rows", ctypes.c_void_p)]


class hh_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("t_setup_ms", ctypes.c_double), ("t_solve_ms", ctypes.c_double),
                ("footprint_bytes", ctypes.c_size_t), ("t_queue_ms", ctypes.c_double),
                ("t_total_ms", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class HHError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2512_12538_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    P = ctypes.POINTER
    sig = {
        "hh_set_allocator": (i, [vp, vp, vp]),
        "hh_footprint": (i, [P(hh_params), P(sz)]),
        "hh_setup": (i, [P(hh_params), vp, P(vp), P(sz)]),
        "hh_solve": (i, [vp, vp, vp, vp, vp, P(hh_stats)]),
        "hh_solve_host": (i, [vp, vp, vp, vp, vp, P(hh_stats)]),
        "hh_residual": (i, [vp, vp, vp, vp, vp, P(d)]),
        "hh_destroy": (None, [vp]),
        "hh_status_string": (ctypes.c_char_p, [i]),
        "hh_node_info": (i, [vp, i, P(i)]),
        "hh_apply_operator": (i, [vp, i, vp, vp, i, vp]),
        "hh_leaf_solve": (i, [vp, i, vp, vp, i, vp]),
        "hh_interface_map": (i, [vp, i, i, vp, vp, i, vp]),
        "hh_get_basis": (i, [vp, i, vp, P(d)]),
        "hh_coarse_apply": (i, [vp, i, vp, vp, vp]),
        "hh_precondition": (i, [vp, vp, vp, vp]),
        "hh_sketch_samples": (i, [vp, i, vp, vp]),
        "hh_profile_enable": (i, [vp, i]),
        "hh_profile_categories": (i, [vp, ctypes.c_uint]),
        "hh_profile_read": (i, [vp, i, P(d), P(ctypes.c_longlong), P(d), P(d)]),
        "hh_launch_count": (ctypes.c_ulonglong, []),
        "hh_residual_noalloc": (i, [i, i, d, vp, vp, vp, vp, P(d)]),
        "hh_debug_set_wait_limit": (i, [ctypes.c_longlong]),
        "hh_autotune_report": (i, [vp, sz, P(sz)]),
        "hh_setup_batch": (i, [P(hh_params), i, vp, P(vp)]),
        "hh_server_create": (i, [sz, i, P(vp)]),
        "hh_server_submit": (i, [vp, P(hh_params), vp, vp, vp, P(ctypes.c_ulonglong)]),
        "hh_server_poll": (i, [vp, ctypes.c_ulonglong, P(i), P(hh_stats)]),
        "hh_server_destroy": (None, [vp]),
        "hh_solve_batch": (i, [P(vp), P(vp), P(vp), P(vp), i, vp, P(hh_stats)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = _load()


def status_string(s: int) -> str:
    return LIB.hh_status_string(int(s)).decode()


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(st: int, where: str, ok=(HH_OK,)):
    if st not in ok:
        raise HHError(st, where)
    return st


def make_params(dim=2, n=255, k=40.0, levels=2, overlap=2, rank=16, oversample=10, n_inner=1,
                tol=1e-10, max_iter=200, precision=HH_PREC_FP64, seed=0, leaf_solver=HH_LEAF_EIGEN,
                outer=HH_OUTER_ORAS, restart=40, flags=0, k_rows=None) -> hh_params:
    if isinstance(precision, str):
        precision = {"fp64": HH_PREC_FP64, "mixed": HH_PREC_MIXED}[precision]
    if isinstance(leaf_solver, str):
        leaf_solver = {"eigen": HH_LEAF_EIGEN, "block": HH_LEAF_BLOCK}[leaf_solver]
    if isinstance(outer, str):
        outer = {"oras": HH_OUTER_ORAS, "gmres": HH_OUTER_GMRES}[outer]
    kr = None
    if k_rows is not None:
        import numpy as np
        kr = np.ascontiguousarray(k_rows, dtype=np.float64)
        if kr.shape != (n + 2,):
            raise ValueError("k_rows needs one wavenumber per grid row (n + 2 values)")
    p = hh_params(dim, n, float(k), levels, overlap, rank, oversample, n_inner, float(tol), max_iter,
                  precision, seed, leaf_solver, outer, restart, flags, None if kr is None else kr.ctypes.data)
    p._k_rows = kr      # the host array must outlive the calls that read it
    return p


# ------------------------------------------------------------------ allocator hook
_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_keep = []


def use_torch_allocator() -> None:
    """Route the library's device allocations through torch's caching allocator."""
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=stream or 0)
        except Exception:
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = _ALLOC_T(_alloc), _FREE_T(_free)
    _keep[:] = [a, f]
    _check(LIB.hh_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p), None),
           "hh_set_allocator")


def hh_set_allocator(alloc=None, free=None, ctx=None) -> int:
    return _check(LIB.hh_set_allocator(alloc, free, ctx), "hh_set_allocator")


# ------------------------------------------------------------------- entry points
def hh_footprint(params: hh_params) -> int:
    b = ctypes.c_size_t()
    _check(LIB.hh_footprint(ctypes.byref(params), ctypes.byref(b)), "hh_footprint")
    return b.value


def hh_setup(params: hh_params, stream=None):
    """Returns (handle, footprint_bytes).  Raises HHError on failure."""
    h = ctypes.c_void_p()
    fp = ctypes.c_size_t()
    _check(LIB.hh_setup(ctypes.byref(params), _stream(stream), ctypes.byref(h), ctypes.byref(fp)), "hh_setup")
    return h, fp.value


def hh_setup_batch(params_list, stream=None) -> list:
    """Sets up len(params_list) problems concurrently; returns their handles."""
    n = len(params_list)
    arr = (hh_params * n)(*params_list)
    hs = (ctypes.c_void_p * n)()
    _check(LIB.hh_setup_batch(arr, n, _stream(stream), hs), "hh_setup_batch")
    return [ctypes.c_void_p(x) for x in hs]


def hh_solve_batch(handles, fs, gs, us, stream=None, allow_noconv=False) -> list:
    """Solves the set-up problems together (lockstep where possible); returns hh_stats
    per problem.  fs, gs, us: device tensors (or pointers), one per handle."""
    n = len(handles)
    VP = ctypes.c_void_p * n
    st = (hh_stats * n)()
    ok = (HH_OK, HH_ENOCONV) if allow_noconv else (HH_OK,)
    _check(LIB.hh_solve_batch(VP(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles]),
                              VP(*[_ptr(x) for x in fs]), VP(*[_ptr(x) for x in gs]), VP(*[_ptr(x) for x in us]),
                              n, _stream(stream), st), "hh_solve_batch", ok)
    return list(st)


def hh_server_create(hbm_budget: int, max_slots: int):
    srv = ctypes.c_void_p()
    _check(LIB.hh_server_create(int(hbm_budget), int(max_slots), ctypes.byref(srv)), "hh_server_create")
    return srv


def hh_server_submit(srv, params: hh_params, f, g, u) -> int:
    """Queues one request; f, g, u device tensors that must stay alive until it finishes."""
    t = ctypes.c_ulonglong()
    _check(LIB.hh_server_submit(srv, ctypes.byref(params), _ptr(f), _ptr(g), _ptr(u), ctypes.byref(t)),
           "hh_server_submit")
    return t.value


def hh_server_poll(srv, ticket: int):
    """None while pending, else (status, hh_stats)."""
    res = ctypes.c_int()
    st = hh_stats()
    r = LIB.hh_server_poll(srv, ctypes.c_ulonglong(ticket), ctypes.byref(res), ctypes.byref(st))
    if r == HH_EPENDING:
        return None
    _check(r, "hh_server_poll")
    return res.value, st


def hh_server_destroy(srv) -> None:
    LIB.hh_server_destroy(srv)


def hh_solve(h, f, g, u, stream=None, allow_noconv=False) -> hh_stats:
    st = hh_stats()
    ok = (HH_OK, HH_ENOCONV) if allow_noconv else (HH_OK,)
    _check(LIB.hh_solve(h, _ptr(f), _ptr(g), _ptr(u), _stream(stream), ctypes.byref(st)), "hh_solve", ok)
    return st


def hh_solve_host(h, f_host, g_host, u_host, stream=None, allow_noconv=False) -> hh_stats:
    """Host arrays: numpy complex128 (C-contiguous) or CPU torch tensors."""
    def hp(a):
        if hasattr(a, "ctypes"):
            return a.ctypes.data
        return a.data_ptr()
    st = hh_stats()
    ok = (HH_OK, HH_ENOCONV) if allow_noconv else (HH_OK,)
    _check(LIB.hh_solve_host(h, hp(f_host), hp(g_host), hp(u_host), _stream(stream), ctypes.byref(st)),
           "hh_solve_host", ok)
    return st


def hh_residual(h, f, g, u, stream=None) -> float:
    r = ctypes.c_double()
    _check(LIB.hh_residual(h, _ptr(f), _ptr(g), _ptr(u), _stream(stream), ctypes.byref(r)), "hh_residual")
    return r.value


def hh_residual_noalloc(dim, n, k, f, g, u, stream=None) -> float:
    """hh_residual without a handle or any device allocation (static scratch)."""
    r = ctypes.c_double()
    _check(LIB.hh_residual_noalloc(int(dim), int(n), float(k), _ptr(f), _ptr(g), _ptr(u), _stream(stream),
                                   ctypes.byref(r)), "hh_residual_noalloc")
    return r.value


def hh_destroy(h) -> None:
    LIB.hh_destroy(h)


def hh_node_info(h, node: int) -> dict:
    a = (ctypes.c_int * 10)()
    _check(LIB.hh_node_info(h, node, a), "hh_node_info")
    keys = ["oa", "ob", "ra", "rb", "level", "parent", "child0", "child1", "Sx", "ifrow"]
    return dict(zip(keys, list(a)))


def hh_apply_operator(h, node, x, y, ncols, stream=None) -> None:
    _check(LIB.hh_apply_operator(h, node, _ptr(x), _ptr(y), ncols, _stream(stream)), "hh_apply_operator")


def hh_leaf_solve(h, leaf, v, x, ncols, stream=None) -> None:
    _check(LIB.hh_leaf_solve(h, leaf, _ptr(v), _ptr(x), ncols, _stream(stream)), "hh_leaf_solve")


def hh_interface_map(h, child, adjoint, x, y, ncols, stream=None) -> None:
    _check(LIB.hh_interface_map(h, child, int(adjoint), _ptr(x), _ptr(y), ncols, _stream(stream)),
           "hh_interface_map")


def hh_get_basis(h, child, V_host=None, sigma_host=None) -> None:
    vp = V_host.ctypes.data if V_host is not None else None
    sp = sigma_host.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if sigma_host is not None else None
    _check(LIB.hh_get_basis(h, child, vp, sp), "hh_get_basis")


def hh_coarse_apply(h, node, r, z, stream=None) -> None:
    _check(LIB.hh_coarse_apply(h, node, _ptr(r), _ptr(z), _stream(stream)), "hh_coarse_apply")


def hh_precondition(h, r, z, stream=None) -> None:
    _check(LIB.hh_precondition(h, _ptr(r), _ptr(z), _stream(stream)), "hh_precondition")


def hh_sketch_samples(h, child, out, stream=None) -> None:
    _check(LIB.hh_sketch_samples(h, child, _ptr(out), _stream(stream)), "hh_sketch_samples")


PROFILE_CATEGORIES = ["factor", "sweep_in", "sweep_recur", "sweep_out", "residual", "coarse_project",
                      "galerkin", "qr", "svd", "leaf_sweep", "coarse_multi"]


def hh_profile_enable(h, enable=True) -> None:
    _check(LIB.hh_profile_enable(h, int(bool(enable))), "hh_profile_enable")


def hh_profile_categories(h, names=None) -> None:
    """Time only the named categories (PROFILE_CATEGORIES); None: all of them."""
    mask = 0xFFFFFFFF if names is None else sum(1 << PROFILE_CATEGORIES.index(n) for n in names)
    _check(LIB.hh_profile_categories(h, ctypes.c_uint(mask)), "hh_profile_categories")


def hh_profile_read(h, work=False) -> dict:
    """{category: (total_ms, launches)} for every profiler category; with work=True
    (total_ms, launches, algorithmic_bytes, algorithmic_flops)."""
    out = {}
    for i, name in enumerate(PROFILE_CATEGORIES):
        ms = ctypes.c_double()
        n = ctypes.c_longlong()
        by = ctypes.c_double()
        fl = ctypes.c_double()
        _check(LIB.hh_profile_read(h, i, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(by), ctypes.byref(fl)),
               "hh_profile_read")
        out[name] = (ms.value, n.value, by.value, fl.value) if work else (ms.value, n.value)
    return out


def hh_launch_count() -> int:
    return int(LIB.hh_launch_count())


def hh_debug_set_wait_limit(polls: int) -> None:
    """Cap the polls of the library's give-up waits (0: give up at once; < 0: defaults)."""
    _check(LIB.hh_debug_set_wait_limit(int(polls)), "hh_debug_set_wait_limit")


def hh_autotune_report() -> list:
    """The autotuner's decisions so far (list of dicts)."""
    import json
    n = ctypes.c_size_t()
    _check(LIB.hh_autotune_report(None, 0, ctypes.byref(n)), "hh_autotune_report")
    buf = ctypes.create_string_buffer(n.value + 1)
    _check(LIB.hh_autotune_report(buf, n.value + 1, ctypes.byref(n)), "hh_autotune_report")
    return json.loads(buf.value.decode())
