"""Failure detection without a GPU fault: every device-side wait of the library is
bounded, and a wait that runs out comes back to the caller as HH_ETIMEOUT with the
context still usable.

hh_debug_set_wait_limit(0) makes the give-up waits give up at once (a wait that
nothing ends, in its testing form): the cooperative grid barrier of the one-column
coarse corrections, and the tensor-core transforms' waits for their operands and MMAs.
The kernels then drain what they have in flight (with the default limits), free their
tensor memory and return.  After the limit is restored, new handles solve correctly in
the same process.
"""
import numpy as np
import pytest

from oracle import direct
from oracle.problem import Problem
from workloads import point_source_rhs, random_complex

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, K = 45, 12.0


@pytest.fixture(scope="module")
def hh():
    from paper_2512_12538_gb300 import build
    build.build()
    import paper_2512_12538_gb300 as m
    return m


def _solve_ok(hh):
    P = Problem(2, N, K)
    f = point_source_rhs(N, 3)
    g = np.zeros((4, P.S), dtype=np.complex128)
    p = hh.make_params(2, N, K, 2, 2, 6, 4, 1, 1e-12, 300, "mixed", 1)
    h, _ = hh.hh_setup(p)
    try:
        u = torch.empty((P.S, P.S), dtype=torch.complex128, device="cuda")
        hh.hh_solve(h, torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), u)
        return float(np.linalg.norm(u.cpu().numpy().reshape(-1) - direct.solve(P, f, g)) /
                     np.linalg.norm(direct.solve(P, f, g)))
    finally:
        hh.hh_destroy(h)


def test_grid_barrier_wait_that_runs_out_reports_timeout(hh):
    """The set-up runs no grid barrier; the solve's coarse corrections do."""
    P = Problem(2, N, K)
    f = torch.from_numpy(point_source_rhs(N, 3)).cuda()
    g = torch.zeros((4, P.S), dtype=torch.complex128, device="cuda")
    p = hh.make_params(2, N, K, 2, 2, 6, 4, 1, 1e-12, 50, "fp64", 1)
    h, _ = hh.hh_setup(p)
    try:
        hh.hh_debug_set_wait_limit(0)
        u = torch.empty((P.S, P.S), dtype=torch.complex128, device="cuda")
        with pytest.raises(hh.HHError) as ei:
            hh.hh_solve(h, f, g, u)
        assert ei.value.status == hh.HH_ETIMEOUT
    finally:
        hh.hh_debug_set_wait_limit(-1)
        hh.hh_destroy(h)
    torch.cuda.synchronize()
    assert _solve_ok(hh) < 1e-8


def test_tensor_core_transform_wait_that_runs_out_reports_timeout(hh):
    """Several right-hand sides in the mixed form take the tensor-core transforms."""
    p = hh.make_params(2, N, K, 2, 2, 6, 4, 1, 1e-12, 50, "mixed", 1)
    h, _ = hh.hh_setup(p)
    try:
        info = hh.hh_node_info(h, 3)
        b, Sx = info["rb"] - info["ra"], info["Sx"]
        v = torch.from_numpy(random_complex((b, Sx, 4), 5)).cuda()
        x = torch.empty_like(v)
        hh.hh_debug_set_wait_limit(0)
        with pytest.raises(hh.HHError) as ei:
            hh.hh_leaf_solve(h, 3, v, x, 4)
        assert ei.value.status == hh.HH_ETIMEOUT
    finally:
        hh.hh_debug_set_wait_limit(-1)
        hh.hh_destroy(h)
    torch.cuda.synchronize()
    assert _solve_ok(hh) < 1e-8
