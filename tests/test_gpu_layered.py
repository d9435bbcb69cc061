"""Layered media on the GPU (Sec. 3.3): k = omega / c(y) varies from grid row to grid row.

The wavenumber of each row enters that row's k^2 term and its impedance terms (the
same reading as the oracle, R16: c alternates c1 = 1 and c0 over 8 equal layers from
y = 0, a row on a layer boundary takes the mean of k^2 of its two layers, omega h = 1).
The library takes it as hh_params.k_rows; 2D leaves then use the explicit-inverse path.
Every step is compared with the oracle's layered operator, and the paper's outer solver
for these problems, GMRES preconditioned by the hierarchical ORAS step, with the
oracle's direct solution.  As in the oracle, the stationary iteration diverges here.
"""
import numpy as np
import pytest

from oracle import direct
from oracle.method import OMethod
from oracle.problem import Problem
from workloads import layered_wavenumber, point_source_rhs, random_complex

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, C0 = 63, 5.0
OMEGA = N + 1.0                          # omega h = 1


@pytest.fixture(scope="module")
def hh():
    from paper_2512_12538_gb300 import build
    build.build()
    import paper_2512_12538_gb300 as m
    return m


@pytest.fixture(scope="module")
def layered():
    kr = layered_wavenumber(N, OMEGA, C0)
    P = Problem(2, N, OMEGA, k_rows=kr)
    O = OMethod(P, 2, 2, 16, 10, seed=1)
    return kr, P, O


def _params(hh, kr, precision, outer="gmres", max_iter=200, tol=1e-12):
    return hh.make_params(2, N, OMEGA, 2, 2, 16, 10, 1, tol, max_iter, precision, 1, "block", outer, 40,
                          k_rows=kr)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a).reshape(-1) - np.asarray(b).reshape(-1)) / np.linalg.norm(b))


def test_layered_operator_on_every_node(hh, layered):
    kr, P, O = layered
    h, _ = hh.hh_setup(_params(hh, kr, "fp64"))
    try:
        for nid in range(len(O.tree)):
            nd = O.tree[nid]
            x = random_complex((nd.b, P.Sx, 2), 50 + nid)
            y = torch.empty((nd.b, P.Sx, 2), dtype=torch.complex128, device="cuda")
            hh.hh_apply_operator(h, nid, torch.from_numpy(x).cuda(), y, 2)
            torch.cuda.synchronize()
            assert _rel(y.cpu().numpy(), O.apply(nid, x)) < 1e-14, nid
    finally:
        hh.hh_destroy(h)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 5e-4)])
def test_layered_leaf_solves_and_interface_maps(hh, layered, precision, tol):
    kr, P, O = layered
    h, _ = hh.hh_setup(_params(hh, kr, precision))
    try:
        for leaf in (3, 4, 5, 6):
            nd = O.tree[leaf]
            v = random_complex((nd.b, P.Sx, 3), leaf)
            x = torch.empty((nd.b, P.Sx, 3), dtype=torch.complex128, device="cuda")
            hh.hh_leaf_solve(h, leaf, torch.from_numpy(v).cuda(), x, 3)
            torch.cuda.synchronize()
            assert _rel(x.cpu().numpy(), O.leaf_solve(leaf, v)) < tol, leaf
        if precision == "fp64":
            for c in (1, 2, 3, 6):
                X = random_complex((P.Sx, 4), 70 + c)
                Y = torch.empty((P.Sx, 4), dtype=torch.complex128, device="cuda")
                hh.hh_interface_map(h, c, 0, torch.from_numpy(X).cuda(), Y, 4)
                torch.cuda.synchronize()
                assert _rel(Y.cpu().numpy(), O.T(c, X)) < 1e-10, c
    finally:
        hh.hh_destroy(h)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-8)])
def test_layered_gmres_solve_matches_the_direct_solution(hh, layered, precision, tol):
    kr, P, O = layered
    f = point_source_rhs(N, 17)
    g = np.zeros((4, P.S), dtype=np.complex128)
    us = direct.solve(P, f, g)
    h, _ = hh.hh_setup(_params(hh, kr, precision))
    try:
        u = torch.empty((P.S, P.S), dtype=torch.complex128, device="cuda")
        st = hh.hh_solve(h, torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), u)
        err = _rel(u.cpu().numpy(), us)
        print(f"layered {precision}: GMRES steps {st.iters}, residual {st.rel_res:.2e}, err {err:.2e}")
        assert err < tol
    finally:
        hh.hh_destroy(h)


def test_layered_stationary_iteration_diverges_as_in_the_oracle(hh, layered):
    kr, P, O = layered
    f = random_complex((P.S, P.S), 17)
    g = np.zeros((4, P.S), dtype=np.complex128)
    h, _ = hh.hh_setup(_params(hh, kr, "fp64", outer="oras", max_iter=12, tol=1e-8))
    try:
        u = torch.empty((P.S, P.S), dtype=torch.complex128, device="cuda")
        st = hh.hh_solve(h, torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), u, allow_noconv=True)
    finally:
        hh.hh_destroy(h)
    _, _, hist = O.solve(P.rhs(f, g), tol=1e-8, maxit=12)
    print(f"stationary after 12 steps: GPU {st.rel_res:.3e}, oracle {hist[-1]:.3e}")
    assert st.rel_res > 10.0 and hist[-1] > 10.0
    assert abs(st.rel_res - hist[-1]) <= 1e-4 * hist[-1]
