"""Pins of the oracle's 2 x 2 box hierarchy (row f2, CPU only).

The facts checked are those the strip method is pinned by, restated on boxes:

* layout: the four children's owned rectangles partition the parent's owned rectangle;
  the parts they own inside the parent's region partition that region; an interior
  child's interface is an L through the cross point;
* T1 (Sec. 1): with full interface spaces and exact sub-solves one coarse-corrected step
  is exact, for the FD scheme and for the paper's Q1 elements;
* T2 (Sec. 3.1 discussion): without coarse correction one hierarchical step equals one
  step of the flat leaf partition;
* T6/T7 (Sec. 2): <T x, y> = <x, T^* y> for leaf children; the randomised SVD equals the
  dense SVD of the explicit interface map when the samples cover;
* with partial ranks, GMRES on the preconditioned system reaches A^{-1} b;
* Table 1 (Sec. 3.1), m = 2: the printed GMRES counts, coarse-free and with coarse
  modes, are reproduced to within one iteration on the paper's own setting
  (`tests/golden/table1_free_space_m2.txt`);
* Table 3 (Sec. 3.3), layered media, m = 2: 15 of the 16 printed counts within one
  iteration and all within two (`tests/golden/table3_layered_c5_m2.txt`);
* Table 4 (Sec. 3.3), layered media with 2 and 3 levels: every coarse-corrected count
  within one iteration (`tests/golden/table4_layered_hierarchical.txt`);
* Table 2 (Sec. 3.1), the hierarchical decomposition with 2 and 3 levels: every
  coarse-corrected count within one iteration (`tests/golden/table2_hierarchical_free_space.txt`).
"""
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import direct
from oracle.boxes import BoxMethod, build_boxes, interface_nodes, owned_in_parent
from oracle.problem import Problem
from workloads import layered_wavenumber_elements, point_source_rhs, random_complex


def test_box_layout_partitions_and_interfaces():
    S, e = 62, 2
    nodes = build_boxes(S, 2, 2 * e)
    assert len(nodes) == 1 + 4 + 16
    for p in nodes.values():
        if p.is_leaf:
            continue
        owned = np.zeros((S, S), int)
        in_region = np.zeros((S, S), int)
        for cid in p.children:
            c = nodes[cid]
            owned[c.oy[0]:c.oy[1], c.ox[0]:c.ox[1]] += 1
            (x0, x1), (y0, y1) = owned_in_parent(nodes, c)
            in_region[y0:y1, x0:x1] += 1
            assert c.gx == (max(0, c.ox[0] - e), min(S, c.ox[1] + e))
            assert c.gy == (max(0, c.oy[0] - e), min(S, c.oy[1] + e))
        assert np.all(owned[p.oy[0]:p.oy[1], p.ox[0]:p.ox[1]] == 1) and owned.sum() == (
            (p.oy[1] - p.oy[0]) * (p.ox[1] - p.ox[0]))
        assert np.all(in_region[p.gy[0]:p.gy[1], p.gx[0]:p.gx[1]] == 1) and in_region.sum() == (
            (p.gy[1] - p.gy[0]) * (p.gx[1] - p.gx[0]))
    # a first-level child meets its siblings along one x side and one y side: an L
    c = nodes[1]
    assert interface_nodes(nodes, c).size == c.nx + c.ny - 1
    # a second-level child inside the grid has siblings on two sides only as well
    assert interface_nodes(nodes, nodes[4 * 4 + 1]).size == nodes[17].nx + nodes[17].ny - 1


@pytest.mark.parametrize("scheme", ["fd", "q1"])
@pytest.mark.parametrize("levels,n", [(1, 26), (2, 46)])
def test_T1_boxes_full_interface_space_one_step_exact(scheme, levels, n):
    P = Problem(2, n, 11.0, scheme=scheme)
    f = random_complex((P.S, P.S), 5)
    g = random_complex((4, P.S), 6)
    M = BoxMethod(P, levels, 2, 10 ** 6, 0, seed=9, exact_subsolves=True)   # rank clamps to |Gamma_c|
    assert direct.rel_err(M.precondition(P.rhs(f, g)), direct.solve(P, f, g)) < 1e-10


@pytest.mark.parametrize("levels,n", [(1, 30), (2, 60)])
def test_T2_boxes_hierarchical_equals_flat_without_coarse(levels, n):
    P = Problem(2, n, 13.0)
    M = BoxMethod(P, levels, 2, 0, 0)
    r = random_complex((P.N,), 21)
    R = r.reshape(P.S, P.S)
    u = np.zeros_like(R)
    for nd in M.nodes.values():
        if nd.is_leaf:
            x = spla.spsolve(M.Atil[nd.id].tocsc(), R[nd.gy[0]:nd.gy[1], nd.gx[0]:nd.gx[1]].reshape(-1))
            x = x.reshape(nd.ny, nd.nx)
            u[nd.oy[0]:nd.oy[1], nd.ox[0]:nd.ox[1]] = \
                x[nd.oy[0] - nd.gy[0]:nd.oy[1] - nd.gy[0], nd.ox[0] - nd.gx[0]:nd.ox[1] - nd.gx[0]]
    assert np.linalg.norm(M.precondition(r) - u.reshape(-1)) <= 1e-13 * np.linalg.norm(u)


def test_T7_boxes_adjoint_identity_for_leaf_children():
    P = Problem(2, 46, 9.0)
    M = BoxMethod(P, 2, 2, 6, 4, seed=12)
    for c in (5, 8, 13, 20):
        assert M.nodes[c].is_leaf
        x = random_complex((M.Gamma[c].size, 2), 3 + c)
        y = random_complex((sum(M.Gamma[s].size for s in M.siblings(c)), 2), 7 + c)
        lhs, rhs = np.vdot(y, M.T(c, x)), np.vdot(M.T_adjoint(c, y), x)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs), c


def test_T6_boxes_rsvd_equals_dense_svd_when_samples_cover():
    P = Problem(2, 26, 9.0)
    M = BoxMethod(P, 1, 2, 10 ** 6, 0, seed=12)
    for c in M.nodes[0].children:
        s_dense = np.linalg.svd(M.T(c, np.eye(M.Gamma[c].size, dtype=complex)), compute_uv=False)
        np.testing.assert_allclose(M.sigma[c], s_dense, rtol=1e-11, atol=1e-13 * s_dense[0])


@pytest.mark.parametrize("levels", [1, 2])
def test_boxes_gmres_with_partial_ranks_reaches_the_solution(levels):
    n = 62
    P = Problem(2, n, 20.0)
    f, g = point_source_rhs(n, 3), np.zeros((4, P.S), complex)
    M = BoxMethod(P, levels, 4, 12, 5, seed=1)
    u, steps, hist = M.solve_gmres(P.rhs(f, g), tol=1e-10, restart=40, maxit=200)
    assert hist[-1] < 1e-10 and steps < 60
    assert direct.rel_err(u, direct.solve(P, f, g)) < 1e-8


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table1_free_space_m2.txt")


def _table1_rows(path=GOLDEN):
    rows = []
    with open(path) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                n, nc, it = (int(t) for t in line.split())
                rows.append((n, nc, it))
    return rows


def test_table1_m2_gmres_counts_reproduced():
    """Q1 elements, element-based 2 x 2 partition extended by two elements (delta = 4h),
    k = 2n with (2n)^2 elements, rank n_c with 5 extra samples, a random discrete
    solution u with f = A u, zero start, GMRES to relative residual 1e-5."""
    rows = _table1_rows()
    assert len(rows) == 16
    got = {}
    for n in sorted({r[0] for r in rows}):
        E = 2 * n
        P = Problem(2, E - 1, float(E), scheme="q1")
        b = P.A() @ random_complex((P.N,), 100 + n)
        for _, nc, _ in (r for r in rows if r[0] == n):
            M = BoxMethod(P, 1, 4, nc, 5, seed=1, partition="elements")
            got[(n, nc)] = M.solve_gmres(b, tol=1e-5, restart=500, maxit=500)[1]
    diffs = {(n, nc): got[(n, nc)] - it for n, nc, it in rows}
    assert all(abs(d) <= 1 for d in diffs.values()), diffs
    # the least n_c the paper lists for three iterations gives three here too
    assert all(got[(n, nc)] == 3 for n, nc, it in rows if it == 3), got
    # and one coarse mode at n = 8 is worse than none, as printed (9 against 7)
    assert got[(8, 1)] > got[(8, 0)]


def test_table3_layered_m2_gmres_counts_reproduced():
    """As Table 1, in the layered medium of Sec. 3.3: c = 1 and c0 = 5 alternating over 8
    equal layers of element rows, c = 1 at y = 0 (the order is not stated; this one fits
    Tables 3 and 4 better), omega = 2n so that k_max h = 1."""
    rows = _table1_rows(os.path.join(os.path.dirname(GOLDEN), "table3_layered_c5_m2.txt"))
    assert len(rows) == 16
    got = {}
    for n in sorted({r[0] for r in rows}):
        E = 2 * n
        omega = float(E)
        P = Problem(2, E - 1, omega, scheme="q1", k_elems=layered_wavenumber_elements(E, omega, 5.0))
        b = P.A() @ random_complex((P.N,), 100 + n)
        for _, nc, _ in (r for r in rows if r[0] == n):
            M = BoxMethod(P, 1, 4, nc, 5, seed=1, partition="elements")
            got[(n, nc)] = M.solve_gmres(b, tol=1e-5, restart=500, maxit=500)[1]
    diffs = [got[(n, nc)] - it for n, nc, it in rows]
    assert max(abs(d) for d in diffs) <= 2, diffs
    assert sum(abs(d) <= 1 for d in diffs) >= 15, diffs


def test_table4_layered_hierarchical_gmres_counts_reproduced():
    """Layered medium with l levels of 2 x 2 boxes (omega = n 2^l), n_c modes at the
    finest level doubling at each coarser level (as in Table 2), n_i = 1."""
    path = os.path.join(os.path.dirname(GOLDEN), "table4_layered_hierarchical.txt")
    rows = []
    with open(path) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append(tuple(int(t) for t in line.split()))
    assert len(rows) == 12
    for n, L, nc, it in rows:
        E = n * 2 ** L
        omega = float(E)
        P = Problem(2, E - 1, omega, scheme="q1", k_elems=layered_wavenumber_elements(E, omega, 5.0))
        b = P.A() @ random_complex((P.N,), 100 + n)
        M = BoxMethod(P, L, 4, [nc * 2 ** (L - j) for j in range(1, L + 1)], 5, seed=1, partition="elements")
        got = M.solve_gmres(b, tol=1e-5, restart=500, maxit=500)[1]
        # coarse-corrected counts within one; the coarse-free ones (19 to 60) within 10%
        assert abs(got - it) <= (1 if nc > 0 else max(2, round(0.1 * it))), (n, L, nc, got, it)


def test_table2_hierarchical_gmres_counts_reproduced():
    """l levels of 2 x 2 boxes, k = n 2^l, n_c modes at the finest level doubling at each
    coarser level, n_i = 1 (the sub-level solves are one coarse-corrected step)."""
    path = os.path.join(os.path.dirname(GOLDEN), "table2_hierarchical_free_space.txt")
    rows = []
    with open(path) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append(tuple(int(t) for t in line.split()))
    assert len(rows) == 12
    diffs = []
    for n, L, nc, it in rows:
        E = n * 2 ** L
        P = Problem(2, E - 1, float(E), scheme="q1")
        b = P.A() @ random_complex((P.N,), 100 + n)
        M = BoxMethod(P, L, 4, [nc * 2 ** (L - j) for j in range(1, L + 1)], 5, seed=1, partition="elements")
        got = M.solve_gmres(b, tol=1e-5, restart=500, maxit=500)[1]
        diffs.append((n, L, nc, got - it))
        if it == 3:
            assert got == 3, (n, L, nc, got)
    assert all(abs(d) <= (1 if nc > 0 else 2) for n, L, nc, d in diffs), diffs
