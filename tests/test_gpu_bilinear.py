"""GPU parity for the paper's bilinear (Q1) finite elements (Sec. 3) on the strip hierarchy.

The handle is set up with HH_FLAG_BILINEAR; the oracle is the same O-method on the oracle's
Q1 problem (`Problem(..., scheme="q1")`: consistent masses, mass-weighted load vector).  Every
step goes through the C-ABI, with the tolerances of tests/test_gpu_parity.py:
* operator on every node 1e-14; residual 1e-12;
* FP64 single steps (leaf solve, interface map and adjoint) 1e-11 / 1e-10, coarse operator
  and one ORAS step 1e-8; complex64 leaf solves 1e-4, coarse operator and ORAS step 1e-3;
* full solves against the direct solution u* = A^{-1} b: FP64 1e-10, mixed 1e-8.
The leaf solves cover the one-launch sweep (one column), the line recursions (3 and 10
columns) and the column recursions (20 columns); the bands are ragged (12-14 rows).
"""
import numpy as np
import pytest

from oracle import direct
from oracle.method import OMethod
from oracle.problem import Problem
from workloads import WORKLOADS, point_source_rhs, problem_inputs, random_complex

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SMALL = dict(n=45, k=12.0, levels=2, overlap=2, rank=6, oversample=4, seed=11)


@pytest.fixture(scope="module")
def hh():
    from paper_2512_12538_gb300 import build
    build.build()
    import paper_2512_12538_gb300 as m
    return m


def rel(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()


def host(x):
    torch.cuda.synchronize()
    return x.cpu().numpy()


def make_pair(hh, precision="fp64", **kw):
    cfg = dict(SMALL)
    cfg.update(kw)
    P = Problem(2, cfg["n"], cfg["k"], scheme="q1")
    O = OMethod(P, cfg["levels"], cfg["overlap"], cfg["rank"], cfg["oversample"], seed=cfg["seed"])
    params = hh.make_params(2, cfg["n"], cfg["k"], cfg["levels"], cfg["overlap"], cfg["rank"], cfg["oversample"], 1,
                            1e-13, 400, precision, cfg["seed"], "eigen", flags=hh.HH_FLAG_BILINEAR)
    h, _ = hh.hh_setup(params)
    return P, O, h


def test_operator_every_node(hh):
    P, O, h = make_pair(hh)
    try:
        for nid in range(len(O.tree)):
            nd = O.tree[nid]
            x = random_complex((nd.b, P.Sx, 3), 200 + nid)
            y = torch.empty_like(dev(x))
            hh.hh_apply_operator(h, nid, dev(x), y, 3)
            assert rel(host(y), O.apply(nid, x)) < 1e-14, nid
    finally:
        hh.hh_destroy(h)


def test_residual_and_load_vector(hh):
    P, O, h = make_pair(hh)
    try:
        f = random_complex((P.S, P.S), 3)
        g = random_complex((4, P.S), 4)
        u = random_complex((P.S, P.S), 5)
        b = P.rhs(f, g)
        want = np.linalg.norm(b - P.A() @ u.reshape(-1)) / np.linalg.norm(b)
        got = hh.hh_residual(h, dev(f), dev(g), dev(u))
        assert abs(got - want) <= 1e-12 * want
        us = direct.solve(P, f, g).reshape(P.S, P.S)
        assert hh.hh_residual(h, dev(f), dev(g), dev(us)) < 1e-13
    finally:
        hh.hh_destroy(h)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-4)])
@pytest.mark.parametrize("ncols", [1, 3, 10, 20])
def test_leaf_solve(hh, precision, tol, ncols):
    # the node buffers hold r + p columns: 20 columns need 20 samples
    P, O, h = make_pair(hh, precision, oversample=14 if ncols > 10 else 4)
    try:
        for leaf in (3, 4, 5, 6):
            nd = O.tree[leaf]
            v = random_complex((nd.b, P.Sx, ncols), 7 * leaf + ncols)
            x = torch.empty_like(dev(v))
            hh.hh_leaf_solve(h, leaf, dev(v), x, ncols)
            assert rel(host(x), O.leaf_solve(leaf, v)) < tol, (leaf, ncols)
    finally:
        hh.hh_destroy(h)


@pytest.mark.parametrize("child", [1, 2, 3, 6])
def test_interface_map_and_adjoint(hh, child):
    P, O, h = make_pair(hh)
    try:
        X = random_complex((P.Sx, 4), 31 + child)
        Y = torch.empty_like(dev(X))
        hh.hh_interface_map(h, child, 0, dev(X), Y, 4)
        assert rel(host(Y), O.T(child, X)) < 1e-10
        hh.hh_interface_map(h, child, 1, dev(X), Y, 4)
        assert rel(host(Y), O.T_adjoint(child, X)) < 1e-10
    finally:
        hh.hh_destroy(h)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-8), ("mixed", 1e-3)])
def test_coarse_operator_and_one_oras_step(hh, precision, tol):
    P, O, h = make_pair(hh, precision)
    try:
        for p in (0, 1, 2):
            nd = O.tree[p]
            rr = random_complex((nd.b, P.Sx, 1), 55 + p)
            z = torch.empty_like(dev(rr))
            hh.hh_coarse_apply(h, p, dev(rr), z)
            assert rel(host(z), O.coarse(p, rr)) < tol, p
        rr = random_complex((P.N,), 77)
        z = torch.empty_like(dev(rr))
        hh.hh_precondition(h, dev(rr), z)
        assert rel(host(z), O.precondition(rr)) < tol
    finally:
        hh.hh_destroy(h)


@pytest.mark.parametrize("outer", ["oras", "gmres"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-8)])
def test_solve_against_direct(hh, precision, tol, outer):
    n, k = 45, 12.0
    P = Problem(2, n, k, scheme="q1")
    f = point_source_rhs(n, 9)
    g = random_complex((4, P.S), 10)
    us = direct.solve(P, f, g)
    s = hh.Solver(2, n, k, 2, 2, 6, 4, tol=1e-13, max_iter=500, precision=precision, seed=3, outer=outer,
                  restart=30, flags=hh.HH_FLAG_BILINEAR)
    u, st = s.solve(dev(f), dev(g))
    s.close()
    assert rel(host(u), us) < tol, st


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-8)])
def test_solve_255_k40_two_levels(hh, precision, tol):
    """The 255 x 255 interior grid, k = 40, 4 leaf bands, r = 16, p = 10, with bilinear elements
    (the 66-row bands take the one-launch sweep)."""
    w = WORKLOADS["helm2d_n255_k40_L2"]
    P = Problem(2, w.n, w.k, scheme="q1")
    f, g = problem_inputs(w)
    us = direct.solve(P, f, g)
    s = hh.Solver(2, w.n, w.k, w.levels, w.overlap, w.rank, w.oversample, tol=1e-12, max_iter=300,
                  precision=precision, seed=1, flags=hh.HH_FLAG_BILINEAR)
    u, st = s.solve(dev(f), dev(g))
    s.close()
    err = rel(host(u), us)
    print(f"q1 255^2 {precision}: {st['iters']} steps, err {err:.2e}")
    assert err < tol, (err, st)


def test_batch_entry_solves_bilinear_problems_one_at_a_time(hh):
    # the lockstep engine takes 5-point problems only; hh_solve_batch solves these in turn
    n, k = 45, 12.0
    P = Problem(2, n, k, scheme="q1")
    hs, fs, gs, us, want = [], [], [], [], []
    for i in range(2):
        f = point_source_rhs(n, 40 + i)
        g = np.zeros((4, P.S), dtype=np.complex128)
        want.append(direct.solve(P, f, g))
        p = hh.make_params(2, n, k, 2, 2, 6, 4, 1, 1e-12, 400, "mixed", 3, "eigen", flags=hh.HH_FLAG_BILINEAR)
        hs.append(hh.hh_setup(p)[0])
        fs.append(dev(f))
        gs.append(dev(g))
        us.append(torch.empty_like(fs[-1]))
    try:
        hh.hh_solve_batch(hs, fs, gs, us)
        for u, w in zip(us, want):
            assert rel(host(u), w) < 1e-8
    finally:
        for h in hs:
            hh.hh_destroy(h)
