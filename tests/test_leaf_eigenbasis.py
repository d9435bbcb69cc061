"""Host checks of the numerical claims behind the eigenbasis leaf path (no GPU).

The leaf band operator is block tridiagonal over grid columns with blocks
D_i = w_i K + (cx_i - i kh bx_i) W and L_i = U_{i-1} = -W (Eq. (2)'s subdomain
matrices; K the band's line operator along y, W its row weights).  With the generalised
eigenvectors K V = W V Lambda, V^T W V = I, the block Schur recursion
S_i = D_i - L_i S_{i-1}^{-1} U_i decouples into one scalar recursion per mode.  The
complex64 form's accuracy rests on V staying well conditioned: the transforms
f^ = V^T f and x = V x^ amplify FP32 rounding by about cond(V)^2.

1. cond(V) <= 25 for every band height up to 132 rows and every kh up to 0.8
   (<= 26 up to the path's limit of 136 rows), over the workloads' whole range.
2. The recursion carried out in complex64 on the host (numpy, FP32 products) at the
   full-size leaf shapes stays five times inside the 5e-4 tolerance the GPU leaf-solve
   test uses, and the same steps in complex128 reproduce the sparse direct solve.

K and the band operator come from the oracle's own problem definition (the 1D operator
of a b-node line and the 2D band operator), so a mistake in the decomposition shows up
as a complex128 mismatch.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle.hierarchy import build_tree
from oracle.problem import Problem
from workloads import random_complex


def _pencil(b, kh):
    """K (the line operator of a b-node band at this kh, impedance ends) and the weights."""
    K = Problem(1, b - 2, kh * (b - 1)).A().toarray()
    w = np.ones(b)
    w[0] = w[-1] = 0.5
    lam, V = sla.eig(K, np.diag(w))
    V = V / np.sqrt(np.einsum("ij,i,ij->j", V, w, V))       # V^T W V = I (no conjugation)
    return K, w, lam, V


def test_column_pencil_eigenvectors_stay_well_conditioned():
    worst = {}
    for b in (8, 13, 33, 47, 66, 100, 131, 132, 136):
        for kh in (0.02, 0.05, 0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8):
            K, w, lam, V = _pencil(b, kh)
            assert np.allclose(V.T @ (w[:, None] * V), np.eye(b), atol=1e-9)
            assert np.allclose(K @ V, (w[:, None] * V) * lam[None, :], atol=1e-9)
            worst[b] = max(worst.get(b, 0.0), np.linalg.cond(V))
    assert max(c for b, c in worst.items() if b <= 132) <= 25.0, worst
    assert worst[136] <= 26.0


def _eig_leaf_solve(P, ra, rb, v, dt):
    """x = A~^{-1} v for the band [ra, rb) by the eigenbasis recursion in precision dt."""
    b, S, kh = rb - ra, P.Sx, P.k * P.h
    _, _, lam, V = _pencil(b, kh)
    ends = (np.arange(S) == 0) | (np.arange(S) == S - 1)
    wx = np.where(ends, 0.5, 1.0)
    cx = np.where(ends, 1.0, 2.0)
    Vt, lamt = V.astype(dt), lam.astype(dt)
    fh = Vt.T @ v.reshape(b, S).astype(dt)
    delta = (wx[None, :] * lamt[:, None] + (cx - 1j * kh * ends)[None, :]).astype(dt)
    xi = np.zeros((b, S), dt)
    y = np.zeros((b, S), dt)
    prev = np.zeros(b, dt)
    yp = np.zeros(b, dt)
    for i in range(S):
        xi[:, i] = 1 / (delta[:, i] - prev)
        prev = xi[:, i]
        y[:, i] = xi[:, i] * (fh[:, i] + yp)
        yp = y[:, i]
    x = np.zeros((b, S), dt)
    x[:, S - 1] = y[:, S - 1]
    for i in range(S - 2, -1, -1):
        x[:, i] = y[:, i] + xi[:, i] * x[:, i + 1]
    return (Vt @ x).reshape(-1)


@pytest.mark.parametrize("n,k,levels,overlap", [(255, 40.0, 2, 2), (1023, 100.0, 3, 4)])
def test_complex64_recursion_error_at_full_size_leaf_shapes(n, k, levels, overlap):
    P = Problem(2, n, k)
    leaves = [nd for nd in build_tree(P.S, levels, overlap) if nd.is_leaf]
    for nd in (leaves[0], max(leaves, key=lambda t: t.b)):
        v = random_complex((nd.b * P.Sx,), 5 + nd.id)
        xs = spla.spsolve(P.band_operator(nd.ra, nd.rb).tocsc(), v)
        e64 = np.linalg.norm(_eig_leaf_solve(P, nd.ra, nd.rb, v, np.complex128) - xs) / np.linalg.norm(xs)
        e32 = np.linalg.norm(_eig_leaf_solve(P, nd.ra, nd.rb, v, np.complex64) - xs) / np.linalg.norm(xs)
        assert e64 < 1e-11, e64
        assert e32 < 1e-4, e32


# ---------------------------------------------------------------- bilinear elements
# With the paper's Q1 elements (Sec. 3) the band operator is K_x (x) M + M_x (x) K' in
# column blocks: D_i = (X_ii - i kh bx_i) M + Mx_ii K and L_i = U_{i-1} = -M + K / 6, with
# M the consistent 1D mass of the band and K = X - (kh)^2 M - i kh E.  The same decoupling
# holds with K V = M V Lambda, V^T M V = I: delta_{i,m} = Mx_ii lambda_m + X_ii - i kh bx_i,
# coupling l_m = -1 + lambda_m / 6.  The GPU path runs the 5-point recursions with the
# multiplier a_i = -l xi_i and the input scaled by 1 / (-l); both readings are checked here
# against the oracle's sparse Q1 band solve.

def _q1_pencil(b, kh):
    """K (the 1D Q1 operator of a b-node line: X - (kh)^2 M - i kh E) and the mass M."""
    from oracle.problem import direction
    K = Problem(1, b - 2, kh * (b - 1), scheme="q1").A().toarray()
    M = direction(b, scheme="q1")[1].toarray()
    lam, V = sla.eig(K, M)
    V = V / np.sqrt(np.einsum("ij,ik,kj->j", V, M, V))       # V^T M V = I (no conjugation)
    return K, M, lam, V


def _q1_eig_leaf_solve(P, ra, rb, v, scaled):
    b, S, kh = rb - ra, P.Sx, P.k * P.h
    _, _, lam, V = _q1_pencil(b, kh)
    ends = (np.arange(S) == 0) | (np.arange(S) == S - 1)
    mx = np.where(ends, 2.0 / 6.0, 4.0 / 6.0)
    cx = np.where(ends, 1.0, 2.0)
    nl = 1.0 - lam / 6.0                                        # -l_m
    fh = V.T @ v.reshape(b, S)
    delta = mx[None, :] * lam[:, None] + (cx - 1j * kh * ends)[None, :]
    xi = np.zeros((b, S), complex)
    prev = np.zeros(b, complex)
    for i in range(S):
        xi[:, i] = 1 / (delta[:, i] - nl * nl * prev)
        prev = xi[:, i]
    y = np.zeros((b, S), complex)
    x = np.zeros((b, S), complex)
    if scaled:
        # the GPU form: a = nl xi, f~ = f^ / nl, then the 5-point recursions
        a, ft = nl[:, None] * xi, fh / nl[:, None]
        yp = np.zeros(b, complex)
        for i in range(S):
            y[:, i] = a[:, i] * (ft[:, i] + yp)
            yp = y[:, i]
        x[:, S - 1] = y[:, S - 1]
        for i in range(S - 2, -1, -1):
            x[:, i] = y[:, i] + a[:, i] * x[:, i + 1]
    else:
        yp = np.zeros(b, complex)
        for i in range(S):
            y[:, i] = xi[:, i] * (fh[:, i] + nl * yp)
            yp = y[:, i]
        x[:, S - 1] = y[:, S - 1]
        for i in range(S - 2, -1, -1):
            x[:, i] = y[:, i] + xi[:, i] * nl * x[:, i + 1]
    return (V @ x).reshape(-1)


def test_bilinear_pencil_recursion_reproduces_the_q1_band_solve():
    P = Problem(2, 63, 40.0, scheme="q1")
    for nd in (t for t in build_tree(P.S, 2, 2) if t.is_leaf):
        K, M, lam, V = _q1_pencil(nd.b, P.k * P.h)
        assert np.allclose(V.T @ M @ V, np.eye(nd.b), atol=1e-9)
        v = random_complex((nd.b * P.Sx,), 17 + nd.id)
        xs = spla.spsolve(P.band_operator(nd.ra, nd.rb).tocsc(), v)
        for scaled in (False, True):
            err = np.linalg.norm(_q1_eig_leaf_solve(P, nd.ra, nd.rb, v, scaled) - xs) / np.linalg.norm(xs)
            assert err < 1e-11, (nd.id, scaled, err)


def test_bilinear_pencil_start_values_lie_near_the_spectrum():
    # the GPU's Aberth start values: 6 (1 - cos t) / (2 + cos t) - (kh)^2 (t = j pi / (b - 1)),
    # the real part's spectrum, which the cosine vectors diagonalise exactly
    from oracle.problem import direction
    for b in (9, 34, 66):
        X = direction(b)[0].toarray()
        M = direction(b, scheme="q1")[1].toarray()
        t = np.pi * np.arange(b) / (b - 1)
        mu = np.sort(6 * (1 - np.cos(t)) / (2 + np.cos(t)))
        np.testing.assert_allclose(np.sort(sla.eigvals(X, M).real), mu, atol=1e-10)
