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
