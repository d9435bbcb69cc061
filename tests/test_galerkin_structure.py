"""The operator structure that the Hermitian-packed FP64 Galerkin matrices rely on (CPU only).

A_c = C^H A~ C (Sec. 1) is formed on the GPU from its upper triangle and the impedance
terms alone.  That is exact when A~ = S + i D with S real symmetric and D real diagonal,
since then C^H S C and C^H D C are Hermitian and, for i < j,
    A_c[j][i] = conj(A_c[i][j]) + 2i conj(H_D[i][j]),   H_D = C^H D C.
These tests pin that structure on the oracle's band operators (Sec. 3.1 rows, one k and
layered k, Sec. 3.3) and the identity itself on random bases. The bilinear elements'
impedance terms couple boundary neighbours (edge masses), so their D is not diagonal: those
bands keep the full-matrix Galerkin kernel.
"""
import numpy as np
import pytest

from oracle.problem import Problem
from workloads import layered_wavenumber, random_complex


def _band(P, ra, rb):
    A = P.band_operator(ra, rb).toarray()
    return A, rb - ra


def _boundary_mask(b, Sx):
    j, i = np.meshgrid(np.arange(b), np.arange(Sx), indexing="ij")
    on = (j == 0) | (j == b - 1)
    if Sx > 1:
        on |= (i == 0) | (i == Sx - 1)
    return on.reshape(-1)


@pytest.mark.parametrize("case", ["2d", "2d_layered", "1d"])
def test_fd_band_is_real_symmetric_plus_boundary_diagonal(case):
    if case == "1d":
        P = Problem(1, 40, 9.0)
    elif case == "2d":
        P = Problem(2, 23, 14.0)
    else:
        P = Problem(2, 31, 14.0, k_rows=layered_wavenumber(31, 14.0, 5.0))
    for ra, rb in ((0, P.Sy), (3, 11), (7, 9)):
        A, b = _band(P, ra, rb)
        S, D = A.real, A.imag
        assert np.array_equal(S, S.T)
        assert np.count_nonzero(D - np.diag(np.diag(D))) == 0
        # the impedance terms sit exactly on the band's boundary points (rows 0 and b - 1,
        # the first and last column), 2 Sx + 2 (b - 2) of them in 2D
        support = np.diag(D) != 0
        assert np.array_equal(support, _boundary_mask(b, P.Sx))
        want = P.Sx if b == 1 else 2 * P.Sx + (2 * (b - 2) if P.Sx > 1 else 0)
        assert support.sum() == want


def test_packed_galerkin_identity_reconstructs_A_c():
    P = Problem(2, 23, 14.0)
    A, b = _band(P, 4, 15)
    n, p = A.shape[0], 10
    C = random_complex((n, p), 5)
    Ac = C.conj().T @ A @ C
    HD = C.conj().T @ np.diag(np.diag(A.imag)) @ C
    R = np.triu(Ac).astype(np.complex128)
    for i in range(p):
        for j in range(i + 1, p):
            R[j, i] = np.conj(R[i, j]) + 2j * np.conj(HD[i, j])
    assert np.max(np.abs(R - Ac)) <= 1e-13 * np.max(np.abs(Ac))
    # and the packing would be wrong without the impedance term: A_c is not Hermitian
    assert np.max(np.abs(Ac - Ac.conj().T)) > 1e-3 * np.max(np.abs(Ac))


def test_bilinear_impedance_terms_are_not_diagonal():
    P = Problem(2, 23, 14.0, scheme="q1")
    A, _ = _band(P, 4, 15)
    D = A.imag
    assert np.count_nonzero(D - np.diag(np.diag(D))) > 0
