"""Pins of the oracle's discretisation and direct solve (CPU only).

The operator is fixed by the continuous problem (Eq. (1), Sec. 3.1), not by its own
formula: exact plane waves must be reproduced at second order, interior rows must
annihilate the discrete plane wave, the matrix must be complex symmetric, band
operators must agree with A away from their artificial boundaries, and the sparse
direct solve must agree with a dense brute-force solve.
"""
import math

import numpy as np
import pytest

from oracle import direct
from oracle.problem import Problem
from workloads import plane_wave_2d, random_complex


def _err_1d_plane_wave(n, k):
    P = Problem(1, n, k)
    x = np.arange(P.S) * P.h
    # u = e^{ikx}: -u'' - k^2 u = 0, -(u'+iku)(0) = -2ik, (u'-iku)(1) = 0   (Eq. (1))
    u = direct.solve(P, np.zeros(P.S), np.array([-2j * k, 0.0]))
    return np.max(np.abs(u - np.exp(1j * k * x)))


def test_1d_plane_wave_second_order():
    k = 10.0
    e = [_err_1d_plane_wave(n, k) for n in (99, 199, 399)]
    assert e[0] < 0.05
    for a, b in zip(e, e[1:]):
        assert 3.6 < a / b < 4.4, e


def _err_2d_plane_wave(n, k, theta):
    P = Problem(2, n, k)
    U, f, g = plane_wave_2d(n, k, theta)
    u = direct.solve(P, f, g).reshape(P.S, P.S)
    return np.max(np.abs(u - U))


def test_2d_plane_wave_second_order():
    k, th = 6.0, 0.37
    e = [_err_2d_plane_wave(n, k, th) for n in (31, 63, 127)]
    assert e[0] < 0.05
    for a, b in zip(e, e[1:]):
        assert 3.5 < a / b < 4.5, e


def _err_2d_manufactured(n, k):
    # u = cos(pi x) exp(2 y) with f = -Lap u - k^2 u and g = d_n u - i k u per side
    P = Problem(2, n, k)
    x = np.arange(P.S) * P.h
    X, Y = np.meshgrid(x, x)                     # [row=y][col=x]
    U = np.cos(math.pi * X) * np.exp(2 * Y)
    lap = (-(math.pi ** 2) + 4.0) * U
    f = -lap - k * k * U
    ux = lambda xx, yy: -math.pi * np.sin(math.pi * xx) * np.exp(2 * yy)
    uy = lambda xx, yy: 2 * np.cos(math.pi * xx) * np.exp(2 * yy)
    uu = lambda xx, yy: np.cos(math.pi * xx) * np.exp(2 * yy)
    g = np.zeros((4, P.S), dtype=complex)
    g[0] = -ux(0 * x, x) - 1j * k * uu(0 * x, x)
    g[1] = ux(1 + 0 * x, x) - 1j * k * uu(1 + 0 * x, x)
    g[2] = -uy(x, 0 * x) - 1j * k * uu(x, 0 * x)
    g[3] = uy(x, 1 + 0 * x) - 1j * k * uu(x, 1 + 0 * x)
    u = direct.solve(P, f, g).reshape(P.S, P.S)
    return np.max(np.abs(u - U))


def test_2d_manufactured_source_second_order():
    e = [_err_2d_manufactured(n, 3.0) for n in (31, 63, 127)]
    for a, b in zip(e, e[1:]):
        assert 3.5 < a / b < 4.5, e


def test_discrete_plane_wave_annihilated_by_interior_rows():
    n, k = 40, 17.0
    P = Problem(2, n, k)
    kx = 0.6 * k
    # discrete dispersion: (2 - 2cos(kx h)) + (2 - 2cos(ky h)) = (kh)^2
    cy = 1 - ((P.kh ** 2) - (2 - 2 * math.cos(kx * P.h))) / 2
    ky = math.acos(cy) / P.h
    x = np.arange(P.S) * P.h
    U = np.exp(1j * (kx * x[None, :] + ky * x[:, None]))
    r = (P.A() @ U.reshape(-1)).reshape(P.S, P.S)
    assert np.max(np.abs(r[1:-1, 1:-1])) < 1e-12
    assert np.max(np.abs(r[0, :])) > 1e-3          # boundary rows are not zero


def test_operator_complex_symmetric_and_band_rows():
    for dim in (1, 2):
        P = Problem(dim, 20, 9.0)
        A = P.A()
        assert abs(A - A.T).max() == 0.0
        ra, rb = 5, 14
        At = P.band_operator(ra, rb).toarray()
        Ad = A.toarray()
        Sx = P.Sx
        rows = np.arange(ra * Sx, rb * Sx)
        sub = Ad[np.ix_(rows, rows)]
        inner = np.arange(Sx, (rb - ra - 1) * Sx)   # rows away from the artificial boundary
        assert np.array_equal(At[inner], sub[inner])
        # artificial boundary rows differ (halved, with the -i kh impedance term)
        assert not np.allclose(At[:Sx], sub[:Sx])


def test_direct_matches_dense_bruteforce():
    for dim, n in ((1, 48), (2, 13)):
        P = Problem(dim, n, 7.5)
        f = random_complex((P.N,), 11)
        g = random_complex((2,) if dim == 1 else (4, P.S), 12)
        u = direct.solve(P, f, g)
        ud = np.linalg.solve(P.A().toarray(), P.rhs(f, g))
        assert direct.rel_err(u, ud) < 1e-13


def test_rhs_weights_corner():
    P = Problem(2, 5, 3.0)
    f = np.zeros((P.S, P.S), complex)
    f[0, 0] = 1.0
    g = np.zeros((4, P.S), complex)
    g[0, 0] = 2.0        # side x = 0 at y = 0
    g[2, 0] = 4.0        # side y = 0 at x = 0
    b = P.rhs(f, g).reshape(P.S, P.S)
    # corner weights w_i = w_j = 1/2: h^2/4 f + h (g_x/2 + g_y/2)
    assert b[0, 0] == pytest.approx(P.h ** 2 / 4 + P.h * (1.0 + 2.0))
