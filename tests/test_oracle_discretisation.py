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
from workloads import layered_wavenumber, plane_wave_2d, random_complex


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


# ------------------------------------------------------- layered media (Sec. 3.3)
def test_constant_row_wavenumbers_give_the_scalar_operator_bit_for_bit():
    for dim in (1, 2):
        P = Problem(dim, 30, 7.0)
        Q = Problem(dim, 30, 7.0, k_rows=np.full(32, 7.0))
        assert abs(P.A() - Q.A()).max() == 0.0
        assert abs(P.band_operator(4, 17) - Q.band_operator(4, 17)).max() == 0.0


def _err_two_layers(n, k1=20.0, k2=8.0):
    """1D, c = 1 on (0, 1/2) and c0 = k1 / k2 on (1/2, 1): an incoming wave from y = 0
    is partly reflected and transmitted.  With u and u' continuous at 1/2 the exact
    solution is e^{i k1 y} + R e^{-i k1 y} below and T e^{i k2 (y - 1/2)} above, with
    R = e^{i k1} (k1 - k2) / (k1 + k2) and T = e^{i k1 / 2} 2 k1 / (k1 + k2)."""
    P = Problem(1, n, k1, k_rows=layered_wavenumber(n, k1, k1 / k2, layers=2))
    y = np.arange(P.S) * P.h
    R = np.exp(1j * k1) * (k1 - k2) / (k1 + k2)
    T = np.exp(0.5j * k1) * 2 * k1 / (k1 + k2)
    U = np.where(y <= 0.5, np.exp(1j * k1 * y) + R * np.exp(-1j * k1 * y), T * np.exp(1j * k2 * (y - 0.5)))
    u = direct.solve(P, np.zeros(P.S), np.array([-2j * k1, 0.0]))
    return np.max(np.abs(u - U))


@pytest.mark.parametrize("ns", [(99, 199, 399), (100, 200, 400)], ids=["interface_on_a_node", "between_nodes"])
def test_two_layer_transmission_second_order(ns):
    """Second order whether the interface falls on a node (that row takes the mean of k^2
    over its two layers) or midway between two.  A wavenumber profile shifted by a row,
    or one-sided at an interface node, converges at first order only."""
    e = [_err_two_layers(n) for n in ns]
    assert e[0] < 0.05
    for a, b in zip(e, e[1:]):
        assert 3.6 < a / b < 4.4, e


def _err_2d_variable_k(n, k0=6.0, a=4.0, b=-3.0):
    """u = e^{i(a x + b y)} with k(y) = k0 (1 + 0.3 sin 2 pi y): f = (a^2 + b^2 - k(y)^2) u,
    g = d_n u - i k u on each side with the local k."""
    h = 1.0 / (n + 1)
    x = np.arange(n + 2) * h
    ky = k0 * (1 + 0.3 * np.sin(2 * math.pi * x))
    P = Problem(2, n, k0, k_rows=ky)
    X, Y = np.meshgrid(x, x)                     # [row=y][col=x]
    U = np.exp(1j * (a * X + b * Y))
    f = (a * a + b * b - ky[:, None] ** 2) * U
    g = np.zeros((4, P.S), dtype=complex)
    g[0] = (-1j * a - 1j * ky) * U[:, 0]        # x = 0, along y
    g[1] = (1j * a - 1j * ky) * U[:, -1]        # x = 1, along y
    g[2] = (-1j * b - 1j * ky[0]) * U[0, :]     # y = 0, along x
    g[3] = (1j * b - 1j * ky[-1]) * U[-1, :]    # y = 1, along x
    u = direct.solve(P, f, g).reshape(P.S, P.S)
    return np.max(np.abs(u - U))


def test_2d_variable_wavenumber_manufactured_second_order():
    e = [_err_2d_variable_k(n) for n in (31, 63, 127)]
    assert e[0] < 0.05
    for a, b in zip(e, e[1:]):
        assert 3.5 < a / b < 4.5, e


def test_layered_operator_complex_symmetric_and_band_rows():
    """Each band operator carries its own rows' wavenumbers: away from its artificial
    boundary it equals A on those rows (a band reading another band's k would not)."""
    n = 30
    P = Problem(2, n, n + 1.0, k_rows=layered_wavenumber(n, n + 1.0, 5.0))   # omega h = 1
    A = P.A()
    assert abs(A - A.T).max() == 0.0
    Ad = A.toarray()
    for ra, rb in ((3, 12), (9, 25), (20, 32)):
        At = P.band_operator(ra, rb).toarray()
        rows = np.arange(ra * P.Sx, rb * P.Sx)
        inner = np.arange(P.Sx, (rb - ra - 1) * P.Sx)
        assert np.array_equal(At[inner], Ad[np.ix_(rows, rows)][inner]), (ra, rb)


# ------------------------------------------------- Q1 bilinear elements (Sec. 3, row f2)
def test_q1_plane_waves_second_order():
    def e1(n, k=10.0):
        P = Problem(1, n, k, scheme="q1")
        x = np.arange(P.S) * P.h
        u = direct.solve(P, np.zeros(P.S), np.array([-2j * k, 0.0]))
        return np.max(np.abs(u - np.exp(1j * k * x)))

    def e2(n, k=6.0, th=0.37):
        P = Problem(2, n, k, scheme="q1")
        U, f, g = plane_wave_2d(n, k, th)
        return np.max(np.abs(direct.solve(P, f, g).reshape(P.S, P.S) - U))

    for e in ([e1(n) for n in (99, 199, 399)], [e2(n) for n in (31, 63, 127)]):
        assert e[0] < 0.05
        for a, b in zip(e, e[1:]):
            assert 3.6 < a / b < 4.4, e


def test_q1_discrete_plane_wave_annihilated_by_interior_rows():
    """Bilinear-element dispersion (Ihlenburg and Babuska): e^{i(tx i + ty j)} solves the
    interior rows when a (4 + 2 cy) / 6 + px (2 - 2 cy) = (kh)^2 px (4 + 2 cy) / 6 with
    a = 2 - 2 cos tx, px = (4 + 2 cos tx) / 6, cy = cos ty.  A wrong mass or stiffness
    entry breaks it; the FD relation does not satisfy it."""
    n, k = 40, 17.0
    P = Problem(2, n, k, scheme="q1")
    kh = k * P.h
    tx = 0.6 * kh
    a, px = 2 - 2 * math.cos(tx), (4 + 2 * math.cos(tx)) / 6
    c0 = a * 4 / 6 + 2 * px - kh * kh * px * 4 / 6
    c1 = a * 2 / 6 - 2 * px - kh * kh * px * 2 / 6
    ty = math.acos(-c0 / c1)
    j = np.arange(P.S)
    U = np.exp(1j * (tx * j[None, :] + ty * j[:, None]))
    r = (P.A() @ U.reshape(-1)).reshape(P.S, P.S)
    assert np.max(np.abs(r[1:-1, 1:-1])) < 1e-12
    r_fd = (Problem(2, n, k).A() @ U.reshape(-1)).reshape(P.S, P.S)
    assert np.max(np.abs(r_fd[1:-1, 1:-1])) > 1e-4


def test_q1_with_lumped_masses_is_the_fd_operator():
    """Replacing each consistent 1D mass matrix by the diagonal of its row sums (mass
    lumping) turns the Q1 operator into the weighted 5-point operator."""
    from oracle.problem import direction, operator
    for dim, n in ((1, 30), (2, 20)):
        P, Q = Problem(dim, n, 9.0, scheme="q1"), Problem(dim, n, 9.0)

        def lump(d):
            X, w, b = d
            return (X, np.asarray(w.sum(axis=1)).reshape(-1), b) if hasattr(w, "tocsr") else d
        A_lumped = operator(P.kh, lump(P._xdir), lump(direction(P.Sy, scheme="q1")))
        assert abs(A_lumped - Q.A()).max() < 1e-15


def test_q1_operator_complex_symmetric_and_band_rows():
    for dim in (1, 2):
        P = Problem(dim, 20, 9.0, scheme="q1")
        A = P.A()
        assert abs(A - A.T).max() == 0.0
        ra, rb = 5, 14
        At = P.band_operator(ra, rb).toarray()
        rows = np.arange(ra * P.Sx, rb * P.Sx)
        inner = np.arange(P.Sx, (rb - ra - 1) * P.Sx)
        assert np.array_equal(At[inner], A.toarray()[np.ix_(rows, rows)][inner])


def test_layered_wavenumber_profile():
    """c alternates 1, c0, 1, ... from y = 0 over equal layers; a row on a layer boundary
    takes the mean of k^2 over its two layers; the top row belongs to the last layer."""
    omega, c0 = 32.0, 5.0
    k = layered_wavenumber(31, omega, c0)          # h = 1/32: four rows per layer
    kb = math.sqrt(0.5 * (omega ** 2 + (omega / c0) ** 2))
    assert k.shape == (33,)
    for j in range(33):
        if j % 4 == 0 and 0 < j < 32:
            assert k[j] == pytest.approx(kb, rel=1e-15), j
        else:
            layer = min(j // 4, 7)
            assert k[j] == (omega if layer % 2 == 0 else omega / c0), j
    # rows that miss the layer boundaries take their layer's value only
    k2 = layered_wavenumber(40, 41.0, 2.0)           # h = 1/41: no row on a boundary
    assert set(np.round(k2, 12)) == {41.0, 20.5}
    # y_j = j h rounds below the boundary for some n; the profile still sees the boundary
    k3 = layered_wavenumber(39, 40.0, 3.0)           # h = 1/40: rows 5, 10, ... on boundaries
    assert all(k3[j] == pytest.approx(math.sqrt(0.5 * (40.0 ** 2 + (40.0 / 3) ** 2))) for j in range(5, 40, 5))
