"""Seeded synthetic inputs for the impedance Helmholtz problem.

The paper's experiments use synthetic data only: a random discrete solution with
f = A u and zero initial guess (Sec. 3.1).  The workloads below follow the same
idea; none needs a dataset.  Every array is complex128 and seeded; the layouts are
the ones the library's C-ABI documents:

* ``f``: ``[S_y][S_x]`` row-major (x fastest); 1D problems use ``[S]``.
* ``g``: ``[4][S]`` impedance data per side, order x=0, x=1, y=0, y=1, each indexed
  along its side; 1D problems use ``[2] = (g0, g1)``.

Grid convention: ``n`` interior nodes per side plus the two impedance boundary
nodes, so ``S = n + 2`` unknowns per side and ``h = 1 / (n + 1)``.

This module contains no part of the solver: only random numbers and the
closed-form inputs (Gaussian sources, plane waves) the tests feed to both sides.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 2512_12538


def random_complex(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Complex array with independent N(0, scale^2) real and imaginary parts."""
    rng = np.random.Generator(np.random.PCG64(seed))
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (scale * (re + 1j * im)).astype(np.complex128)


def point_source_rhs(n: int, seed: int, n_src: int = 8, width_h: float = 2.0) -> np.ndarray:
    """Sum of ``n_src`` Gaussian point sources on the unit square, sampled on the grid.

    f(x) = sum_s a_s exp(-|x - x_s|^2 / (2 sigma^2)) with sigma = width_h * h,
    complex amplitudes a_s with N(0,1) real and imaginary parts and centres x_s
    uniform in (0,1)^2.  Returns ``[S][S]`` complex128 (rows = y).
    """
    S = n + 2
    h = 1.0 / (n + 1)
    rng = np.random.Generator(np.random.PCG64(seed))
    amp = rng.standard_normal(n_src) + 1j * rng.standard_normal(n_src)
    ctr = rng.uniform(0.0, 1.0, size=(n_src, 2))
    sigma = width_h * h
    x = np.arange(S) * h
    f = np.zeros((S, S), dtype=np.complex128)
    for s in range(n_src):
        gx = np.exp(-((x - ctr[s, 0]) ** 2) / (2 * sigma * sigma))
        gy = np.exp(-((x - ctr[s, 1]) ** 2) / (2 * sigma * sigma))
        f += amp[s] * np.outer(gy, gx)
    return f


def layered_wavenumber(n: int, omega: float, c0: float, layers: int = 8, c1: float = 1.0) -> np.ndarray:
    """Wavenumber of each grid row for the layered medium of Sec. 3.3: k(y) = omega / c(y)
    with c alternating c1, c0, c1, ... over `layers` equal layers of y in [0, 1], from
    y = 0 up.  A row inside a layer takes that layer's k.  A row on a layer boundary
    (y_j = l / layers) takes the mean of k^2 over its two layers: its nodal control volume
    straddles both, and the mean keeps the scheme second order there.  Returns S = n + 2
    values."""
    h = 1.0 / (n + 1)
    t = np.arange(n + 2) * h * layers
    kl = omega / np.where(np.arange(layers) % 2 == 0, c1, c0)
    nearest = np.rint(t).astype(int)
    on_boundary = (np.abs(t - nearest) < 1e-9) & (nearest > 0) & (nearest < layers)
    inside = np.minimum(np.floor(t + 1e-9).astype(int), layers - 1)
    k = kl[inside]
    below, above = kl[np.clip(nearest - 1, 0, layers - 1)], kl[np.clip(nearest, 0, layers - 1)]
    return np.where(on_boundary, np.sqrt(0.5 * (below * below + above * above)), k)


def layered_wavenumber_elements(E: int, omega: float, c0: float, layers: int = 8, c1: float = 1.0,
                                first: str = "c1") -> np.ndarray:
    """Wavenumber of each of the E rows of elements (bilinear elements, E per side) for the
    layered medium of Sec. 3.3: k = omega / c(y) with c alternating over `layers` equal
    layers, `first` ("c0" or "c1") at y = 0.  E must be a multiple of `layers`."""
    if E % layers:
        raise ValueError("E must be a multiple of the number of layers")
    layer = np.arange(E) // (E // layers)
    even = c0 if first == "c0" else c1
    odd = c1 if first == "c0" else c0
    return omega / np.where(layer % 2 == 0, even, odd)


def plane_wave_2d(n: int, k: float, theta: float):
    """Continuous plane wave u = exp(i k (cos t x + sin t y)) with matching data.

    Returns (u_exact [S][S], f = 0, g [4][S]) where g = d_n u - i k u on each side
    (outward normals -x, +x, -y, +y).  The discrete solution converges to u at
    second order, which pins the discretisation independently of its derivation.
    """
    S = n + 2
    h = 1.0 / (n + 1)
    x = np.arange(S) * h
    kx, ky = k * math.cos(theta), k * math.sin(theta)
    U = np.exp(1j * (kx * x[None, :] + ky * x[:, None]))
    g = np.zeros((4, S), dtype=np.complex128)
    # side x=0: points (0, y_j); d_n u = -u_x
    g[0] = (-1j * kx - 1j * k) * np.exp(1j * ky * x)
    # side x=1: points (1, y_j); d_n u = +u_x
    g[1] = (1j * kx - 1j * k) * np.exp(1j * (kx + ky * x))
    # side y=0: points (x_i, 0); d_n u = -u_y
    g[2] = (-1j * ky - 1j * k) * np.exp(1j * kx * x)
    # side y=1: points (x_i, 1); d_n u = +u_y
    g[3] = (1j * ky - 1j * k) * np.exp(1j * (kx * x + ky))
    return U, np.zeros((S, S), dtype=np.complex128), g


@dataclasses.dataclass(frozen=True)
class Workload:
    """One named synthetic workload: problem, method parameters and RHS recipe."""

    name: str
    dim: int
    n: int
    k: float
    levels: int
    overlap: int
    rank: int
    oversample: int
    n_inner: int = 1
    rhs: str = "point_sources"      # "point_sources" | "random"

    @property
    def S(self) -> int:
        return self.n + 2

    @property
    def h(self) -> float:
        return 1.0 / (self.n + 1)


WORKLOADS = {
    # 1D, n = 1000 interior points, k = 20 pi, two overlapping subdomains with
    # 4 shared points, a-harmonic coarse space (one vector per subdomain).
    "helm1d_n1000_k20pi": Workload("helm1d_n1000_k20pi", 1, 1000, 20 * math.pi, 1, 4, 1, 0,
                                   rhs="random"),
    # 2D 255x255 interior grid, k = 40, 2-level binary strip hierarchy
    # (4 leaf strips), overlap 2 rows, sketch rank 16 with oversampling 10.
    "helm2d_n255_k40_L2": Workload("helm2d_n255_k40_L2", 2, 255, 40.0, 2, 2, 16, 10),
    # 2D 1023x1023, k = 100, 3-level hierarchy (8 leaf strips), overlap 4 rows,
    # rank 32, oversampling 10.
    "helm2d_n1023_k100_L3": Workload("helm2d_n1023_k100_L3", 2, 1023, 100.0, 3, 4, 32, 10),
}


def problem_inputs(w: Workload, index: int = 0):
    """Seeded (f, g) for workload ``w``; ``index`` selects an independent draw."""
    seed = BASE_SEED + 1000 * index + w.n
    if w.dim == 1:
        f = random_complex((w.S,), seed)
        g = random_complex((2,), seed + 1)
        return f, g
    if w.rhs == "random":
        f = random_complex((w.S, w.S), seed)
    else:
        f = point_source_rhs(w.n, seed)
    g = np.zeros((4, w.S), dtype=np.complex128)
    return f, g


def batch_problems(count: int, seed: int = BASE_SEED + 7, sides=(63, 127, 191, 255), kh=(0.3, 0.6),
                   levels: int = 2, overlap: int = 2, rank: int = 16, oversample: int = 8):
    """The batching-form workload: ``count`` independent 2D problems.

    Grid sides n drawn uniformly from ``sides``, k such that k h is uniform in ``kh``
    (h = 1/(n+1)), a ``levels``-level strip hierarchy, overlap, rank and oversampling as
    given (512 problems with these defaults is the batch configuration).  Each problem
    gets its own seeded point-source right-hand side and zero impedance data.  Returns a
    list of (Workload, f, g).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        n = int(sides[int(rng.integers(len(sides)))])
        k = float(rng.uniform(kh[0], kh[1]) * (n + 1))
        w = Workload(f"batch{i}_n{n}", 2, n, k, levels, overlap, rank, oversample)
        f = point_source_rhs(n, seed + 17 * (i + 1))
        g = np.zeros((4, n + 2), dtype=np.complex128)
        out.append((w, f, g))
    return out
