"""Discrete impedance Helmholtz problem (oracle side; test infrastructure only).

Continuous problem: -Delta u - k^2 u = f with d_n u - i k u = g on the boundary
(Eq. (1) in 1D, Sec. 3.1 in 2D).  The paper discretises with Q1 finite elements;
this build uses second-order finite differences on nodes x_i = i h, i = 0..S-1,
h = 1/(n+1), S = n+2, with the impedance condition imposed through a ghost node
eliminated by the centred difference of d_n u, and every row scaled by h^2 times
the nodal weights w_i w_j (w = 1/2 on boundary nodes, 1 inside).  The scaling keeps
the matrix complex symmetric (A = A^T), which the adjoint solves rely on.

Row (i, j) (i along x, j along y):

    (A u)_ij = w_j X_i(u_.j) + w_i Y_j(u_i.) - (k_j h)^2 w_i w_j u_ij
               - i k_j h (w_j bx_i + w_i by_j) u_ij
    b_ij     = h^2 w_i w_j f_ij + h (w_j gx_ij + w_i gy_ij)

k_j is the wavenumber of grid row j: the constant k, or, for the layered media of
Sec. 3.3 (k = omega / c(y), piecewise constant in y), its value at y_j.  It enters
only the diagonal, so A stays complex symmetric.

X is the second difference along x (2u_i - u_{i-1} - u_{i+1} inside, u_0 - u_1 and
u_{S-1} - u_{S-2} at the ends), bx_i flags the two x-boundary nodes, and gx is the
impedance datum of the x-side the node lies on; Y, by, gy likewise along y.  A 1D
problem is the same formula with the x-direction absent (X = 0, w_x = 1, bx = 0).

A subdomain operator A~_i (Eq. (2)) is the same formula on a band of rows
[ra, rb): its first and last rows take the boundary treatment with zero impedance
data, i.e. -(u' + iku) = 0 and (u' - iku) = 0 on the artificial boundary (Sec. 1).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def direction(n: int, present: bool = True, scheme: str = "fd"):
    """Line operator pieces for one direction of ``n`` nodes: (X, w, boundary flags).

    X is the (halved-at-the-ends) second difference, w the nodal weights and the
    flags mark the two end nodes.  An absent direction (1D problems) contributes
    X = 0, w = 1 and no boundary term.

    scheme "q1" (the bilinear elements of Sec. 3): X is the same (h times the 1D
    stiffness matrix) and w becomes the consistent 1D mass matrix over h,
    tridiag(1, 4, 1) / 6 with 2/6 at the two ends.  Its row sums are the FD weights:
    the FD scheme is Q1 with lumped masses.
    """
    if not present:
        return sp.csr_matrix((1, 1), dtype=np.float64), np.ones(1), np.zeros(1)
    if n < 2:
        raise ValueError("a present direction needs at least two nodes")
    main = np.full(n, 2.0)
    main[0] = main[-1] = 1.0
    off = -np.ones(n - 1)
    X = sp.diags([off, main, off], [-1, 0, 1], format="csr")
    bnd = np.zeros(n)
    bnd[0] = bnd[-1] = 1.0
    if scheme == "q1":
        d = np.full(n, 4.0 / 6.0)
        d[0] = d[-1] = 2.0 / 6.0
        o = np.full(n - 1, 1.0 / 6.0)
        return X, sp.diags([o, d, o], [-1, 0, 1], format="csr"), bnd
    if scheme != "fd":
        raise ValueError("scheme must be 'fd' or 'q1'")
    w = np.ones(n)
    w[0] = w[-1] = 0.5
    return X, w, bnd


def operator(kh, xdir, ydir) -> sp.csr_matrix:
    """Assemble the weighted 5-point operator for a rectangle of nodes.

    kh is k h, one value or one per y node (row).  Unknowns are ordered row-major,
    index = j * Sx + i (x fastest), so Kronecker products read kron(y-part, x-part).
    """
    Xx, wx, bx = xdir
    Yy, wy, by = ydir
    if sp.issparse(wy):
        # Q1: consistent masses; the element wavenumber is one constant
        khs = np.unique(np.asarray(kh, dtype=np.float64))
        if khs.size != 1:
            raise ValueError("the Q1 scheme takes one constant wavenumber")
        q = float(khs[0])
        Wx = wx if sp.issparse(wx) else sp.diags(wx)
        A = (sp.kron(wy, Xx) + sp.kron(Yy, Wx)
             - (q * q) * sp.kron(wy, Wx)
             - 1j * q * (sp.kron(wy, sp.diags(bx)) + sp.kron(sp.diags(by), Wx)))
        return sp.csr_matrix(A, dtype=np.complex128)
    khy = np.broadcast_to(np.asarray(kh, dtype=np.float64), wy.shape)
    Wx, Wy = sp.diags(wx), sp.diags(wy)
    # the weights are 1/2 or 1 and the flags 0 or 1, so with a constant kh every entry
    # equals (kh kh) w_j w_i and kh (w_j bx_i + by_j w_i) to the last bit
    A = (sp.kron(Wy, Xx) + sp.kron(Yy, Wx)
         - sp.kron(sp.diags(wy * (khy * khy)), Wx)
         - 1j * (sp.kron(sp.diags(wy * khy), sp.diags(bx)) + sp.kron(sp.diags(by * khy), Wx)))
    return sp.csr_matrix(A, dtype=np.complex128)


def weighted_mass_q1(w_elem: np.ndarray) -> sp.csr_matrix:
    """The 1D Q1 mass matrix over h with a weight per element, sum_e w_e [2 1; 1 2] / 6
    assembled over the nodes (constant weights give w times the consistent mass)."""
    w_elem = np.asarray(w_elem, dtype=np.float64)
    n = w_elem.size + 1
    d = np.zeros(n)
    d[:-1] += 2.0 * w_elem / 6.0
    d[1:] += 2.0 * w_elem / 6.0
    o = w_elem / 6.0
    return sp.diags([o, d, o], [-1, 0, 1], format="csr")


def operator_q1_layered(kh_elem, xdir) -> sp.csr_matrix:
    """Q1 operator on a rectangle whose wavenumber is constant on each row of elements
    (layered media, Sec. 3.3): kh_elem holds k h for the ny - 1 element rows.  The k^2
    mass term and the impedance edge masses on the x sides take the element weights; the
    impedance rows on the y sides take the wavenumber of their adjacent element row."""
    Xx, wx, bx = xdir
    kh_elem = np.asarray(kh_elem, dtype=np.float64)
    Yy, My, by = direction(kh_elem.size + 1, scheme="q1")
    Wx = wx if sp.issparse(wx) else sp.diags(wx)
    kb = np.zeros(kh_elem.size + 1)
    kb[0], kb[-1] = kh_elem[0], kh_elem[-1]
    A = (sp.kron(My, Xx) + sp.kron(Yy, Wx)
         - sp.kron(weighted_mass_q1(kh_elem * kh_elem), Wx)
         - 1j * (sp.kron(weighted_mass_q1(kh_elem), sp.diags(bx)) + sp.kron(sp.diags(by * kb), Wx)))
    return sp.csr_matrix(A, dtype=np.complex128)


class Problem:
    """Grid and discrete operators for one impedance Helmholtz problem.

    dim: 1 or 2.  n: interior nodes per side.  k: wavenumber.
    Vectors are flattened row-major [S_y][S_x]; S_x = 1 in 1D.
    """

    def __init__(self, dim: int, n: int, k: float, k_rows=None, scheme: str = "fd", k_elems=None):
        """k_rows (optional): the wavenumber of each grid row j = 0..S-1 (layered media,
        Sec. 3.3); k is then only a label.  Without it every row has k.  scheme: "fd"
        (the weighted 5-point scheme) or "q1" (bilinear elements, one constant k, or with
        k_elems one k per row of elements, S - 1 values, for layered media)."""
        if dim not in (1, 2):
            raise ValueError("dim must be 1 or 2")
        if scheme not in ("fd", "q1"):
            raise ValueError("scheme must be 'fd' or 'q1'")
        self.scheme = scheme
        self.dim, self.n, self.k = dim, n, float(k)
        self.S = n + 2
        self.h = 1.0 / (n + 1)
        self.kh = self.k * self.h
        self.Sy = self.S
        self.Sx = self.S if dim == 2 else 1
        if k_rows is None:
            self.k_rows = np.full(self.Sy, self.k)
        else:
            self.k_rows = np.asarray(k_rows, dtype=np.float64).copy()
            if self.k_rows.shape != (self.Sy,) or not np.all(np.isfinite(self.k_rows)) or np.any(self.k_rows < 0):
                raise ValueError("k_rows must hold one finite k >= 0 per grid row")
        self.kh_rows = self.k_rows * self.h
        if scheme == "q1" and np.unique(self.k_rows).size != 1:
            raise ValueError("the Q1 scheme takes its layers as k_elems")
        self.k_elems = None
        if k_elems is not None:
            self.k_elems = np.asarray(k_elems, dtype=np.float64).copy()
            if scheme != "q1" or k_rows is not None or self.k_elems.shape != (self.Sy - 1,):
                raise ValueError("k_elems: one k per row of elements, with the Q1 scheme")
        self._xdir = direction(self.Sx, present=(dim == 2), scheme=scheme)

    @property
    def N(self) -> int:
        return self.Sx * self.Sy

    def band_operator(self, ra: int, rb: int) -> sp.csr_matrix:
        """A~ on rows [ra, rb): impedance (Robin, zero data) rows at both band ends."""
        if self.k_elems is not None:
            return operator_q1_layered(self.k_elems[ra:rb - 1] * self.h, self._xdir)
        return operator(self.kh_rows[ra:rb], self._xdir, direction(rb - ra, scheme=self.scheme))

    def box_operator(self, x0: int, x1: int, y0: int, y1: int) -> sp.csr_matrix:
        """A~ on the rectangle of nodes [x0, x1) x [y0, y1) (2D): impedance rows with zero
        data on its four sides; the whole grid gives A."""
        xdir = direction(x1 - x0, scheme=self.scheme)
        if self.k_elems is not None:
            return operator_q1_layered(self.k_elems[y0:y1 - 1] * self.h, xdir)
        return operator(self.kh_rows[y0:y1], xdir, direction(y1 - y0, scheme=self.scheme))

    def A(self) -> sp.csr_matrix:
        """The global operator A (the band covering every row)."""
        return self.band_operator(0, self.Sy)

    def rhs(self, f: np.ndarray, g: np.ndarray) -> np.ndarray:
        """b = h^2 w_i w_j f + h (w_j gx + w_i gy), flattened row-major.  For Q1 the
        weights are the consistent mass matrices: b = h^2 (M_y F M_x^T) + h (edge masses
        applied to g)."""
        if self.scheme == "q1":
            return self._rhs_q1(f, g)
        h = self.h
        _, wx, _ = self._xdir
        _, wy, _ = direction(self.Sy)
        f = np.asarray(f, dtype=np.complex128).reshape(self.Sy, self.Sx)
        b = (h * h) * wy[:, None] * wx[None, :] * f
        g = np.asarray(g, dtype=np.complex128)
        if self.dim == 1:
            b[0, 0] += h * g[0]
            b[-1, 0] += h * g[1]
        else:
            g = g.reshape(4, self.S)
            b[:, 0] += h * wy * g[0]        # side x = 0, indexed along y
            b[:, -1] += h * wy * g[1]       # side x = 1
            b[0, :] += h * wx * g[2]        # side y = 0, indexed along x
            b[-1, :] += h * wx * g[3]       # side y = 1
        return b.reshape(-1)

    def _rhs_q1(self, f: np.ndarray, g: np.ndarray) -> np.ndarray:
        h = self.h
        _, mx, _ = self._xdir
        _, my, _ = direction(self.Sy, scheme="q1")
        f = np.asarray(f, dtype=np.complex128).reshape(self.Sy, self.Sx)
        g = np.asarray(g, dtype=np.complex128)
        if self.dim == 1:
            b = (h * h) * (my @ f)
            b[0, 0] += h * g[0]                 # a boundary point carries no edge mass
            b[-1, 0] += h * g[1]
            return b.reshape(-1)
        b = (h * h) * (my @ (mx @ f.T).T)
        g = g.reshape(4, self.S)
        b[:, 0] += h * (my @ g[0])              # side x = 0, indexed along y
        b[:, -1] += h * (my @ g[1])             # side x = 1
        b[0, :] += h * (mx @ g[2])              # side y = 0, indexed along x
        b[-1, :] += h * (mx @ g[3])             # side y = 1
        return b.reshape(-1)
