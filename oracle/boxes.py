"""2 x 2 box hierarchy for the hierarchical ORAS method (oracle side; test
infrastructure only).

The paper's experiments (Sec. 3) partition (0,1)^2 into m x m boxes and each box
again into boxes; with [2 x 2, 2 x 2, ...] every subdomain has four children.  The
partition is first non-overlapping, then extended outward from the non-overlapping
interfaces.  This module restates the strip method of `method.OMethod` on boxes.

Readings (the strip readings, per axis):

* a node owning [ox0, ox1) x [oy0, oy1) splits each axis at its midpoint; child
  (ix, iy) owns the quarter (ix, iy) and has id 4 p + 1 + 2 iy + ix;
* every non-root region is the owned rectangle extended by e = overlap / 2 nodes on
  each side, clipped to the grid;
* inside its parent's region a child owns the part on its side of both split lines
  (the parent's overlap nodes belong to the adjacent child), so the restricted
  prolongations compose to those of the flat leaf partition;
* the interface Gamma_c of child c is the set of nodes on the sides of c's region that
  are not sides of its parent's region: its artificial boundary towards its siblings,
  an L through the cross point for a 2 x 2 split.  Data enter by injection,
  B_c^T g = g on Gamma_c.  The parent's own artificial boundary belongs to A~_p
  (Sec. 1, Sec. 2);
* T_c = (B_s A~_s R_s P_c M_c B_c^T)_s stacked over the three siblings s, with B_s the
  restriction to Gamma_s (Sec. 2: the output data of c for its neighbours).  This is
  the paper's B_{c,s} = B_s A~_s R_s P_c with the restricted prolongation P_c, taken
  literally: a sibling's interface runs through parts of c's region that other
  siblings own, and the iteration never passes c's values there on.  (The strips use
  R_c^T in place of P_c: identical there for e >= 2, better for e = 1.)  With this
  form the coarse-free and coarse-corrected GMRES counts of Table 1 for m = 2 are
  reproduced to within one iteration.  At a cross point every sibling whose interface
  passes through it gets its own value;
* A~ on a box is the same weighted operator on that rectangle, with impedance rows
  (zero data) on all four sides (Sec. 1).

Vectors on a node's region are arrays V[y, x, col] local to the region.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from .method import OMethod
from .problem import Problem
from .sketch import gaussian_sketch


@dataclasses.dataclass
class Box:
    id: int
    level: int
    ox: tuple          # owned nodes [x0, x1), global
    oy: tuple
    gx: tuple          # region nodes [x0, x1), global
    gy: tuple
    parent: int = -1
    children: tuple = ()

    @property
    def nx(self) -> int:
        return self.gx[1] - self.gx[0]

    @property
    def ny(self) -> int:
        return self.gy[1] - self.gy[0]

    @property
    def is_leaf(self) -> bool:
        return not self.children


def build_boxes(S: int, levels: int, overlap: int, partition: str = "nodes") -> dict:
    """Nodes by id: root 0 owns the S x S grid; children of p are 4p+1 .. 4p+4.

    partition "nodes": regions are the owned node ranges extended by e = overlap / 2
    nodes on each side.  partition "elements" (the experiments of Sec. 3): the
    non-overlapping partition is by elements, so a box's elements span its owned nodes
    and the first node of the next box; they are extended by e elements on each side
    (overlap delta = 2 e h), i.e. nodes [ox0 - e, ox1 + e + 1), clipped to the grid."""
    if levels < 0:
        raise ValueError("levels must be >= 0")
    if levels > 0 and (overlap < 2 or overlap % 2):
        raise ValueError("overlap must be even and >= 2")
    if partition not in ("nodes", "elements"):
        raise ValueError("partition must be 'nodes' or 'elements'")
    e = overlap // 2
    hi = e + 1 if partition == "elements" else e
    nodes = {0: Box(0, 0, (0, S), (0, S), (0, S), (0, S))}
    for lev in range(levels):
        for p in [nd for nd in nodes.values() if nd.level == lev]:
            mx = p.ox[0] + (p.ox[1] - p.ox[0]) // 2
            my = p.oy[0] + (p.oy[1] - p.oy[0]) // 2
            kids = []
            for iy, (y0, y1) in enumerate(((p.oy[0], my), (my, p.oy[1]))):
                for ix, (x0, x1) in enumerate(((p.ox[0], mx), (mx, p.ox[1]))):
                    cid = 4 * p.id + 1 + 2 * iy + ix
                    if min(x1 - x0, y1 - y0) < (2 * e + 2 if partition == "nodes" else e + 1):
                        raise ValueError(f"box {cid} owns {x1 - x0} x {y1 - y0} nodes: too few for the overlap")
                    nodes[cid] = Box(cid, lev + 1, (x0, x1), (y0, y1), (max(0, x0 - e), min(S, x1 + hi)),
                                     (max(0, y0 - e), min(S, y1 + hi)), p.id)
                    kids.append(cid)
            p.children = tuple(kids)
    return nodes


def owned_in_parent(nodes: dict, c: Box) -> tuple:
    """((x0, x1), (y0, y1)), global: the part of the parent's region child c owns."""
    p = nodes[c.parent]
    q = c.id - 4 * p.id - 1
    ix, iy = q % 2, q // 2
    mx = nodes[p.children[0]].ox[1]
    my = nodes[p.children[0]].oy[1]
    xs = (p.gx[0], mx) if ix == 0 else (mx, p.gx[1])
    ys = (p.gy[0], my) if iy == 0 else (my, p.gy[1])
    return xs, ys


def interface_nodes(nodes: dict, c: Box) -> np.ndarray:
    """Flat indices (y * nx + x, local to c's region) of Gamma_c, in row-major order."""
    p = nodes[c.parent]
    ys, xs = np.meshgrid(np.arange(c.ny), np.arange(c.nx), indexing="ij")
    on = np.zeros((c.ny, c.nx), dtype=bool)
    if c.gx[0] > p.gx[0]:
        on |= xs == 0
    if c.gx[1] < p.gx[1]:
        on |= xs == c.nx - 1
    if c.gy[0] > p.gy[0]:
        on |= ys == 0
    if c.gy[1] < p.gy[1]:
        on |= ys == c.ny - 1
    return np.flatnonzero(on.reshape(-1))


class BoxMethod:
    """Set-up (leaf factorisation, sketches, coarse spaces) and the iteration on 2 x 2
    boxes.  Same steps as `method.OMethod` (Eqs. (2)-(3), Sec. 2), on rectangles."""

    def __init__(self, prob: Problem, levels: int, overlap: int, rank: int, oversample: int,
                 n_inner: int = 1, seed: int = 0, exact_subsolves: bool = False, partition: str = "nodes"):
        if prob.dim != 2:
            raise ValueError("boxes need a 2D problem")
        self.prob = prob
        self.levels = levels
        self.n_inner = n_inner
        self.seed = seed
        # rank: one value for every level, or a sequence giving the children of level j
        # (j = 1 .. levels) rank[j - 1] modes each
        self.ranks = list(rank) if np.ndim(rank) else [int(rank)] * max(levels, 1)
        self.rank, self.oversample = max(self.ranks), oversample
        self.nodes = build_boxes(prob.S, levels, overlap, partition)
        self.A = prob.A()
        self.Atil = {nd.id: self._box_operator(nd) for nd in self.nodes.values()}
        self.Gamma = {nd.id: interface_nodes(self.nodes, nd) for nd in self.nodes.values() if nd.id != 0}
        self.lu = {}
        for nd in self.nodes.values():
            if nd.id != 0 and (nd.is_leaf or exact_subsolves):
                self.lu[nd.id] = spla.splu(self.Atil[nd.id].tocsc())
        self.V, self.sigma, self.C, self.Ac, self.Ac_lu = {}, {}, {}, {}, {}
        for lev in reversed(range(levels)):
            if self.ranks[lev] <= 0:
                continue
            for p in self.nodes.values():
                if p.level == lev and not p.is_leaf:
                    self._build_coarse(p.id)

    def _box_operator(self, nd: Box):
        if nd.id == 0:
            return self.A
        return self.prob.box_operator(nd.gx[0], nd.gx[1], nd.gy[0], nd.gy[1])

    # ------------------------------------------------------------------ helpers
    def _zeros(self, nid: int, k: int) -> np.ndarray:
        nd = self.nodes[nid]
        return np.zeros((nd.ny, nd.nx, k), dtype=np.complex128)

    def apply(self, nid: int, V: np.ndarray) -> np.ndarray:
        nd, k = self.nodes[nid], V.shape[2]
        return (self.Atil[nid] @ V.reshape(nd.ny * nd.nx, k)).reshape(nd.ny, nd.nx, k)

    def apply_adjoint(self, nid: int, V: np.ndarray) -> np.ndarray:
        nd, k = self.nodes[nid], V.shape[2]
        return (self.Atil[nid].getH() @ V.reshape(nd.ny * nd.nx, k)).reshape(nd.ny, nd.nx, k)

    def _slice(self, p: int, c: int):
        """Child c's region inside parent p's region arrays."""
        P, Cn = self.nodes[p], self.nodes[c]
        return (slice(Cn.gy[0] - P.gy[0], Cn.gy[1] - P.gy[0]), slice(Cn.gx[0] - P.gx[0], Cn.gx[1] - P.gx[0]))

    def _restrict(self, p: int, c: int, V: np.ndarray) -> np.ndarray:
        return V[self._slice(p, c)]

    def _prolong_add(self, p: int, c: int, Wp: np.ndarray, Wc: np.ndarray) -> None:
        """Wp += P_c Wc: only the part of p's region that c owns."""
        P, Cn = self.nodes[p], self.nodes[c]
        (x0, x1), (y0, y1) = owned_in_parent(self.nodes, Cn)
        Wp[y0 - P.gy[0]:y1 - P.gy[0], x0 - P.gx[0]:x1 - P.gx[0]] += \
            Wc[y0 - Cn.gy[0]:y1 - Cn.gy[0], x0 - Cn.gx[0]:x1 - Cn.gx[0]]

    def _inject(self, c: int, X: np.ndarray) -> np.ndarray:
        """B_c^T X: interface data onto Gamma_c, zero elsewhere."""
        U = self._zeros(c, X.shape[1])
        U.reshape(-1, X.shape[1])[self.Gamma[c]] = X
        return U

    def _trace(self, c: int, U: np.ndarray) -> np.ndarray:
        """B_c U: the values on Gamma_c."""
        return U.reshape(-1, U.shape[2])[self.Gamma[c]]

    # ------------------------------------------------------------ sub-level solve
    def M(self, nid: int, V: np.ndarray) -> np.ndarray:
        """A~_nid^{-1} V: exact for leaves (and with exact sub-solves), else n_i sub-level
        iterations of Eqs. (2)-(3) over the four children."""
        if nid in self.lu:
            nd, k = self.nodes[nid], V.shape[2]
            return self.lu[nid].solve(V.reshape(nd.ny * nd.nx, k)).reshape(nd.ny, nd.nx, k)
        W = np.zeros_like(V)
        for it in range(self.n_inner):
            R = V - self.apply(nid, W) if it else V
            W = W + self.sweep(nid, R)
            if nid in self.C:
                W = W + self.coarse(nid, V - self.apply(nid, W))
        return W

    def M_adjoint(self, nid: int, V: np.ndarray) -> np.ndarray:
        if nid in self.lu:
            nd, k = self.nodes[nid], V.shape[2]
            return self.lu[nid].solve(V.reshape(nd.ny * nd.nx, k), trans="H").reshape(nd.ny, nd.nx, k)
        return np.conj(self.M(nid, np.conj(V)))

    def sweep(self, nid: int, R: np.ndarray) -> np.ndarray:
        """sum_c P_c M_c R_c R over the four children (Eq. (2))."""
        W = np.zeros_like(R)
        for c in self.nodes[nid].children:
            self._prolong_add(nid, c, W, self.M(c, self._restrict(nid, c, R)))
        return W

    def coarse(self, nid: int, R: np.ndarray) -> np.ndarray:
        """C_p A_c^{-1} C_p^H R (Eq. (3))."""
        C = self.C[nid]
        nd, k = self.nodes[nid], R.shape[2]
        Cf = C.reshape(nd.ny * nd.nx, -1)
        y = sla.lu_solve(self.Ac_lu[nid], Cf.conj().T @ R.reshape(nd.ny * nd.nx, k))
        return (Cf @ y).reshape(nd.ny, nd.nx, k)

    # ------------------------------------------------------- interface maps (Sec. 2)
    def siblings(self, c: int) -> list:
        return [s for s in self.nodes[self.nodes[c].parent].children if s != c]

    def T(self, c: int, X: np.ndarray) -> np.ndarray:
        """T_c X, stacked over the siblings s in id order: B_s A~_s R_s P_c M_c B_c^T X."""
        p = self.nodes[c].parent
        Wp = self._zeros(p, X.shape[1])
        self._prolong_add(p, c, Wp, self.M(c, self._inject(c, X)))
        return np.concatenate([self._trace(s, self.apply(s, self._restrict(p, s, Wp))) for s in self.siblings(c)])

    def _prolong_adjoint(self, p: int, c: int, Zp: np.ndarray) -> np.ndarray:
        """P_c^H Zp: the part of p's region that c owns, placed in c's region."""
        P, Cn = self.nodes[p], self.nodes[c]
        (x0, x1), (y0, y1) = owned_in_parent(self.nodes, Cn)
        Zc = self._zeros(c, Zp.shape[2])
        Zc[y0 - Cn.gy[0]:y1 - Cn.gy[0], x0 - Cn.gx[0]:x1 - Cn.gx[0]] = \
            Zp[y0 - P.gy[0]:y1 - P.gy[0], x0 - P.gx[0]:x1 - P.gx[0]]
        return Zc

    def T_adjoint(self, c: int, Y: np.ndarray) -> np.ndarray:
        """T_c^* Y = B_c M_c^H P_c^H sum_s R_s^T A~_s^H B_s^T Y_s."""
        p = self.nodes[c].parent
        Zp = self._zeros(p, Y.shape[1])
        at = 0
        for s in self.siblings(c):
            n = self.Gamma[s].size
            Zp[self._slice(p, s)] += self.apply_adjoint(s, self._inject(s, Y[at:at + n]))
            at += n
        return self._trace(c, self.M_adjoint(c, self._prolong_adjoint(p, c, Zp)))

    def rsvd(self, c: int):
        """Dominant right singular vectors of T_c by the randomised SVD (Sec. 2)."""
        g = self.Gamma[c].size
        rank = self.ranks[self.nodes[c].level - 1]
        m = min(rank + self.oversample, g)
        r = min(rank, m)
        Y = self.T(c, gaussian_sketch(self.seed, c, g, m))
        Q, R = np.linalg.qr(Y)
        d = np.diag(R)
        ph = np.where(np.abs(d) > 0, d / np.where(np.abs(d) > 0, np.abs(d), 1), 1)
        Z = self.T_adjoint(c, Q * ph[None, :])
        _, s, Vh = np.linalg.svd(Z.conj().T, full_matrices=False)
        return Vh.conj().T[:, :r], s

    def extend(self, c: int, V: np.ndarray) -> np.ndarray:
        """C_c = P_c M_c B_c^T V_c on the parent's region."""
        p = self.nodes[c].parent
        Cp = self._zeros(p, V.shape[1])
        self._prolong_add(p, c, Cp, self.M(c, self._inject(c, V)))
        return Cp

    def _build_coarse(self, p: int) -> None:
        blocks = []
        for c in self.nodes[p].children:
            V, s = self.rsvd(c)
            self.V[c], self.sigma[c] = V, s
            blocks.append(self.extend(c, V))
        C = np.concatenate(blocks, axis=2)
        nd = self.nodes[p]
        Cf = C.reshape(nd.ny * nd.nx, -1)
        self.C[p] = C
        self.Ac[p] = Cf.conj().T @ (self.Atil[p] @ Cf)     # A_c = C^H A~_p C (Sec. 1)
        self.Ac_lu[p] = sla.lu_factor(self.Ac[p])

    # --------------------------------------------------------------- the iteration
    def precondition(self, r: np.ndarray) -> np.ndarray:
        """One coarse-corrected step from zero on the global residual r: Eqs. (2)-(3)
        with u^(n-1) = 0 at the root (the sub-levels take their n_i iterations)."""
        S = self.prob.S
        if self.levels == 0:
            return spla.spsolve(self.A.tocsc(), r)
        R = r.reshape(S, S, 1)
        W = self.sweep(0, R)
        if 0 in self.C:
            W = W + self.coarse(0, R - self.apply(0, W))
        return W.reshape(-1)

    # the outer iterations only need A and the preconditioner
    solve = OMethod.solve
    solve_gmres = OMethod.solve_gmres
