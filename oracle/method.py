"""O-method: the hierarchical ORAS iteration with randomised-SVD coarse spaces.

Oracle side, test infrastructure only.  Plain FP64 complex; sparse LU (SuperLU),
dense QR/SVD (LAPACK) and dense LU are used as library steps.  Vectors on a node's
region are arrays V[row, x, col] with row local to the node's band of rows.

Paper passages followed (Gander, Jiang & Zhang):

* Eq. (2): one-level ORAS sweep  u~ = sum_i P_i A~_i^{-1} R_i (f - A u).  The printed
  equation drops the previous iterate; read (as the zero-initial-guess case shows)
  u~^(n) = u^(n-1) + sum_i P_i A~_i^{-1} R_i (f - A u^(n-1)).
* Eq. (3): coarse correction u = u~ + C A_c^{-1} C^H (f - A u~), A_c = C^H A C (Sec. 1).
* R_i: identity restriction to the subdomain; P_i: restricted prolongation (ORAS),
  zero outside the rows the subdomain owns, sum_i P_i R_i = I (Sec. 1).
* A~_i: the subdomain operator with zero impedance data on artificial boundaries
  (Sec. 1; algebraic form Sec. 2).
* Hierarchy (Sec. 1): a subdomain problem is itself solved by Eqs. (2)-(3) over its
  children; with n_i iterations from zero at the sub-level (Sec. 2, Sec. 3: "a few
  steps of the sublevel iteration", n_i per level).  The coarse basis at the upper
  level therefore "contains iterative errors".
* Interface map (Sec. 2): T_c = B_{c,s} A~_c^{-1} B_c^T with B_{c,s} = B_s A~_s R_s P_c.
  Reading: B_{c,s} = B_s A~_s R_s R_c^T (unrestricted extension) -- equal to the
  paper's definition when the overlap leaves the trace rows inside c's owned rows,
  and well defined for the one-row extension (e = 1) as well.  Only the sibling's
  interface counts: the parent's own artificial boundary belongs to A~_p.
* Randomised SVD (Sec. 2): apply T_c to samples, orthogonalise, apply T_c^*, SVD;
  keep the dominant right singular vectors V_c (Halko-Martinsson-Tropp basic
  scheme).  Euclidean inner product (Sec. 2).  For an internal child the solve is
  the inexact sub-level iteration M_c; its adjoint is read as conj o M_c o conj
  (exact for leaves, where A~ is complex symmetric).
* Coarse vectors C_c = P_c A~_c^{-1} B_c^T V_c and C = (C_c) (Sec. 2); in 1D the
  interface has one node and C_c is the a-harmonic extension of Eqs. (4)-(5).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from .hierarchy import build_tree, interface_row, owned_in_parent, sibling
from .problem import Problem
from .sketch import gaussian_sketch


class OMethod:
    """Set-up (leaf factorisation, sketches, coarse spaces) and the iteration."""

    def __init__(self, prob: Problem, levels: int, overlap: int, rank: int, oversample: int,
                 n_inner: int = 1, seed: int = 0, exact_subsolves: bool = False):
        self.prob = prob
        self.Sx = prob.Sx
        self.levels = levels
        self.n_inner = n_inner
        self.seed = seed
        self.tree = build_tree(prob.Sy, levels, overlap)
        # samples and kept modes, clamped to the interface dimension (one row of Sx nodes)
        self.m = min(rank + oversample, self.Sx)
        self.r = min(rank, self.m)
        self.A = prob.A()
        self.Atil = {nd.id: prob.band_operator(nd.ra, nd.rb) for nd in self.tree}
        self.lu = {}
        for nd in self.tree:
            if nd.id != 0 and (nd.is_leaf or exact_subsolves):
                self.lu[nd.id] = spla.splu(self.Atil[nd.id].tocsc())
        self.V, self.sigma, self.C, self.Ac, self.Ac_lu = {}, {}, {}, {}, {}
        if self.r > 0:
            for lev in reversed(range(levels)):
                for p in self.tree:
                    if p.level == lev and not p.is_leaf:
                        self._build_coarse(p.id)

    # ------------------------------------------------------------------ helpers
    def _zeros(self, nid: int, k: int) -> np.ndarray:
        return np.zeros((self.tree[nid].b, self.Sx, k), dtype=np.complex128)

    def apply(self, nid: int, V: np.ndarray) -> np.ndarray:
        """A~_nid V (A for the root)."""
        b, k = self.tree[nid].b, V.shape[2]
        return (self.Atil[nid] @ V.reshape(b * self.Sx, k)).reshape(b, self.Sx, k)

    def apply_adjoint(self, nid: int, V: np.ndarray) -> np.ndarray:
        """A~_nid^H V."""
        b, k = self.tree[nid].b, V.shape[2]
        return (self.Atil[nid].getH() @ V.reshape(b * self.Sx, k)).reshape(b, self.Sx, k)

    def _restrict(self, p: int, c: int, V: np.ndarray) -> np.ndarray:
        """R_c: rows of child c's region out of parent p's vector."""
        P, Cn = self.tree[p], self.tree[c]
        return V[Cn.ra - P.ra:Cn.rb - P.ra]

    def _prolong_add(self, p: int, c: int, Wp: np.ndarray, Wc: np.ndarray) -> None:
        """Wp += P_c Wc: only the rows c owns inside p (restricted prolongation)."""
        P, Cn = self.tree[p], self.tree[c]
        a, b = owned_in_parent(self.tree, Cn)
        Wp[a - P.ra:b - P.ra] += Wc[a - Cn.ra:b - Cn.ra]

    # ------------------------------------------------------------ sub-level solve
    def leaf_solve(self, nid: int, V: np.ndarray) -> np.ndarray:
        b, k = self.tree[nid].b, V.shape[2]
        X = self.lu[nid].solve(V.reshape(b * self.Sx, k))
        return X.reshape(b, self.Sx, k)

    def M(self, nid: int, V: np.ndarray) -> np.ndarray:
        """Approximate A~_nid^{-1} V: exact for leaves, else n_i sub-level iterations."""
        if nid in self.lu:
            return self.leaf_solve(nid, V)
        nd = self.tree[nid]
        W = np.zeros_like(V)
        for it in range(self.n_inner):
            R = V - self.apply(nid, W) if it else V
            W = W + self.sweep(nid, R)
            if self.r > 0:
                W = W + self.coarse(nid, V - self.apply(nid, W))
        return W

    def M_adjoint(self, nid: int, V: np.ndarray) -> np.ndarray:
        """Adjoint solve: A~^{-H} for leaves; conj o M o conj for internal nodes."""
        if nid in self.lu:
            b, k = self.tree[nid].b, V.shape[2]
            return self.lu[nid].solve(V.reshape(b * self.Sx, k), trans="H").reshape(b, self.Sx, k)
        return np.conj(self.M(nid, np.conj(V)))

    def sweep(self, nid: int, R: np.ndarray) -> np.ndarray:
        """One ORAS sweep over the children of nid: sum_c P_c M_c R_c R (Eq. (2))."""
        W = np.zeros_like(R)
        for c in self.tree[nid].children:
            self._prolong_add(nid, c, W, self.M(c, self._restrict(nid, c, R)))
        return W

    def coarse(self, nid: int, R: np.ndarray) -> np.ndarray:
        """C_p A_c^{-1} C_p^H R on node nid's region (Eq. (3))."""
        C = self.C[nid]
        b, k = self.tree[nid].b, R.shape[2]
        Cf = C.reshape(b * self.Sx, -1)
        y = sla.lu_solve(self.Ac_lu[nid], Cf.conj().T @ R.reshape(b * self.Sx, k))
        return (Cf @ y).reshape(b, self.Sx, k)

    # ------------------------------------------------------- interface maps (Sec. 2)
    def T(self, c: int, X: np.ndarray) -> np.ndarray:
        """T_c X = B_s A~_s R_s R_c^T M_c B_c^T X; X is Sx x k interface data."""
        Cn = self.tree[c]
        p, s = Cn.parent, sibling(self.tree, Cn)
        U = self._zeros(c, X.shape[1])
        U[interface_row(self.tree, Cn) - Cn.ra] = X
        W = self.M(c, U)
        Wp = self._zeros(p, X.shape[1])
        Wp[Cn.ra - self.tree[p].ra:Cn.rb - self.tree[p].ra] = W
        Ws = self._restrict(p, s.id, Wp)
        return self.apply(s.id, Ws)[interface_row(self.tree, s) - s.ra]

    def T_adjoint(self, c: int, Y: np.ndarray) -> np.ndarray:
        """T_c^* Y = B_c M_c^H R_c R_s^T A~_s^H B_s^T Y."""
        Cn = self.tree[c]
        p, s = Cn.parent, sibling(self.tree, Cn)
        Z = self._zeros(s.id, Y.shape[1])
        Z[interface_row(self.tree, s) - s.ra] = Y
        Z = self.apply_adjoint(s.id, Z)
        Zp = self._zeros(p, Y.shape[1])
        Zp[s.ra - self.tree[p].ra:s.rb - self.tree[p].ra] = Z
        W = self.M_adjoint(c, self._restrict(p, c, Zp))
        return W[interface_row(self.tree, Cn) - Cn.ra]

    def rsvd(self, c: int):
        """Dominant right singular vectors of T_c by the randomised SVD (Sec. 2)."""
        Om = gaussian_sketch(self.seed, c, self.Sx, self.m)
        Y = self.T(c, Om)
        Q, R = np.linalg.qr(Y)                      # Householder QR (LAPACK)
        d = np.diag(R)
        ph = np.where(np.abs(d) > 0, d / np.where(np.abs(d) > 0, np.abs(d), 1), 1)
        Q = Q * ph[None, :]                         # R with real positive diagonal
        Z = self.T_adjoint(c, Q)                    # Z = T^* Q, so Z^H = Q^H T
        _, s, Vh = np.linalg.svd(Z.conj().T, full_matrices=False)
        return Vh.conj().T[:, :self.r], s

    def extend(self, c: int, V: np.ndarray) -> np.ndarray:
        """C_c = P_c M_c B_c^T V_c, returned on the parent's region."""
        Cn = self.tree[c]
        U = self._zeros(c, V.shape[1])
        U[interface_row(self.tree, Cn) - Cn.ra] = V
        W = self.M(c, U)
        Cp = self._zeros(Cn.parent, V.shape[1])
        self._prolong_add(Cn.parent, c, Cp, W)
        return Cp

    def _build_coarse(self, p: int) -> None:
        blocks = []
        for c in self.tree[p].children:
            V, s = self.rsvd(c)
            self.V[c], self.sigma[c] = V, s
            blocks.append(self.extend(c, V))
        C = np.concatenate(blocks, axis=2)
        b = self.tree[p].b
        Cf = C.reshape(b * self.Sx, -1)
        G = self.Atil[p] @ Cf                       # A~_p C   (A at the root)
        self.C[p] = C
        self.Ac[p] = Cf.conj().T @ G                # A_c = C^H A C (Sec. 1)
        self.Ac_lu[p] = sla.lu_factor(self.Ac[p])

    # --------------------------------------------------------------- the iteration
    def precondition(self, r: np.ndarray) -> np.ndarray:
        """One coarse-corrected ORAS step from zero: Eqs. (2)-(3) with u^(n-1) = 0."""
        if self.levels == 0:
            return spla.spsolve(self.A.tocsc(), r)
        R = r.reshape(self.prob.Sy, self.Sx, 1)
        W = self.sweep(0, R)
        if self.r > 0:
            W = W + self.coarse(0, R - self.apply(0, W))
        return W.reshape(-1)

    def solve_gmres(self, b: np.ndarray, tol: float = 1e-12, restart: int = 40, maxit: int = 400, M=None):
        """GMRES on the Schwarz-preconditioned system (Sec. 3), right-preconditioned by
        M (default: `precondition`, one coarse-corrected ORAS step from zero) and
        restarted every `restart` steps.  Each cycle minimises ||b - A u|| over
        u_0 + M K(A M, r_0): Arnoldi with modified Gram-Schmidt, the small least-squares
        problem by a library solve.  The preconditioned vectors are kept (flexible
        form), so u = u_0 + Z y needs no second application of M.  A cycle ends at the
        restart length, at a residual estimate below tol, or at a breakdown; the true
        residual then decides.  Returns (u, steps, history of relative residual
        estimates, one per step, after the initial 1)."""
        M = self.precondition if M is None else M
        u = np.zeros_like(b)
        nb = np.linalg.norm(b)
        if nb == 0.0:
            return u, 0, [0.0]
        hist = [1.0]
        steps = 0
        while steps < maxit:
            r = b - self.A @ u
            beta = np.linalg.norm(r)
            if beta / nb < tol:
                break
            V = [r / beta]
            Z = []
            H = np.zeros((restart + 1, restart), dtype=np.complex128)
            y = np.zeros(0, dtype=np.complex128)
            for j in range(restart):
                z = M(V[j])
                Z.append(z)
                w = self.A @ z
                for i in range(j + 1):
                    H[i, j] = np.vdot(V[i], w)
                    w = w - H[i, j] * V[i]
                H[j + 1, j] = np.linalg.norm(w)
                e1 = np.zeros(j + 2, dtype=np.complex128)
                e1[0] = beta
                y = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)[0]
                est = np.linalg.norm(e1 - H[:j + 2, :j + 1] @ y) / nb
                steps += 1
                hist.append(est)
                if est < tol or H[j + 1, j] == 0.0 or steps >= maxit:
                    break
                V.append(w / H[j + 1, j])
            u = u + sum(Z[i] * y[i] for i in range(len(y)))
        return u, steps, hist

    def solve(self, b: np.ndarray, tol: float = 1e-12, maxit: int = 200, u0=None):
        """u^(n) = u^(n-1) + precondition(b - A u^(n-1)) until ||b - Au|| < tol ||b||."""
        u = np.zeros_like(b) if u0 is None else u0.copy()
        nb = np.linalg.norm(b)
        hist = []
        it = 0
        while True:
            r = b - self.A @ u
            hist.append(np.linalg.norm(r) / nb)
            if hist[-1] < tol or it >= maxit or not np.isfinite(hist[-1]):
                break
            u = u + self.precondition(r)
            it += 1
        return u, it, hist
