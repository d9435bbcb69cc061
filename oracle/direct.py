"""O-direct: the discrete solution u* = A^{-1} b (oracle side; test infrastructure only).

The hierarchical ORAS iteration is a stationary iteration whose fixed point is the
solution of A u = f (Eqs. (2)-(3)); this module computes that fixed point by its
definition, a direct sparse LU solve (SuperLU) of the assembled system.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .problem import Problem


def solve(prob: Problem, f: np.ndarray, g: np.ndarray) -> np.ndarray:
    """u* with A u* = b(f, g), flattened row-major [S_y][S_x].

    The column ordering (minimum degree on A^T + A) only limits the fill of the LU
    factors; it is not part of the method.  With it the 1023 x 1023 interior grid
    (1,050,625 unknowns) factors in seconds rather than minutes.
    """
    lu = spla.splu(prob.A().tocsc(), permc_spec="MMD_AT_PLUS_A")
    return lu.solve(prob.rhs(f, g))


def rel_err(u: np.ndarray, u_star: np.ndarray) -> float:
    """||u - u*||_2 / ||u*||_2 over every node."""
    u = np.asarray(u).reshape(-1)
    u_star = np.asarray(u_star).reshape(-1)
    return float(np.linalg.norm(u - u_star) / np.linalg.norm(u_star))
