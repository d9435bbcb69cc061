"""The 1023 x 1023, k = 100, three-level workload at full size (1,050,625 unknowns, eight
leaf bands of 130 to 132 rows, rank 32, oversampling 10), in both precision forms.

Each solution returned through the C-ABI is compared element by element with the
oracle's direct solution u* = A^{-1} b (sparse LU with a fill-reducing ordering, about
15 s on the host): relative error at most 1e-8 for the mixed form and 1e-10 for the FP64
form (the targets of the relative-error metric, C8 reading).

A second check holds at any size: the oracle's own sparse operator applied to the
returned u gives a relative residual below the tolerance that agrees with the one the
library reports.  Both residuals are FP64 sums of a 5-point stencil and b, so each entry
carries rounding of at most about 16 eps (|b| + |A| |u|) (six complex terms); their
difference is bounded by twice that, in the 2-norm relative to ||b||.  The bound is
computed from the data.
"""
import numpy as np
import pytest

from oracle import direct
from oracle.problem import Problem
from workloads import WORKLOADS, problem_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# stopping tolerances on the FP64 relative residual; the errors they give are far below
# the targets (printed by each run)
TOL = {"mixed": 1e-9, "fp64": 1e-11}
ERR = {"mixed": 1e-8, "fp64": 1e-10}


@pytest.fixture(scope="module")
def hh():
    from paper_2512_12538_gb300 import build
    build.build()
    import paper_2512_12538_gb300 as m
    return m


@pytest.fixture(scope="module")
def case():
    w = WORKLOADS["helm2d_n1023_k100_L3"]
    f, g = problem_inputs(w)
    P = Problem(2, w.n, w.k)
    A = P.A()
    b = P.rhs(f, g)
    u_star = direct.solve(P, f, g)
    return w, f, g, A, b, u_star


@pytest.mark.parametrize("precision,outer", [("mixed", "oras"), ("mixed", "gmres"), ("fp64", "oras")])
def test_full_size_three_level_solution_matches_the_direct_solution(hh, case, precision, outer):
    w, f, g, A, b, u_star = case
    tol = TOL[precision]
    p = hh.make_params(2, w.n, w.k, w.levels, w.overlap, w.rank, w.oversample, w.n_inner, tol, 800, precision, 1,
                       "eigen", outer, 40)
    h, _ = hh.hh_setup(p)
    try:
        u = torch.empty((w.S, w.S), dtype=torch.complex128, device="cuda")
        st = hh.hh_solve(h, torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), u)
        uh = u.cpu().numpy().reshape(-1)
    finally:
        hh.hh_destroy(h)
    assert np.isfinite(uh).all() and np.linalg.norm(uh) > 0
    err = direct.rel_err(uh, u_star)
    nb = np.linalg.norm(b)
    rr = float(np.linalg.norm(b - A @ uh) / nb)
    eps = np.finfo(np.float64).eps
    bound = float(np.linalg.norm(16 * eps * (np.abs(b) + abs(A) @ np.abs(uh))) / nb)
    print(f"{precision}/{outer}: iters={st.iters} err={err:.3e} reported={st.rel_res:.3e} oracle={rr:.3e} "
          f"rounding bound={bound:.1e}")
    assert err <= ERR[precision]
    assert st.rel_res < tol
    assert abs(rr - st.rel_res) <= 2 * bound
    assert rr < tol + 2 * bound
