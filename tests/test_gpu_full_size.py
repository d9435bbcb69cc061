"""The 1023 x 1023, k = 100, three-level workload at full size (1,050,625 unknowns, eight
leaf bands of up to 132 rows, rank 32, oversampling 10), in the complex64 form.

The oracle's direct solve does not finish in seconds at this size, so the check is a
property that holds at any size: the solution returned through the C-ABI satisfies the
discrete system, judged by the oracle's own sparse operator and right-hand side in FP64.
That residual must be below the tolerance, and it must agree with the residual the
library reports.

Both residuals are FP64 sums of a 5-point stencil and b, so each entry carries rounding of
at most about 16 eps (|b| + |A| |u|) (six complex terms). Their difference is bounded by
twice that, in the 2-norm relative to ||b||. The bound is computed from the data.
"""
import numpy as np
import pytest

from oracle.problem import Problem
from workloads import WORKLOADS, problem_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-9


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
    return w, f, g, A, b


@pytest.mark.parametrize("outer", ["oras", "gmres"])
def test_full_size_three_level_solution_satisfies_the_oracle_system(hh, case, outer):
    w, f, g, A, b = case
    p = hh.make_params(2, w.n, w.k, w.levels, w.overlap, w.rank, w.oversample, w.n_inner, TOL, 600, "mixed", 1,
                       "eigen", outer, 40)
    h, _ = hh.hh_setup(p)
    try:
        u = torch.empty((w.S, w.S), dtype=torch.complex128, device="cuda")
        st = hh.hh_solve(h, torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), u)
        uh = u.cpu().numpy().reshape(-1)
    finally:
        hh.hh_destroy(h)
    assert np.isfinite(uh).all() and np.linalg.norm(uh) > 0
    nb = np.linalg.norm(b)
    rr = float(np.linalg.norm(b - A @ uh) / nb)
    eps = np.finfo(np.float64).eps
    bound = float(np.linalg.norm(16 * eps * (np.abs(b) + abs(A) @ np.abs(uh))) / nb)
    print(f"{outer}: iters={st.iters} reported={st.rel_res:.3e} oracle={rr:.3e} rounding bound={bound:.1e}")
    assert st.rel_res < TOL
    assert abs(rr - st.rel_res) <= 2 * bound
    assert rr < TOL + 2 * bound
