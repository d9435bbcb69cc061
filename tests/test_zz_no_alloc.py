"""hh_residual_noalloc (the allocation-free relative residual) against hh_residual and
against the oracle's ||b - A u|| / ||b|| (its sparse operator and right-hand side, FP64).

Collected last on purpose: it must pass both in a fresh process, where its first call
also does the per-device set-up, and after every other test has run.
"""
import numpy as np
import pytest

from oracle.problem import Problem
from workloads.generators import random_complex

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hh():
    from paper_2512_12538_gb300 import build
    build.build()
    import paper_2512_12538_gb300 as m
    return m


def test_rejects_sizes_beyond_the_static_scratch(hh):
    # host-side checks only: nothing reaches the device
    cap = hh.HH_NOALLOC_MAX_ROWS
    for dim in (1, 2):
        with pytest.raises(hh.HHError) as ei:
            hh.hh_residual_noalloc(dim, cap - 1, 10.0, None, None, None, stream=0)
        assert ei.value.status == hh.HH_ETOOLARGE
    assert "scratch" in hh.status_string(hh.HH_ETOOLARGE)


def _inputs(seed, S, Sx, gl):
    f = torch.from_numpy(random_complex((S, Sx), seed)).cuda()
    g = torch.from_numpy(random_complex((gl,) if gl == 2 else (4, S), seed + 1000)).cuda()
    u = torch.from_numpy(random_complex((S, Sx), seed + 2000)).cuda()
    return f, g, u


CASES = [
    # dim, n, k, levels, overlap, rank, oversample
    (2, 45, 12.0, 2, 2, 6, 4),
    (2, 255, 40.0, 2, 2, 16, 10),
    (1, 1000, 62.83, 1, 4, 1, 0),
]


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"d{c[0]}n{c[1]}")
def test_noalloc_matches_hh_residual_on_two_calls_in_a_row(hh, case):
    dim, n, k, levels, overlap, rank, over = case
    S = n + 2
    Sx = S if dim == 2 else 1
    first = _inputs(11, S, Sx, 4 if dim == 2 else 2)
    second = _inputs(12, S, Sx, 4 if dim == 2 else 2)
    p = hh.make_params(dim, n, k, levels, overlap, rank, over, 1, 1e-10, 100, "fp64", 0)
    h, _ = hh.hh_setup(p)
    try:
        want = [hh.hh_residual(h, *first), hh.hh_residual(h, *second)]
    finally:
        hh.hh_destroy(h)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    got = [hh.hh_residual_noalloc(dim, n, k, *first), hh.hh_residual_noalloc(dim, n, k, *second)]
    again = hh.hh_residual_noalloc(dim, n, k, *first)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    for a, b in zip(got, want):
        assert np.isfinite(a) and a > 0
        assert abs(a - b) <= 1e-12 * b, (a, b)
    assert again == got[0]       # fixed summation order: bit-identical on a repeat


@pytest.mark.gpu
def test_noalloc_zero_rhs_and_exact_solution(hh):
    # b = 0 gives 0 (as hh_residual does); u = 0 gives exactly 1
    n, k = 45, 12.0
    S = n + 2
    z = torch.zeros((S, S), dtype=torch.complex128, device="cuda")
    gz = torch.zeros((4, S), dtype=torch.complex128, device="cuda")
    f, g, _ = _inputs(13, S, S, 4)
    assert hh.hh_residual_noalloc(2, n, k, z, gz, f) == 0.0
    assert hh.hh_residual_noalloc(2, n, k, f, g, z) == pytest.approx(1.0, abs=1e-15)


@pytest.mark.gpu
@pytest.mark.parametrize("dim,n,k", [(2, 45, 12.0), (2, 1023, 100.0), (1, 1000, 62.83),
                                     (1, 16382, 500.0), (1, 16381, 500.0)],
                         ids=["d2n45", "d2n1023", "d1n1000", "d1_at_cap", "d1_below_cap"])
def test_noalloc_matches_the_oracle_residual(hh, dim, n, k):
    """The oracle's residual of random data, up to the largest size the static scratch
    takes (n + 2 = HH_NOALLOC_MAX_ROWS grid rows: more rows than the launch has warps, so
    the kernel's grid-stride loop runs).  Both sides sum in FP64 in different orders:
    1e-12 relative."""
    S = n + 2
    assert S <= hh.HH_NOALLOC_MAX_ROWS
    Sx = S if dim == 2 else 1
    f = random_complex((S, Sx), 21)
    g = random_complex((4, S) if dim == 2 else (2,), 22)
    u = random_complex((S, Sx), 23)
    P = Problem(dim, n, k)
    b = P.rhs(f.reshape(-1) if dim == 1 else f, g)
    want = float(np.linalg.norm(b - P.A() @ u.reshape(-1)) / np.linalg.norm(b))
    d = [torch.from_numpy(x).cuda() for x in (f, g, u)]
    got = [hh.hh_residual_noalloc(dim, n, k, *d) for _ in range(2)]
    for a in got:
        assert abs(a - want) <= 1e-12 * want, (a, want)
    assert got[0] == got[1]
