"""The bench's stopping tolerance reaches relative error 1e-8 on the bench workload, in
both precision forms and with a 10x margin, and the tracing hooks the bench relies on work."""
import numpy as np
import pytest

from oracle import direct
from oracle.problem import Problem
from workloads import WORKLOADS, problem_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hh():
    from paper_2512_12538_gb300 import build
    build.build()
    import paper_2512_12538_gb300 as m
    return m


@pytest.fixture(scope="module")
def case():
    import bench
    w = WORKLOADS[bench.WORKLOAD]
    f, g = problem_inputs(w)
    P = Problem(2, w.n, w.k)
    return bench, w, f, g, direct.solve(P, f, g)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_bench_tolerance_gives_rel_err_1e8_with_margin(hh, case, precision):
    bench, w, f, g, us = case
    p = hh.make_params(2, w.n, w.k, w.levels, w.overlap, w.rank, w.oversample, w.n_inner, bench.TOL,
                       bench.MAX_ITER, precision, 1, outer=bench.OUTER, restart=bench.RESTART)
    h, _ = hh.hh_setup(p)
    try:
        u = torch.empty((w.S, w.S), dtype=torch.complex128, device="cuda")
        st = hh.hh_solve(h, torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), u)
        err = direct.rel_err(u.cpu().numpy(), us)
        print(f"{precision}: iters={st.iters} rel_res={st.rel_res:.2e} err={err:.2e}")
        # the metric asks for 1e-8; the bench's tolerance must keep a 10x margin
        assert err <= 1e-9
    finally:
        hh.hh_destroy(h)


def test_profiler_and_launch_counter(hh, case):
    bench, w, f, g, us = case
    p = hh.make_params(2, 45, 12.0, 2, 2, 6, 4, 1, 1e-10, 300, "mixed", 0)
    n0 = hh.hh_launch_count()
    hh.hh_profile_enable(None, True)
    h, _ = hh.hh_setup(p)
    hh.hh_profile_enable(None, False)
    try:
        P = Problem(2, 45, 12.0)
        fd = torch.zeros((P.S, P.S), dtype=torch.complex128, device="cuda")
        fd[10, 10] = 1.0
        gd = torch.zeros((4, P.S), dtype=torch.complex128, device="cuda")
        u = torch.empty_like(fd)
        st = hh.hh_solve(h, fd, gd, u)
        prof = hh.hh_profile_read(h)
        work = hh.hh_profile_read(h, work=True)
        assert work["sweep_recur"][2] > 0 and work["sweep_in"][3] > 0 and work["coarse_project"][2] > 0
        assert work["leaf_sweep"][2] > 0 and work["leaf_sweep"][3] > 0
        assert prof["factor"][1] == 1 and prof["factor"][0] > 0
        for stage in ("sweep_in", "sweep_recur", "sweep_out"):
            assert prof[stage][1] == 6                   # 3 multi-vector sketch passes per level
        assert prof["leaf_sweep"][1] == st.iters         # one single-vector sweep per iteration
        assert prof["galerkin"][1] == 3 and prof["svd"][1] == 2 and prof["qr"][1] == 2
        assert hh.hh_launch_count() - n0 > 50
    finally:
        hh.hh_destroy(h)
