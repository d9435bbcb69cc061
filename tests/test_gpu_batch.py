"""Batching form (many independent problems set up and solved together) against the
direct solution and against the same problems solved one at a time."""
import numpy as np
import pytest

from oracle import direct
from oracle.problem import Problem
from workloads import Workload, batch_problems, point_source_rhs

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hh():
    from paper_2512_12538_gb300 import build
    build.build()
    import paper_2512_12538_gb300 as m
    return m


def _params(hh, probs, precision="mixed", outer="oras"):
    return [hh.make_params(2, w.n, w.k, w.levels, w.overlap, w.rank, w.oversample, 1, 1e-10, 400, precision, 1 + i,
                           outer=outer) for i, (w, f, g) in enumerate(probs)]


def test_setup_batch_rejects_invalid_parameters(hh):
    # host-side validation: nothing reaches the device
    probs = batch_problems(2, sides=(63,))
    ps = _params(hh, probs)
    ps[1] = hh.make_params(2, 63, 20.0, 2, 3, 16, 8)        # odd overlap
    with pytest.raises(hh.HHError) as ei:
        hh.hh_setup_batch(ps, stream=0)
    assert ei.value.status == hh.HH_EINVAL


def _solve_batch(hh, probs, params):
    hs = hh.hh_setup_batch(params)
    try:
        us = [torch.empty((w.S, w.S), dtype=torch.complex128, device="cuda") for (w, f, g) in probs]
        sts = hh.hh_solve_batch(hs, [torch.from_numpy(f).cuda() for (w, f, g) in probs],
                                [torch.from_numpy(g).cuda() for (w, f, g) in probs], us)
        return [u.cpu().numpy() for u in us], sts
    finally:
        for h in hs:
            hh.hh_destroy(h)


def _solve_alone(hh, w, f, g, p):
    h, _ = hh.hh_setup(p)
    try:
        u = torch.empty((w.S, w.S), dtype=torch.complex128, device="cuda")
        st = hh.hh_solve(h, torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), u, allow_noconv=True)
        return u.cpu().numpy(), st
    finally:
        hh.hh_destroy(h)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol,count", [("mixed", 1e-8, 16), ("fp64", 1e-10, 8)])
def test_batch_matches_direct_and_solo(hh, precision, tol, count):
    """The batch configuration's whole range: grid sides 63 to 255 and k h drawn from
    [0.3, 0.6].  Every problem's result is compared with u*.  Each problem is also solved
    alone by the stationary iteration: where that converges in as many steps as the
    problem took in the batch, the lockstep arithmetic is the same per problem, so the
    two iterates agree up to the order of the partial sums (1e-12).  Problems whose
    stationary iteration stalls or diverges are handed to GMRES inside the batch, so
    their batch and solo runs differ; for those the comparison with u* decides."""
    sides = (63, 127, 191, 255) if precision == "mixed" else (63, 127, 191)
    probs = batch_problems(count, sides=sides, kh=(0.3, 0.6))
    params = _params(hh, probs, precision)
    got, sts = _solve_batch(hh, probs, params)
    same = 0
    for i, (w, f, g) in enumerate(probs):
        us = direct.solve(Problem(2, w.n, w.k), f, g).reshape(w.S, w.S)
        err = _rel(got[i], us)
        kh = w.k / (w.n + 1)
        print(f"{w.name} kh={kh:.3f}: iters {sts[i].iters}, err {err:.2e}")
        assert sts[i].rel_res < 1e-10
        assert err < tol, (w.name, sts[i].iters)
        alone, st1 = _solve_alone(hh, w, f, g, params[i])
        if st1.rel_res < 1e-10 and st1.iters == sts[i].iters:
            assert _rel(got[i], alone) < 1e-12
            same += 1
    assert same >= count // 2, same


@pytest.mark.gpu
def test_batch_with_a_non_lockstep_member_solves_one_by_one(hh):
    probs = batch_problems(3, sides=(63, 127))
    params = _params(hh, probs)
    params[1] = _params(hh, [probs[1]], outer="gmres")[0]
    got, sts = _solve_batch(hh, probs, params)
    for i, (w, f, g) in enumerate(probs):
        us = direct.solve(Problem(2, w.n, w.k), f, g).reshape(w.S, w.S)
        assert _rel(got[i], us) < 1e-8


@pytest.mark.gpu
def test_batch_rescues_problems_the_stationary_iteration_does_not_converge(hh):
    # n = 63 with k h = 0.47 and 0.57: the stationary ORAS iteration with n_i = 1 diverges
    # there (its residual grows); the batch hands such problems to flexible GMRES
    probs = batch_problems(3, sides=(127,), kh=(0.3, 0.35))
    for n, kh in ((63, 0.47), (63, 0.57)):
        w = Workload(f"div_n{n}", 2, n, kh * (n + 1), 2, 2, 16, 8)
        probs.append((w, point_source_rhs(n, 99 + n), np.zeros((4, n + 2), dtype=np.complex128)))
    got, sts = _solve_batch(hh, probs, _params(hh, probs))
    for i, (w, f, g) in enumerate(probs):
        us = direct.solve(Problem(2, w.n, w.k), f, g).reshape(w.S, w.S)
        assert sts[i].rel_res < 1e-10
        assert _rel(got[i], us) < 1e-8, (w.name, sts[i].iters)
