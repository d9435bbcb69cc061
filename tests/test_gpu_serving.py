"""Serving form: requests of different sizes arriving while others are in flight give
the same results as when each is solved alone, and admission respects the HBM budget."""
import time

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


def test_server_rejects_invalid_arguments(hh):
    for budget, slots in ((0, 4), (1 << 30, 0), (1 << 30, 5000)):
        with pytest.raises(hh.HHError) as ei:
            hh.hh_server_create(budget, slots)
        assert ei.value.status == hh.HH_EINVAL


def _params(hh, w, i, outer="oras"):
    return hh.make_params(2, w.n, w.k, w.levels, w.overlap, w.rank, w.oversample, 1, 1e-10, 400, "mixed", 1 + i,
                          outer=outer)


def _wait(hh, srv, tickets, timeout_s=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        assert time.time() - t0 < timeout_s, "requests did not finish"
        for i, t in enumerate(tickets):
            if i in out:
                continue
            r = hh.hh_server_poll(srv, t)
            if r is not None:
                out[i] = r
        time.sleep(0.0005)
    return [out[i] for i in range(len(tickets))]


def _alone(hh, w, f, g, p):
    h, _ = hh.hh_setup(p)
    try:
        u = torch.empty((w.S, w.S), dtype=torch.complex128, device="cuda")
        st = hh.hh_solve(h, torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), u, allow_noconv=True)
        return u.cpu().numpy(), st
    finally:
        hh.hh_destroy(h)


@pytest.mark.gpu
def test_served_results_equal_solo_results(hh):
    """Requests of every serving size (sides 63 to 1023; k h from 0.3 to 0.6 on the small
    ones, the 3-level hierarchy with r = 32 on 511 and 1023) arriving while others are in
    flight.  Each result is compared with u*; where the request's stationary iteration
    alone converges in as many steps as it took in the server, the served result equals
    the solo one to 1e-12 (the same arithmetic, summed in another order)."""
    probs = batch_problems(8, sides=(63, 127, 255), kh=(0.3, 0.6))
    # one request the lockstep iteration does not take (GMRES outer) and one whose
    # stationary iteration diverges (handed to GMRES)
    w = Workload("div", 2, 63, 0.47 * 64, 2, 2, 16, 8)
    probs.append((w, point_source_rhs(63, 123), np.zeros((4, 65), dtype=np.complex128)))
    for n, k in ((511, 150.0), (1023, 100.0)):
        w = Workload(f"big{n}", 2, n, k, 3, 4, 32, 10)
        probs.append((w, point_source_rhs(n, 7 + n), np.zeros((4, n + 2), dtype=np.complex128)))
    outers = ["oras"] * len(probs)
    outers[2] = "gmres"
    params = [_params(hh, w, i, outers[i]) for i, (w, f, g) in enumerate(probs)]
    fs = [torch.from_numpy(f).cuda() for (w, f, g) in probs]
    gs = [torch.from_numpy(g).cuda() for (w, f, g) in probs]
    us = [torch.zeros((w.S, w.S), dtype=torch.complex128, device="cuda") for (w, f, g) in probs]
    torch.cuda.synchronize()
    srv = hh.hh_server_create(16 << 30, 16)
    try:
        tickets = []
        for i in range(len(probs)):
            tickets.append(hh.hh_server_submit(srv, params[i], fs[i], gs[i], us[i]))
            time.sleep(0.002)   # later requests arrive while earlier ones iterate
        res = _wait(hh, srv, tickets)
    finally:
        hh.hh_server_destroy(srv)
    same = 0
    for i, (w, f, g) in enumerate(probs):
        st, stats = res[i]
        assert st == hh.HH_OK and stats.rel_res < 1e-10, (w.name, st)
        got = us[i].cpu().numpy()
        ud = direct.solve(Problem(2, w.n, w.k), f, g).reshape(w.S, w.S)
        err = np.linalg.norm(got - ud) / np.linalg.norm(ud)
        print(f"{w.name} kh={w.k / (w.n + 1):.3f} {outers[i]}: iters {stats.iters}, err {err:.2e}")
        assert err < 1e-8
        if outers[i] == "oras":
            alone, st1 = _alone(hh, w, f, g, params[i])
            if st1.rel_res < 1e-10 and st1.iters == stats.iters:
                assert np.linalg.norm(got - alone) / np.linalg.norm(alone) < 1e-12
                same += 1
        assert stats.t_total_ms >= stats.t_queue_ms >= 0.0
    assert same >= len(probs) // 2, same


@pytest.mark.gpu
def test_admission_keeps_footprints_within_budget(hh):
    probs = batch_problems(3, sides=(127,), kh=(0.3, 0.35))
    params = [_params(hh, w, i) for i, (w, f, g) in enumerate(probs)]
    fp = max(hh.hh_footprint(p) for p in params)
    fs = [torch.from_numpy(f).cuda() for (w, f, g) in probs]
    gs = [torch.from_numpy(g).cuda() for (w, f, g) in probs]
    us = [torch.zeros((w.S, w.S), dtype=torch.complex128, device="cuda") for (w, f, g) in probs]
    torch.cuda.synchronize()
    srv = hh.hh_server_create(int(1.5 * fp), 8)   # room for one request at a time
    try:
        with pytest.raises(hh.HHError) as ei:       # larger than the whole budget
            big = hh.make_params(2, 255, 40.0, 2, 2, 16, 10)
            hh.hh_server_submit(srv, big, fs[0], gs[0], us[0])
        assert ei.value.status == hh.HH_ENOMEM
        tickets = [hh.hh_server_submit(srv, params[i], fs[i], gs[i], us[i]) for i in range(3)]
        res = _wait(hh, srv, tickets)
    finally:
        hh.hh_server_destroy(srv)
    assert all(st == hh.HH_OK for st, _ in res)
    # admitted one after another: the last waited for the first two
    assert res[2][1].t_queue_ms > 0.0


@pytest.mark.gpu
def test_requests_cycling_through_few_slots(hh):
    # more requests than slots: problems join the lockstep iteration while others leave
    probs = batch_problems(20, sides=(63, 127), kh=(0.3, 0.35))
    params = [_params(hh, w, i) for i, (w, f, g) in enumerate(probs)]
    fs = [torch.from_numpy(f).cuda() for (w, f, g) in probs]
    gs = [torch.from_numpy(g).cuda() for (w, f, g) in probs]
    us = [torch.zeros((w.S, w.S), dtype=torch.complex128, device="cuda") for (w, f, g) in probs]
    torch.cuda.synchronize()
    srv = hh.hh_server_create(8 << 30, 3)
    try:
        tickets = [hh.hh_server_submit(srv, params[i], fs[i], gs[i], us[i]) for i in range(len(probs))]
        res = _wait(hh, srv, tickets)
    finally:
        hh.hh_server_destroy(srv)
    for i, (w, f, g) in enumerate(probs):
        st, stats = res[i]
        assert st == hh.HH_OK, (w.name, st)
        ud = direct.solve(Problem(2, w.n, w.k), f, g).reshape(w.S, w.S)
        got = us[i].cpu().numpy()
        assert np.linalg.norm(got - ud) / np.linalg.norm(ud) < 1e-8
