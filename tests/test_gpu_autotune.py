"""The sweep autotuner: the first use of each shape times the candidates on the device
and keeps the faster; the report lists every decision with its measured times.  The
choice changes speed only: solutions agree with the direct solution whatever it picks."""
import numpy as np
import pytest

from oracle import direct
from oracle.problem import Problem
from workloads import point_source_rhs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hh():
    from paper_2512_12538_gb300 import build
    build.build()
    import paper_2512_12538_gb300 as m
    return m


def test_autotuner_records_both_candidates_and_solutions_stay_exact(hh):
    n, k = 127, 40.0
    P = Problem(2, n, k)
    f = point_source_rhs(n, 5)
    g = np.zeros((4, P.S), dtype=np.complex128)
    p = hh.make_params(2, n, k, 2, 2, 16, 10, 1, 1e-12, 400, "mixed", 1)
    h, _ = hh.hh_setup(p)
    try:
        u = torch.empty((P.S, P.S), dtype=torch.complex128, device="cuda")
        hh.hh_solve(h, torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), u)
        assert direct.rel_err(u.cpu().numpy(), direct.solve(P, f, g)) < 1e-8
    finally:
        hh.hh_destroy(h)
    rep = hh.hh_autotune_report()
    print(rep)
    tr = [e for e in rep if e["what"].startswith("transform") and e["Sx"] == n + 2]
    assert {e["what"] for e in tr} == {"transform_in", "transform_out"}
    for e in tr:
        assert e["cuda_cores_ms"] > 0 and e["tensor_cores_ms"] > 0
        faster = "tensor_cores" if e["tensor_cores_ms"] < e["cuda_cores_ms"] else "cuda_cores"
        assert e["chosen"] == faster
    cl = [e for e in rep if e["what"] == "fused_sweep_cluster" and e["Sx"] == n + 2]
    for e in cl:
        assert e["chosen"] in (8, 16) and e["cluster16_ms"] > 0 and e["cluster8_ms"] > 0
    # a second handle of the same shapes reuses the decisions
    h, _ = hh.hh_setup(p)
    hh.hh_destroy(h)
    assert len(hh.hh_autotune_report()) == len(rep)
