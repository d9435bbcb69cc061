"""Interface-map spectrum diagnostics on the GPU (Sec. 2, the discussion of Fig. 4).

The randomised SVD of each interface map T_c runs on the GPU during the set-up; its
r + p singular values come back through hh_get_basis.  Two diagnostics are checked
against the oracle:

1. The count of singular values above a fixed level (1e-2) follows the paper's trend:
   at hk = 1 it grows about linearly with k (about doubling per doubling of n).  The
   GPU's count from its sketch (64 samples) equals the count from the oracle's dense SVD
   of the explicitly formed T_c, within one value at the sample edge.
2. The gain of the interface map, ||T_c g||^2 / ||g||^2 for interface data g, and of the
   round trip through both siblings (T_s T_c: data on c's interface, through c and then
   through s back to c), computed from the GPU's interface maps, equals the oracle's:
   the quantity the paper compares with the contraction of the Despres iteration.
"""
import numpy as np
import pytest

from oracle.method import OMethod
from oracle.problem import Problem
from workloads import random_complex

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LEVEL = 1e-2


@pytest.fixture(scope="module")
def hh():
    from paper_2512_12538_gb300 import build
    build.build()
    import paper_2512_12538_gb300 as m
    return m


def _gpu_sigma(hh, n, k, overlap, precision="fp64"):
    """The GPU sketch's singular values of T_1 (64 samples: r = 32, p = 32)."""
    m = min(64, n + 2)
    r = min(32, m // 2)
    p = hh.make_params(2, n, k, 1, overlap, r, m - r, 1, 1e-10, 10, precision, 7)
    h, _ = hh.hh_setup(p)
    try:
        V = np.zeros((n + 2, r), dtype=np.complex128)
        sig = np.zeros(m)
        hh.hh_get_basis(h, 1, V, sig)
        return sig
    finally:
        hh.hh_destroy(h)


def _dense_sigma(n, k, overlap):
    M = OMethod(Problem(2, n, k), 1, overlap, 1, 0, seed=1)
    return np.linalg.svd(M.T(1, np.eye(M.Sx, dtype=complex)), compute_uv=False)


def test_singular_value_counts_grow_linearly_with_k_at_hk_1(hh):
    counts = []
    for n in (15, 31, 63):
        k = n + 1.0                                      # h k = 1
        s_gpu = _gpu_sigma(hh, n, k, 4)
        s_dense = _dense_sigma(n, k, 4)
        c_gpu, c_dense = int((s_gpu > LEVEL).sum()), int((s_dense > LEVEL).sum())
        print(f"n={n} k={k}: sigma > {LEVEL}: GPU sketch {c_gpu}, dense {c_dense}; "
              f"sigma_0 GPU {s_gpu[0]:.6e} dense {s_dense[0]:.6e}")
        assert c_dense < len(s_gpu)                      # the sketch's samples cover the count
        assert abs(c_gpu - c_dense) <= 1
        if len(s_gpu) == len(s_dense):
            # samples span the whole interface: the sketch's values are T's own
            np.testing.assert_allclose(s_gpu, s_dense, rtol=1e-8, atol=1e-10 * s_dense[0])
        else:
            # fewer samples than the interface dimension: the sketch's values interlace
            # below T's (sigma_i(Q^H T) <= sigma_i(T)), close for the leading ones
            assert np.all(s_gpu <= s_dense[:len(s_gpu)] * (1 + 1e-10) + 1e-13)
            assert s_gpu[0] >= s_dense[0] * (1 - 1e-4)
        counts.append(c_gpu)
    for a, b in zip(counts, counts[1:]):
        assert 1.6 < b / a < 2.4, counts


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_interface_map_gains_match_the_oracle(hh, precision, tol):
    n, k = 63, 40.0
    P = Problem(2, n, k)
    O = OMethod(P, 2, 2, 8, 4, seed=3)
    p = hh.make_params(2, n, k, 2, 2, 8, 4, 1, 1e-10, 10, precision, 3)
    h, _ = hh.hh_setup(p)
    try:
        G = random_complex((P.Sx, 8), 41)
        for c, s in ((3, 4), (5, 6), (1, 2)):
            y = torch.empty((P.Sx, 8), dtype=torch.complex128, device="cuda")
            z = torch.empty_like(y)
            hh.hh_interface_map(h, c, 0, torch.from_numpy(G).cuda(), y, 8)
            hh.hh_interface_map(h, s, 0, y, z, 8)
            torch.cuda.synchronize()
            Y, Z = y.cpu().numpy(), z.cpu().numpy()
            gain = (np.linalg.norm(Y, axis=0) / np.linalg.norm(G, axis=0)) ** 2
            trip = (np.linalg.norm(Z, axis=0) / np.linalg.norm(G, axis=0)) ** 2
            Yo = O.T(c, G)
            gain_o = (np.linalg.norm(Yo, axis=0) / np.linalg.norm(G, axis=0)) ** 2
            trip_o = (np.linalg.norm(O.T(s, Yo), axis=0) / np.linalg.norm(G, axis=0)) ** 2
            print(f"{precision} child {c}: gain {gain.mean():.4e} (oracle {gain_o.mean():.4e}), "
                  f"round trip {trip.mean():.4e} (oracle {trip_o.mean():.4e})")
            np.testing.assert_allclose(gain, gain_o, rtol=tol)
            np.testing.assert_allclose(trip, trip_o, rtol=tol)
    finally:
        hh.hh_destroy(h)
