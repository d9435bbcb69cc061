"""Leaf solves at the full-size leaf shapes, through the C-ABI, against the oracle.

The subdomain solves x = A~_leaf^{-1} v of Eq. (2) at the shapes the named workloads
actually run:
* 255 x 255 interior grid, 2 levels, overlap 2: four bands of 65 and 66 rows, 257 columns;
* 1023 x 1023 interior grid, 3 levels, overlap 4: eight bands of 130 to 132 rows, 1025
  columns.
Both leaf paths (the Schur recursion in the column eigenbasis, and explicit inverses with
block substitution), both precision forms, and one right-hand side (the ORAS sweep) as
well as r + p of them (the sketch).  With r + p columns the eigenbasis path runs its
multi-column kernels (transform, recursions, transform back) rather than the one-launch
single-vector sweep, so both are covered at these sizes.

The oracle's leaf solve is a sparse LU of the same band operator (R3 reading: the band's
rows with impedance rows and zero data on its artificial boundaries).

Tolerances (relative 2-norm error over the whole block): FP64 1e-11, as for the small
bands (rounding times the band's condition number).  Complex64: FP32 rounding (6e-8)
amplified by the band's condition number and, on the eigenbasis path, by cond(V)^2 of
the column-pencil eigenvectors (at most 25 here, `tests/test_leaf_eigenbasis.py`):
5e-4 on both paths.  The same recursion carried out in complex64 on the host gives
1.1e-5 at the 66-row bands and 5.2e-5 at the 132-row bands (`test_leaf_eigenbasis.py`).
"""
import numpy as np
import pytest

from oracle.method import OMethod
from oracle.problem import Problem
from workloads import WORKLOADS, random_complex

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = {"n255": WORKLOADS["helm2d_n255_k40_L2"], "n1023": WORKLOADS["helm2d_n1023_k100_L3"]}
TOL = {"fp64": 1e-11, "mixed": 5e-4}


@pytest.fixture(scope="module")
def hh():
    from paper_2512_12538_gb300 import build
    build.build()
    import paper_2512_12538_gb300 as m
    return m


_oracles = {}


def _oracle(name):
    """The oracle with its leaf bands factored (no coarse spaces: rank 0)."""
    if name not in _oracles:
        w = SHAPES[name]
        P = Problem(2, w.n, w.k)
        _oracles[name] = (P, OMethod(P, w.levels, w.overlap, 0, 0))
    return _oracles[name]


# mixed form, eigenbasis path: the multi-vector transforms as the autotuner picks them
# (flags 0), forced onto the CUDA cores (HH_FLAG_CUDA_CORE_SWEEPS) and forced onto the
# tensor cores (HH_FLAG_TENSOR_CORE_SWEEPS)
CASES = [(ls, pr, 0) for ls in ("eigen", "block") for pr in ("fp64", "mixed")] + [("eigen", "mixed", 2),
                                                                                  ("eigen", "mixed", 4)]


@pytest.mark.parametrize("name", ["n255", "n1023"])
@pytest.mark.parametrize("leaf_solver,precision,flags", CASES, ids=lambda c: str(c))
def test_leaf_solve_at_full_size_shapes(hh, name, leaf_solver, precision, flags):
    w = SHAPES[name]
    if leaf_solver == "block" and precision == "fp64" and name == "n1023":
        # a 132 x 132 complex128 inverse does not fit one block's shared memory: the
        # library rejects the parameters (checked below) rather than running it
        p = hh.make_params(2, w.n, w.k, w.levels, w.overlap, w.rank, w.oversample, 1, 1e-10, 10, precision, 1,
                           leaf_solver)
        with pytest.raises(hh.HHError) as ei:
            hh.hh_setup(p)
        assert ei.value.status == hh.HH_EINVAL
        return
    P, O = _oracle(name)
    p = hh.make_params(2, w.n, w.k, w.levels, w.overlap, w.rank, w.oversample, 1, 1e-10, 10, precision, 1,
                       leaf_solver, flags=flags)
    h, _ = hh.hh_setup(p)
    m = w.rank + w.oversample
    try:
        leaves = [nd.id for nd in O.tree if nd.is_leaf]
        rows = sorted({O.tree[i].b for i in leaves})
        assert rows == ([65, 66] if name == "n255" else [130, 131, 132])
        for leaf in leaves:
            nd = O.tree[leaf]
            for nc in (1, m):
                v = random_complex((nd.b, P.Sx, nc), 1000 * leaf + nc)
                x = torch.empty((nd.b, P.Sx, nc), dtype=torch.complex128, device="cuda")
                hh.hh_leaf_solve(h, leaf, torch.from_numpy(v).cuda(), x, nc)
                torch.cuda.synchronize()
                want = O.leaf_solve(leaf, v)
                err = float(np.linalg.norm(x.cpu().numpy() - want) / np.linalg.norm(want))
                print(f"{name} {leaf_solver} {precision} flags={flags} leaf {leaf} (b={nd.b}) nc={nc}: {err:.2e}")
                assert err < TOL[precision], (leaf, nc, err)
    finally:
        hh.hh_destroy(h)
