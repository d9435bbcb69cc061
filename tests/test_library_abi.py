"""CPU-side checks of the C-ABI library: it builds, loads, and exports every entry point
declared in include/hh.h; host-only calls validate parameters (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "hh.h")) as fh:
        src = fh.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hh_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def hh():
    from paper_2512_12538_gb300 import build
    build.build()
    import paper_2512_12538_gb300 as m
    return m


def test_every_declared_symbol_exported(hh):
    names = _declared()
    assert "hh_setup" in names and "hh_solve" in names
    lib = ctypes.CDLL(hh.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(hh):
    for s in (0, -1, -2, -3, -4, -5, -6, -7):
        assert hh.status_string(s) and hh.status_string(s) != "unknown status"


def test_footprint_host_only_and_validation(hh):
    p = hh.make_params(dim=2, n=255, k=40.0, levels=2, overlap=2, rank=16, oversample=10, leaf_solver="block")
    fp = hh.hh_footprint(p)
    # at least the FP64 explicit leaf inverses: 4 leaves x 257 columns x 65^2 x 16 bytes
    assert fp > 4 * 257 * 65 * 65 * 16
    pm = hh.make_params(dim=2, n=255, k=40.0, levels=2, overlap=2, rank=16, oversample=10, precision="mixed",
                        leaf_solver="block")
    assert hh.hh_footprint(pm) < fp
    pe = hh.make_params(dim=2, n=255, k=40.0, levels=2, overlap=2, rank=16, oversample=10)
    assert hh.hh_footprint(pe) < fp          # the eigenbasis path stores b^2 + Sx b per leaf
    bad = [dict(overlap=3), dict(overlap=0), dict(levels=0), dict(n=2), dict(rank=0), dict(k=-1.0),
           dict(n=20, levels=4), dict(rank=40, oversample=0), dict(dim=3), dict(n_inner=0), dict(tol=0.0),
           dict(leaf_solver=7), dict(outer=3), dict(outer=1, restart=0), dict(outer=1, restart=65),
           dict(n=1023, levels=2), dict(levels=7, n=4000), dict(flags=16), dict(flags=6), dict(flags=0x80000000)]
    for kw in bad:
        args = dict(dim=2, n=255, k=40.0, levels=2, overlap=2, rank=16, oversample=10)
        args.update(kw)
        with pytest.raises(hh.HHError) as ei:
            hh.hh_footprint(hh.make_params(**args))
        assert ei.value.status == hh.HH_EINVAL, kw


def test_block_leaf_path_band_limits(hh):
    # host-side validation only.  The explicit-inverse leaf path takes bands taller than
    # the eigenbasis path's 136 rows, up to what one b x b inverse in shared memory
    # allows: 169 rows in complex64, 119 in complex128.  n = 1200 with 3 levels gives
    # bands of about 154 rows; n = 1023 with 2 levels about 260.
    def fp(n, levels, precision, leaf_solver):
        p = hh.make_params(dim=2, n=n, k=100.0, levels=levels, overlap=4, rank=16, oversample=8,
                           precision=precision, leaf_solver=leaf_solver)
        return hh.hh_footprint(p)

    assert fp(1200, 3, "mixed", "block") > 0
    for n, levels, precision, leaf_solver in ((1200, 3, "mixed", "eigen"), (1200, 3, "fp64", "block"),
                                              (1023, 2, "mixed", "block")):
        with pytest.raises(hh.HHError) as ei:
            fp(n, levels, precision, leaf_solver)
        assert ei.value.status == hh.HH_EINVAL
    assert fp(1023, 3, "mixed", "block") > 0 and fp(1023, 3, "fp64", "eigen") > 0


def test_footprint_1d(hh):
    p = hh.make_params(dim=1, n=1000, k=62.83, levels=1, overlap=4, rank=1, oversample=0)
    assert 0 < hh.hh_footprint(p) < 64 << 20


def test_layered_media_parameters(hh):
    # host-side validation only: one positive finite wavenumber per grid row, and 2D
    # leaves on the explicit-inverse path
    import numpy as np
    kr = np.full(65, 64.0)
    assert hh.hh_footprint(hh.make_params(2, 63, 64.0, 2, 2, 16, 10, leaf_solver="block", k_rows=kr)) > 0
    assert hh.hh_footprint(hh.make_params(1, 63, 64.0, 1, 4, 1, 0, k_rows=kr)) > 0
    bad = kr.copy()
    bad[7] = -1.0
    for p in (hh.make_params(2, 63, 64.0, 2, 2, 16, 10, leaf_solver="eigen", k_rows=kr),
              hh.make_params(2, 63, 64.0, 2, 2, 16, 10, leaf_solver="block", k_rows=bad)):
        with pytest.raises(hh.HHError) as ei:
            hh.hh_footprint(p)
        assert ei.value.status == hh.HH_EINVAL
    with pytest.raises(ValueError):
        hh.make_params(2, 63, 64.0, 2, 2, 16, 10, leaf_solver="block", k_rows=kr[:-1])


def test_bilinear_element_parameters(hh):
    # host-side validation only: the bilinear elements (HH_FLAG_BILINEAR) take 2D problems on
    # the eigenbasis leaves with one wavenumber; their per-mode scales add b per leaf
    import numpy as np
    q1 = hh.HH_FLAG_BILINEAR
    base = hh.hh_footprint(hh.make_params(2, 255, 40.0, 2, 2, 16, 10))
    assert hh.hh_footprint(hh.make_params(2, 255, 40.0, 2, 2, 16, 10, flags=q1)) >= base
    assert hh.hh_footprint(hh.make_params(2, 255, 40.0, 2, 2, 16, 10, precision="mixed",
                                          flags=q1 | hh.HH_FLAG_TENSOR_CORE_SWEEPS)) > 0
    kr = np.full(65, 64.0)
    for p in (hh.make_params(1, 255, 40.0, 1, 4, 1, 0, flags=q1),
              hh.make_params(2, 255, 40.0, 2, 2, 16, 10, leaf_solver="block", flags=q1),
              hh.make_params(2, 63, 64.0, 2, 2, 16, 10, k_rows=kr, flags=q1),
              hh.make_params(2, 63, 64.0, 2, 2, 16, 10, leaf_solver="block", k_rows=kr, flags=q1)):
        with pytest.raises(hh.HHError) as ei:
            hh.hh_footprint(p)
        assert ei.value.status == hh.HH_EINVAL
