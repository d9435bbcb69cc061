"""The ctypes binding agrees with include/hh.h: every enum constant and macro has the
header's value, every status has its own message, and the parameter and statistics
structs have the header's field order, offsets and sizes as a C compiler lays them out.
Host only: the library is loaded, nothing is computed."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hh.h")


def _header():
    with open(HEADER) as fh:
        return re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)


def _enum_values(src):
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(HH_[A-Z_0-9]+)\s*=\s*(-?\d+)", src)}


def _struct_fields(src, name):
    m = re.search(r"typedef\s+struct\s*\{([^{}]*)\}\s*" + name + r"\s*;", src)
    assert m, name
    return re.findall(r"\b([a-z_][a-z_0-9]*)\s*;", m.group(1))


@pytest.fixture(scope="module")
def hh():
    from paper_2512_12538_gb300 import build
    build.build()
    import paper_2512_12538_gb300 as m
    return m


def test_enum_constants_match_the_header(hh):
    from paper_2512_12538_gb300 import _lib
    vals = _enum_values(_header())
    assert len(vals) >= 16
    for name, v in vals.items():
        assert getattr(_lib, name) == v, name
    macro = re.search(r"#define\s+HH_NOALLOC_MAX_ROWS\s+(\d+)", _header())
    assert macro and _lib.HH_NOALLOC_MAX_ROWS == int(macro.group(1))
    for name in ("HH_FLAG_COARSE_FP32", "HH_FLAG_CUDA_CORE_SWEEPS", "HH_FLAG_TENSOR_CORE_SWEEPS", "HH_FLAG_BILINEAR"):
        flag = re.search(r"#define\s+" + name + r"\s+(\d+)u", _header())
        assert flag and getattr(_lib, name) == int(flag.group(1)), name


def test_every_status_has_its_own_message(hh):
    codes = sorted(v for k, v in _enum_values(_header()).items()
                   if k in ("HH_OK",) or re.fullmatch(r"HH_E[A-Z]+", k))
    assert codes == list(range(-9, 1))
    msgs = [hh.status_string(c) for c in codes]
    assert all(m and m != "unknown status" for m in msgs)
    assert len(set(msgs)) == len(msgs)
    assert hh.status_string(-100) == "unknown status"
    assert hh.status_string(7) == "unknown status"


@pytest.mark.parametrize("struct", ["hh_params", "hh_stats"])
def test_struct_field_order_matches_the_header(hh, struct):
    from paper_2512_12538_gb300 import _lib
    cls = getattr(_lib, struct)
    assert [f for f, _ in cls._fields_] == _struct_fields(_header(), struct)


def test_struct_offsets_match_the_c_compiler(hh, tmp_path):
    """Offsets and sizes from gcc, compiled against the header itself."""
    from paper_2512_12538_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = _header()
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "hh.h"', "int main(void) {"]
    for struct in ("hh_params", "hh_stats"):
        lines.append(f'printf("{struct} size %zu\\n", sizeof({struct}));')
        for f in _struct_fields(src, struct):
            lines.append(f'printf("{struct} {f} %zu\\n", offsetof({struct}, {f}));')
    lines += ["return 0;", "}"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in filter(None, out):
        s, f, v = line.split()
        got[(s, f)] = int(v)
    for struct in ("hh_params", "hh_stats"):
        cls = getattr(_lib, struct)
        assert ctypes.sizeof(cls) == got[(struct, "size")], struct
        for f, _ in cls._fields_:
            assert getattr(cls, f).offset == got[(struct, f)], (struct, f)
