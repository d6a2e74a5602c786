"""The C-ABI library builds, loads and exports every entry point of include/mra.h.

No compute call is made here, so these tests need no GPU.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mra.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mra_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1507_04789_gb300 import build, mra
    if not os.path.exists(mra.LIB_PATH):
        build.build()
    return ctypes.CDLL(mra.LIB_PATH)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mra_build", "mra_loglik", "mra_predict", "mra_free", "mra_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared in mra.h but not exported: {missing}"


def test_binding_signatures_load(lib):
    from paper_1507_04789_gb300 import mra
    L = mra.load_library()
    assert L.mra_last_error() is not None


def test_argument_errors_need_no_gpu(lib):
    """Invalid configurations are rejected on the host before any CUDA call."""
    from paper_1507_04789_gb300 import mra
    import numpy as np
    with pytest.raises(mra.MRAError) as ei:
        mra.Handle(np.zeros((4, 2)), np.zeros(4), M=2, r=16, J=3)
    assert ei.value.code == mra.MRA_ERR_ARG
    with pytest.raises(mra.MRAError) as ei:
        mra.Handle(np.zeros((4, 2)), np.zeros(4), M=2, r=65)
    assert ei.value.code == mra.MRA_ERR_ARG
    with pytest.raises(mra.MRAError):
        mra.Handle(np.zeros((4, 2)), np.zeros(4), M=13, r=16)


@pytest.mark.parametrize("M,J,prec", [(2, (2, 6), "fp64"), (2, (4, 8), "emu"), (2, (16, 16), "emu"),
                                      (7, (16,) * 6 + (4,), "fp64"), (1, (1,), "fp64")])
def test_level_varying_J_errors_need_no_gpu(lib, M, J, prec):
    """Level-varying J (Sec. 2.2): each J_m in {2, 4, 8, 16}, J_M (the leaves'
    level) 2 or 4 in the emulated form, at most 2^24 leaves; rejected on the host."""
    from paper_1507_04789_gb300 import mra
    import numpy as np
    with pytest.raises(mra.MRAError) as ei:
        mra.Handle(np.zeros((4, 2)), np.zeros(4), M=M, r=16, J=J, precision=prec)
    assert ei.value.code == mra.MRA_ERR_ARG
    with pytest.raises(ValueError):
        mra.Handle(np.zeros((4, 2)), np.zeros(4), M=3, r=16, J=(2, 4))   # one J_m per level


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structs have the header's size and field offsets
    (a C program compiled against include/mra.h prints them)."""
    import shutil
    import subprocess
    from paper_1507_04789_gb300 import mra
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"mra_config": mra.MraConfig, "mra_params": mra.MraParams, "mra_stats_t": mra.MraStats}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "mra.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, f, v = line.split()
        got[(cname, f)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
