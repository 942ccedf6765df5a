"""The C-ABI library builds, loads and exports every symbol include/dloops.h declares (CPU)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    nvcc = os.path.exists("/usr/local/cuda/bin/nvcc")
    from paper_1012_5168_gb300 import build
    if not os.path.exists(build.LIB) and not nvcc:
        pytest.skip("no CUDA toolkit to build the library")
    return build.build()


def _declared():
    text = open(os.path.join(ROOT, "include", "dloops.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dl_[a-z_0-9]+)\s*\(", text)))


def test_header_symbols_exported(libpath):
    declared = _declared()
    assert len(declared) >= 20
    lib = ctypes.CDLL(libpath)
    for name in declared:
        assert hasattr(lib, name), name
    import paper_1012_5168_gb300 as dl
    assert sorted(dl.SYMBOLS) == declared


def test_status_strings_without_gpu(libpath):
    import paper_1012_5168_gb300 as dl
    L = dl.lib()
    assert L.dl_status_string(0) == b"ok"
    assert L.dl_status_string(4) == b"not converged"
    # argument checks happen before any CUDA call
    h = ctypes.c_void_p()
    assert L.dl_create(ctypes.byref(h), (ctypes.c_int * 4)(4, 4, 3, 4), -1, None) == dl.EINVAL
    assert L.dl_create(ctypes.byref(h), (ctypes.c_int * 4)(4, 4, 4, 4), 0, None) == dl.EINVAL
    assert L.dl_create(None, (ctypes.c_int * 4)(4, 4, 4, 4), -1, None) == dl.EINVAL


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1012_5168_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f


def test_struct_layouts_match_the_binding(tmp_path):
    """sizeof and field offsets of the ABI structs, from the C compiler, equal the ctypes mirrors."""
    import shutil
    import subprocess
    import paper_1012_5168_gb300 as dl
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = {"dl_solve_params": dl.SolveParams, "dl_solve_stats": dl.SolveStats, "dl_smear": dl.Smear,
               "dl_timing": dl.Timing}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "dloops.h"', "int main(void) {"]
    for name, py in mirrors.items():
        lines.append(f'printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in py._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    for name, py in mirrors.items():
        assert got[(name, "sizeof")] == ctypes.sizeof(py), name
        for field, _ in py._fields_:
            assert got[(name, field)] == getattr(py, field).offset, (name, field)


def test_build_compiles_every_unit():
    """Every CUDA translation unit under csrc/ is in the build (and nothing else)."""
    from paper_1012_5168_gb300 import build
    units = sorted(f for f in os.listdir(build.CSRC) if f.endswith(".cu"))
    assert sorted(build.UNITS) == units
