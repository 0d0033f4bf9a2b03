"""The C ABI library builds, loads and exports every symbol include/f3r.h declares.

Runs without a GPU: no compute call is made.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(f3r_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libf3r():
    from paper_2505_20719_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(libf3r):
    names = _declared("f3r.h")
    assert "f3r_setup" in names and "f3r_solve" in names and "f3r_spmv" in names
    for name in names:
        assert hasattr(libf3r, name), name


def test_default_params_without_gpu(libf3r):
    from paper_2505_20719_gb300 import f3r
    p = f3r.default_params()
    assert (p.nlevels, p.m[0], p.m[1], p.m[2], p.rich_m, p.c) == (3, 100, 8, 4, 2, 64)
    assert (p.a_prec[0], p.a_prec[1], p.a_prec[2], p.rich_a_prec) == (f3r.F64, f3r.F32, f3r.F16, f3r.F16)
    assert (p.v_prec[0], p.v_prec[1], p.v_prec[2], p.rich_v_prec) == (f3r.F64, f3r.F32, f3r.F32, f3r.F16)
    assert p.tol == 1e-9 and p.max_outer == 300 and p.cgs_passes == 2


def test_status_strings(libf3r):
    libf3r.f3r_status_str.restype = ctypes.c_char_p
    assert libf3r.f3r_status_str(0) == b"ok"
    assert libf3r.f3r_status_str(4) == b"not converged"


def test_setup_rejects_bad_arguments_before_touching_the_gpu(libf3r):
    from paper_2505_20719_gb300 import f3r
    h = ctypes.c_void_p()
    # n <= 0 is rejected by argument checks alone
    code = libf3r.f3r_setup(ctypes.byref(h), 0, 0, None, None, None, None, None)
    assert code == f3r.ERR_ARG


def test_cuda_sources_target_sm103a_only():
    from paper_2505_20719_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    src = os.path.join(ROOT, "paper_2505_20719_gb300", "csrc")
    for f in os.listdir(src):
        text = open(os.path.join(src, f)).read()
        assert "oracle" not in text.lower() or f.endswith(".md"), f


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs have the C compiler's size
    and field offsets (compiled against include/f3r.h with gcc)."""
    import shutil
    import subprocess

    from paper_2505_20719_gb300 import f3r

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"f3r_params": f3r.Params, "f3r_stats": f3r.Stats, "f3r_system_desc": f3r.SystemDesc,
               "f3r_batch_result": f3r.BatchResult}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "f3r.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for line in out:
        if not line:
            continue
        cname, key, value = line.split()
        py = structs[cname]
        want = ctypes.sizeof(py) if key == "size" else getattr(py, key).offset
        assert int(value) == want, (cname, key, value, want)
        seen += 1
    assert seen == sum(1 + len(py._fields_) for py in structs.values())
