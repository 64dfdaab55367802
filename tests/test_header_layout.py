"""The Python binding's view of include/mf.h: every parameter struct passed
by pointer has the same size and field offsets in the binding's ctypes mirror
as in the header compiled by the host C compiler, and the binding's status
codes, form numbers and radial-kernel numbers equal the header's enums."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

import paper_2508_04172_gb300 as mf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mf.h")

# C struct name -> ctypes mirror in the binding
MIRRORS = {
    "mf_mlp_train_params": mf.MlpTrainParams,
    "mf_surrogate_params": mf.SurrogateParams,
    "mf_wave": mf.Wave,
    "mf_ns_params": mf.NsParams,
    "mf_ns_result": mf.NsResult,
}


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{HEADER}"', "int main(void) {"]
    for cname, py in MIRRORS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    p = subprocess.run([cc, "-std=c11", "-Wall", "-o", str(exe), str(src)], capture_output=True, text=True)
    assert p.returncode == 0, p.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {}
    for ln in out.splitlines():
        cname, field, val = ln.split()
        got[(cname, field)] = int(val)
    return got


def test_ctypes_mirrors_match_the_header(tmp_path):
    got = _c_layout(tmp_path)
    for cname, py in MIRRORS.items():
        assert ctypes.sizeof(py) == got[(cname, "size")], cname
        for fname, _ in py._fields_:
            assert getattr(py, fname).offset == got[(cname, fname)], (cname, fname)


def _enum_values(prefix):
    src = open(HEADER).read()
    return {m.group(1): int(m.group(2)) for m in re.finditer(rf"\b({prefix}\w+)\s*=\s*(-?\d+)", src)}


def test_status_codes_match_the_header():
    codes = _enum_values("MF_E_")
    codes.update(_enum_values("MF_OK"))
    assert codes, "no status codes parsed"
    for name, val in codes.items():
        assert getattr(mf, name) == val, name


def test_form_and_kernel_numbers_match_the_header():
    forms = _enum_values("MF_FORM_")
    assert {("MF_FORM_" + k.upper()): v for k, v in mf.FORMS.items()} == forms
    kernels = _enum_values("MF_RBF_")
    assert {("MF_RBF_" + k.upper()): i for i, k in enumerate(mf.RBF_KERNELS)} == kernels


def test_noalloc_limit_is_the_declared_one():
    src = open(HEADER).read()
    m = re.search(r"#define\s+MF_NOALLOC_MAX_PARTIAL\s+(\d+)", src)
    assert m and int(m.group(1)) == 4194304 == 16 * 1024 * 1024 // 4
