"""The ctypes mirrors of the C ABI's structs match the header's layout.

A small C program, compiled with the host's gcc against include/smsm.h, prints the size
and every field offset of smsm_opts, smsm_params, smsm_report and smsm_tune_report, and
the values of the flag and status constants; the binding's ctypes structures and
constants must agree field by field (a drift would pass wrong parameters through the ABI
without any error).  Host only.
"""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_1901_01893_gb300 import smsm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "smsm_opts": smsm.Opts,
    "smsm_params": smsm.Params,
    "smsm_report": smsm.Report,
    "smsm_tune_report": smsm.TuneReport,
}
# ctypes field name -> C field name where they differ
RENAME = {"lambda_": "lambda"}
CONSTANTS = ["SMSM_FLAG_GENERIC_KERNELS", "SMSM_FLAG_PER_COIL_NORMAL", "SMSM_FLAG_CLUSTER_EIG",
             "SMSM_ERR_EIG_UNCONVERGED", "SMSM_PRECISION_BF16_SPLIT", "SMSM_MODE_NULLSPACE"]


def _program():
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "smsm.h"', "int main(void) {"]
    for cname, cls in STRUCTS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            c_f = RENAME.get(fname, fname)
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {c_f}));')
    for k in CONSTANTS:
        lines.append(f'  printf("const {k} %d\\n", (int){k});')
    lines += ["  return 0;", "}"]
    return "\n".join(lines) + "\n"


@pytest.fixture(scope="module")
def layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text(_program())
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    res = {}
    for line in out.splitlines():
        a, b, v = line.split()
        res[(a, b)] = int(v)
    return res


@pytest.mark.parametrize("cname", list(STRUCTS))
def test_struct_layout_matches_header(layout, cname):
    cls = STRUCTS[cname]
    assert ctypes.sizeof(cls) == layout[(cname, "size")]
    for fname, _ in cls._fields_:
        assert getattr(cls, fname).offset == layout[(cname, fname)], (cname, fname)


def test_constants_match_header(layout):
    for k in CONSTANTS:
        assert getattr(smsm, k) == layout[("const", k)], k
