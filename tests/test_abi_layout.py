"""The ctypes mirror of include/tsvd.h against the header itself, on CPU: a small C
program compiled with gcc prints sizeof and offsetof of every struct field and the
value of every #define, and the binding must agree with each one."""

import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

from paper_2403_06218_gb300 import _capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tsvd.h")

STRUCTS = {
    "tsvd_matrix": _capi.TsvdMatrix,
    "tsvd_opts": _capi.TsvdOpts,
    "tsvd_info": _capi.TsvdInfo,
    "tsvd_backward_opts": _capi.TsvdBackwardOpts,
    "tsvd_backward_info": _capi.TsvdBackwardInfo,
}


def _header_defines():
    out = {}
    for line in open(HEADER):
        m = re.match(r"#define\s+(TSVD_[A-Z0-9_]+)\s+(\S.*?)\s*(/\*.*)?$", line)
        if m and m.group(1) != "TSVD_H_":
            out[m.group(1)] = m.group(2)
    return out


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tsvd.h"', "int main(void) {"]
    for cname, cls in STRUCTS.items():
        lines.append(f'  printf("size {cname} %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("off {cname} {field} %zu\\n", offsetof({cname}, {field}));')
    for name in _header_defines():
        lines.append(f'  printf("def {name} %lld\\n", (long long)({name}));')
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    sizes, offs, defs = {}, {}, {}
    for line in out.splitlines():
        kind, *rest = line.split()
        if kind == "size":
            sizes[rest[0]] = int(rest[1])
        elif kind == "off":
            offs[(rest[0], rest[1])] = int(rest[2])
        else:
            defs[rest[0]] = int(rest[1])
    return sizes, offs, defs


@pytest.mark.parametrize("cname", sorted(STRUCTS))
def test_struct_layout_matches_the_header(c_layout, cname):
    sizes, offs, _ = c_layout
    cls = STRUCTS[cname]
    assert C.sizeof(cls) == sizes[cname], cname
    for field, _ in cls._fields_:
        assert getattr(cls, field).offset == offs[(cname, field)], (cname, field)


def test_constants_match_the_header(c_layout):
    _, _, defs = c_layout
    mirrored = {name: getattr(_capi, name) for name in defs if hasattr(_capi, name)}
    # every status code, enumeration and limit the binding uses is mirrored
    for name in ("TSVD_OK", "TSVD_NOT_CONVERGED", "TSVD_ERR_INVALID_ARG", "TSVD_ERR_NONFINITE", "TSVD_ERR_CUDA",
                 "TSVD_ERR_WORKSPACE", "TSVD_ERR_TIMEOUT", "TSVD_ERR_UNSUPPORTED", "TSVD_DENSE", "TSVD_CSR",
                 "TSVD_F64", "TSVD_F32", "TSVD_DEVICE", "TSVD_HOST", "TSVD_METHOD_RSVD", "TSVD_METHOD_BLANCZOS",
                 "TSVD_PREC_FP64", "TSVD_PREC_MIXED", "TSVD_MAX_BLOCK", "TSVD_MAX_SMALL_SVD", "TSVD_FLAG_PROFILE",
                 "TSVD_NOALLOC_SCRATCH_BYTES"):
        assert name in mirrored, name
    for name, value in mirrored.items():
        assert value == defs[name], name
    # the kernel-class names follow the TSVD_K_* indices
    assert defs["TSVD_K_COUNT"] == len(_capi.KERNEL_CLASSES)
    for idx, cls in enumerate(_capi.KERNEL_CLASSES):
        key = {"a_products": "TSVD_K_APROD"}.get(cls, "TSVD_K_" + cls.upper())
        assert defs[key] == idx, cls
    assert _capi.TsvdInfo.prof_ms.size == 8 * defs["TSVD_K_COUNT"]
