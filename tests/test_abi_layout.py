"""The ctypes binding against the C header (no GPU): every struct has the C layout (size and the
offset of every field, compiled by gcc from include/ls.h), every constant has the header's value,
and every function is declared with the header's number of parameters."""
import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

from paper_1910_13844_gb300 import _abi

STRUCTS = ["ls_grid", "ls_options", "ls_stats", "ls_server_options", "ls_request", "ls_kernel_times",
           "ls_result", "ls_tune"]
CONSTANTS = [n for n in dir(_abi) if re.fullmatch(r"LS_[A-Z0-9_]+", n) and isinstance(getattr(_abi, n), int)]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory, repo_root):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    d = tmp_path_factory.mktemp("layout")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ls.h"', "int main(void) {"]
    for s in STRUCTS:
        lines.append(f'  printf("size {s} %zu\\n", sizeof({s}));')
        for name, _ in getattr(_abi, s)._fields_:
            lines.append(f'  printf("offset {s}.{name} %zu\\n", offsetof({s}, {name}));')
    for n in CONSTANTS:
        lines.append(f'  printf("const {n} %lld\\n", (long long){n});')
    lines.append('  printf("const LS_K_COUNT %d\\n", (int)LS_K_COUNT);')
    lines += ["  return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(repo_root, "include"), str(src),
                    "-o", str(exe)], check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        kind, key, val = line.split()
        table[(kind, key)] = int(val)
    return table


@pytest.mark.parametrize("name", STRUCTS)
def test_struct_layout_matches_the_header(c_layout, name):
    cls = getattr(_abi, name)
    assert C.sizeof(cls) == c_layout[("size", name)]
    for field, _ in cls._fields_:
        assert getattr(cls, field).offset == c_layout[("offset", f"{name}.{field}")], field


def test_constants_match_the_header(c_layout):
    assert CONSTANTS, "no constants found in the binding"
    for n in CONSTANTS:
        assert getattr(_abi, n) == c_layout[("const", n)], n
    # the per-kind arrays of ls_kernel_times and the binding's kind names have LS_K_COUNT entries
    assert len(_abi.LS_K_NAMES) == c_layout[("const", "LS_K_COUNT")]


def _prototypes(header_text):
    text = re.sub(r"/\*.*?\*/", " ", header_text, flags=re.S)
    text = re.sub(r"#[^\n]*", " ", text)
    protos = {}
    for m in re.finditer(r"\b(ls_[a-z0-9_]+)\s*\(([^;{}]*?)\)\s*;", text):
        name, params = m.group(1), " ".join(m.group(2).split())
        protos[name] = 0 if params in ("", "void") else params.count(",") + 1
    return protos


def test_every_function_has_the_header_parameter_count(repo_root):
    protos = _prototypes(open(os.path.join(repo_root, "include", "ls.h")).read())
    assert set(protos) == set(_abi.SIGNATURES)
    for name, (_, argtypes) in _abi.SIGNATURES.items():
        assert len(argtypes) == protos[name], name
