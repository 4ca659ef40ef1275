"""The public header is plain C (C99, compiled with gcc -pedantic) and the
Python mirrors of its structs (RunCfg, BatchItem, Tanner) have the same size
and field offsets as the C compiler gives them.  No GPU needed."""
import ctypes
import os
import shutil
import subprocess

import pytest

import paper_2212_06985_gb300 as t3d

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MIRRORS = {"t3d_run_cfg": t3d.RunCfg, "t3d_batch_item": t3d.BatchItem, "t3d_tanner": t3d.Tanner}
KINDS = sorted(t3d.KERNEL_KINDS)


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    d = tmp_path_factory.mktemp("abi")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "toric3d.h"', 'int main(void) {']
    for cname, py in MIRRORS.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    for name in KINDS:
        lines.append(f'    printf("kind {name} %d\\n", (int)T3D_K_{name.upper()});')
    lines.append('    printf("kind count %d\\n", (int)T3D_K_COUNT);')
    lines += ['    return 0;', '}']
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe)], check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        cname, field, value = line.split()
        layout[(cname, field)] = int(value)
    return layout


@pytest.mark.parametrize("cname", sorted(MIRRORS))
def test_python_mirror_matches_c_layout(c_layout, cname):
    py = MIRRORS[cname]
    assert ctypes.sizeof(py) == c_layout[(cname, "size")]
    for fname, _ in py._fields_:
        assert getattr(py, fname).offset == c_layout[(cname, fname)], fname


def test_kernel_kinds_match_c_enum(c_layout):
    for name, value in t3d.KERNEL_KINDS.items():
        assert c_layout[("kind", name)] == value, name
    assert c_layout[("kind", "count")] == len(t3d.KERNEL_KINDS)
