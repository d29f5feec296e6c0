"""The ctypes mirrors of the C structs match the headers byte for byte: a small
C program compiled against include/pic.h (and the oracle's header) prints the
size of every struct and the offset of every field the bindings declare."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

import oracle as O
import paper_1801_00972_gb300 as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _layout_c(header, structs):
    lines = ["#include <stddef.h>", "#include <stdio.h>", f'#include "{header}"', "int main(void) {"]
    for cname, pyname, cls in structs:
        lines.append(f'  printf("{pyname} sizeof %zu\\n", sizeof({cname}));')
        for field in cls._fields_:
            f = field[0]
            lines.append(f'  printf("{pyname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    return "\n".join(lines) + "\n"


def _measure(tmp_path, header, incdir, structs):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text(_layout_c(header, structs))
    subprocess.run([cc, "-std=c99", "-I", incdir, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        name, field, value = line.split()
        got[(name, field)] = int(value)
    return got


def _check(got, structs):
    for _, pyname, cls in structs:
        assert got[(pyname, "sizeof")] == C.sizeof(cls), pyname
        for field in cls._fields_:
            assert got[(pyname, field[0])] == getattr(cls, field[0]).offset, (pyname, field[0])


def test_library_structs_match_pic_h(tmp_path):
    structs = [("pic_mesh", "pic_mesh", P.pic_mesh), ("pic_electrodes", "pic_electrodes", P.pic_electrodes),
               ("pic_gas", "pic_gas", P.pic_gas), ("pic_grains", "pic_grains", P.pic_grains),
               ("pic_run", "pic_run", P.pic_run), ("pic_tuning", "pic_tuning", P.pic_tuning)]
    _check(_measure(tmp_path, "pic.h", os.path.join(ROOT, "include"), structs), structs)


def test_oracle_config_matches_its_header(tmp_path):
    structs = [("orc_cfg", "orc_cfg", O.Cfg)]
    _check(_measure(tmp_path, "pic_oracle.h", os.path.join(ROOT, "oracle"), structs), structs)
