"""The binding's ctypes structures have the layout of the C structures in
include/jslam.h: a small C program, compiled here against the header,
prints sizeof and offsetof of every field the binding declares, and each
must equal ctypes' size and offset (a field added, dropped, reordered or
retyped on one side only fails here, on the CPU)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2410_04090_gb300 import jslam

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PAIRS = [("jslam_config", jslam.Config), ("jslam_image", jslam.Image), ("jslam_stereo_job", jslam.StereoJob),
         ("jslam_keypoints", jslam.Keypoints), ("jslam_matches", jslam.Matches), ("jslam_refined", jslam.Refined),
         ("jslam_level_view", jslam.LevelView), ("jslam_tuning", jslam.Tuning), ("jslam_skip_view", jslam.SkipView)]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("layout")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "jslam.h"', "int main(void) {"]
    for cname, cls in PAIRS:
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                           "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True)
    return {(a, b): int(c) for a, b, c in (ln.split() for ln in out.splitlines())}


@pytest.mark.parametrize("cname,cls", PAIRS, ids=[c for c, _ in PAIRS])
def test_struct_layout_matches_the_header(c_layout, cname, cls):
    assert ctypes.sizeof(cls) == c_layout[cname, "sizeof"], cname
    for fname, _ in cls._fields_:
        assert getattr(cls, fname).offset == c_layout[cname, fname], (cname, fname)
