"""The binding agrees with include/jslam.h.  Structures: a small C program,
compiled here against the header, prints sizeof and offsetof of every field
the binding declares, and each must equal ctypes' size and offset.
Functions: every prototype's arguments and result have the kinds the
binding declares.  A field or argument added, dropped, reordered or retyped
on one side only fails here, on the CPU."""
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


CONSTANTS = {"JSLAM_OK": "OK", "JSLAM_ERR_ARG": "ERR_ARG", "JSLAM_ERR_CUDA": "ERR_CUDA", "JSLAM_ERR_NOMEM": "ERR_NOMEM",
             "JSLAM_ERR_CAPACITY": "ERR_CAPACITY", "JSLAM_ERR_TIMEOUT": "ERR_TIMEOUT", "JSLAM_ERR_STATE": "ERR_STATE",
             "JSLAM_MEM_DEVICE": "MEM_DEVICE", "JSLAM_MEM_HOST": "MEM_HOST"}


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
    for name in CONSTANTS:
        lines.append(f'  printf("const {name} %d\\n", (int){name});')
    lines += ["  return 0;", "}"]
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                           "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True)
    return {(a, b): int(c) for a, b, c in (ln.split() for ln in out.splitlines())}


def test_constants_match_the_header(c_layout):
    for cname, pyname in CONSTANTS.items():
        assert getattr(jslam, pyname) == c_layout["const", cname], cname


@pytest.mark.parametrize("cname,cls", PAIRS, ids=[c for c, _ in PAIRS])
def test_struct_layout_matches_the_header(c_layout, cname, cls):
    assert ctypes.sizeof(cls) == c_layout[cname, "sizeof"], cname
    for fname, _ in cls._fields_:
        assert getattr(cls, fname).offset == c_layout[cname, fname], (cname, fname)


def _c_kind(decl):
    d = " ".join(decl.replace("const", " ").split())
    if "*" in d:
        return "ptr"
    t = d.rsplit(" ", 1)[0] if " " in d else d
    return {"int32_t": "i32", "int": "i32", "float": "f32", "double": "f64", "size_t": "size",
            "jslam_status": "i32", "void": "void"}.get(t, "struct:" + t)


def _ctypes_kind(t):
    if t is None:
        return "void"
    if t in (ctypes.c_void_p, ctypes.c_char_p) or getattr(t, "_type_", None) is not None and \
            isinstance(t, type) and issubclass(t, ctypes._Pointer):
        return "ptr"
    names = {cls: c for c, cls in PAIRS}
    if t in names:
        return "struct:" + names[t]
    if t is ctypes.c_size_t:  # checked before the integers: an alias of c_ulong here
        return "size"
    return {ctypes.c_int32: "i32", ctypes.c_float: "f32", ctypes.c_double: "f64"}[t]


def test_prototypes_match_the_binding():
    """Every entry point the header declares has, in the binding, the same
    number of arguments and the same kind (pointer, 32-bit integer, float,
    double, size_t or a structure by value) at every position, and the same
    kind of result."""
    import re
    text = open(os.path.join(ROOT, "include", "jslam.h")).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    protos = re.findall(r"\b(jslam_status|void|int32_t|const char\s*\*)\s*(jslam_\w+)\s*\(([^;{]*?)\)\s*;", text,
                        flags=re.S)
    lib = jslam.lib()
    seen = set()
    for ret, name, params in protos:
        params = [p.strip() for p in params.split(",")]
        want = [] if params == ["void"] else [_c_kind(p) for p in params]
        fn = getattr(lib, name)
        got = [_ctypes_kind(t) for t in fn.argtypes]
        assert got == want, (name, got, want)
        rk = "ptr" if "*" in ret else _c_kind(ret + " r")
        assert _ctypes_kind(fn.restype) == rk, (name, fn.restype, ret)
        seen.add(name)
    assert seen == set(jslam.SYMBOLS)


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No fallback: with the compiled library absent, the first call into the
    binding raises (and names the build step), in a fresh process state."""
    monkeypatch.setattr(jslam, "LIB_PATH", str(tmp_path / "libjslam.so"))
    monkeypatch.setattr(jslam, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        jslam.lib()
    with pytest.raises(RuntimeError, match="missing"):
        jslam.Frontend(max_width=64, max_height=64, max_feats=10)
